// estimate.cpp -- Algorithm 1's outer loop: how many colourings a (1 +- epsilon)
// estimate with confidence 1 - delta needs, and the median of group means over
// them (arXiv 1804.09764, Section 2.1, Algorithm 1 and Eq. 3).
//
// The paper states N_iter = O(e^k log(1/delta) / epsilon^2) and t = O(log(1/delta))
// groups without constants; the constants here follow from the variance bound
// and the two tail inequalities given with cc_iterations_for in include/cc.h
// (k^k/k! <= e^k, so the count is within the paper's O(.)).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "runtime.h"

using namespace cc;

namespace {

// exact copies (little-endian 64-bit limbs) to the nearest double
double limbs_to_double(const uint64_t *x, int L)
{
    double v = 0;
    for (int l = L - 1; l >= 0; l--) v = v * 18446744073709551616.0 + (double)x[l];
    return v;
}

}  // namespace

extern "C" {

cc_status cc_iterations_for(int32_t k, double epsilon, double delta, int64_t *n_iter, int32_t *groups)
{
    if (!n_iter || !groups) return fail(CC_ERR_INVALID_ARG, "NULL output");
    if (k < 1 || k > kMaxK) return fail(CC_ERR_K_RANGE, "k must be in 1..16");
    if (!(epsilon > 0) || !(delta > 0 && delta < 1) || !std::isfinite(epsilon))
        return fail(CC_ERR_INVALID_ARG, "need epsilon > 0 and 0 < delta < 1");
    // 1/p = k^k / k!, accumulated as a product of k/i
    double inv_p = 1;
    for (int i = 1; i <= k; i++) inv_p *= (double)k / i;
    const double s = std::max(1.0, std::ceil(4.0 * (inv_p - 1.0) / (epsilon * epsilon)));
    const double t = std::max(1.0, std::ceil(8.0 * std::log(1.0 / delta)));
    if (!(s * t < 4.611686018427387904e18) || t > 2147483647.0)
        return fail(CC_ERR_CAPACITY, "sample size exceeds 2^62 colourings");
    *n_iter = (int64_t)s * (int64_t)t;
    *groups = (int32_t)t;
    return CC_OK;
}

cc_status cc_estimate(cc_ctx *ctx, cc_graph_id g, cc_template_id t, uint64_t seed, int64_t first_iter,
                      double epsilon, double delta, int64_t max_iter, cc_estimate_result *out)
{
    if (!ctx || !out) return fail(CC_ERR_INVALID_ARG, "ctx or out is NULL");
    if (first_iter < 0) return fail(CC_ERR_INVALID_ARG, "first_iter < 0");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    auto tit = c->templates.find(t);
    if (tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown template");
    const int k = tit->second->k;
    int64_t n = 0;
    int32_t groups = 0;
    cc_status rc = cc_iterations_for(k, epsilon, delta, &n, &groups);
    if (rc != CC_OK) return rc;
    if (max_iter > 0 && n > max_iter)
        return fail(CC_ERR_CAPACITY, "the estimate needs " + std::to_string(n) + " colourings > max_iter " +
                                         std::to_string(max_iter));
    const int64_t s = n / groups;
    const auto t0 = std::chrono::steady_clock::now();
    cudaSetDevice(c->device);
    double kk = std::pow((double)k, (double)k), kf = 1;
    for (int i = 2; i <= k; i++) kf *= i;
    constexpr int kChunk = 4096, kCap = 4;
    std::vector<uint64_t> counts((size_t)kChunk * kCap);
    std::vector<double> gsum(groups, 0.0);
    double total = 0, dev = 0;
    for (int64_t j0 = 0; j0 < n; j0 += kChunk) {
        CountJob job;
        job.seed = seed;
        job.first_iter = first_iter + j0;
        job.n_iter = (int32_t)std::min<int64_t>(kChunk, n - j0);
        job.mom_groups = 1;
        job.width_bits = -1;
        cc_result r;
        std::memset(&r, 0, sizeof r);
        rc = count_sync(c, g, t, job, counts.data(), kCap, nullptr, nullptr, &r);
        if (rc != CC_OK) return rc;
        if (!r.exact) return fail(CC_ERR_WIDTH, "counts are not exact");
        dev += r.device_seconds;
        for (int j = 0; j < job.n_iter; j++) {
            const double est = limbs_to_double(&counts[(size_t)j * kCap], kCap) * (kk / kf);
            gsum[(j0 + j) / s] += est;
            total += est;
        }
    }
    std::vector<double> means(groups);
    for (int i = 0; i < groups; i++) means[i] = gsum[i] / (double)s;
    std::sort(means.begin(), means.end());
    std::memset(out, 0, sizeof *out);
    out->k = k;
    out->groups = groups;
    out->n_iter = n;
    out->per_group = s;
    out->estimate = (groups % 2) ? means[groups / 2] : 0.5 * (means[groups / 2 - 1] + means[groups / 2]);
    out->mean = total / (double)n;
    out->min_group_mean = means.front();
    out->max_group_mean = means.back();
    out->device_seconds = dev;
    out->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return CC_OK;
}

}  // extern "C"
