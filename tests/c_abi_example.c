/*
 * A C caller of the library (include/cc.h), no Python involved: a triangle
 * with a pendant vertex, the 3-vertex path counted over four colourings.  The
 * graph has exactly 5 copies of the path (sum over vertices of C(deg, 2)), and
 * the estimate of Eq. 3 averages k^k/k! times the colourful copies.
 *
 * Build:  gcc -std=c11 -I include tests/c_abi_example.c \
 *             -L paper_1804_09764_gb300/_build -lcc_gb300 \
 *             -Wl,-rpath,paper_1804_09764_gb300/_build -o c_abi_example
 * Run on a GPU: ./c_abi_example
 */
#include <stdint.h>
#include <stdio.h>

#include "cc.h"

static int check(cc_status s, const char *what)
{
    if (s != CC_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, cc_status_string(s), cc_last_error());
        return 1;
    }
    return 0;
}

int main(void)
{
    cc_options opt;
    cc_default_options(&opt);
    opt.hbm_budget_bytes = 1ull << 30; /* the library allocates this arena itself */
    cc_ctx *ctx = NULL;
    if (check(cc_create(&ctx, &opt), "cc_create")) return 1;

    /* edges 0-1, 1-2, 2-0, 2-3, both directions in CSR */
    const int64_t row_ptr[5] = {0, 2, 4, 7, 8};
    const int32_t col_idx[8] = {1, 2, 0, 2, 0, 1, 3, 2};
    const int32_t path3[4] = {0, 1, 1, 2};
    cc_graph_id g;
    cc_template_id t;
    uint64_t counts[4 * 4]; /* 4 colourings x up to 4 limbs */
    cc_result res;
    int rc = check(cc_graph_load_csr(ctx, 4, row_ptr, col_idx, CC_VALIDATE, &g), "cc_graph_load_csr") ||
             check(cc_template_load(ctx, 3, path3, -1, &t), "cc_template_load") ||
             check(cc_count(ctx, g, t, 7, 4, counts, 4, &res), "cc_count");
    if (!rc) {
        for (int j = 0; j < 4; j++)
            printf("colouring %d: %llu colourful copies\n", j, (unsigned long long)counts[4 * j]);
        printf("estimate %.3f (the graph holds 5 copies), |Aut| = %lld\n", res.estimate, (long long)res.aut);
    }
    cc_destroy(ctx);
    return rc;
}
