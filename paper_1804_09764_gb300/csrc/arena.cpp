// arena.cpp -- best-fit sub-allocator over the device arena.
//
// Every device buffer of the library (graphs, count tables, per-plan
// workspaces) is carved from one allocation whose size is the HBM budget, so
// "fits the budget" is exactly "the arena can place it".  Free blocks are kept
// by offset and coalesced on release.
#include "runtime.h"

namespace cc {

namespace {
constexpr uint64_t kAlign = 256;
inline uint64_t round_up(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
}  // namespace

void Arena::init(char *base, uint64_t bytes)
{
    base_ = base;
    cap_ = bytes / kAlign * kAlign;
    free_.clear();
    used_.clear();
    if (cap_) free_[0] = cap_;
    free_total_ = cap_;
}

void *Arena::alloc(uint64_t bytes)
{
    uint64_t need = round_up(bytes ? bytes : 1);
    auto best = free_.end();
    for (auto it = free_.begin(); it != free_.end(); ++it)
        if (it->second >= need && (best == free_.end() || it->second < best->second)) best = it;
    if (best == free_.end()) return nullptr;
    uint64_t off = best->first, sz = best->second;
    free_.erase(best);
    if (sz > need) free_[off + need] = sz - need;
    used_[off] = need;
    free_total_ -= need;
    return base_ + off;
}

void Arena::free(void *p)
{
    if (!p) return;
    uint64_t off = (uint64_t)((char *)p - base_);
    auto it = used_.find(off);
    if (it == used_.end()) return;
    uint64_t sz = it->second;
    used_.erase(it);
    free_total_ += sz;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {
        sz += nx->second;
        free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
        --pv;
        if (pv->first + pv->second == off) {
            pv->second += sz;
            return;
        }
    }
    free_[off] = sz;
}

uint64_t Arena::largest_free() const
{
    uint64_t m = 0;
    for (auto &kv : free_) m = kv.second > m ? kv.second : m;
    return m;
}

}  // namespace cc
