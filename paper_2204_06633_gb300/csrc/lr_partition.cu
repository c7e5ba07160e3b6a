// Multi-GPU partitioning of the response (host only: no device, context or plan is touched).
//
// The response shards two ways (one process per GPU, no collective on the data path):
//  - across sources: the sources of a batch (or the walkers of a sampler) are independent, so
//    they are dealt to ranks by a length-balanced greedy rule and each rank runs its own batched
//    launch;
//  - across time for one long source: disjoint output ranges per rank; every rank computes its
//    range widened by the TDI reach on each side (the link series a TDI output reads, Eqs.
//    tdi1/tdi2) and keeps its own outputs, so the only exchange is the replicated strain halo at
//    set-up.  Adjoint partials then add: the sky-angle gradients as three numbers, the strain
//    gradients where the ranks' input windows overlap.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "lisaresp.h"

extern "C" {

LR_API int lr_partition_sources(int64_t S, const int64_t *lengths, int ranks, int *rank_of, int64_t *load)
{
    if (S < 0 || ranks < 1 || (S > 0 && (!lengths || !rank_of))) return LR_ERR_INVALID_ARG;
    for (int64_t s = 0; s < S; ++s)
        if (lengths[s] < 0) return LR_ERR_INVALID_ARG;
    std::vector<int64_t> order((size_t)S);
    std::iota(order.begin(), order.end(), (int64_t)0);
    // longest first; equal lengths in index order (a total order: every rank gets the same deal)
    std::sort(order.begin(), order.end(), [lengths](int64_t a, int64_t b) {
        return lengths[a] != lengths[b] ? lengths[a] > lengths[b] : a < b;
    });
    std::vector<int64_t> tot((size_t)ranks, 0);
    for (int64_t s : order) {
        int best = 0;
        for (int r = 1; r < ranks; ++r)
            if (tot[(size_t)r] < tot[(size_t)best]) best = r;  // least loaded, lowest rank on ties
        rank_of[s] = best;
        tot[(size_t)best] += lengths[s];
    }
    if (load)
        for (int r = 0; r < ranks; ++r) load[r] = tot[(size_t)r];
    return LR_OK;
}

LR_API int lr_partition_time(int64_t n, int64_t halo_left, int64_t halo_right, int64_t align, int ranks, int rank,
                             lr_time_shard *out)
{
    if (!out || n < 0 || halo_left < 0 || halo_right < 0 || align < 1 || ranks < 1 || rank < 0 || rank >= ranks)
        return LR_ERR_INVALID_ARG;
    // owned ranges: whole units of `align` outputs dealt as evenly as possible, in rank order; the
    // extra units go to the last ranks, which also hold the (possibly partial) last unit, so the
    // owned counts differ by at most `align`
    const int64_t units = (n + align - 1) / align;
    const int64_t per = units / ranks, extra = units % ranks, plain = ranks - extra;
    const int64_t u0 = (int64_t)rank * per + std::max<int64_t>(0, rank - plain);
    const int64_t u1 = u0 + per + (rank >= plain ? 1 : 0);
    const int64_t first = std::min(n, u0 * align), end = std::min(n, u1 * align);
    out->first = first;
    out->count = end - first;
    // computed span: the owned range widened by the halos, the edges rounded out to `align` (so
    // the span's tiles are the unsplit run's tiles) and clamped to [0, n)
    int64_t lo = first - halo_left, hi = end + halo_right;
    lo = lo <= 0 ? 0 : (lo / align) * align;
    hi = hi >= n ? n : std::min(n, ((hi + align - 1) / align) * align);
    if (out->count == 0) lo = hi = first;
    out->lo = lo;
    out->hi = hi;
    return LR_OK;
}

}  // extern "C"
