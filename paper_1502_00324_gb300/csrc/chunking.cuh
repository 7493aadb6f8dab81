// chunking.cuh -- column chunking of the contraction's work items, shared by
// the host step driver and the device-side step plan of graph-captured
// encodes (the same arithmetic on both sides gives the same items).
#pragma once

#include <cstdint>

namespace fic {

// Column chunking of the contraction: work items are (M tile, chunk of
// column tiles).  Chunk counts stay <= 16 x SMs / M tiles, which bounds the
// partial-best buffers.
__host__ __device__ inline int64_t max_chunks(int sm_count, int64_t n_mtiles, int64_t n_ct)
{
    int64_t cap = (16LL * sm_count + n_mtiles - 1) / n_mtiles;
    if (cap > 4096) cap = 4096;
    if (cap > n_ct) cap = n_ct;
    return cap < 1 ? 1 : cap;
}

// A problem alone in its launch: the chunk count that minimises the
// estimated makespan over one item per SM (waves x tiles per item, plus a
// per-item cost of refilling the pipeline, refill tiles).
__host__ __device__ inline void choose_chunks_alone(int sm_count, int64_t n_mtiles, int64_t n_ct,
                                                    int refill, int* n_chunks, int* per_chunk)
{
    const int64_t slots = sm_count;
    const double item_cost = (double)refill;  // in tiles
    int64_t best_nc = 1;
    double best = 1e300;
    const int64_t max_nc = max_chunks(sm_count, n_mtiles, n_ct);
    for (int64_t nc = 1; nc <= max_nc; ++nc) {
        const int64_t per = (n_ct + nc - 1) / nc;
        const int64_t ncs = (n_ct + per - 1) / per;
        if (ncs != nc) continue;
        const int64_t waves = (n_mtiles * nc + slots - 1) / slots;
        const double cost = (double)waves * ((double)per + item_cost);
        if (cost < best - 1e-9) {
            best = cost;
            best_nc = nc;
        }
    }
    *n_chunks = (int)best_nc;
    *per_chunk = (int)((n_ct + best_nc - 1) / best_nc);
}

// Several problems in one launch: items of about tiles_per_item column
// tiles (total tiles / (16 / refill x SMs)), so the persistent CTAs stay
// balanced.
__host__ __device__ inline void choose_chunks_shared(int sm_count, int64_t n_mtiles, int64_t n_ct,
                                                     double tiles_per_item, int* n_chunks,
                                                     int* per_chunk)
{
    int64_t per = (int64_t)(tiles_per_item + 0.5);
    if (per < 1) per = 1;
    if (per > n_ct) per = n_ct;
    int64_t nc = (n_ct + per - 1) / per;
    const int64_t cap = max_chunks(sm_count, n_mtiles, n_ct);
    if (nc > cap) nc = cap;
    per = (n_ct + nc - 1) / nc;
    nc = (n_ct + per - 1) / per;
    *n_chunks = (int)nc;
    *per_chunk = (int)per;
}

}  // namespace fic
