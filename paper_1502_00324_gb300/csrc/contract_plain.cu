// contract_plain.cu -- the CUDA-core form of the search: C' = A' . D'^T with
// int32 multiply-adds in registers, fused with the scoring epilogue.
//
// A' rows are (range, isometry) pairs holding T_k^-1(r) - 128 (the isometry
// moved to the range side: sum r . T_k(d') = sum T_k^-1(r) . d', Sec. 2);
// D' rows are pool domains holding d' - 510.  Both come in the tile layout of
// common.cuh.  One block owns a 128-row M tile (16 ranges x 8 isometries)
// and a chunk of 128-column tiles; thread (ty, tx) owns range ty of the tile
// (its 8 isometry rows) and the column groups 4tx..4tx+3 and 64+4tx..64+4tx+3
// of each tile.
#include "epilogue.cuh"
#include "kernels.h"

namespace fic {

template <int K, int NS>
__global__ void __launch_bounds__(256)
contract_plain_kernel(const Problem* __restrict__ probs, int n_probs,
                      const int* __restrict__ n_items_dev, const __grid_constant__ StepParams sp)
{
    // one block per work item; M tiles vary fastest (item_coords), so a
    // range's earlier chunks finish before its later ones start (the grid
    // is an upper bound when the item count is in device memory)
    if (n_items_dev && (int)blockIdx.x >= *n_items_dev) return;
    const Problem& Q = probs[find_problem(probs, n_probs, (int)blockIdx.x)];
    const __half* __restrict__ A = Q.A;
    const __half* __restrict__ D = Q.D;
    const float* __restrict__ cf = Q.cf;
    const ColExact* __restrict__ ci = Q.ci;
    const RowConst* __restrict__ rc = Q.rc;
    Best* __restrict__ part = Q.part;
    long long* __restrict__ gbest = Q.gbest;
    const int64_t rows_pad = Q.rows_pad, cols_pad = Q.cols_pad;
    const int R = Q.R, dn = Q.dn, ctiles_per_chunk = Q.per_chunk, n_ctiles = Q.n_ct,
              n_chunks = Q.n_chunks;
    const int local = (int)blockIdx.x - Q.item_start;
    int chunk, mtile;
    item_coords(Q, local, chunk, mtile);
    __shared__ __align__(16) int sA[16][128];
    __shared__ __align__(16) int sD[16][128];
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int range = mtile * kRangesPerTile + ty;
    const RowConst r = range < R ? rc[range] : RowConst{0, 0, 0.f, 0.f};
    // flat ranges are resolved in the split step (h = p^2 Vd)
    const bool valid = range < R && !range_is_flat(r, sp.n);
    const float inv_n = 1.0f / (float)sp.n;

    // thresholds are per range: the 8 isometries of a thread and the 16
    // threads of a range share theirs every tile, together with the best key
    // other chunks of the range have published (read one tile ahead)
    long long* const gb = gbest + range;
    RowState st[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        row_state_init(st[i]);
        if (valid) row_state_seed(st[i], gb, inv_n, r.delta);
    }
    long long gseen = valid ? __ldcg(gb) : kNoCandidate;
    long long gpub = kNoCandidate;

    const int ct0 = chunk * ctiles_per_chunk;
    const int ct1 = min(n_ctiles, ct0 + ctiles_per_chunk);
    const int lrow = tid & 127, lkg = tid >> 7;

    for (int ct = ct0; ct < ct1; ++ct) {
        int acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0;

#pragma unroll 1
        for (int kc = 0; kc < K / 16; ++kc) {
            const int k0 = kc * 16 + lkg * 8;
            const uint4 va = *reinterpret_cast<const uint4*>(
                A + tile_off((int64_t)mtile * kMTile + lrow, k0, rows_pad, K));
            const uint4 vd = *reinterpret_cast<const uint4*>(
                D + tile_off((int64_t)ct * 128 + lrow, k0, cols_pad, K));
            const __half* ha = reinterpret_cast<const __half*>(&va);
            const __half* hd = reinterpret_cast<const __half*>(&vd);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                sA[lkg * 8 + e][lrow] = __half2int_rn(ha[e]);
                sD[lkg * 8 + e][lrow] = __half2int_rn(hd[e]);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int4 a0 = *reinterpret_cast<const int4*>(&sA[k][ty * 8]);
                const int4 a1 = *reinterpret_cast<const int4*>(&sA[k][ty * 8 + 4]);
                const int av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const int4 d0 = *reinterpret_cast<const int4*>(&sD[k][4 * tx]);
                const int4 d1 = *reinterpret_cast<const int4*>(&sD[k][64 + 4 * tx]);
                const int dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * dv[j];
            }
            __syncthreads();
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = (float)acc[i][j];
                epi_groups<NS, 2>(st[i], x, cf, ct * 32 + tx, 16, 0, (unsigned)i, -r.a, r.delta,
                                  inv_n, r.sr, ci, dn, &sp);
            }
        }
        float t = gseen < kNoCandidate ? thr_from_h(gseen, inv_n, r.delta) : st[0].thr;
        long long hmin = st[0].h;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            t = fminf(t, st[i].thr);
            hmin = min(hmin, st[i].h);
        }
#pragma unroll
        for (int m = 1; m < 16; m <<= 1) t = fminf(t, __shfl_xor_sync(0xffffffffu, t, m));
#pragma unroll
        for (int i = 0; i < 8; ++i) st[i].thr = t;
        if (valid) {
            gseen = __ldcg(gb);
            if (hmin < gpub) {
                atomicMin(gb, hmin);
                gpub = hmin;
            }
        }
    }
    if (valid)
#pragma unroll
        for (int i = 0; i < 8; ++i) row_state_publish(st[i], gb);
    // best over the 8 isometries held by this thread, then over the 16 threads
    long long h = st[0].h;
    unsigned idx = st[0].idx;
#pragma unroll
    for (int i = 1; i < 8; ++i)
        if (key_less(st[i].h, st[i].idx, h, idx)) {
            h = st[i].h;
            idx = st[i].idx;
        }
#pragma unroll
    for (int m = 1; m < 16; m <<= 1) key_min_shfl(h, idx, m);
    if (tx == 0 && valid) {
        Best b;
        b.h = h;
        b.idx = idx;
        b.pad = 0;
        part[(int64_t)range * n_chunks + chunk] = b;
    }
}

template <int K>
static cudaError_t launch_plain_k(const ContractArgs& a, cudaStream_t s)
{
    if (a.n_items == 0) return cudaSuccess;
    switch (a.sp.ns) {
        case 1: contract_plain_kernel<K, 1><<<a.n_items, 256, 0, s>>>(a.probs, a.n_probs, a.n_items_dev, a.sp); break;
        case 2: contract_plain_kernel<K, 2><<<a.n_items, 256, 0, s>>>(a.probs, a.n_probs, a.n_items_dev, a.sp); break;
        case 3: contract_plain_kernel<K, 3><<<a.n_items, 256, 0, s>>>(a.probs, a.n_probs, a.n_items_dev, a.sp); break;
        default: contract_plain_kernel<K, 0><<<a.n_items, 256, 0, s>>>(a.probs, a.n_probs, a.n_items_dev, a.sp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_contract_plain(const ContractArgs& a, cudaStream_t s)
{
    switch (a.K) {
        case 16: return launch_plain_k<16>(a, s);
        case 64: return launch_plain_k<64>(a, s);
        case 256: return launch_plain_k<256>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fic
