// contract_tc.cu -- the tensor-core form of the search on sm_103a:
// C' = A' . D'^T on tcgen05 (kind::f16, FP16 operands, FP32 accumulators in
// tensor memory), fused with the exact scoring/argmin epilogue.
//
// A' rows: (range, isometry) pairs holding T_k^-1(r) - 128 (the isometry is
// applied on the range side because sum d' and sum d'^2 are isometry
// invariant and sum r . T_k(d') = sum T_k^-1(r) . d', Sec. 2); D' rows: pool
// domains holding d' - 510.  With |r - 128| <= 128, |d' - 510| <= 510 and
// n <= 256 terms every partial sum is an integer below 2^24, so the FP32
// accumulators hold C' exactly.
//
// One persistent CTA per SM walks work items (128-row M tile, chunk of
// 256-column N tiles).  Warp roles:
//   warp 0      one thread issues bulk async copies (the TMA engine): the
//               A tile once per item, then per N tile its column constants
//               and its K-blocks of D' into a ring of shared-memory stages;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32
//               accumulators); one thread issues tcgen05.mma per K step and
//               tcgen05.commit to release stages and publish accumulators;
//   warps 2-9   epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one
//               row per thread) for one half of the 256 columns, 64 columns
//               per tcgen05.ld, hands the accumulator back as soon as the
//               last chunk is in registers, and runs the filter/exact argmin
//               of epilogue.cuh.
// Work items are ordered column-chunk-major, so the CTAs running at one
// time share a few D' chunks in L2 instead of streaming all of D'.
// Every mbarrier wait is bounded (cycle counter); on expiry the kernel records
// FIC_ETIMEOUT in the error word, drains its own copies and MMAs, frees TMEM
// and returns.
#include <cstdio>

#include "epilogue.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace fic {
namespace {
using namespace tc;

#ifndef FIC_TC_EPI_WARPS
#define FIC_TC_EPI_WARPS 8
#endif
#ifndef FIC_TC_NTILE
#define FIC_TC_NTILE 256
#endif
constexpr int kEpiWarps = FIC_TC_EPI_WARPS;     // epilogue warps, a multiple of 4
constexpr int kN = FIC_TC_NTILE;                // MMA N = pool columns per tile
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kColsPerEpiWarp = kN * 4 / kEpiWarps;
constexpr int kEpiBlocks = kColsPerEpiWarp / 32;      // 32-column blocks per tile
constexpr int kPartsPerChunk = kEpiWarps / 4;         // partials per (range, column chunk)
// Registers live in four 16K-entry files, one per SM sub-partition, and the
// warps of a block are dealt round-robin to the sub-partitions.
constexpr int kWarpsPerSubPartition = (kThreads / 32 + 3) / 4;
constexpr int kMaxRegsRaw = 16384 / (32 * kWarpsPerSubPartition) / 8 * 8;
constexpr int kMaxRegs = kMaxRegsRaw > 255 ? 255 : kMaxRegsRaw;
constexpr uint32_t kTmemCols = 512;

// Launch parameters; per-image data comes from the problem table (A rows
// are (range, isometry) pairs, row 8 range + k; gbest per range).
struct TcParams {
    const Problem* probs;
    int n_probs, n_items;
    const int* n_items_dev;  // device item count (graph-captured steps), else null
    int* err;
    int nstage, ncf;
};

template <int K, int NS>
__global__ void __maxnreg__(kMaxRegs)
contract_tc_kernel(const __grid_constant__ TcParams P, const __grid_constant__ StepParams sp)
{
    constexpr int KB = K < 64 ? K : 64;
    constexpr int NKB = K / KB;
    constexpr uint32_t kAKBBytes = 128u * KB * 2u;     // one K-block of the A tile
    constexpr uint32_t kBStageBytes = (uint32_t)kN * KB * 2u;  // one K-block of a D tile
    constexpr uint32_t kSbo = KB * 16u;                // 8-row group stride
    constexpr uint32_t kIdesc = idesc_f16_f32(128, kN);
    const uint32_t cf_bytes = (uint32_t)kN * (uint32_t)sp.cw * 4u;
    const int nstage = P.nstage;
    const int ncf = P.ncf;  // column-constant tiles in flight (ring)

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = sA + NKB * kAKBBytes;
    uint8_t* sCF = sB + (size_t)nstage * kBStageBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sCF + (size_t)ncf * cf_bytes);
    // barrier slots: A tile, D stages, accumulators, constant tiles, drain
    const uint32_t b_base = smem_u32(bars);
    const uint32_t a_full = b_base, a_empty = b_base + 8;
    auto full = [&](int s) { return b_base + 16 + 8u * s; };
    auto empty = [&](int s) { return b_base + 16 + 8u * (nstage + s); };
    const uint32_t b_acc = b_base + 16 + 16u * nstage;
    auto tfull = [&](int a) { return b_acc + 8u * a; };
    auto tempty = [&](int a) { return b_acc + 16 + 8u * a; };
    const uint32_t b_cf = b_acc + 32;
    auto cff = [&](int c) { return b_cf + 8u * c; };
    auto cfe = [&](int c) { return b_cf + 8u * (ncf + c); };
    const uint32_t drain = b_cf + 16u * ncf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 + 2 * nstage + 4 + 2 * ncf + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int s = 0; s < nstage; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), kEpiWarps);
        }
        for (int c = 0; c < ncf; ++c) {
            mbar_init(cff(c), 1);
            mbar_init(cfe(c), kEpiWarps);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    int* err = P.err;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // the whole warp walks the schedule; one elected lane issues copies
        int64_t it = 0, cfi = 0, icount = 0;
        int sidx = 0, cidx = 0;          // ring positions of it and cfi
        uint32_t sphase = 0, cphase = 0; // and their parities
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            const int local = item - Q.item_start;
            int chunk, mtile;
            item_coords(Q, local, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            // operand pointers in registers: the waits' memory clobbers would
            // otherwise reload them from the problem table on every tile
            const float* const qcf = Q.cf;
            const __half* const qD = Q.D;
            const int64_t qcols = Q.cols_pad;
            if (!(ok = mbar_wait_warp(a_empty, (uint32_t)((icount & 1) ^ 1), err, kWaitCycles))) break;
            if (elect_one()) {
                mbar_expect_tx(a_full, NKB * kAKBBytes);
                for (int kb = 0; kb < NKB; ++kb)
                    bulk_g2s(smem_u32(sA + kb * kAKBBytes),
                             Q.A + ((int64_t)kb * Q.rows_pad * KB + (int64_t)mtile * 128 * KB),
                             kAKBBytes, a_full);
            }
            __syncwarp();
            ++icount;
            for (int ct = ct0; ct < ct1 && ok; ++ct) {
                if (!(ok = mbar_wait_warp(cfe(cidx), cphase ^ 1, err, kWaitCycles))) break;
                if (elect_one()) {
                    mbar_expect_tx(cff(cidx), cf_bytes);
                    bulk_g2s(smem_u32(sCF + (size_t)cidx * cf_bytes), qcf + (int64_t)ct * kN * sp.cw,
                             cf_bytes, cff(cidx));
                }
                __syncwarp();
                ++cfi;
                if (++cidx == ncf) {
                    cidx = 0;
                    cphase ^= 1;
                }
                for (int kb = 0; kb < NKB; ++kb) {
                    if (!(ok = mbar_wait_warp(empty(sidx), sphase ^ 1, err, kWaitCycles))) break;
                    if (elect_one()) {
                        mbar_expect_tx(full(sidx), kBStageBytes);
                        bulk_g2s(smem_u32(sB + (size_t)sidx * kBStageBytes),
                                 qD + ((int64_t)kb * qcols * KB + (int64_t)ct * kN * KB),
                                 kBStageBytes, full(sidx));
                    }
                    __syncwarp();
                    ++it;
                    if (++sidx == nstage) {
                        sidx = 0;
                        sphase ^= 1;
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            // drain: let every copy this warp armed land before exit
            for (int64_t j = (it > nstage ? it - nstage : 0); j < it; ++j)
                mbar_wait(full((int)(j % nstage)), (uint32_t)((j / nstage) & 1), err + 1,
                          kDrainCycles);
            if (icount > 0) mbar_wait(a_full, (uint32_t)((icount - 1) & 1), err + 1, kDrainCycles);
            for (int64_t j = (cfi > ncf ? cfi - ncf : 0); j < cfi; ++j)
                mbar_wait(cff((int)(j % ncf)), (uint32_t)((j / ncf) & 1), err + 1, kDrainCycles);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        const uint64_t a_desc = smem_desc(smem_u32(sA), 128u, kSbo);
        int64_t tcount = 0, icount = 0;
        int sidx = 0;                    // D' stage ring position
        uint32_t sphase = 0;             // and its parity
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            int chunk, mtile;
            item_coords(Q, item - Q.item_start, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            if (!(ok = mbar_wait_warp(a_full, (uint32_t)(icount & 1), err, kWaitCycles))) break;
            tc_fence_after();
            for (int ct = ct0; ct < ct1 && ok; ++ct) {
                const int acc = (int)(tcount & 1);
                const uint32_t ph = (uint32_t)((tcount >> 1) & 1);
                if (!(ok = mbar_wait_warp(tempty(acc), ph ^ 1, err, kWaitCycles))) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)acc * 256u;  // 256-column slots
                for (int kb = 0; kb < NKB; ++kb) {
                    if (!(ok = mbar_wait_warp(full(sidx), sphase, err, kWaitCycles))) break;
                    tc_fence_after();
                    const uint64_t ak = desc_add(a_desc, (uint32_t)kb * kAKBBytes);
                    const uint64_t bk =
                        smem_desc(smem_u32(sB + (size_t)sidx * kBStageBytes), 128u, kSbo);
                    if (elect_one()) {
#pragma unroll
                        for (int j = 0; j < KB / 16; ++j)
                            tc_mma_f16(d_tmem, desc_add(ak, 256u * j), desc_add(bk, 256u * j), kIdesc,
                                       (kb | j) != 0 ? 1u : 0u);
                        tc_commit(empty(sidx));
                    }
                    __syncwarp();
                    if (++sidx == nstage) {
                        sidx = 0;
                        sphase ^= 1;
                    }
                }
                if (!ok) break;
                if (elect_one()) tc_commit(tfull(acc));
                __syncwarp();
                ++tcount;
            }
            if (!ok) break;
            if (elect_one()) tc_commit(a_empty);
            __syncwarp();
            ++icount;
        }
        // every issued MMA has finished before TMEM is released
        if (elect_one()) tc_commit(drain);
        __syncwarp();
        mbar_wait(drain, 0, err + 1, kWaitCycles);
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - 2;
        const int quad = warp & 3;          // TMEM lanes 32 quad .. 32 quad + 31
        const int cq = e >> 2;              // column slice cq of a tile
        const float inv_n = 1.0f / (float)sp.n;
        int64_t tcount = 0;
        int cidx = 0;                    // constants ring position
        uint32_t cphase = 0;             // and its parity
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            const int local = item - Q.item_start;
            int chunk, mtile;
            item_coords(Q, local, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            const ColExact* qci = Q.ci;
            const int qdn = Q.dn;
            const int row = mtile * 128 + quad * 32 + lane;
            const int range = row >> 3;
            const unsigned iso = (unsigned)(row & 7);
            const RowConst r = range < Q.R ? Q.rc[range] : RowConst{0, 0, 0.f, 0.f};
            // flat ranges are resolved in the split step (h = p^2 Vd)
            const bool valid = range < Q.R && !range_is_flat(r, sp.n);
            RowState st;
            row_state_init(st);
            // thresholds are per range: the 8 isometry lanes of a range share
            // theirs every tile, and the best key that other chunks of the
            // range have published is read one tile ahead
            long long* const gb = Q.gbest + range;
            if (valid) row_state_seed(st, gb, inv_n, r.delta);
            long long gseen = valid ? __ldcg(gb) : kNoCandidate;
            long long gpub = kNoCandidate;
            for (int ct = ct0; ct < ct1; ++ct) {
                if (gseen < kNoCandidate) st.thr = fminf(st.thr, thr_from_h(gseen, inv_n, r.delta));
                st.thr = fminf(st.thr, __shfl_xor_sync(0xffffffffu, st.thr, 1));
                st.thr = fminf(st.thr, __shfl_xor_sync(0xffffffffu, st.thr, 2));
                st.thr = fminf(st.thr, __shfl_xor_sync(0xffffffffu, st.thr, 4));
                if (valid) gseen = __ldcg(gb);
                const int acc = (int)(tcount & 1);
                const uint32_t ph = (uint32_t)((tcount >> 1) & 1);
                const int cb = cidx;
                if (!(ok = mbar_wait(tfull(acc), ph, err, kWaitCycles))) break;
                if (!(ok = mbar_wait(cff(cb), cphase, err, kWaitCycles))) break;
                tc_fence_after();
                const float* cfs = reinterpret_cast<const float*>(sCF + (size_t)cb * cf_bytes);
                const uint32_t tb = tmem_base + ((uint32_t)(quad * 32) << 16) +
                                    (uint32_t)(acc * 256 + cq * kColsPerEpiWarp);  // 256-column slots
#pragma unroll 1
                for (int b = 0; b < kEpiBlocks; ++b) {
                    float x[32];
                    __syncwarp();
                    tmem_ld32_issue(tb + 32u * b, x);
                    tmem_wait32(x);
                    if (b == kEpiBlocks - 1) {
                        // the accumulator is in registers: hand TMEM back to the MMA
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty(acc));
                    }
                    if (valid)
                        epi_groups<NS, 8>(st, x, cfs, (cq * kColsPerEpiWarp + 32 * b) / 4, 1,
                                          ct * kN, iso, -r.a, r.delta, inv_n, r.sr, qci, qdn,
                                          &sp);
                }
                if (st.h < gpub) {
                    atomicMin(gb, st.h);
                    gpub = st.h;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(cfe(cb));
                ++tcount;
                if (++cidx == ncf) {
                    cidx = 0;
                    cphase ^= 1;
                }
            }
            if (!ok) break;
            if (valid) row_state_publish(st, gb);
            // best over the 8 isometries of each range (lanes 8j .. 8j+7)
            long long h = st.h;
            unsigned idx = st.idx;
            key_min_shfl(h, idx, 1);
            key_min_shfl(h, idx, 2);
            key_min_shfl(h, idx, 4);
            if (valid && (lane & 7) == 0) {
                Best b;
                b.h = h;
                b.idx = idx;
                b.pad = 0;
                Q.part[(int64_t)range * (kPartsPerChunk * Q.n_chunks) + kPartsPerChunk * chunk + cq] = b;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols)
                     : "memory");
    }
}

constexpr size_t kSmemBudget = 220 * 1024;
constexpr size_t kSmemMinForOneCta = 120 * 1024;  // > half an SM: one CTA per SM

template <int K>
size_t tc_layout(int cw, int* nstage_out, int* ncf_out)
{
    constexpr int KB = K < 64 ? K : 64;
    const size_t a_bytes = (size_t)128 * K * 2;
    const size_t stage = (size_t)kN * KB * 2;
    const size_t cf_tile = (size_t)kN * cw * 4;
    const int ncf = cf_tile <= 4096 ? 8 : 2;  // deep ring for the usual 1-3 S values
    const size_t fixed = a_bytes + (size_t)ncf * cf_tile + 1024;
    int ns = (int)((kSmemBudget - fixed) / stage);
    if (ns > 8) ns = 8;
    if (ns < 2) ns = 2;
    *nstage_out = ns;
    *ncf_out = ncf;
    size_t total = fixed + (size_t)ns * stage;
    if (total < kSmemMinForOneCta) total = kSmemMinForOneCta;
    return total;
}

template <int K, int NS>
cudaError_t launch_tc_kns(const ContractArgs& a, cudaStream_t s)
{
    int nstage = 0, ncf = 0;
    const size_t smem = tc_layout<K>(a.sp.cw, &nstage, &ncf);
    auto kern = contract_tc_kernel<K, NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    TcParams P;
    P.probs = a.probs;
    P.n_probs = a.n_probs;
    P.n_items = a.n_items;
    P.n_items_dev = a.n_items_dev;
    P.err = a.err;
    P.nstage = nstage;
    P.ncf = ncf;
    const int grid = P.n_items < a.grid_ctas ? P.n_items : a.grid_ctas;
    kern<<<grid, kThreads, smem, s>>>(P, a.sp);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_tc_k(const ContractArgs& a, cudaStream_t s)
{
    switch (a.sp.ns) {
        case 1: return launch_tc_kns<K, 1>(a, s);
        case 2: return launch_tc_kns<K, 2>(a, s);
        case 3: return launch_tc_kns<K, 3>(a, s);
        default: return launch_tc_kns<K, 0>(a, s);
    }
}

}  // namespace

cudaError_t launch_contract_tc(const ContractArgs& a, cudaStream_t s)
{
    switch (a.K) {
        case 16: return launch_tc_k<16>(a, s);
        case 64: return launch_tc_k<64>(a, s);
        case 256: return launch_tc_k<256>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

int contract_tc_parts_per_chunk() { return kPartsPerChunk; }
int contract_tc_ntile() { return kN; }

size_t contract_tc_smem_bytes(int K)
{
    int ns = 0, ncf = 0;
    switch (K) {
        case 16: return tc_layout<16>(3, &ns, &ncf);
        case 64: return tc_layout<64>(3, &ns, &ncf);
        case 256: return tc_layout<256>(3, &ns, &ncf);
        default: return 0;
    }
}

}  // namespace fic
