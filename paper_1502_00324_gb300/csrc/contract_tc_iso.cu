// contract_tc_iso.cu -- tensor-core search for 2x2, 4x4 and 8x8 ranges with
// the isometry in the accumulator index.
//
// For one range and one pool domain the 8 isometries share sum d', sum d'^2,
// Vd and the range sums, so the filter of epilogue.cuh,
//   f(k, s) = beta_s - 8 p_s q (C'_k - a m_c),
// is decreasing in C'_k: min over k of f(k, s) = f(max over k of C'_k, s).
// The rounded filter is monotone too (each step is one monotone rounding),
// so evaluating it once on max_k C'_k gives exactly the smallest of the eight
// per-isometry filter values.  Holding all 8 isometries of a range in one
// thread therefore costs one max per element plus the filter per column.
//
// Layout: TMEM lane = range (M = 128 ranges per tile), one accumulator per
// isometry.  A (T_k^-1 r - 128 for k = 0..7, iso-major rows k * Rpad + range)
// stays resident in shared memory for a work item: 8 x 128 x K halves (32 KB
// at K = 16, 128 KB at K = 64).  Per pool tile the MMA issuer runs passes of
// a few isometries, each into one of four 128-column TMEM slots (see
// IsoShape), so the epilogue of one pass overlaps the MMAs of the next three.
//
// Warp roles: warp 0 bulk-copies (TMA engine) the A tiles, the D' stages and
// the column-constant tiles; warp 1 owns TMEM and issues tcgen05.mma /
// tcgen05.commit; warps 2-9 are the epilogue (warp w: TMEM lanes 32 (w % 4)
// .. +31, one half of a tile's columns).  Every mbarrier wait is bounded
// (tc_common.cuh).
#include "epilogue.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace fic {
namespace {
using namespace tc;

// Tile shape by K: N pool columns per tile and PASS isometries per
// accumulator pass; one pass fills a TMEM slot of PASS x N columns and the
// 512 columns hold 512 / (PASS N) slots.  (Four 128-column slots with N = 32
// measured slower than two 256-column slots: the per-tile costs double.)
template <int K> struct IsoShape;
template <> struct IsoShape<16> { static constexpr int N = 64, PASS = 4; };
template <> struct IsoShape<64> { static constexpr int N = 64, PASS = 4; };
// Epilogue decompositions (chosen by the tuner): EPI = 8 warps reading 16
// columns per TMEM load, or EPI = 16 warps reading 8 columns per load (more
// warps to hide latency, fewer registers each).
template <int EPI> struct IsoEpi {
    static constexpr int kEpiWarps = EPI;                    // 4 x column slices
    static constexpr int kThreads = 32 * (2 + EPI);
    static constexpr int kPartsPerChunk = EPI / 4;           // one per column slice
    static constexpr int kChunk = EPI == 16 ? 8 : 16;        // columns per TMEM load
    static constexpr int kWarpsPerSubPartition = (kThreads / 32 + 3) / 4;
    static constexpr int kMaxRegs = 16384 / (32 * kWarpsPerSubPartition) / 8 * 8;
};
constexpr uint32_t kTmemCols = 512;    // all of TMEM: 512 / (PASS N) slots
constexpr int kMaxSlots = 4;

// Launch parameters; per-image data comes from the problem table (A is
// iso-major: row k * (rows_pad / 8) + range; gbest and partials per range).
struct IsoParams {
    const Problem* probs;
    int n_probs, n_items;
    const int* n_items_dev;  // device item count (graph-captured steps), else null
    int* err;
    int nstage, ncf;
};

__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int P, int W>
__device__ __forceinline__ float iso_max(const float (&x)[P][W], int i)
{
    // two instructions for four values: one 2-input and one 3-input maximum
    if constexpr (P == 4) return fmax3(x[0][i], x[1][i], fmaxf(x[2][i], x[3][i]));
    else return fmaxf(x[0][i], x[1][i]);
}

// Filter pass over W columns (W / 4 groups of 4) x P isometries of one
// range: the minimum of each group (gm, for pass 2) and of the block.
template <int NS, int P, int W>
__device__ __forceinline__ float iso_pass1(const float (&x)[P][W], const float* __restrict__ cf,
                                           int g0, float na, const StepParams& sp,
                                           float (&gm)[W / 4])
{
    constexpr int cw = 1 + NS;
    const uint64_t nak = pk2(na, na);
    uint64_t nk[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) nk[s] = pk2(-sp.kf[s], -sp.kf[s]);
#pragma unroll
    for (int g = 0; g < W / 4; ++g) {
        float c[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) c[e] = iso_max<P, W>(x, 4 * g + e);
        const float4* cg = reinterpret_cast<const float4*>(cf + (size_t)(g0 + g) * cw * 4);
        const float4 m = cg[0];
        const uint64_t t01 = fma2(nak, pk2(m.x, m.y), pk2(c[0], c[1]));
        const uint64_t t23 = fma2(nak, pk2(m.z, m.w), pk2(c[2], c[3]));
        float g01 = __int_as_float(0x7f800000), g23 = g01;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float4 b = cg[1 + s];
            float f0, f1, f2, f3;
            upk2(fma2(nk[s], t01, pk2(b.x, b.y)), f0, f1);
            upk2(fma2(nk[s], t23, pk2(b.z, b.w)), f2, f3);
            g01 = fmin3(g01, f0, f1);
            g23 = fmin3(g23, f2, f3);
        }
        gm[g] = fminf(g01, g23);
    }
    float mn = gm[0];
#pragma unroll
    for (int g = 1; g < W / 4; ++g) mn = fminf(mn, gm[g]);
    return mn;
}

// Exact re-scoring of the candidates of a 16-column block whose filter is
// within 2 delta of the block minimum mn and under the range's threshold
// (ci: the tile's exact column sums, staged in shared memory with its
// filter constants, indexed by the column within the tile).
// Candidates of one range arrive out of index order across passes, so a
// candidate is skipped only when its lower bound proves h > h* (index below
// the best) or h > h* - 1 (index above it).
template <int NS, int P, int W>
__device__ __forceinline__ void iso_pass2(RowState& st, const float (&x)[P][W], float mn,
                                          const float (&gm)[W / 4],
                                          const float* __restrict__ cf, int g0, int col_base,
                                          int iso_base, float na, float delta, float inv_n,
                                          int sr, const ColExact* __restrict__ ci, int dn,
                                          const StepParams* __restrict__ spp)
{
    // Compact code on purpose: this path is rare, and fully unrolled it
    // would be thousands of instructions that miss the instruction cache on
    // every entry while the other warps of the CTA wait for this one's TMEM
    // slot.  The chunk goes to a local copy, indexed in rolled loops.
    const StepParams& sp = *spp;
    constexpr int cw = 1 + NS;
    float te = fminf(st.thr, __fadd_ru(mn, 2.0f * delta));
    unsigned gmask = 0;
#pragma unroll
    for (int g = 0; g < W / 4; ++g) gmask |= (gm[g] <= te) ? (1u << g) : 0u;
    if (!gmask) return;
    float xl[P * W];
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
        for (int c = 0; c < W; ++c) xl[j * W + c] = x[j][c];
#pragma unroll 1
    for (; gmask; gmask &= gmask - 1) {
        const int g = __ffs(gmask) - 1;
        const float* cg = cf + (size_t)(g0 + g) * cw * 4;
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
            const int c = 4 * g + e;
            float cmax = xl[c];
#pragma unroll
            for (int j = 1; j < P; ++j) cmax = fmaxf(cmax, xl[j * W + c]);
            float fm = __int_as_float(0x7f800000);
#pragma unroll
            for (int s = 0; s < NS; ++s) fm = fminf(fm, col_filter(cg, e, na, cmax, sp, s));
            if (!(fm <= te)) continue;
            const int col = (g0 + g) * 4 + e + col_base;
#pragma unroll 1
            for (int j = 0; j < P; ++j) {
                const unsigned iso = (unsigned)(iso_base + j);
                const float xj = xl[j * W + c];
                float fj = __int_as_float(0x7f800000), lo = fj;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const float tp = __fmaf_rn(na, cg[e], xj);
                    const float beta = cg[(1 + s) * 4 + e];
                    const float f = __fmaf_rn(-sp.kf[s], tp, beta);
                    const float err = 0x1p-22f * __fmaf_ru(sp.kf[s], fabsf(tp), beta);
                    fj = fminf(fj, f);
                    lo = fminf(lo, __fsub_rd(f, err));
                }
                if (!(fj <= te)) continue;
                if (st.h != kNoCandidate) {
                    const long long bound =
                        pack_idx((unsigned)col, iso, 0) > st.idx ? st.h - 1 : st.h;
                    if (lo > __ll2float_ru(bound) * inv_n) continue;
                }
                st = exact_col(st, xj, cg, e, col, iso, na, delta, inv_n, sr,
                               ci + (g0 + g) * 4 + e, dn, spp, te);
                te = fminf(te, st.thr);
            }
        }
    }
}

// 4 x 8 columns of TMEM (4 accumulators 'stride' columns apart), one wait.
__device__ __forceinline__ void tmem_load_iso(uint32_t taddr, uint32_t stride, float (&x)[4][8])
{
    tmem_ld8_issue(taddr, x[0]);
    tmem_ld8_issue(taddr + stride, x[1]);
    tmem_ld8_issue(taddr + 2 * stride, x[2]);
    tmem_ld8_issue(taddr + 3 * stride, x[3]);
    tmem_wait4x8(x[0], x[1], x[2], x[3]);
}

// P x 16 columns of TMEM (P accumulators 'stride' columns apart), one wait.
template <int P>
__device__ __forceinline__ void tmem_load_iso(uint32_t taddr, uint32_t stride, float (&x)[P][16])
{
    if constexpr (P == 4) {
        tmem_ld16_issue(taddr, x[0]);
        tmem_ld16_issue(taddr + stride, x[1]);
        tmem_ld16_issue(taddr + 2 * stride, x[2]);
        tmem_ld16_issue(taddr + 3 * stride, x[3]);
        tmem_wait4x16(x[0], x[1], x[2], x[3]);
    } else {
        tmem_ld16_issue(taddr, x[0]);
        tmem_ld16_issue(taddr + stride, x[1]);
        tmem_wait2x16(x[0], x[1]);
    }
}

template <int K, int NS, int EPI>
__global__ void __maxnreg__(IsoEpi<EPI>::kMaxRegs)
contract_tc_iso_kernel(const __grid_constant__ IsoParams P, const __grid_constant__ StepParams sp)
{
    constexpr int kEpiWarps = IsoEpi<EPI>::kEpiWarps;
    constexpr int kPartsPerChunk = IsoEpi<EPI>::kPartsPerChunk;
    constexpr int kChunk = IsoEpi<EPI>::kChunk;
    static_assert(K == 16 || K == 64, "one K-block per tile");
    constexpr int kN = IsoShape<K>::N;                // pool columns per tile
    constexpr int kPass = IsoShape<K>::PASS;          // isometries per pass
    constexpr int kPasses = 8 / kPass;
    constexpr int kSlotCols = kPass * kN;             // TMEM columns per pass
    constexpr int kSlots = 512 / kSlotCols;
    constexpr int kWarpCols = kN / (kEpiWarps / 4);   // columns per epilogue warp and tile
    constexpr uint32_t kAIsoBytes = 128u * K * 2u;    // one isometry's A tile
    constexpr uint32_t kBStageBytes = (uint32_t)kN * K * 2u;
    constexpr uint32_t kSbo = K * 16u;                // 8-row group stride
    constexpr uint32_t kIdesc = idesc_f16_f32(128, kN);
    // constants ring: per tile the filter constants, then the exact column sums
    const uint32_t cfc_bytes = (uint32_t)kN * (uint32_t)sp.cw * 4u;
    const uint32_t cf_bytes = cfc_bytes + (uint32_t)kN * (uint32_t)sizeof(ColExact);
    const int nstage = P.nstage, ncf = P.ncf;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = sA + 8 * kAIsoBytes;
    uint8_t* sCF = sB + (size_t)nstage * kBStageBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sCF + (size_t)ncf * cf_bytes);
    const uint32_t b_base = smem_u32(bars);
    const uint32_t a_full = b_base, a_empty = b_base + 8;
    auto full = [&](int s) { return b_base + 16 + 8u * s; };
    auto empty = [&](int s) { return b_base + 16 + 8u * (nstage + s); };
    const uint32_t b_acc = b_base + 16 + 16u * nstage;
    auto tfull = [&](int a) { return b_acc + 8u * a; };
    auto tempty = [&](int a) { return b_acc + 8u * kMaxSlots + 8u * a; };
    const uint32_t b_cf = b_acc + 16u * kMaxSlots;
    auto cff = [&](int c) { return b_cf + 8u * c; };
    auto cfe = [&](int c) { return b_cf + 8u * (ncf + c); };
    const uint32_t drain = b_cf + 16u * ncf;
    uint32_t* tmem_slot =
        reinterpret_cast<uint32_t*>(bars + 2 + 2 * nstage + 2 * kMaxSlots + 2 * ncf + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int s = 0; s < nstage; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < kSlots; ++a) {
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
            const int64_t rpad = Q.rows_pad / 8;
            // operand pointers in registers: the waits' memory clobbers would
            // otherwise reload them from the problem table on every tile
            const float* const qcf = Q.cf;
            const ColExact* const qci = Q.ci;
            const __half* const qD = Q.D;
            if (!(ok = mbar_wait_warp(a_empty, (uint32_t)((icount & 1) ^ 1), err, kWaitCycles))) break;
            if (elect_one()) {
                mbar_expect_tx(a_full, 8 * kAIsoBytes);
                for (int k = 0; k < 8; ++k)
                    bulk_g2s(smem_u32(sA + k * kAIsoBytes),
                             Q.A + ((int64_t)k * rpad + (int64_t)mtile * 128) * K, kAIsoBytes,
                             a_full);
            }
            __syncwarp();
            ++icount;
            for (int ct = ct0; ct < ct1 && ok; ++ct) {
                if (!(ok = mbar_wait_warp(cfe(cidx), cphase ^ 1, err, kWaitCycles))) break;
                if (elect_one()) {
                    mbar_expect_tx(cff(cidx), cf_bytes);
                    bulk_g2s(smem_u32(sCF + (size_t)cidx * cf_bytes), qcf + (int64_t)ct * kN * sp.cw,
                             cfc_bytes, cff(cidx));
                    bulk_g2s(smem_u32(sCF + (size_t)cidx * cf_bytes + cfc_bytes),
                             qci + (int64_t)ct * kN, cf_bytes - cfc_bytes, cff(cidx));
                }
                __syncwarp();
                ++cfi;
                if (++cidx == ncf) {
                    cidx = 0;
                    cphase ^= 1;
                }
                if (!(ok = mbar_wait_warp(empty(sidx), sphase ^ 1, err, kWaitCycles))) break;
                if (elect_one()) {
                    mbar_expect_tx(full(sidx), kBStageBytes);
                    bulk_g2s(smem_u32(sB + (size_t)sidx * kBStageBytes), qD + (int64_t)ct * kN * K,
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
        // warp-uniform schedule with precomputed descriptors; one elected lane
        // issues the MMAs and commits
        const uint64_t a_desc = smem_desc(smem_u32(sA), 128u, kSbo);
        int64_t icount = 0;
        int sidx = 0, slot = 0;          // D' stage and TMEM slot positions
        uint32_t sphase = 0, tphase = 0; // and their parities
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
                if (!(ok = mbar_wait_warp(full(sidx), sphase, err, kWaitCycles))) break;
                tc_fence_after();
                const uint64_t b_desc =
                    smem_desc(smem_u32(sB + (size_t)sidx * kBStageBytes), 128u, kSbo);
#pragma unroll
                for (int pass = 0; pass < kPasses; ++pass) {
                    if (!(ok = mbar_wait_warp(tempty(slot), tphase ^ 1, err, kWaitCycles))) break;
                    tc_fence_after();
                    if (elect_one()) {
#pragma unroll
                        for (int j = 0; j < kPass; ++j) {
                            const uint32_t d_tmem = tmem_base + (uint32_t)(slot * kSlotCols + j * kN);
                            const uint64_t aj = desc_add(a_desc, (uint32_t)(pass * kPass + j) * kAIsoBytes);
#pragma unroll
                            for (int kk = 0; kk < K / 16; ++kk)
                                tc_mma_f16(d_tmem, desc_add(aj, 256u * kk), desc_add(b_desc, 256u * kk),
                                           kIdesc, kk != 0 ? 1u : 0u);
                        }
                        tc_commit(tfull(slot));
                    }
                    __syncwarp();
                    if (++slot == kSlots) {
                        slot = 0;
                        tphase ^= 1;
                    }
                }
                if (!ok) break;
                if (elect_one()) tc_commit(empty(sidx));  // every pass read this stage
                __syncwarp();
                if (++sidx == nstage) {
                    sidx = 0;
                    sphase ^= 1;
                }
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
        const int quad = warp & 3;   // TMEM lanes (ranges) 32 quad .. +31
        const int hsel = e >> 2;     // column slice of a tile
        const float inv_n = 1.0f / (float)sp.n;
        int cidx = 0, slot = 0;          // constants ring and TMEM slot positions
        uint32_t cphase = 0, tphase = 0; // and their parities
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            const int local = item - Q.item_start;
            int chunk, mtile;
            item_coords(Q, local, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            const int qdn = Q.dn;
            const int range = mtile * 128 + quad * 32 + lane;
            const RowConst r = range < Q.R ? Q.rc[range] : RowConst{0, 0, 0.f, 0.f};
            // flat ranges are resolved in the split step (h = p^2 Vd)
            const bool valid = range < Q.R && !range_is_flat(r, sp.n);
            RowState st;
            row_state_init(st);
            long long* const gb = Q.gbest + range;  // in a register for the whole item
            if (valid) row_state_seed(st, gb, inv_n, r.delta);
            // the best key other chunks of this range have published, read one
            // tile ahead; this chunk publishes its own improvements per tile
            long long gseen = valid ? __ldcg(gb) : kNoCandidate;
            long long gpub = kNoCandidate;
            for (int ct = ct0; ct < ct1; ++ct) {
                if (gseen < kNoCandidate) st.thr = fminf(st.thr, thr_from_h(gseen, inv_n, r.delta));
                if (valid) gseen = __ldcg(gb);
                if (!(ok = mbar_wait(cff(cidx), cphase, err, kWaitCycles))) break;
                const float* cfs = reinterpret_cast<const float*>(sCF + (size_t)cidx * cf_bytes);
                const ColExact* cis =
                    reinterpret_cast<const ColExact*>(sCF + (size_t)cidx * cf_bytes + cfc_bytes);
#pragma unroll
                for (int pass = 0; pass < kPasses; ++pass) {
                    if (!(ok = mbar_wait(tfull(slot), tphase, err, kWaitCycles))) break;
                    tc_fence_after();
                    const uint32_t tb = tmem_base + ((uint32_t)(quad * 32) << 16) +
                                        (uint32_t)(slot * kSlotCols + hsel * kWarpCols);
#pragma unroll
                    for (int ch = 0; ch < kWarpCols / kChunk; ++ch) {
                        float x[kPass][kChunk];
                        __syncwarp();
                        tmem_load_iso(tb + (uint32_t)(kChunk * ch), (uint32_t)kN, x);
                        if (ch == kWarpCols / kChunk - 1) {
                            // the pass is in registers: hand the slot back to the MMA
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(tempty(slot));
                        }
                        if (valid) {
                            const int g0 = (hsel * kWarpCols + kChunk * ch) / 4;
                            float gm[kChunk / 4];
                            const float mn = iso_pass1<NS, kPass, kChunk>(x, cfs, g0, -r.a, sp, gm);
                            if (mn <= st.thr)
                                iso_pass2<NS, kPass, kChunk>(st, x, mn, gm, cfs, g0, ct * kN,
                                                             pass * kPass, -r.a, r.delta, inv_n,
                                                             r.sr, cis, qdn, &sp);
                        }
                    }
                    if (++slot == kSlots) {
                        slot = 0;
                        tphase ^= 1;
                    }
                }
                if (!ok) break;
                if (st.h < gpub) {
                    atomicMin(gb, st.h);
                    gpub = st.h;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(cfe(cidx));
                if (++cidx == ncf) {
                    cidx = 0;
                    cphase ^= 1;
                }
            }
            if (!ok) break;
            if (valid) {
                row_state_publish(st, gb);
                Best b;
                b.h = st.h;
                b.idx = st.idx;
                b.pad = 0;
                Q.part[(int64_t)range * (kPartsPerChunk * Q.n_chunks) + kPartsPerChunk * chunk +
                       hsel] = b;
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
size_t iso_layout(int cw, int* nstage_out, int* ncf_out)
{
    constexpr int kN = IsoShape<K>::N;
    const size_t a_bytes = (size_t)8 * 128 * K * 2;
    const size_t stage = (size_t)kN * K * 2;
    const size_t cf_tile = (size_t)kN * cw * 4 + (size_t)kN * sizeof(ColExact);
    const int ncf = 16;
    const size_t fixed = a_bytes + (size_t)ncf * cf_tile + 1024;
    int ns = (int)((kSmemBudget - fixed) / stage);
    if (ns > 16) ns = 16;
    if (ns < 2) ns = 2;
    *nstage_out = ns;
    *ncf_out = ncf;
    size_t total = fixed + (size_t)ns * stage;
    if (total < kSmemMinForOneCta) total = kSmemMinForOneCta;
    return total;
}

template <int K, int NS, int EPI>
cudaError_t launch_iso_kns(const ContractArgs& a, cudaStream_t s)
{
    int nstage = 0, ncf = 0;
    const size_t smem = iso_layout<K>(a.sp.cw, &nstage, &ncf);
    auto kern = contract_tc_iso_kernel<K, NS, EPI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    IsoParams P;
    P.probs = a.probs;
    P.n_probs = a.n_probs;
    P.n_items = a.n_items;
    P.n_items_dev = a.n_items_dev;
    P.err = a.err;
    P.nstage = nstage;
    P.ncf = ncf;
    const int grid = P.n_items < a.grid_ctas ? P.n_items : a.grid_ctas;
    kern<<<grid, IsoEpi<EPI>::kThreads, smem, s>>>(P, a.sp);
    return cudaGetLastError();
}

template <int K, int EPI>
cudaError_t launch_iso_ke(const ContractArgs& a, cudaStream_t s)
{
    switch (a.sp.ns) {
        case 1: return launch_iso_kns<K, 1, EPI>(a, s);
        case 2: return launch_iso_kns<K, 2, EPI>(a, s);
        case 3: return launch_iso_kns<K, 3, EPI>(a, s);
        default: return cudaErrorInvalidValue;  // larger S sets use the row kernel
    }
}

template <int K>
cudaError_t launch_iso_k(const ContractArgs& a, cudaStream_t s)
{
    return a.variant == 1 ? launch_iso_ke<K, 16>(a, s) : launch_iso_ke<K, 8>(a, s);
}

}  // namespace

bool contract_tc_iso_supports(int K, int ns) { return (K == 16 || K == 64) && ns >= 1 && ns <= 3; }
int contract_tc_iso_parts_per_chunk(int variant)
{
    return variant == 1 ? IsoEpi<16>::kPartsPerChunk : IsoEpi<8>::kPartsPerChunk;
}
int contract_tc_iso_ntile(int K) { return K == 16 ? IsoShape<16>::N : IsoShape<64>::N; }

cudaError_t launch_contract_tc_iso(const ContractArgs& a, cudaStream_t s)
{
    switch (a.K) {
        case 16: return launch_iso_k<16>(a, s);
        case 64: return launch_iso_k<64>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fic
