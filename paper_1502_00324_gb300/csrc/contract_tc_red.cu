// contract_tc_red.cu -- tensor-core search for 2x2, 4x4 and 8x8 ranges with the
// isometries on the domain side and their maximum taken by the
// tensor-memory load (tcgen05.ld.red, an sm_103a instruction).
//
// The eight isometries of Sec. 2 permute the pixels of a block, so
// sum r . T_k(d') = sum T_k^-1(r) . d': the MMA can take the ranges as they
// are (A: 128 ranges x K) and the domains in all eight isometries (B: 32
// domains x 8, row 8 c + k = T_k(d'_c)).  A tile's accumulator then holds,
// in TMEM lane = range, the eight isometries of domain c in the eight
// consecutive columns 8 c .. 8 c + 7, and one tcgen05.ld.red.max of those
// columns returns the eight values together with their maximum.  The filter
// of epilogue.cuh is decreasing in C'_k (p >= 0) and each of its roundings
// is monotone, so its value at the maximum is the smallest of the eight
// (the argument of the isometry-in-accumulator kernel): one filter per
// (range, domain) and no instruction for the maximum.
//
// The transformed domains are built in shared memory by two producer warps
// from the gathered pool operand: each 32-bit word of a copy holds two
// pixels and is one byte permute of two source words (or a source word
// itself).  The copies are written in the canonical K-major, no-swizzle
// layout with the 8-row group stride padded by 16 bytes, which spreads a
// warp's 16-byte stores (one domain per lane) over distinct bank groups.
//
// Warp roles: warp 0 bulk-copies (TMA engine) the A tile of a work item,
// the raw pool tiles and the column constants; warp 1 owns TMEM and issues
// tcgen05.mma / tcgen05.commit; warps 2-3 build the transformed B stages
// (alternate tiles); warps 4-11 are the epilogue (warp w: TMEM lanes
// 32 (w % 4) .. +31, the tiles of parity (w - 4) / 4 with all their
// domains).  Every mbarrier wait is bounded (tc_common.cuh).
#include "epilogue.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace fic {
namespace {
using namespace tc;

constexpr int kDom = 32;                    // pool domains per tile
constexpr int kTileN = 8 * kDom;            // accumulator columns per tile (MMA N)
constexpr int kSlots = 2;                   // TMEM slots of kTileN columns
constexpr uint32_t kTmemCols = kSlots * kTileN;
constexpr int kXformWarps = 2;
constexpr int kFirstEpiWarp = 2 + kXformWarps;

// Epilogue: 8 warps = 4 lane quarters x 2 tile parities.  Warp (q, p) takes
// the tiles t with t % 2 == p, all 32 domains of each in batches of kBatch,
// so the two warps of a lane quarter alternate tiles and TMEM slots (slot p)
// and each slot is handed back by 4 warps.
constexpr int kEpiWarps = 8;
constexpr int kParts = 2;               // partial bests per (range, chunk): one per parity
constexpr int kBatch = 8;               // domains per batch of TMEM loads
constexpr int kThreads = 32 * (kFirstEpiWarp + kEpiWarps);
constexpr int kMaxRegs = 65536 / kThreads / 8 * 8;
static_assert(kSlots == 2 && kEpiWarps == 8, "two parities, one TMEM slot each");

struct RedParams {
    const Problem* probs;
    int n_probs, n_items;
    const int* n_items_dev;  // device item count (graph-captured steps), else null
    int* err;
    int nraw, nstage, ncf;
};

// 32 lanes x 8 columns with their maximum (per lane, over the 8 columns).
__device__ __forceinline__ void tmem_ldred8(uint32_t taddr, float (&v)[8], float& mx)
{
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x8.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, %8, [%9];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7]), "=f"(mx)
        : "r"(taddr));
}

// Waits for this thread's outstanding tcgen05.ld of a batch (8 domains x 8
// isometries and 8 maxima); every register is an operand, so no use moves
// above the wait.
__device__ __forceinline__ void tmem_wait_batch(float (&x)[8][8], float (&mx)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(x[0][0]), "+f"(x[0][1]), "+f"(x[0][2]), "+f"(x[0][3]), "+f"(x[0][4]), "+f"(x[0][5]), "+f"(x[0][6]), "+f"(x[0][7]),
                   "+f"(x[1][0]), "+f"(x[1][1]), "+f"(x[1][2]), "+f"(x[1][3]), "+f"(x[1][4]), "+f"(x[1][5]), "+f"(x[1][6]), "+f"(x[1][7]),
                   "+f"(x[2][0]), "+f"(x[2][1]), "+f"(x[2][2]), "+f"(x[2][3]), "+f"(x[2][4]), "+f"(x[2][5]), "+f"(x[2][6]), "+f"(x[2][7]),
                   "+f"(x[3][0]), "+f"(x[3][1]), "+f"(x[3][2]), "+f"(x[3][3]), "+f"(x[3][4]), "+f"(x[3][5]), "+f"(x[3][6]), "+f"(x[3][7]),
                   "+f"(x[4][0]), "+f"(x[4][1]), "+f"(x[4][2]), "+f"(x[4][3]), "+f"(x[4][4]), "+f"(x[4][5]), "+f"(x[4][6]), "+f"(x[4][7]),
                   "+f"(x[5][0]), "+f"(x[5][1]), "+f"(x[5][2]), "+f"(x[5][3]), "+f"(x[5][4]), "+f"(x[5][5]), "+f"(x[5][6]), "+f"(x[5][7]),
                   "+f"(x[6][0]), "+f"(x[6][1]), "+f"(x[6][2]), "+f"(x[6][3]), "+f"(x[6][4]), "+f"(x[6][5]), "+f"(x[6][6]), "+f"(x[6][7]),
                   "+f"(x[7][0]), "+f"(x[7][1]), "+f"(x[7][2]), "+f"(x[7][3]), "+f"(x[7][4]), "+f"(x[7][5]), "+f"(x[7][6]), "+f"(x[7][7])
                 :
                 : "memory");
    asm volatile(""
                 : "+f"(mx[0]), "+f"(mx[1]), "+f"(mx[2]), "+f"(mx[3]), "+f"(mx[4]), "+f"(mx[5]),
                   "+f"(mx[6]), "+f"(mx[7]));
}

// Makes this thread's generic-proxy shared-memory writes visible to the
// async proxy (the tensor core reads the B stages through it).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Source pixel (row-major index in the B x B block) of pixel t of T_k(x):
// T_k = mirror^b o rot^m, m = k & 3, b = k >= 4, rot(x)[i][j] = x[B-1-j][i],
// mirror(x)[i][j] = x[i][B-1-j] (the index maps of the range prep).
__host__ __device__ constexpr int iso_src_pixel(int B, int k, int t)
{
    int i = t / B, j = t % B;
    if (k >= 4) j = B - 1 - j;
    for (int m = 0; m < (k & 3); ++m) {
        const int u = i;
        i = B - 1 - j;
        j = u;
    }
    return i * B + j;
}

// Build-time checks of the map against the definitions above: each T_k is
// a permutation of the B x B pixels, rot^4 and mirror^2 are the identity,
// and a few entries written out from rot(x)[i][j] = x[B-1-j][i] and
// mirror(x)[i][j] = x[i][B-1-j].
__host__ __device__ constexpr bool iso_map_is_permutation(int B, int k)
{
    for (int s = 0; s < B * B; ++s) {
        int hits = 0;
        for (int t = 0; t < B * B; ++t) hits += iso_src_pixel(B, k, t) == s ? 1 : 0;
        if (hits != 1) return false;
    }
    return true;
}
__host__ __device__ constexpr bool iso_maps_ok(int B)
{
    for (int k = 0; k < 8; ++k)
        if (!iso_map_is_permutation(B, k)) return false;
    for (int t = 0; t < B * B; ++t) {
        // four quarter turns, and rot^2 applied twice, give back every pixel
        int u = t;
        for (int r = 0; r < 4; ++r) u = iso_src_pixel(B, 1, u);
        if (u != t || iso_src_pixel(B, 2, iso_src_pixel(B, 2, t)) != t) return false;
        // the mirror is an involution
        if (iso_src_pixel(B, 4, iso_src_pixel(B, 4, t)) != t) return false;
    }
    return true;
}
static_assert(iso_maps_ok(2) && iso_maps_ok(4) && iso_maps_ok(8), "isometry maps");
static_assert(iso_src_pixel(4, 1, 1) == 8, "rot(x)[0][1] = x[2][0]");
static_assert(iso_src_pixel(4, 4, 0) == 3, "mirror(x)[0][0] = x[0][3]");
static_assert(iso_src_pixel(4, 5, 1) == 4, "mirror o rot (x)[0][1] = x[1][0]: the transpose");
static_assert(iso_src_pixel(8, 7, 0) == 63, "mirror o rot^3 (x)[0][0] = x[7][7]");

// Word w (pixels 2w, 2w + 1) of T_k(x), x given as K/2 words of two halves
// (pixels past B x B are the zero padding of K).
template <int B, int k, int w, int NW>
__device__ __forceinline__ uint32_t iso_word(const uint32_t (&x)[NW])
{
    constexpr int s0 = iso_src_pixel(B, k, 2 * w), s1 = iso_src_pixel(B, k, 2 * w + 1);
    if constexpr (2 * w >= B * B) {
        return 0u;  // K padding beyond the B x B pixels (2 x 2 ranges)
    } else if constexpr (s0 / 2 == s1 / 2 && (s0 & 1) == 0 && (s1 & 1) == 1) {
        return x[s0 / 2];
    } else {
        constexpr uint32_t lo = (s0 & 1) ? 0x32u : 0x10u;  // half s0 of word s0/2 -> bytes 0-1
        constexpr uint32_t hi = (s1 & 1) ? 0x76u : 0x54u;  // half s1 of word s1/2 -> bytes 2-3
        return __byte_perm(x[s0 / 2], x[s1 / 2], lo | (hi << 8));
    }
}

// Writes copy k of one domain: its K/8 core-matrix rows of 16 bytes, chunk
// kc (pixels 8 kc .. 8 kc + 7) at dst + kc * 128 (dst: the domain's 8-row
// group plus row k).
template <int B, int k, int kc, int NW>
__device__ __forceinline__ void store_chunks(uint8_t* dst, const uint32_t (&x)[NW])
{
    if constexpr (kc < NW / 4) {
        uint4 v;
        v.x = iso_word<B, k, 4 * kc + 0, NW>(x);
        v.y = iso_word<B, k, 4 * kc + 1, NW>(x);
        v.z = iso_word<B, k, 4 * kc + 2, NW>(x);
        v.w = iso_word<B, k, 4 * kc + 3, NW>(x);
        *reinterpret_cast<uint4*>(dst + k * 16 + kc * 128) = v;
        store_chunks<B, k, kc + 1, NW>(dst, x);
    }
}

// All eight copies of one domain (rows 8 c + k of the B stage).
template <int B, int k, int NW>
__device__ __forceinline__ void store_copies(uint8_t* dst, const uint32_t (&x)[NW])
{
    if constexpr (k < 8) {
        store_chunks<B, k, 0, NW>(dst, x);
        store_copies<B, k + 1, NW>(dst, x);
    }
}

// The filter constants of G groups of 4 domains (m_c, then beta_s per S),
// read into registers ahead of the TMEM wait.
template <int NS, int G>
__device__ __forceinline__ void red_consts(const float* __restrict__ cf, int g0,
                                           float4 (&cc)[G][1 + NS])
{
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int j = 0; j < 1 + NS; ++j)
            cc[g][j] = reinterpret_cast<const float4*>(cf + (size_t)(g0 + g) * (1 + NS) * 4)[j];
}

// Filter of G groups of 4 domains, each given by its maximum over the
// eight isometries (c): the minimum of each group (gm) and of all.
template <int NS, int G>
__device__ __forceinline__ float red_pass1(const float (&c)[4 * G], const float4 (&cc)[G][1 + NS],
                                           float na, const StepParams& sp, float (&gm)[G])
{
    const uint64_t nak = pk2(na, na);
    uint64_t nk[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) nk[s] = pk2(-sp.kf[s], -sp.kf[s]);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const float4 m = cc[g][0];
        const uint64_t t01 = fma2(nak, pk2(m.x, m.y), pk2(c[4 * g], c[4 * g + 1]));
        const uint64_t t23 = fma2(nak, pk2(m.z, m.w), pk2(c[4 * g + 2], c[4 * g + 3]));
        float g01 = __int_as_float(0x7f800000), g23 = g01;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float4 b = cc[g][1 + s];
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
    for (int g = 1; g < G; ++g) mn = fminf(mn, gm[g]);
    return mn;
}

// 32 lanes x 8 columns, waited for (the values of one domain in the exact
// re-score below).
__device__ __forceinline__ void tmem_ld8_wait(uint32_t taddr, float (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                   "+f"(v[6]), "+f"(v[7])
                 :
                 : "memory");
}

// Exact re-scoring of the candidates of a batch of 4 G domains (maxima c)
// whose filter is within 2 delta of the batch minimum mn and under the
// range's threshold.  Entered by the whole warp (cand: this lane has a
// candidate): for each domain that some lane still needs, the warp reads its
// eight isometries back from TMEM (tb: the batch's first column), so no
// value of the batch stays in registers after the filter.  cf/ci: the
// tile's filter constants and exact column sums, indexed by the domain
// within the tile.  Candidates arrive out of index order across tiles, so a
// candidate is skipped only when its lower bound proves h > h* (index below
// the best) or h > h* - 1 (index above it).
template <int NS, int G>
__device__ __forceinline__ void red_rescore(RowState& st, bool cand, const float (&c)[4 * G], float mn,
                                         const float (&gm)[G], uint32_t tb,
                                         const float* __restrict__ cf, int g0, int col_base,
                                         float na, float delta, float inv_n, int sr,
                                         const ColExact* __restrict__ ci, int dn,
                                         const StepParams* __restrict__ spp)
{
    const StepParams& sp = *spp;
    constexpr int cw = 1 + NS;
    float te = cand ? fminf(st.thr, __fadd_ru(mn, 2.0f * delta)) : -__int_as_float(0x7f800000);
    // h*/n and (h* - 1)/n rounded up, converted again only when the best changes
    long long hc = kNoCandidate;
    float hb_eq = 0.0f, hb_below = 0.0f;
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        float gmg = gm[0];
#pragma unroll
        for (int j = 1; j < G; ++j)
            if (g == j) gmg = gm[j];
        if (!__any_sync(0xffffffffu, gmg <= te)) continue;
        const float* cg = cf + (size_t)(g0 + g) * cw * 4;
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
            const int d = 4 * g + e;
            float cmax = c[0];
#pragma unroll
            for (int j = 1; j < 4 * G; ++j)
                if (d == j) cmax = c[j];
            float fm = __int_as_float(0x7f800000);
#pragma unroll
            for (int s = 0; s < NS; ++s) fm = fminf(fm, col_filter(cg, e, na, cmax, sp, s));
            const bool need = fm <= te;
            if (!__any_sync(0xffffffffu, need)) continue;
            float v[8];
            __syncwarp();
            tmem_ld8_wait(tb + (uint32_t)(8 * d), v);  // the whole warp reads the domain
            if (need) {
            const int col = (g0 + g) * 4 + e + col_base;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float xj = v[k];
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
                    if (st.h != hc) {
                        hc = st.h;
                        hb_eq = __ll2float_ru(hc) * inv_n;
                        hb_below = __ll2float_ru(hc - 1) * inv_n;
                    }
                    if (lo > (pack_idx((unsigned)col, (unsigned)k, 0) > st.idx ? hb_below : hb_eq))
                        continue;
                }
                st = exact_col_inl(st, xj, cg, e, col, (unsigned)k, na, delta, inv_n, sr,
                                   ci + (g0 + g) * 4 + e, dn, spp, te);
                te = fminf(te, st.thr);
            }
            }
        }
    }
}

// Out-of-line entry of the re-score, which is rare: scalar arguments and the
// row state by value, so that the kernel's live registers are saved once per
// entry and nothing of the caller has to live in memory.
template <int NS>
__device__ __noinline__ RowState red_rescore_call(RowState st, bool cand, float c0, float c1, float c2,
                                                  float c3, float c4, float c5, float c6, float c7,
                                                  float mn, float gm0, float gm1, uint32_t tb,
                                                  const float* __restrict__ cf, int g0, int col_base,
                                                  float na, float delta, float inv_n, int sr,
                                                  const ColExact* __restrict__ ci, int dn,
                                                  const StepParams* __restrict__ spp)
{
    const float c[8] = {c0, c1, c2, c3, c4, c5, c6, c7};
    const float gm[2] = {gm0, gm1};
    red_rescore<NS, 2>(st, cand, c, mn, gm, tb, cf, g0, col_base, na, delta, inv_n, sr, ci, dn, spp);
    return st;
}

template <int B>
struct RedLayout {
    static constexpr int K = k_pad(B * B);
    static constexpr int NW = K / 2;                        // 32-bit words per domain
    static constexpr uint32_t kAbytes = 128u * K * 2u;      // A tile (128 ranges)
    static constexpr uint32_t kRawBytes = (uint32_t)kDom * K * 2u;
    static constexpr uint32_t kSboB = K * 16u + 16u;        // padded 8-row group stride
    static constexpr uint32_t kStageBytes = (uint32_t)kDom * kSboB;
};

template <int B, int NS>
__global__ void __maxnreg__(kMaxRegs)
contract_tc_red_kernel(const __grid_constant__ RedParams P, const __grid_constant__ StepParams sp)
{
    using Lay = RedLayout<B>;
    constexpr int K = Lay::K;
    static_assert(K == 16 || K == 64, "one K-block per tile");
    constexpr int NW = Lay::NW;
    constexpr uint32_t kIdesc = idesc_f16_f32(128, kTileN);
    const uint32_t cfc_bytes = (uint32_t)kDom * (uint32_t)sp.cw * 4u;
    const uint32_t cf_bytes = cfc_bytes + (uint32_t)kDom * (uint32_t)sizeof(ColExact);
    const int nraw = P.nraw, nstage = P.nstage, ncf = P.ncf;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = sA + Lay::kAbytes;
    uint8_t* sRaw = sB + (size_t)nstage * Lay::kStageBytes;
    uint8_t* sCF = sRaw + (size_t)nraw * Lay::kRawBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sCF + (size_t)ncf * cf_bytes);
    const uint32_t b_base = smem_u32(bars);
    const uint32_t a_full = b_base, a_empty = b_base + 8;
    auto rfull = [&](int r) { return b_base + 16 + 8u * r; };
    auto rempty = [&](int r) { return b_base + 16 + 8u * (nraw + r); };
    const uint32_t b_stage = b_base + 16 + 16u * nraw;
    auto bfull = [&](int s) { return b_stage + 8u * s; };
    auto bempty = [&](int s) { return b_stage + 8u * (nstage + s); };
    const uint32_t b_acc = b_stage + 16u * nstage;
    auto tfull = [&](int a) { return b_acc + 8u * a; };
    auto tempty = [&](int a) { return b_acc + 8u * kSlots + 8u * a; };
    const uint32_t b_cf = b_acc + 16u * kSlots;
    auto cff = [&](int c) { return b_cf + 8u * c; };
    auto cfe = [&](int c) { return b_cf + 8u * (ncf + c); };
    const uint32_t drain = b_cf + 16u * ncf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 + 2 * nraw + 2 * nstage +
                                                      2 * kSlots + 2 * ncf + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int r = 0; r < nraw; ++r) {
            mbar_init(rfull(r), 1);
            mbar_init(rempty(r), 1);
        }
        for (int s = 0; s < nstage; ++s) {
            mbar_init(bfull(s), 1);
            mbar_init(bempty(s), 1);
        }
        for (int a = 0; a < kSlots; ++a) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), kEpiWarps / kSlots);
        }
        for (int c = 0; c < ncf; ++c) {
            mbar_init(cff(c), 1);
            mbar_init(cfe(c), kEpiWarps / 2);  // the 4 warps of tile parity c % 2
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
        int64_t rt = 0, cfi = 0, icount = 0;
        int ridx = 0, cidx = 0;          // ring positions of rt and cfi
        uint32_t rphase = 0, cphase = 0; // and their parities
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            int chunk, mtile;
            item_coords(Q, item - Q.item_start, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            // operand pointers in registers: the waits' memory clobbers would
            // otherwise reload them from the problem table on every tile
            const float* const qcf = Q.cf;
            const ColExact* const qci = Q.ci;
            const __half* const qD = Q.D;
            if (!(ok = mbar_wait_warp(a_empty, (uint32_t)((icount & 1) ^ 1), err, kWaitCycles))) break;
            if (elect_one()) {
                // isometry 0 of the iso-major range operand: the ranges as they are
                mbar_expect_tx(a_full, Lay::kAbytes);
                bulk_g2s(smem_u32(sA), Q.A + (int64_t)mtile * 128 * K, Lay::kAbytes, a_full);
            }
            __syncwarp();
            ++icount;
            for (int ct = ct0; ct < ct1 && ok; ++ct) {
                if (!(ok = mbar_wait_warp(cfe(cidx), cphase ^ 1, err, kWaitCycles))) break;
                if (elect_one()) {
                    mbar_expect_tx(cff(cidx), cf_bytes);
                    bulk_g2s(smem_u32(sCF + (size_t)cidx * cf_bytes), qcf + (int64_t)ct * kDom * sp.cw,
                             cfc_bytes, cff(cidx));
                    bulk_g2s(smem_u32(sCF + (size_t)cidx * cf_bytes + cfc_bytes),
                             qci + (int64_t)ct * kDom, cf_bytes - cfc_bytes, cff(cidx));
                }
                __syncwarp();
                ++cfi;
                if (++cidx == ncf) {
                    cidx = 0;
                    cphase ^= 1;
                }
                if (!(ok = mbar_wait_warp(rempty(ridx), rphase ^ 1, err, kWaitCycles))) break;
                if (elect_one()) {
                    mbar_expect_tx(rfull(ridx), Lay::kRawBytes);
                    bulk_g2s(smem_u32(sRaw + (size_t)ridx * Lay::kRawBytes),
                             qD + (int64_t)ct * kDom * K, Lay::kRawBytes, rfull(ridx));
                }
                __syncwarp();
                ++rt;
                if (++ridx == nraw) {
                    ridx = 0;
                    rphase ^= 1;
                }
            }
        }
        if (!ok && lane == 0) {
            // drain: let every copy this warp armed land before exit
            for (int64_t j = (rt > nraw ? rt - nraw : 0); j < rt; ++j)
                mbar_wait(rfull((int)(j % nraw)), (uint32_t)((j / nraw) & 1), err + 1, kDrainCycles);
            if (icount > 0) mbar_wait(a_full, (uint32_t)((icount - 1) & 1), err + 1, kDrainCycles);
            for (int64_t j = (cfi > ncf ? cfi - ncf : 0); j < cfi; ++j)
                mbar_wait(cff((int)(j % ncf)), (uint32_t)((j / ncf) & 1), err + 1, kDrainCycles);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        const uint64_t a_desc = smem_desc(smem_u32(sA), 128u, K * 16u);
        int64_t icount = 0;
        int sidx = 0, slot = 0;          // B stage and TMEM slot positions
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
                if (!(ok = mbar_wait_warp(bfull(sidx), sphase, err, kWaitCycles))) break;
                if (!(ok = mbar_wait_warp(tempty(slot), tphase ^ 1, err, kWaitCycles))) break;
                tc_fence_after();
                if (elect_one()) {
                    const uint64_t b_desc = smem_desc(smem_u32(sB + (size_t)sidx * Lay::kStageBytes),
                                                      128u, Lay::kSboB);
                    const uint32_t d_tmem = tmem_base + (uint32_t)(slot * kTileN);
#pragma unroll
                    for (int kk = 0; kk < K / 16; ++kk)
                        tc_mma_f16(d_tmem, desc_add(a_desc, 256u * kk), desc_add(b_desc, 256u * kk),
                                   kIdesc, kk != 0 ? 1u : 0u);
                    tc_commit(tfull(slot));
                    tc_commit(bempty(sidx));
                }
                __syncwarp();
                if (++slot == kSlots) {
                    slot = 0;
                    tphase ^= 1;
                }
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
    } else if (warp < kFirstEpiWarp) {
        // ------------------------------------------------------------ B stages
        // every tile's ring positions are tracked; this warp builds the tiles
        // of its parity: lane c transforms domain c of the tile
        const int me = warp - 2;
        int64_t t = 0;
        int ridx = 0, sidx = 0;
        uint32_t rphase = 0, sphase = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            int chunk, mtile;
            item_coords(Q, item - Q.item_start, chunk, mtile);
            const int ct0 = chunk * Q.per_chunk;
            const int ct1 = min(Q.n_ct, ct0 + Q.per_chunk);
            for (int ct = ct0; ct < ct1; ++ct, ++t) {
                if ((int)(t % kXformWarps) == me) {
                    if (!(ok = mbar_wait_warp(rfull(ridx), rphase, err, kWaitCycles))) break;
                    // raw tile in the operand layout: domain c, pixels 8 kc .. 8 kc + 7 at
                    // (c / 8) * 16 K + kc * 128 + (c % 8) * 16 bytes
                    uint32_t x[NW];
                    const uint8_t* raw = sRaw + (size_t)ridx * Lay::kRawBytes +
                                         (size_t)(lane >> 3) * 16 * K + (size_t)(lane & 7) * 16;
#pragma unroll
                    for (int kc = 0; kc < K / 8; ++kc) {
                        const uint4 v = *reinterpret_cast<const uint4*>(raw + kc * 128);
                        x[4 * kc + 0] = v.x;
                        x[4 * kc + 1] = v.y;
                        x[4 * kc + 2] = v.z;
                        x[4 * kc + 3] = v.w;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(rempty(ridx));
                    if (!(ok = mbar_wait_warp(bempty(sidx), sphase ^ 1, err, kWaitCycles))) break;
                    store_copies<B, 0, NW>(sB + (size_t)sidx * Lay::kStageBytes + (size_t)lane * Lay::kSboB,
                                            x);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bfull(sidx));
                }
                if (++ridx == nraw) {
                    ridx = 0;
                    rphase ^= 1;
                }
                if (++sidx == nstage) {
                    sidx = 0;
                    sphase ^= 1;
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - kFirstEpiWarp;
        const int quad = warp & 3;   // TMEM lanes (ranges) 32 quad .. +31
        const int par = e >> 2;      // this warp's tiles: t % 2 == par, TMEM slot par
        const float inv_n = 1.0f / (float)sp.n;
        int cidx = 0;                // constants ring position of tile t
        uint32_t cphase = 0;         // and its parity
        uint32_t tphase = 0;         // phase of this warp's TMEM slot
        int64_t t = 0;               // tile counter of the CTA
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const Problem& Q = P.probs[find_problem(P.probs, P.n_probs, item)];
            int chunk, mtile;
            item_coords(Q, item - Q.item_start, chunk, mtile);
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
            // the best key other warps and chunks of this range have published,
            // read one tile ahead; this warp publishes its improvements per tile
            long long gseen = valid ? __ldcg(gb) : kNoCandidate;
            long long gpub = kNoCandidate, gthr = kNoCandidate;
            for (int ct = ct0; ct < ct1; ++ct, ++t) {
                if ((int)(t & 1) == par) {
                    if (gseen < gthr) {
                        // a better key than the one already in the threshold
                        st.thr = fminf(st.thr, thr_from_h(gseen, inv_n, r.delta));
                        gthr = gseen;
                    }
                    if (valid) gseen = __ldcg(gb);
                    if (!(ok = mbar_wait(cff(cidx), cphase, err, kWaitCycles))) break;
                    const float* cfs = reinterpret_cast<const float*>(sCF + (size_t)cidx * cf_bytes);
                    const ColExact* cis =
                        reinterpret_cast<const ColExact*>(sCF + (size_t)cidx * cf_bytes + cfc_bytes);
                    if (!(ok = mbar_wait(tfull(par), tphase, err, kWaitCycles))) break;
                    tc_fence_after();
                    const uint32_t tb = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(par * kTileN);
#pragma unroll
                    for (int bt = 0; bt < kDom / kBatch; ++bt) {
                        float x[kBatch][8], mx[kBatch];
                        __syncwarp();
#pragma unroll
                        for (int d = 0; d < kBatch; ++d)
                            tmem_ldred8(tb + (uint32_t)(8 * (bt * kBatch + d)), x[d], mx[d]);
                        // the batch's filter constants load while the TMEM reads are in flight
                        const int g0 = bt * kBatch / 4;
                        float4 cc[kBatch / 4][1 + NS];
                        red_consts<NS, kBatch / 4>(cfs, g0, cc);
                        tmem_wait_batch(x, mx);
                        float gm[kBatch / 4];
                        const float mn = red_pass1<NS, kBatch / 4>(mx, cc, -r.a, sp, gm);
                        const bool cand = valid && mn <= st.thr;
                        static_assert(kBatch == 8, "the re-score entry takes 8 maxima");
                        if (__any_sync(0xffffffffu, cand))
                            st = red_rescore_call<NS>(st, cand, mx[0], mx[1], mx[2], mx[3], mx[4],
                                                      mx[5], mx[6], mx[7], mn, gm[0], gm[1],
                                                      tb + (uint32_t)(8 * bt * kBatch), cfs, g0,
                                                      ct * kDom, -r.a, r.delta, inv_n, r.sr, cis,
                                                      qdn, &sp);
                    }
                    // the tile's candidates are scored: hand the slot back to the MMA
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty(par));
                    tphase ^= 1;
                    if (st.h < gpub) {
                        atomicMin(gb, st.h);
                        gpub = st.h;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(cfe(cidx));
                }
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
                Q.part[(int64_t)range * (kParts * Q.n_chunks) + kParts * chunk + par] = b;
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
constexpr size_t kSmemMinForOneCta = 120 * 1024;  // > half an SM: one CTA (and TMEM owner) per SM

template <int B>
size_t red_layout(int cw, int* nraw_out, int* nstage_out, int* ncf_out)
{
    using Lay = RedLayout<B>;
    const size_t cf_tile = (size_t)kDom * cw * 4 + (size_t)kDom * sizeof(ColExact);
    constexpr int ncf = 16;  // even: constants entry c serves the tiles of parity c % 2
    static_assert(ncf % 2 == 0, "constants ring of whole tile pairs");
    const int nraw = Lay::K == 64 ? 8 : 16;
    const size_t fixed = Lay::kAbytes + (size_t)nraw * Lay::kRawBytes + (size_t)ncf * cf_tile + 1024;
    int ns = (int)((kSmemBudget - fixed) / Lay::kStageBytes);
    if (ns > 8) ns = 8;
    if (ns < 2) ns = 2;
    *nraw_out = nraw;
    *nstage_out = ns;
    *ncf_out = ncf;
    const size_t total = fixed + (size_t)ns * Lay::kStageBytes;
    return total < kSmemMinForOneCta ? kSmemMinForOneCta : total;
}

template <int B, int NS>
cudaError_t launch_red_kns(const ContractArgs& a, cudaStream_t s)
{
    int nraw = 0, nstage = 0, ncf = 0;
    const size_t smem = red_layout<B>(a.sp.cw, &nraw, &nstage, &ncf);
    auto kern = contract_tc_red_kernel<B, NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    RedParams P;
    P.probs = a.probs;
    P.n_probs = a.n_probs;
    P.n_items = a.n_items;
    P.n_items_dev = a.n_items_dev;
    P.err = a.err;
    P.nraw = nraw;
    P.nstage = nstage;
    P.ncf = ncf;
    const int grid = P.n_items < a.grid_ctas ? P.n_items : a.grid_ctas;
    kern<<<grid, kThreads, smem, s>>>(P, a.sp);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_red_b(const ContractArgs& a, cudaStream_t s)
{
    switch (a.sp.ns) {
        case 1: return launch_red_kns<B, 1>(a, s);
        case 2: return launch_red_kns<B, 2>(a, s);
        case 3: return launch_red_kns<B, 3>(a, s);
        default: return cudaErrorInvalidValue;  // larger S sets use the row kernel
    }
}

}  // namespace

bool contract_tc_red_supports(int n, int ns)
{
    return (n == 4 || n == 16 || n == 64) && ns >= 1 && ns <= 3;
}
int contract_tc_red_ntile() { return kDom; }
int contract_tc_red_parts_per_chunk() { return kParts; }

cudaError_t launch_contract_tc_red(const ContractArgs& a, cudaStream_t s)
{
    switch (a.sp.n) {
        case 4: return launch_red_b<2>(a, s);
        case 16: return launch_red_b<4>(a, s);
        case 64: return launch_red_b<8>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fic
