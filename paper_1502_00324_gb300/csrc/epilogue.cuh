// epilogue.cuh -- per-row scoring and argmin over a block of contraction
// outputs, shared by the tensor-core and the CUDA-core engines.
//
// For each candidate (pool column c, S index s) of a row (range x isometry)
// the exact selection key is h = p^2 Vd - 8 p q Crd (an int64; the eq. 1
// score at the eq. 3 offset is 16 q^2 Vr + h).  The epilogue first evaluates
// an FP32 filter f ~ h/n with a proven error bound delta (common.cuh); only
// candidates that can tie or beat the row's best are re-scored exactly,
// keeping the lexicographically smallest (h, pool index, isometry, S index).
//
// Filter, per element: t' = C' - a m_c (= Crd/n exactly), f_s = beta_s - 8 p q t'.
// Both are single-rounding FMAs, evaluated two columns at a time with the
// packed fma.rn.f32x2 (each lane an IEEE round-to-nearest FMA).
//
// Column constants are stored in groups of 4 columns: for group g the
// constant j of its 4 columns is the float4 at cf + (g * cw + j) * 4, with
// j = 0 for m_c and j = 1 + s for beta_s (cw = 1 + |S|); padded columns
// carry beta = +inf.
#pragma once

#include "common.cuh"

namespace fic {

struct RowState {
    float thr;        // no candidate with filter value > thr can win
    unsigned idx;     // best packed (pool index, isometry, S index)
    long long h;      // best exact key so far
};

__device__ __forceinline__ void row_state_init(RowState& st)
{
    st.thr = __int_as_float(0x7f800000);  // +inf
    st.h = kNoCandidate;
    st.idx = 0xffffffffu;
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// (d.lo, d.hi) = (a.lo * b.lo + c.lo, a.hi * b.hi + c.hi), each rounded once.
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Filter values of one column (scalar form, same roundings as the packed one).
__device__ __forceinline__ float col_filter(const float* __restrict__ cg, int e, float na,
                                            float x, const StepParams& sp, int s)
{
    const float tp = __fmaf_rn(na, cg[e], x);                // C' - a m
    return __fmaf_rn(-sp.kf[s], tp, cg[(1 + s) * 4 + e]);   // beta - 8pq t'
}

// Exact re-scoring of one column for the S values whose filter passes te.
static __device__ __forceinline__ RowState exact_col_inl(RowState st, float x,
                                                        const float* __restrict__ cg, int e, int col,
                                                        unsigned iso, float na, float delta,
                                                        float inv_n, int sr,
                                                        const ColExact* __restrict__ cep, int dn,
                                                        const StepParams* __restrict__ spp, float te)
{
    const StepParams& sp = *spp;
    if (col >= dn) return st;
    const ColExact ce = *cep;  // this column's sums
    const int cprime = __float2int_rn(x);
    for (int s = 0; s < sp.ns; ++s) {
        const float f = col_filter(cg, e, na, x, sp, s);
        if (!(f <= te)) continue;
        const long long h = exact_h(cprime, sr, ce.sd, ce.sd2, sp.n, sp.p[s], sp.q);
        const unsigned idx = pack_idx((unsigned)col, iso, (unsigned)s);
        if (key_less(h, idx, st.h, st.idx)) {
            st.h = h;
            st.idx = idx;
            st.thr = thr_from_h(h, inv_n, delta);
            te = fminf(te, st.thr);
        }
    }
    return st;
}

// The same out of line: it runs rarely, and a call keeps the caller's
// register arrays statically indexed.
static __device__ __noinline__ RowState exact_col(RowState st, float x, const float* __restrict__ cg,
                                           int e, int col, unsigned iso, float na, float delta,
                                           float inv_n, int sr, const ColExact* __restrict__ cep,
                                           int dn, const StepParams* __restrict__ spp, float te)
{
    return exact_col_inl(st, x, cg, e, col, iso, na, delta, inv_n, sr, cep, dn, spp, te);
}

// Process NG groups of 4 consecutive columns of one row: group g holds
// x[4g .. 4g+3], its constants start at cf + (g0 + g * gstride) * cw * 4 and
// its first pool column is (g0 + g * gstride) * 4 + col_base.
// NS = 1..3 selects the unrolled packed path; NS = 0 handles any |S| <= 16.
template <int NS, int NG>
__device__ __forceinline__ float epi_pass1(const float (&x)[4 * NG], const float* __restrict__ cf,
                                           int g0, int gstride, float na,
                                           const StepParams* __restrict__ spp)
{
    const StepParams& sp = *spp;
    const int cw = (NS == 0) ? sp.cw : 1 + NS;
    // pass 1: block minimum of the filter (four independent min chains)
    float mn0 = __int_as_float(0x7f800000), mn1 = mn0, mn2 = mn0, mn3 = mn0;
    if constexpr (NS >= 1 && NS <= 3) {
        const uint64_t nak = pk2(na, na);
        uint64_t nk[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) nk[s] = pk2(-sp.kf[s], -sp.kf[s]);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const float4* cg = reinterpret_cast<const float4*>(cf + (size_t)(g0 + g * gstride) * cw * 4);
            const float4 m = cg[0];
            const uint64_t t01 = fma2(nak, pk2(m.x, m.y), pk2(x[4 * g], x[4 * g + 1]));
            const uint64_t t23 = fma2(nak, pk2(m.z, m.w), pk2(x[4 * g + 2], x[4 * g + 3]));
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float4 b = cg[1 + s];
                float f0, f1, f2, f3;
                upk2(fma2(nk[s], t01, pk2(b.x, b.y)), f0, f1);
                upk2(fma2(nk[s], t23, pk2(b.z, b.w)), f2, f3);
                if (g & 1) {
                    mn2 = fmin3(mn2, f0, f1);
                    mn3 = fmin3(mn3, f2, f3);
                } else {
                    mn0 = fmin3(mn0, f0, f1);
                    mn1 = fmin3(mn1, f2, f3);
                }
            }
        }
    } else {
        for (int g = 0; g < NG; ++g) {
            const float* cg = cf + (size_t)(g0 + g * gstride) * cw * 4;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                for (int s = 0; s < sp.ns; ++s) mn0 = fminf(mn0, col_filter(cg, e, na, x[4 * g + e], sp, s));
        }
    }
    return fminf(fminf(mn0, mn1), fminf(mn2, mn3));
}

// Pass 2, for a block whose minimum mn is <= st.thr: the candidates within
// 2 delta of mn and under thr are re-scored exactly (groups are screened
// with the packed filter, elements one by one).
template <int NS, int NG>
__device__ __forceinline__ void epi_pass2(RowState& st, const float (&x)[4 * NG], float mn,
                                       const float* __restrict__ cf, int g0, int gstride,
                                       int col_base, unsigned iso, float na, float delta,
                                       float inv_n, int sr, const ColExact* __restrict__ ci,
                                       int dn, const StepParams* __restrict__ spp)
{
    const StepParams& sp = *spp;
    const int cw = (NS == 0) ? sp.cw : 1 + NS;

    float te = fminf(st.thr, __fadd_ru(mn, 2.0f * delta));
    const int ns = (NS == 0) ? sp.ns : NS;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const float* cg = cf + (size_t)(g0 + g * gstride) * cw * 4;
        const int col0 = (g0 + g * gstride) * 4 + col_base;
        float gm = __int_as_float(0x7f800000);
        if constexpr (NS >= 1 && NS <= 3) {
            const uint64_t nak = pk2(na, na);
            const float4 m = reinterpret_cast<const float4*>(cg)[0];
            const uint64_t t01 = fma2(nak, pk2(m.x, m.y), pk2(x[4 * g], x[4 * g + 1]));
            const uint64_t t23 = fma2(nak, pk2(m.z, m.w), pk2(x[4 * g + 2], x[4 * g + 3]));
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float4 b = reinterpret_cast<const float4*>(cg)[1 + s];
                const uint64_t nk = pk2(-sp.kf[s], -sp.kf[s]);
                float f0, f1, f2, f3;
                upk2(fma2(nk, t01, pk2(b.x, b.y)), f0, f1);
                upk2(fma2(nk, t23, pk2(b.z, b.w)), f2, f3);
                gm = fmin3(gm, f0, f1);
                gm = fmin3(gm, f2, f3);
            }
        } else {
            gm = -__int_as_float(0x7f800000);
        }
        if (!(gm <= te)) continue;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float fm = __int_as_float(0x7f800000);
            for (int s = 0; s < ns; ++s) fm = fminf(fm, col_filter(cg, e, na, x[4 * g + e], sp, s));
            if (fm <= te) {
                // Later columns of this row's sweep lose ties, so they win only
                // with h <= h* - 1.  With this element's own error bound
                // (4u (8pq|t'| + beta), twice the first-order bound; exactly 0
                // for a flat domain) a lower bound f - err above (h* - 1)/n
                // proves it cannot win.
                if (st.h != kNoCandidate) {
                    float lo = __int_as_float(0x7f800000);
                    for (int s = 0; s < ns; ++s) {
                        const float tp = __fmaf_rn(na, cg[e], x[4 * g + e]);
                        const float beta = cg[(1 + s) * 4 + e];
                        const float f = __fmaf_rn(-sp.kf[s], tp, beta);
                        const float err = 0x1p-22f * __fmaf_ru(sp.kf[s], fabsf(tp), beta);
                        lo = fminf(lo, __fsub_rd(f, err));
                    }
                    if (lo > __ll2float_ru(st.h - 1) * inv_n) continue;
                }
                st = exact_col(st, x[4 * g + e], cg, e, col0 + e, iso, na, delta, inv_n, sr,
                               ci + col0 + e, dn, spp, te);
                te = fminf(te, st.thr);
            }
        }
    }
}

// Pass 1 then, when the block can hold a winner, pass 2.
template <int NS, int NG>
__device__ __forceinline__ void epi_groups(RowState& st, const float (&x)[4 * NG],
                                           const float* __restrict__ cf, int g0, int gstride,
                                           int col_base, unsigned iso, float na, float delta,
                                           float inv_n, int sr, const ColExact* __restrict__ ci,
                                           int dn, const StepParams* __restrict__ spp)
{
    const float mn = epi_pass1<NS, NG>(x, cf, g0, gstride, na, spp);
    if (mn <= st.thr)
        epi_pass2<NS, NG>(st, x, mn, cf, g0, gstride, col_base, iso, na, delta, inv_n, sr, ci,
                          dn, spp);
}

// Seed a row's threshold from the best exact key another column chunk has
// published for it (any such key belongs to a real candidate, so it is >=
// the row's true minimum and the seeded threshold still admits the argmin).
__device__ __forceinline__ void row_state_seed(RowState& st, const long long* gbest, float inv_n,
                                               float delta)
{
    const long long g = __ldcg(gbest);
    if (g < kNoCandidate) st.thr = thr_from_h(g, inv_n, delta);
}

__device__ __forceinline__ void row_state_publish(const RowState& st, long long* gbest)
{
    if (st.h < kNoCandidate) atomicMin(gbest, st.h);
}

__device__ __forceinline__ void key_min_shfl(long long& h, unsigned& idx, int lane_mask)
{
    const long long oh = __shfl_xor_sync(0xffffffffu, h, lane_mask);
    const unsigned oi = __shfl_xor_sync(0xffffffffu, idx, lane_mask);
    if (key_less(oh, oi, h, idx)) {
        h = oh;
        idx = oi;
    }
}

}  // namespace fic
