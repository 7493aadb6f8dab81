// epilogue.cuh -- per-row scoring and argmin over a block of contraction
// outputs, shared by the tensor-core and the CUDA-core engines.
//
// For each candidate (pool column c, S index s) of a row (range x isometry)
// the exact selection key is h = p^2 Vd - 8 p q Crd (an int64; the eq. 1
// score at the eq. 3 offset is 16 q^2 Vr + h).  The epilogue first evaluates
// an FP32 filter f ~ h/n with a proven error bound delta (common.cuh); only
// candidates that can tie or beat the row's best are re-scored exactly,
// keeping the lexicographically smallest (h, pool index, isometry, S index).
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

// Column constants: cf[c * cw] = m_c (= sum D' / n), cf[c * cw + 1 + s] =
// beta_s (= fl(p_s^2 Vd / n)); padded columns carry beta = +inf.
// Returns min over s of the filter values; f[] receives them.
template <int NS>
__device__ __forceinline__ float filter_vals(const float* __restrict__ cfc, float a, float x,
                                             const StepParams& sp, float* f)
{
    if constexpr (NS >= 1 && NS <= 3) {
        const float4 c = *reinterpret_cast<const float4*>(cfc);
        const float t = __fmaf_rn(a, c.x, -x);
        f[0] = __fmaf_rn(sp.kf[0], t, c.y);
        if constexpr (NS == 1) return f[0];
        f[1] = __fmaf_rn(sp.kf[1], t, c.z);
        if constexpr (NS == 2) return fminf(f[0], f[1]);
        f[2] = __fmaf_rn(sp.kf[2], t, c.w);
        return fminf(f[0], fminf(f[1], f[2]));
    } else {
        const float t = __fmaf_rn(a, cfc[0], -x);
        float m = __int_as_float(0x7f800000);
        for (int s = 0; s < sp.ns; ++s) {
            f[s] = __fmaf_rn(sp.kf[s], t, cfc[1 + s]);
            m = fminf(m, f[s]);
        }
        return m;
    }
}

// Exact re-scoring of one column for the S values whose filter passes te.
// Out of line: it runs rarely, and a call keeps the caller's register
// arrays statically indexed.
template <int NS>
__device__ __noinline__ RowState exact_col(RowState st, float x, const float* __restrict__ cfc,
                                           int col, unsigned iso, float a, float delta,
                                           float inv_n, int sr, const ColExact* __restrict__ ci,
                                           int dn, const StepParams* __restrict__ spp, float te)
{
    const StepParams& sp = *spp;
    if (col >= dn) return st;
    float f[NS == 0 ? 16 : NS];
    filter_vals<NS>(cfc, a, x, sp, f);
    const ColExact ce = ci[col];
    const int cprime = __float2int_rn(x);
    const int ns = NS == 0 ? sp.ns : NS;
    for (int s = 0; s < ns; ++s) {
        if (!(f[s] <= te)) continue;
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

// Process NCOL outputs x[j] of one row.  The constants of x[j] are at
// cf + (cf_col0 + j * cstride) * cw; its pool column is col0 + j * cstride.
// NS = 1..3 selects the unrolled path; NS = 0 handles any sp.ns <= 16.
template <int NS, int NCOL>
__device__ __forceinline__ void epi_block(RowState& st, const float (&x)[NCOL],
                                          const float* __restrict__ cf, int cf_col0, int col0,
                                          int cstride, unsigned iso, float a, float delta,
                                          float inv_n, int sr, const ColExact* __restrict__ ci,
                                          int dn, const StepParams* __restrict__ spp)
{
    const StepParams& sp = *spp;
    constexpr int NSV = (NS == 0) ? 16 : NS;
    // pass 1: block minimum of the filter
    float mn0 = __int_as_float(0x7f800000), mn1 = mn0;
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
        const float* cfc = cf + (size_t)(cf_col0 + j * cstride) * sp.cw;
        if constexpr (NS == 2) {
            const float4 c = *reinterpret_cast<const float4*>(cfc);
            const float t = __fmaf_rn(a, c.x, -x[j]);
            const float f0 = __fmaf_rn(sp.kf[0], t, c.y);
            const float f1 = __fmaf_rn(sp.kf[1], t, c.z);
            if (j & 1) mn1 = fmin3(mn1, f0, f1);
            else mn0 = fmin3(mn0, f0, f1);
        } else {
            float f[NSV];
            const float m = filter_vals<NS>(cfc, a, x[j], sp, f);
            if (j & 1) mn1 = fminf(mn1, m);
            else mn0 = fminf(mn0, m);
        }
    }
    const float mn = fminf(mn0, mn1);
    if (!(mn <= st.thr)) return;
    // pass 2: candidates within 2 delta of the block minimum and under thr
    float te = fminf(st.thr, __fadd_ru(mn, 2.0f * delta));
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
        const float* cfc = cf + (size_t)(cf_col0 + j * cstride) * sp.cw;
        float f[NSV];
        const float m = filter_vals<NS>(cfc, a, x[j], sp, f);
        if (m <= te) {
            st = exact_col<NS>(st, x[j], cfc, col0 + j * cstride, iso, a, delta, inv_n, sr, ci,
                               dn, spp, te);
            te = fminf(te, st.thr);
        }
    }
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
