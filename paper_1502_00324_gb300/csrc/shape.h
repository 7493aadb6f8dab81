// shape.h -- the shape of one quadtree step under a tuning choice (kernel
// family, tile width, partial-best slots, chunk refill cost) and the layout
// sizes that follow from it.  Internal to libfic.so; shared by the eager
// step driver and graph-captured encodes.
#pragma once

#include <cstdint>
#include <cstring>

#include "engine.h"
#include "kernels.h"

namespace fic {

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Pool operands up to this size take the diagonal chunk order (item_coords):
// concurrent work items then read different column chunks, which costs no
// HBM traffic while the operand stays in L2.
constexpr double kDiagMaxPoolBytes = 48.0 * 1024 * 1024;

inline StepParams make_step(const fic_sset& s, int n)
{
    StepParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.n = n;
    sp.q = s.q;
    sp.ns = s.n_s;
    sp.cw = 1 + s.n_s;  // m_c and one beta per S, in groups of 4 columns
    for (int i = 0; i < s.n_s; ++i) {
        sp.p[i] = s.p[i];
        sp.kf[i] = (float)(8LL * s.p[i] * s.q);
    }
    return sp;
}

// Engine-dependent shape of one quadtree step under a tuning choice.
struct StepShape {
    int B, n2, K;
    StepParams sp;
    bool iso;            // iso-major range operand (isometry or domain-side kernel)
    bool red;            // domain-side isometries, maximum by the TMEM load
    int64_t tile_w;      // pool columns per tile
    int parts_per_chunk; // partial bests per (range, column chunk)
    int refill;          // chunking: per-item refill cost in tiles
    int epi;             // isometry kernel epilogue variant
};

inline StepShape step_shape(const fic_params& p, int lvl, const TuneChoice& v)
{
    StepShape h;
    h.B = p.B_max >> lvl;
    h.n2 = h.B * h.B;
    h.K = k_pad(h.n2);
    h.sp = make_step(p.S_sets[lvl], h.n2);
    // isometry-in-accumulator kernel: ranges in TMEM lanes, one accumulator
    // per isometry (iso-major A); row kernel: rows are (range, isometry)
    const bool tc = p.engine == FIC_ENGINE_TENSOR;
    h.red = tc && v.iso == 2 && contract_tc_red_supports(h.n2, h.sp.ns);
    h.iso = h.red || (tc && v.iso == 1 && contract_tc_iso_supports(h.K, h.sp.ns));
    h.tile_w = h.red   ? contract_tc_red_ntile()
               : h.iso ? contract_tc_iso_ntile(h.K)
                       : (tc ? contract_tc_ntile() : kPlainNTile);
    h.epi = v.epi;
    h.parts_per_chunk = h.red   ? contract_tc_red_parts_per_chunk()
                        : h.iso ? contract_tc_iso_parts_per_chunk(h.epi)
                                : (tc ? contract_tc_parts_per_chunk() : 1);
    h.refill = v.refill > 0 ? v.refill : 2;
    return h;
}

// Default (untuned) shape: the domain-side isometry kernel where it applies
// (2x2 .. 8x8 steps with |S| <= 3), else the row kernel.
inline TuneChoice default_choice() { return TuneChoice{2, 2, 0}; }

inline int64_t rows_pad_for(const StepShape& h, int64_t R)
{
    return h.iso ? 8 * round_up(R, 128) : round_up(8 * R, kMTile);
}

inline int64_t mtiles_for(const StepShape& h, int64_t rows_pad)
{
    return h.iso ? rows_pad / 8 / 128 : rows_pad / kMTile;
}

}  // namespace fic
