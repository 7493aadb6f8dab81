// common.cuh -- shared device-side definitions of the range-domain search.
//
// Notation (arXiv 1502.00324, Sec. 2 and eq. 1-3): a range r is a B x B block
// (n = B*B pixels); a domain is a 2B x 2B block decimated 2x2, carried here as
// the B x B array d' of 2x2 pixel SUMS (0..1020), so d = d'/4.  With
// S = p/q and the optimal offset of eq. 3, eq. 1 becomes the exact integer
//   score = 16 q^2 n E = 16 q^2 Vr - 8 p q Crd + p^2 Vd,
//   Vr = n sum r^2 - (sum r)^2, Crd = n sum r d' - sum r sum d',
//   Vd = n sum d'^2 - (sum d')^2.
// Selection only needs h = p^2 Vd - 8 p q Crd (Vr is fixed per range).
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace fic {

// ---------------------------------------------------------------------------
// Operand centring.  The contraction runs on A' = r - 128 (|A'| <= 128) and
// D' = d' - 510 (|D'| <= 510): every product is at most 65,280 in magnitude
// and every partial sum over n <= 256 terms at most 16,711,680 < 2^24, so
// FP16 operands with FP32 accumulation give the exact integer C' = sum A'D'.
// sum r d' = C' + 510 sum r + 128 sum d' - 65280 n.
// ---------------------------------------------------------------------------
constexpr int kRangeCentre = 128;
constexpr int kDomainCentre = 510;

// ---------------------------------------------------------------------------
// Operand tile layout (both A = ranges x isometries and D = pool domains):
// the canonical K-major, no-swizzle layout of tcgen05 shared-memory operands,
// laid out the same way in global memory so that a tile is one contiguous
// bulk copy.  K (= n, padded to a multiple of 16) is cut into K-blocks of
// KB = min(K, 64) elements; inside a K-block, 8-row groups follow each other,
// and inside a group the KB/8 "core matrices" (8 rows x 8 halves = 128 B)
// follow each other along K.
//   half offset(row, k) = (k / KB) * rows_pad * KB + (row / 8) * 8 * KB
//                         + ((k % KB) / 8) * 64 + (row % 8) * 8 + (k % 8)
// Core-matrix strides: along K (LBO) 128 B; along rows (SBO) 16 * KB B.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int k_pad(int n) { return n < 16 ? 16 : n; }
__host__ __device__ constexpr int k_block(int K) { return K < 64 ? K : 64; }

__host__ __device__ inline int64_t tile_off(int64_t row, int k, int64_t rows_pad, int K)
{
    const int KB = k_block(K);
    return (int64_t)(k / KB) * rows_pad * KB + (row >> 3) * 8 * KB +
           ((k % KB) >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Tiles: the M tile is 128 rows = 16 ranges x 8 isometries (row = 8 range +
// isometry, so each range is one 8-row group).  The pool is padded to a
// multiple of kColPad so that any N tile of 128, 192 or 256 columns divides it.
constexpr int kMTile = 128;
constexpr int kRangesPerTile = kMTile / 8;
constexpr int kColPad = 768;

// ---------------------------------------------------------------------------
// Per-range and per-domain constants.
// ---------------------------------------------------------------------------
struct RowConst {       // one per active range
    int sr;             // sum r
    int sr2;            // sum r^2
    float a;            // sum A' = sum r - 128 n (exact in FP32)
    float delta;        // bound on |filter - h/n| over all candidates
};

// A flat range (all pixels equal, Vr = 0) has Crd = 0 against every domain,
// so h = p^2 Vd for every candidate: its best mapping is the pool's smallest
// Vd, resolved from one pool-wide key instead of in the contraction.
__host__ __device__ inline bool range_is_flat(const RowConst& r, int n)
{
    return (long long)n * r.sr2 == (long long)r.sr * r.sr;
}

struct ColExact {       // one per pool domain
    int sd;             // sum d'
    int sd2;            // sum d'^2 (<= 256 * 1020^2 < 2^31)
};

// Best candidate of a range (or of a range over one column chunk).
// idx packs (pool index << 7) | (isometry << 4) | S index.
struct Best {
    long long h;
    unsigned idx;
    unsigned pad;
};

constexpr long long kNoCandidate = 0x7f7f7f7f7f7f7f7fLL;  // byte-fill value: memset 0x7f

__host__ __device__ inline unsigned pack_idx(unsigned c, unsigned k, unsigned s)
{
    return (c << 7) | (k << 4) | s;
}

// The key keeps 25 bits for the pool index, so a step's padded pool must
// stay within 2^25 columns; validate_params rejects larger pools.
constexpr int64_t kMaxPoolColumns = (int64_t)1 << 25;
// The device-wide scan (pool compaction, split requeue, record order) takes
// at most kMaxScanTiles tiles of kScanTileItems elements.
constexpr int64_t kScanTileItems = 4096;
constexpr int64_t kMaxScanTiles = 4096;
constexpr int64_t kMaxScanCount = kScanTileItems * kMaxScanTiles;

__device__ __forceinline__ bool key_less(long long h1, unsigned i1, long long h2, unsigned i2)
{
    return h1 < h2 || (h1 == h2 && i1 < i2);
}

// Exact selection key h = p^2 Vd - 8 p q Crd from the centred contraction C'.
__device__ __forceinline__ long long exact_h(int cprime, int sr, int sd, int sd2, int n, int p, int q)
{
    const long long srd = (long long)cprime + 510LL * sr + 128LL * sd - 65280LL * n;
    const long long crd = (long long)n * srd - (long long)sr * sd;
    const long long vd = (long long)n * sd2 - (long long)sd * sd;
    return (long long)p * p * vd - 8LL * p * q * crd;
}

// ---------------------------------------------------------------------------
// One image's quadtree step inside a grouped contraction launch.  Work items
// of problem p are item_start .. item_start + n_mtiles * n_chunks - 1, chunk
// major (item_coords).
// ---------------------------------------------------------------------------
struct Problem {
    const __half* A;      // range operand (layout of the engine)
    const __half* D;      // pool operand
    const float* cf;      // column filter constants
    const ColExact* ci;   // exact column sums
    const RowConst* rc;   // per active range
    Best* part;           // partial bests: range * parts_per_range + slot
    long long* gbest;     // shared best key per row (or per range)
    int64_t rows_pad;     // rows of A
    int64_t cols_pad;     // pool columns, padded
    int R, dn;            // active ranges, pool size
    int n_mtiles, n_ct;   // M tiles, N tiles
    int n_chunks, per_chunk;
    int item_start;
    int diag;             // 1: M tile m starts at column chunk m * n_chunks / n_mtiles
};

// Column chunk and M tile of item 'local' of problem Q.  Items run chunk
// major; with Q.diag each M tile's sequence starts at the chunk whose pool
// domains lie at about the same image position as its ranges (ranges and
// pool are both in raster order), where a range's best match tends to be,
// so its threshold is tight from the first tiles on.
__device__ __forceinline__ void item_coords(const Problem& Q, int local, int& chunk, int& mtile)
{
    mtile = local % Q.n_mtiles;
    chunk = local / Q.n_mtiles;
    if (Q.diag) {
        chunk += (int)((long long)mtile * Q.n_chunks / Q.n_mtiles);
        if (chunk >= Q.n_chunks) chunk -= Q.n_chunks;
    }
}

// Counts of a step that a graph-captured encode keeps in device memory (null
// members: the host values passed alongside are the counts).  Grids are
// sized for the host values, which are then upper bounds.
struct StepCounts {
    const uint32_t* R = nullptr;          // active ranges
    const uint32_t* dn = nullptr;         // pool size
    const uint32_t* n_parts = nullptr;    // partial bests per range
    const uint32_t* code_base = nullptr;  // records emitted before this step
};

__host__ __device__ inline int64_t round_up64(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

__device__ __forceinline__ int find_problem(const Problem* __restrict__ probs, int n, int item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].item_start <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// FP32 filter.  For column c and S_s = p_s/q the filter value is
//   f = fma(-8 p q, t', beta_s),  t' = fma(-a, m_c, C'),
// with a = sum A' (exact), m_c = sum D'/n (exact), beta_s = fl(p^2 Vd / n).
// Exactly, t' = Crd/n and f = h/n; each of the three roundings is relative
// 2^-24, so
//   |f - h/n| <= (2u + u^2) (8 p q |Crd|/n + p^2 Vd/n),  u = 2^-24,
// and |Crd| <= sqrt(Vr Vd) (Cauchy-Schwarz).  RowConst.delta holds twice
// that bound, maximised over the step's S set and the pool's largest Vd.
// A candidate can only tie or beat the best h* so far if f <= h*/n + delta,
// and inside one tile only if f <= (tile minimum of f) + 2 delta.
// ---------------------------------------------------------------------------
struct StepParams {
    int n;              // B*B
    int q;
    int ns;             // number of S values
    int cw;             // constants per column: m_c and one beta per S (1 + ns)
    int p[16];
    float kf[16];       // 8 p q
};

__device__ __forceinline__ float thr_from_h(long long h, float inv_n, float delta)
{
    return __fadd_ru(__ll2float_ru(h) * inv_n, delta);
}

// Device error word: 0 ok; otherwise the first failure recorded.
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;

}  // namespace fic
