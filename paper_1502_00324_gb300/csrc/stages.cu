// stages.cu -- the step kernels around the contraction: domain entropy and
// pool compaction, operand gathers, quadtree split/requeue, record ordering
// and the decoder pass.
#include <cfloat>

#include "common.cuh"
#include "fic.h"
#include "kernels.h"

namespace fic {

// ---------------------------------------------------------------------------
// Isometry index maps (Sec. 2: rotations by 90 degrees clockwise, and each
// rotation mirrored).  T_k = mirror^b o rot^m with m = k & 3, b = k >= 4;
// rot(x)[i][j] = x[B-1-j][i], mirror(x)[i][j] = x[i][B-1-j].
// ---------------------------------------------------------------------------

// Source of T_k(x)[i][j] in x.
__device__ __forceinline__ void iso_fwd_src(int i, int j, int k, int B, int& si, int& sj)
{
    if (k >= 4) j = B - 1 - j;
    for (int m = 0; m < (k & 3); ++m) {
        const int t = i;
        i = B - 1 - j;
        j = t;
    }
    si = i;
    sj = j;
}

// Source of T_k^-1(x)[i][j] in x; T_k^-1 = rot^-m o mirror^b and
// rot^-1(x)[i][j] = x[j][B-1-i].
__device__ __forceinline__ void iso_inv_src(int i, int j, int k, int B, int& si, int& sj)
{
    for (int m = 0; m < (k & 3); ++m) {
        const int t = i;
        i = j;
        j = B - 1 - t;
    }
    if (k >= 4) j = B - 1 - j;
    si = i;
    sj = j;
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// ---------------------------------------------------------------------------
// Eq. 5-6 entropy, in bits, from integer counts:
//   H = log2(P) - (1/P) sum_g q_g log2 q_g,  P = 4n pixels of the 2B x 2B block.
// The sum runs in fixed point: a table holds round(q log2 q 2^49) as int64
// (built with CUDA's log2; q <= 1024), so the sum over the bins is exact,
// independent of order, and equal count multisets give identical H.  The
// sum of one block is below 1024 * 10 * 2^49 < 2^63.
// ---------------------------------------------------------------------------
constexpr double kEntScale = 562949953421312.0;  // 2^49

__global__ void entropy_table_kernel(long long* T, int count)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) T[q] = q == 0 ? 0LL : llrint((double)q * log2((double)q) * kEntScale);
}

// One warp per run of kRun positions along x (one row of positions): the
// 256-bin histogram of the first window in shared memory, then the window
// slides by L: the L leftmost columns leave, L new columns enter.  Each count
// change q -> q +- 1 changes the fixed-point sum by +-(T[q + 1] - T[q]) (the
// difference table dq, exact), so a lane only adds its own deltas; its
// running share after each position goes to shared memory, and at the end
// of the run lane j sums the 32 shares of position j, evaluates H and
// writes its outputs (coalesced, one FP64 evaluation per lane in parallel).
//   thr mode (keys == NULL): flags[pos] = H > thr; near counts |H - thr| < 1e-9.
//   top mode (keys != NULL): keys[pos] = (2^24 - 1 - Hq) << 40 | pos with
//     Hq = floor(H 2^20 + 1/2) (larger entropy, then lower index, first), and
//     flags[pos] = 1 when H 2^20 + 1/2 is within 1e-6 of an integer (a
//     rounding step could move the position: counted later near the cut).
constexpr int kRun = 32;
constexpr int kEntWarps = 4;
constexpr int64_t kEntMaxBlocks = 152 * 8;  // blocks loop over the runs beyond this

__global__ void __launch_bounds__(32 * kEntWarps)
entropy_kernel(const uint8_t* __restrict__ img, int N, int B, int L, int per, double thr,
               const long long* __restrict__ T, uint32_t* __restrict__ flags,
               double* __restrict__ Hout, unsigned long long* __restrict__ keys,
               unsigned long long* __restrict__ near)
{
    __shared__ long long dq[kEntTableCount - 1];               // T[q + 1] - T[q]
    __shared__ unsigned hist[kEntWarps][256];
    __shared__ long long share[kEntWarps][kRun][kRun + 1];     // [position][lane], padded
    const int S = 2 * B, P = S * S;
    for (int q = threadIdx.x; q < P; q += blockDim.x) dq[q] = T[q + 1] - T[q];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int runs_per_row = (per + kRun - 1) / kRun;
    const int64_t n_runs = (int64_t)runs_per_row * per;
    unsigned* h = hist[w];
    const double log2P = (double)ilog2(P);
    const int mc = L < S ? L : S;  // columns that leave and enter per slide
    const int m = mc * S;
    for (int64_t run = (int64_t)blockIdx.x * kEntWarps + w; run < n_runs;
         run += (int64_t)gridDim.x * kEntWarps) {
        const int iy = (int)(run / runs_per_row);
        const int ix0 = (int)(run % runs_per_row) * kRun;
        const int ix1 = min(per, ix0 + kRun);
        const int y = iy * L;
#pragma unroll
        for (int b = 0; b < 8; ++b) h[lane * 8 + b] = 0;
        __syncwarp();
        long long part = 0;  // this lane's share of sum T[q]
        {
            const int x = ix0 * L;
            for (int t = lane; t < P; t += 32) {
                const unsigned g = img[(int64_t)(y + t / S) * N + x + t % S];
                part += dq[atomicAdd(&h[g], 1u)];
            }
        }
        for (int ix = ix0; ix < ix1; ++ix) {
            if (ix > ix0) {
                // slide by L: columns x - L .. x - L + mc - 1 leave, x + S - mc ..
                // x + S - 1 enter (L >= S: the whole window is replaced)
                const int x = ix * L;
                __syncwarp();
                for (int t = lane; t < m; t += 32) {
                    const int r = t / mc, c = t % mc;
                    const unsigned g = img[(int64_t)(y + r) * N + (x - L) + c];
                    part -= dq[atomicSub(&h[g], 1u) - 1u];
                }
                __syncwarp();
                for (int t = lane; t < m; t += 32) {
                    const int r = t / mc, c = t % mc;
                    const unsigned g = img[(int64_t)(y + r) * N + (x + S - mc) + c];
                    part += dq[atomicAdd(&h[g], 1u)];
                }
            }
            share[w][ix - ix0][lane] = part;
        }
        __syncwarp();
        bool is_near = false;
        if (ix0 + lane < ix1) {
            long long tot = 0;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) tot += share[w][lane][l];
            const int64_t pos = (int64_t)iy * per + ix0 + lane;
            const double H = log2P - (double)tot / kEntScale / (double)P;
            if (Hout) Hout[pos] = H;
            if (keys) {
                const double hx = H * 1048576.0 + 0.5;
                const double fl = floor(hx);
                const unsigned long long hq = (unsigned long long)fl;
                keys[pos] = ((0xFFFFFFull - hq) << 40) | (unsigned long long)pos;
                flags[pos] = (hx - fl < 1e-6 || hx - fl > 1.0 - 1e-6) ? 1u : 0u;
            } else {
                flags[pos] = H > thr ? 1u : 0u;
                is_near = fabs(H - thr) < 1e-9;
            }
        }
        const unsigned nb = __ballot_sync(0xffffffffu, is_near);
        if (lane == 0 && nb) atomicAdd(near, (unsigned long long)__popc(nb));
        __syncwarp();  // the next run reuses this warp's histogram and shares
    }
}

// ---------------------------------------------------------------------------
// Top-DN selection: the k-th smallest of n distinct 64-bit keys by an MSD
// radix select (8 passes of 8 bits; the state lives on the device, so the
// passes need no host synchronisation), then the admission flags.
// ---------------------------------------------------------------------------
struct SelectState {
    unsigned long long prefix;  // digits fixed so far (the k-th key at the end)
    long long k;                // rank still to find among keys with the prefix
};

__global__ void select_init_kernel(SelectState* st, long long k, unsigned* hist)
{
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->k = k;
    }
    hist[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(256)
select_hist_kernel(const unsigned long long* __restrict__ keys, int64_t n,
                   const SelectState* __restrict__ st, int shift, unsigned* __restrict__ hist)
{
    __shared__ unsigned sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long pre = st->prefix;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const unsigned long long key = keys[i];
        const bool match = shift == 56 || ((key ^ pre) >> (shift + 8)) == 0;
        if (match) atomicAdd(&sh[(key >> shift) & 0xff], 1u);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

__global__ void __launch_bounds__(256)
select_pick_kernel(SelectState* st, int shift, unsigned* hist)
{
    __shared__ unsigned c[256];
    const int d = threadIdx.x;
    c[d] = hist[d];
    __syncthreads();
    if (d == 0) {
        long long k = st->k, below = 0;
        int digit = 255;
        for (int i = 0; i < 256; ++i) {
            if (below + (long long)c[i] >= k) {
                digit = i;
                break;
            }
            below += c[i];
        }
        st->prefix |= (unsigned long long)digit << shift;
        st->k = k - below;
    }
    __syncthreads();
    hist[d] = 0;
}

// flags[i] = keys[i] <= k-th key; near counts the positions whose rounded
// entropy could move by one step (flag set by the entropy kernel) and whose
// step is within one of the cut.
__global__ void select_flags_kernel(const unsigned long long* __restrict__ keys, int64_t n,
                                    const SelectState* __restrict__ st,
                                    uint32_t* __restrict__ flags,
                                    unsigned long long* __restrict__ near)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long key = keys[i];
    const long long hb = (long long)(st->prefix >> 40), hq = (long long)(key >> 40);
    if (flags[i] && hq >= hb - 1 && hq <= hb + 1) atomicAdd(near, 1ull);
    flags[i] = key <= st->prefix ? 1u : 0u;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of uint32 (pool compaction, split requeue,
// record ordering).  Tiles of 4096 elements: per-tile sums, one-block scan
// of the tile sums, then a per-tile scan with the tile offset.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileItems, "scan tile size");

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t wtot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? wsum[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, si, d);
            if (lane >= d) si += o;
        }
        if (lane < nw) wsum[lane] = si - s;
        if (lane == 31) wtot = si;  // lanes >= nw add 0: lane 31 holds the total
    }
    __syncthreads();
    const uint32_t res = wsum[w] + inc - v;
    if (total) *total = wtot;
    __syncthreads();
    return res;
}

// n_dev (optional): the count in device memory, at most n (graph-captured
// steps size their grids for n and read the actual count here).
__device__ __forceinline__ int64_t dev_count(int64_t n, const uint32_t* n_dev)
{
    return n_dev ? min(n, (int64_t)*n_dev) : n;
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ n_dev,
                   uint32_t* __restrict__ sums)
{
    n = dev_count(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t g = base + i;
        if (g < n) s += in[g];
    }
    uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
scan_top_kernel(uint32_t* __restrict__ sums, int nb, uint32_t* __restrict__ total)
{
    // 1024 threads x 4 consecutive items -> up to 4096 tiles
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int g = threadIdx.x * 4 + i;
        v[i] = g < nb ? sums[g] : 0u;
        s += v[i];
    }
    uint32_t tot;
    uint32_t off = block_excl_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int g = threadIdx.x * 4 + i;
        if (g < nb) sums[g] = off;
        off += v[i];
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                  const uint32_t* __restrict__ n_dev, const uint32_t* __restrict__ sums)
{
    n = dev_count(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t g = base + i;
        v[i] = g < n ? in[g] : 0u;
        s += v[i];
    }
    uint32_t off = block_excl_scan(s, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t g = base + i;
        if (g < n) out[g] = off;
        off += v[i];
    }
}

int64_t scan_tmp_words(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                        uint32_t* total, cudaStream_t s, int* launches, const uint32_t* n_dev)
{
    if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kMaxScanTiles) return cudaErrorInvalidValue;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, tmp);
    scan_top_kernel<<<1, 1024, 0, s>>>(tmp, (int)nb, total);
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, n_dev, tmp);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pool list (Sec. 3.3: domain coordinates kept in a list; the list index is
// the address): admitted positions in raster order, packed x | y << 16.
// ---------------------------------------------------------------------------
__global__ void pool_scatter_kernel(const uint32_t* __restrict__ flags,
                                    const uint32_t* __restrict__ pos, int64_t n_pos, int per,
                                    int L, uint32_t* __restrict__ pool_xy)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pos || !flags[i]) return;
    const uint32_t x = (uint32_t)((i % per) * L), y = (uint32_t)((i / per) * L);
    pool_xy[pos[i]] = x | (y << 16);
}

cudaError_t launch_entropy_table(long long* T, int count, cudaStream_t s)
{
    entropy_table_kernel<<<(count + 255) / 256, 256, 0, s>>>(T, count);
    return cudaGetLastError();
}

cudaError_t launch_entropy(const uint8_t* img, int N, int B, int L, int per, double thr,
                           const long long* T, uint32_t* flags, double* H,
                           unsigned long long* keys, unsigned long long* near, cudaStream_t s)
{
    const int64_t npos = (int64_t)per * per;
    if (npos == 0) return cudaSuccess;
    const int64_t runs = (int64_t)per * ((per + kRun - 1) / kRun);
    const int64_t blocks = (runs + kEntWarps - 1) / kEntWarps;
    const int grid = (int)(blocks < kEntMaxBlocks ? blocks : kEntMaxBlocks);
    entropy_kernel<<<grid, 32 * kEntWarps, 0, s>>>(img, N, B, L, per, thr, T, flags, H, keys,
                                                   near);
    return cudaGetLastError();
}

size_t select_state_bytes() { return sizeof(SelectState) + 256 * sizeof(unsigned); }

__global__ void fill_u32_kernel(uint32_t* __restrict__ a, int64_t n, uint32_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

cudaError_t launch_fill_u32(uint32_t* a, int64_t n, uint32_t v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_u32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, n, v);
    return cudaGetLastError();
}

cudaError_t launch_top_select(const unsigned long long* keys, int64_t n, int64_t k,
                              void* state, uint32_t* flags, unsigned long long* near,
                              cudaStream_t s, int* launches)
{
    SelectState* st = static_cast<SelectState*>(state);
    unsigned* hist = reinterpret_cast<unsigned*>(st + 1);
    if (n <= 0) return cudaSuccess;
    select_init_kernel<<<1, 256, 0, s>>>(st, k, hist);
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1184) blocks = 1184;
    for (int shift = 56; shift >= 0; shift -= 8) {
        select_hist_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, n, st, shift, hist);
        select_pick_kernel<<<1, 256, 0, s>>>(st, shift, hist);
    }
    select_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, st, flags, near);
    if (launches) *launches += 18;
    return cudaGetLastError();
}

cudaError_t launch_pool_scatter(const uint32_t* flags, const uint32_t* pos, int64_t n_pos,
                                int per, int L, uint32_t* pool_xy, cudaStream_t s)
{
    if (n_pos == 0) return cudaSuccess;
    pool_scatter_kernel<<<(unsigned)((n_pos + 255) / 256), 256, 0, s>>>(flags, pos, n_pos, per,
                                                                        L, pool_xy);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2x2 box sums S2[y][x] = img[y][x] + img[y][x+1] + img[y+1][x] + img[y+1][x+1]
// (pitch N, x, y < N - 1): the decimated value d' of every domain at every
// step is one S2 entry, so the image is summed once per encode.
// ---------------------------------------------------------------------------
__global__ void box2_kernel(const uint8_t* __restrict__ img, int N, uint16_t* __restrict__ s2)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= N - 1 || y >= N - 1) return;
    const uint8_t* p0 = img + (int64_t)y * N + x;
    s2[(int64_t)y * N + x] = (uint16_t)((int)p0[0] + p0[1] + p0[N] + p0[N + 1]);
}

// Top-level active ranges: every B_max block in raster order (Sec. 2).
__global__ void init_ranges_kernel(uint32_t* __restrict__ act, int tops, int B_max)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)tops * tops) return;
    const uint32_t x = (uint32_t)((i % tops) * B_max), y = (uint32_t)((i / tops) * B_max);
    act[i] = x | (y << 16);
}

cudaError_t launch_init_ranges(uint32_t* act, int tops, int B_max, cudaStream_t s)
{
    const int64_t n = (int64_t)tops * tops;
    if (n == 0) return cudaSuccess;
    init_ranges_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(act, tops, B_max);
    return cudaGetLastError();
}

cudaError_t launch_box2(const uint8_t* img, int N, uint16_t* s2, cudaStream_t s)
{
    if (N < 2) return cudaSuccess;
    dim3 grid((unsigned)((N - 1 + 255) / 256), (unsigned)(N - 1));
    box2_kernel<<<grid, 256, 0, s>>>(img, N, s2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Domain gather (Sec. 2 decimation): for pool column c, the B x B array of
// 2x2 sums d' (d'[i][j] = S2[y + 2i][x + 2j]) is written centred (d' - 510,
// FP16, exact) into the tile layout, with sum d', sum d'^2 and the filter
// constants m_c, beta_s.  K/8 threads per column, each producing one 16-byte
// row of a core matrix.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256)
gather_kernel(const uint16_t* __restrict__ box, int N, int B, int L, int per,
              const uint32_t* __restrict__ pool_xy, int64_t dn, int64_t cols_pad,
              const uint32_t* __restrict__ dn_dev, StepParams sp, __half* __restrict__ D,
              float* __restrict__ cf, ColExact* __restrict__ ci)
{
    // Thread t: column c = block's first + 8 (t / (8 G)) + t % 8, k-group
    // (t / 8) % G.  Eight consecutive threads write eight consecutive
    // columns' 16-byte rows of one core matrix: 128 contiguous bytes.
    constexpr int G = K / 8;
    constexpr int kCols = 256 / G;  // columns per block (256 threads)
    __shared__ int s_sum[kCols], s_sq[kCols];
    const int t = threadIdx.x;
    const int cl = t & 7, kg = (t >> 3) % G, cgp = t / (8 * G);
    const int64_t c0 = (int64_t)blockIdx.x * kCols;
    const int64_t c = c0 + cgp * 8 + cl;
    if (t < kCols) {
        s_sum[t] = 0;
        s_sq[t] = 0;
    }
    // columns in use: the padded pool (cols_pad stays the layout's stride)
    int64_t cols = cols_pad;
    if (dn_dev) {
        dn = dev_count(dn, dn_dev);
        cols = min(cols_pad, round_up64(dn > 0 ? dn : 1, kColPad));
    }
    __syncthreads();
    if (c0 >= cols) return;  // whole block past the used columns (cols % kCols == 0)
    const bool real = c < dn;
    int x = 0, y = 0;
    if (real) {
        if (pool_xy) {
            const uint32_t v = pool_xy[c];
            x = (int)(v & 0xffffu);
            y = (int)(v >> 16);
        } else {
            const uint32_t cu = (uint32_t)c, pu = (uint32_t)per;  // c < 2^31
            x = (int)(cu % pu) * L;
            y = (int)(cu / pu) * L;
        }
    }
    const int n = B * B, lb = __ffs(B) - 1;  // B is a power of two
    const uint16_t* __restrict__ base = box + (int64_t)y * N + x;
    int sum = 0, sq = 0;
    __align__(16) __half hv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = kg * 8 + e;
        int val = 0;
        if (real && k < n) {
            const int i = k >> lb, j = k & (B - 1);
            const int d = base[2 * i * N + 2 * j];
            sum += d;
            sq += d * d;
            val = d - kDomainCentre;
        }
        hv[e] = __int2half_rn(val);
    }
    *reinterpret_cast<uint4*>(D + tile_off(c, kg * 8, cols_pad, K)) =
        *reinterpret_cast<const uint4*>(hv);
    if (real) {
        atomicAdd(&s_sum[c - c0], sum);
        atomicAdd(&s_sq[c - c0], sq);
    }
    __syncthreads();
    if (t >= kCols) return;
    // constants in groups of 4 columns: constant j of column cc at
    // cf[((cc / 4) * cw + j) * 4 + cc % 4]
    const int64_t cc = c0 + t;
    float* grp = cf + (cc >> 2) * sp.cw * 4 + (cc & 3);
    if (cc < dn) {
        const int sd = s_sum[t], sd2 = s_sq[t];
        const long long vd = (long long)n * sd2 - (long long)sd * sd;
        grp[0] = (float)(sd - kDomainCentre * n) * (1.0f / (float)n);
        for (int u = 0; u < sp.ns; ++u)
            grp[(1 + u) * 4] =
                __double2float_rn((double)sp.p[u] * sp.p[u] * (double)vd / (double)n);
        ci[cc] = ColExact{sd, sd2};
    } else {
        grp[0] = 0.0f;
        for (int u = 0; u < sp.ns; ++u) grp[(1 + u) * 4] = __int_as_float(0x7f800000);
        ci[cc] = ColExact{0, 0};
    }
}

// Pool-wide reductions over the per-domain sums: max Vd and the key
// (Vd << 24 | c) of the smallest Vd (first index on ties; Vd < 2^36,
// c < 2^24).  Grid-stride; one atomic per block.
__global__ void __launch_bounds__(256)
pool_stats_kernel(const ColExact* __restrict__ ci, int64_t dn, const uint32_t* __restrict__ dn_dev,
                  int n, unsigned long long* __restrict__ vd_max,
                  unsigned long long* __restrict__ vd_min_key)
{
    dn = dev_count(dn, dn_dev);
    unsigned long long mx = 0, mn = ~0ull;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < dn;
         c += (int64_t)gridDim.x * blockDim.x) {
        const ColExact e = ci[c];
        const unsigned long long vd =
            (unsigned long long)((long long)n * e.sd2 - (long long)e.sd * e.sd);
        mx = vd > mx ? vd : mx;
        const unsigned long long key = (vd << 24) | (unsigned long long)c;
        mn = key < mn ? key : mn;
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const unsigned long long omx = __shfl_xor_sync(0xffffffffu, mx, m);
        const unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn, m);
        mx = omx > mx ? omx : mx;
        mn = omn < mn ? omn : mn;
    }
    __shared__ unsigned long long smx[8], smn[8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smx[w] = mx;
        smn[w] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mx = smx[i] > mx ? smx[i] : mx;
            mn = smn[i] < mn ? smn[i] : mn;
        }
        atomicMax(vd_max, mx);
        atomicMin(vd_min_key, mn);
    }
}

cudaError_t launch_gather(const uint16_t* s2img, int N, int B, int L, int per,
                          const uint32_t* pool_xy, int64_t dn, int64_t cols_pad, int K,
                          const StepParams& sp, __half* D, float* cf, ColExact* ci,
                          unsigned long long* vd_max, unsigned long long* vd_min_key,
                          cudaStream_t s, const uint32_t* dn_dev)
{
    // 256 threads cover 256 / (K / 8) columns (8, 32 or 128), which divides kColPad
    const unsigned blocks = (unsigned)(cols_pad / (256 / (K / 8)));
    switch (K) {
        case 16:
            gather_kernel<16><<<blocks, 256, 0, s>>>(s2img, N, B, L, per, pool_xy, dn, cols_pad,
                                                     dn_dev, sp, D, cf, ci);
            break;
        case 64:
            gather_kernel<64><<<blocks, 256, 0, s>>>(s2img, N, B, L, per, pool_xy, dn, cols_pad,
                                                     dn_dev, sp, D, cf, ci);
            break;
        case 256:
            gather_kernel<256><<<blocks, 256, 0, s>>>(s2img, N, B, L, per, pool_xy, dn, cols_pad,
                                                      dn_dev, sp, D, cf, ci);
            break;
        default: return cudaErrorInvalidValue;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // pool-wide max Vd (filter bound) and (min Vd, first index) key (flat ranges)
    if (dn > 0) {
        pool_stats_kernel<<<256, 256, 0, s>>>(ci, dn, dn_dev, B * B, vd_max, vd_min_key);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Range prep: for active range rho and isometry k, row 8 rho + k holds
// T_k^-1(r) - 128 (so that sum r . T_k(d') = sum T_k^-1(r) . d'); plus the
// isometry-invariant sums and the filter error bound.  One warp per range.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
range_prep_kernel(const uint8_t* __restrict__ img, int N, int B, const uint32_t* __restrict__ act,
                  int R, const uint32_t* __restrict__ R_dev, int Rpad, int64_t rows_pad, int K,
                  StepParams sp, const unsigned long long* __restrict__ vd_max, int iso_major,
                  __half* __restrict__ A, RowConst* __restrict__ rc)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rho = blockIdx.x * 8 + w;
    int rlim = Rpad;
    if (R_dev) {
        // ranges in use: up to the M tiles that cover the R active ones
        R = (int)dev_count(R, R_dev);
        rlim = min(Rpad, (int)round_up64(R, 128));
    }
    if (rho >= rlim) return;
    const int n = B * B, G = K / 8;
    const bool real = rho < R;
    int rx = 0, ry = 0;
    if (real) {
        const uint32_t v = act[rho];
        rx = (int)(v & 0xffffu);
        ry = (int)(v >> 16);
    }
    int sr = 0, sr2 = 0;
    if (real)
        for (int t = lane; t < n; t += 32) {
            const int v = img[(int64_t)(ry + t / B) * N + rx + t % B];
            sr += v;
            sr2 += v * v;
        }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, m);
        sr2 += __shfl_xor_sync(0xffffffffu, sr2, m);
    }
    for (int v = lane; v < 8 * G; v += 32) {
        const int k = v / G, kg = v % G;
        __align__(16) __half hv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int kk = kg * 8 + e;
            int val = 0;
            if (real && kk < n) {
                int si, sj;
                iso_inv_src(kk / B, kk % B, k, B, si, sj);
                val = (int)img[(int64_t)(ry + si) * N + rx + sj] - kRangeCentre;
            }
            hv[e] = __int2half_rn(val);
        }
        const int64_t row = iso_major ? (int64_t)k * Rpad + rho : (int64_t)rho * 8 + k;
        *reinterpret_cast<uint4*>(A + tile_off(row, kg * 8, rows_pad, K)) =
            *reinterpret_cast<const uint4*>(hv);
    }
    if (lane == 0) {
        RowConst r{0, 0, 0.0f, 0.0f};
        if (real) {
            const double u = 0x1p-24;
            const double vr = (double)((long long)n * sr2 - (long long)sr * sr);
            const double vdm = (double)(*vd_max);
            int pm = 0;
            for (int t = 0; t < sp.ns; ++t) pm = max(pm, sp.p[t]);
            const double bound = (2.0 * u + u * u) *
                                 (8.0 * pm * sp.q * sqrt(vr * vdm) + (double)pm * pm * vdm) /
                                 (double)n;
            r.sr = sr;
            r.sr2 = sr2;
            r.a = (float)(sr - kRangeCentre * n);
            r.delta = __double2float_ru(2.0 * bound);
        }
        rc[rho] = r;
    }
}

cudaError_t launch_range_prep(const uint8_t* img, int N, int B, const uint32_t* act, int R,
                              int64_t rows_pad, int K, const StepParams& sp,
                              const unsigned long long* vd_max, int iso_major, __half* A,
                              RowConst* rc, cudaStream_t s, const uint32_t* R_dev)
{
    const int Rpad = (int)(rows_pad / 8);
    if (Rpad == 0) return cudaSuccess;
    range_prep_kernel<<<(Rpad + 7) / 8, 256, 0, s>>>(img, N, B, act, R, R_dev, Rpad, rows_pad, K,
                                                     sp, vd_max, iso_major, A, rc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Split / requeue (Sec. 2): reduce the per-chunk partial bests, then split
// iff the step is not the last and the RMS error exceeds the tolerance,
//   sqrt(E/n) > e16/16  <=>  256 score > 16 q^2 n^2 e16^2,
// score = 16 q^2 Vr + h.  The last step always stores its best mapping.
// ---------------------------------------------------------------------------
__global__ void split_decide_kernel(const Best* __restrict__ part, int n_chunks,
                                    const RowConst* __restrict__ rc, int R, int n, StepParams sp,
                                    int e16, int last, int dn,
                                    const unsigned long long* __restrict__ vd_min_key,
                                    Best* __restrict__ best, uint32_t* __restrict__ split,
                                    StepCounts dc)
{
    const int rho = blockIdx.x * blockDim.x + threadIdx.x;
    if (dc.R) R = (int)dev_count(R, dc.R);
    if (dc.dn) dn = (int)dev_count(dn, dc.dn);
    if (dc.n_parts) n_chunks = (int)*dc.n_parts;
    if (rho >= R) return;
    const RowConst r = rc[rho];
    long long h = kNoCandidate;
    unsigned idx = 0xffffffffu;
    if (dn > 0 && range_is_flat(r, n)) {
        // h = p_s^2 Vd over all (c, k, s): k = 0; c = the first smallest-Vd
        // domain, or c = 0 when p_s = 0 (then every domain gives h = 0)
        const unsigned long long key = *vd_min_key;
        const long long vdmin = (long long)(key >> 24);
        const unsigned cmin = (unsigned)(key & 0xffffffu);
        for (int s = 0; s < sp.ns; ++s) {
            const long long ps = sp.p[s];
            const long long hs = ps == 0 ? 0 : ps * ps * vdmin;
            const unsigned is = pack_idx(ps == 0 ? 0u : cmin, 0u, (unsigned)s);
            if (key_less(hs, is, h, idx)) {
                h = hs;
                idx = is;
            }
        }
    } else {
        for (int c = 0; c < n_chunks; ++c) {
            const Best b = part[(int64_t)rho * n_chunks + c];
            if (key_less(b.h, b.idx, h, idx)) {
                h = b.h;
                idx = b.idx;
            }
        }
    }
    const int q = sp.q;
    bool sp_;
    if (dn == 0 || h == kNoCandidate) {
        sp_ = !last;
    } else {
        const long long vr = (long long)n * r.sr2 - (long long)r.sr * r.sr;
        const long long qq = (long long)q * q;
        const long long score = 16LL * qq * vr + h;
        const long long lim = 16LL * qq * n * n * (long long)e16 * e16;
        sp_ = !last && 256LL * score > lim;
    }
    Best b;
    b.h = h;
    b.idx = idx;
    b.pad = 0;
    best[rho] = b;
    split[rho] = sp_ ? 1u : 0u;
}

__global__ void split_scatter_kernel(const uint32_t* __restrict__ act, const Best* __restrict__ best,
                                     const uint32_t* __restrict__ split,
                                     const uint32_t* __restrict__ split_pos,
                                     const RowConst* __restrict__ rc, int R, int B, int level,
                                     const uint32_t* __restrict__ pool_xy, int per, int L, int dn,
                                     uint32_t* __restrict__ next_act, fic_code* __restrict__ codes,
                                     int64_t code_base, StepCounts dc)
{
    const int rho = blockIdx.x * blockDim.x + threadIdx.x;
    if (dc.R) R = (int)dev_count(R, dc.R);
    if (dc.dn) dn = (int)dev_count(dn, dc.dn);
    if (dc.code_base) code_base = *dc.code_base;
    if (rho >= R) return;
    const uint32_t v = act[rho];
    const uint32_t x = v & 0xffffu, y = v >> 16;
    if (split[rho]) {
        const uint32_t hb = (uint32_t)B / 2;
        uint32_t* o = next_act + 4 * (int64_t)split_pos[rho];
        o[0] = x | (y << 16);
        o[1] = (x + hb) | (y << 16);
        o[2] = x | ((y + hb) << 16);
        o[3] = (x + hb) | ((y + hb) << 16);
        return;
    }
    const int n = B * B;
    const Best b = best[rho];
    fic_code c;
    c.rx = (uint16_t)x;
    c.ry = (uint16_t)y;
    c.level = (uint8_t)level;
    const int oq = rc[rho].sr / (2 * n);
    c.o_q = (uint8_t)(oq > 127 ? 127 : oq);
    if (dn == 0 || b.h == kNoCandidate) {
        c.iso = 0;
        c.s_idx = 0xff;
        c.dx = 0;
        c.dy = 0;
        c.pool_idx = 0xffffffffu;
    } else {
        const uint32_t col = b.idx >> 7;
        c.iso = (uint8_t)((b.idx >> 4) & 7);
        c.s_idx = (uint8_t)(b.idx & 15);
        c.pool_idx = col;
        if (pool_xy) {
            const uint32_t pv = pool_xy[col];
            c.dx = (uint16_t)(pv & 0xffffu);
            c.dy = (uint16_t)(pv >> 16);
        } else {
            c.dx = (uint16_t)((col % (uint32_t)per) * L);
            c.dy = (uint16_t)((col / (uint32_t)per) * L);
        }
    }
    codes[code_base + rho - (int64_t)split_pos[rho]] = c;
}

cudaError_t launch_split_decide(const Best* part, int n_chunks, const RowConst* rc, int R,
                                int n, const StepParams& sp, int e16, int last, int dn,
                                const unsigned long long* vd_min_key, Best* best,
                                uint32_t* split, cudaStream_t s, const StepCounts& dc)
{
    if (R == 0) return cudaSuccess;
    split_decide_kernel<<<(R + 255) / 256, 256, 0, s>>>(part, n_chunks, rc, R, n, sp, e16, last,
                                                        dn, vd_min_key, best, split, dc);
    return cudaGetLastError();
}

cudaError_t launch_split_scatter(const uint32_t* act, const Best* best, const uint32_t* split,
                                 const uint32_t* split_pos, const RowConst* rc, int R, int B,
                                 int level, const uint32_t* pool_xy, int per, int L, int dn,
                                 uint32_t* next_act, void* codes, int64_t code_base,
                                 cudaStream_t s, const StepCounts& dc)
{
    if (R == 0) return cudaSuccess;
    split_scatter_kernel<<<(R + 255) / 256, 256, 0, s>>>(
        act, best, split, split_pos, rc, R, B, level, pool_xy, per, L, dn, next_act,
        static_cast<fic_code*>(codes), code_base, dc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Record order (Sec. 3.3): top-level ranges in raster order, then the
// quadtree depth first in TL, TR, BL, BR order.  Leaves tile the image, so
// that order is the order of their top-left finest cells under the key
// (top-level raster index, Morton code with the row bit above the column bit).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread_bits(uint32_t v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void order_mark_kernel(const fic_code* __restrict__ codes, int64_t n_codes,
                                  const uint32_t* __restrict__ n_dev, int N, int B_max, int B_min,
                                  uint32_t* __restrict__ cellmap, uint32_t* __restrict__ cellflag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dev_count(n_codes, n_dev)) return;
    const fic_code c = codes[i];
    const int cpt = B_max / B_min;  // finest cells per top-level side
    const int cx = c.rx / B_min, cy = c.ry / B_min;
    const int tops = N / B_max;
    const int64_t top = (int64_t)(cy / cpt) * tops + cx / cpt;
    const uint32_t morton = (spread_bits((uint32_t)(cy % cpt)) << 1) | spread_bits((uint32_t)(cx % cpt));
    const int64_t z = top * cpt * cpt + morton;
    cellmap[z] = (uint32_t)i;
    cellflag[z] = 1u;
}

__global__ void order_gather_kernel(const fic_code* __restrict__ codes,
                                    const uint32_t* __restrict__ cellmap,
                                    const uint32_t* __restrict__ cellflag,
                                    const uint32_t* __restrict__ rank, int64_t n_cells,
                                    fic_code* __restrict__ out)
{
    const int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= n_cells || !cellflag[z]) return;
    out[rank[z]] = codes[cellmap[z]];
}

cudaError_t launch_order_mark(const void* codes, int64_t n_codes, int N, int B_max, int B_min,
                              uint32_t* cellmap, uint32_t* cellflag, cudaStream_t s,
                              const uint32_t* n_dev)
{
    if (n_codes == 0) return cudaSuccess;
    order_mark_kernel<<<(unsigned)((n_codes + 255) / 256), 256, 0, s>>>(
        static_cast<const fic_code*>(codes), n_codes, n_dev, N, B_max, B_min, cellmap, cellflag);
    return cudaGetLastError();
}

cudaError_t launch_order_gather(const void* codes, const uint32_t* cellmap,
                                const uint32_t* cellflag, const uint32_t* rank, int64_t n_cells,
                                void* out, cudaStream_t s)
{
    if (n_cells == 0) return cudaSuccess;
    order_gather_kernel<<<(unsigned)((n_cells + 255) / 256), 256, 0, s>>>(
        static_cast<const fic_code*>(codes), cellmap, cellflag, rank, n_cells,
        static_cast<fic_code*>(out));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Decoder pass (Sec. 2: each range rebuilt from its domain and mapping):
//   pixel = clamp(floor(((2 o_q + 1) 4qn + p (n T(d')_ij - sum d') + 2qn) / (4qn)), 0, 255)
// i.e. (2 o_q + 1) + S (d - mean d) with d = T(d')/4, rounded half up.
// One warp per record; *changed is set when any pixel differs from src.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
decode_pass_kernel(const fic_code* __restrict__ codes, int64_t n_codes, DecodeS ds,
                   const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int N,
                   unsigned* __restrict__ changed)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ci = (int64_t)blockIdx.x * 8 + w;
    if (ci >= n_codes) return;
    const fic_code c = codes[ci];
    const int B = ds.B_max >> c.level, n = B * B;
    bool diff = false;
    if (c.s_idx == 0xff) {
        for (int t = lane; t < n; t += 32) {
            const int64_t o = (int64_t)(c.ry + t / B) * N + c.rx + t % B;
            const uint8_t v = (uint8_t)(2 * c.o_q + 1);
            diff |= src[o] != v;
            dst[o] = v;
        }
    } else {
        // sum d' over the domain (isometry invariant)
        long long sd = 0;
        for (int t = lane; t < n; t += 32) {
            const uint8_t* p0 = src + (int64_t)(c.dy + 2 * (t / B)) * N + c.dx + 2 * (t % B);
            sd += (int)p0[0] + p0[1] + p0[N] + p0[N + 1];
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, m);
        const long long p = ds.p[c.level][c.s_idx], q = ds.q[c.level];
        const long long den = 4 * q * n;
        for (int t = lane; t < n; t += 32) {
            const int i = t / B, j = t % B;
            int si, sj;
            iso_fwd_src(i, j, c.iso, B, si, sj);
            const uint8_t* p0 = src + (int64_t)(c.dy + 2 * si) * N + c.dx + 2 * sj;
            const long long d = (int)p0[0] + p0[1] + p0[N] + p0[N + 1];
            const long long num = (2LL * c.o_q + 1) * den + p * ((long long)n * d - sd) + den / 2;
            long long v = num >= 0 ? num / den : -((-num + den - 1) / den);
            v = v < 0 ? 0 : (v > 255 ? 255 : v);
            const int64_t o = (int64_t)(c.ry + i) * N + c.rx + j;
            diff |= src[o] != (uint8_t)v;
            dst[o] = (uint8_t)v;
        }
    }
    if (__any_sync(0xffffffffu, diff) && lane == 0) atomicOr(changed, 1u);
}

// ---------------------------------------------------------------------------
// Stored stream records (Sec. 3.3, Fig. 7, eq. 8): step (2 bits), mean
// (7 bits), then when the step's pool is not empty isometry (3 bits),
// address (ceil(log2 DN) bits) and S index (ceil(log2 |S|) bits), most
// significant bit first.  Sizes first, then (after an exclusive scan of
// the sizes) every record ORs its bits into 32-bit words in which stream
// bit b is word b / 32, bit 31 - b % 32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pack_record(const fic_code& c, const PackLevels& pl, uint64_t* v)
{
    const int l = c.level;
    uint64_t x = ((uint64_t)l << 7) | (uint64_t)(c.o_q & 0x7f);
    int nb = 9;
    if (pl.has_pool[l]) {
        x = (x << 3) | (uint64_t)(c.iso & 7);
        x = (x << pl.addr_bits[l]) | (uint64_t)c.pool_idx;
        x = (x << pl.s_bits[l]) | (uint64_t)c.s_idx;
        nb += 3 + pl.addr_bits[l] + pl.s_bits[l];
    }
    *v = x;
    return nb;
}

__global__ void pack_sizes_kernel(const fic_code* __restrict__ codes, int64_t n, PackLevels pl,
                                  uint32_t* __restrict__ sizes)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t v;
    sizes[i] = (uint32_t)pack_record(codes[i], pl, &v);
}

__global__ void pack_write_kernel(const fic_code* __restrict__ codes, int64_t n, PackLevels pl,
                                  const uint32_t* __restrict__ offs, uint32_t* __restrict__ words)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t v;
    int nb = pack_record(codes[i], pl, &v);
    uint32_t b = offs[i];
    while (nb > 0) {
        const int room = 32 - (int)(b & 31);
        const int take = nb < room ? nb : room;
        const uint32_t part = (uint32_t)((v >> (nb - take)) & ((1ull << take) - 1ull));
        atomicOr(&words[b >> 5], part << (room - take));
        nb -= take;
        b += (uint32_t)take;
    }
}

cudaError_t launch_pack_records(const void* codes, int64_t n, const PackLevels& pl,
                                uint32_t* sizes, uint32_t* offs, uint32_t* scan_tmp,
                                uint32_t* total_bits, uint32_t* words, int64_t n_words,
                                cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(words, 0, sizeof(uint32_t) * (size_t)(n_words ? n_words : 1), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaMemsetAsync(total_bits, 0, sizeof(uint32_t), s);
    const fic_code* c = static_cast<const fic_code*>(codes);
    const unsigned g = (unsigned)((n + 255) / 256);
    pack_sizes_kernel<<<g, 256, 0, s>>>(c, n, pl, sizes);
    e = launch_scan(sizes, offs, n, scan_tmp, total_bits, s, nullptr);
    if (e != cudaSuccess) return e;
    pack_write_kernel<<<g, 256, 0, s>>>(c, n, pl, offs, words);
    return cudaGetLastError();
}

cudaError_t launch_decode_pass(const void* codes, int64_t n_codes, const DecodeS& ds,
                               const uint8_t* src, uint8_t* dst, int N, unsigned* changed,
                               cudaStream_t s)
{
    if (n_codes == 0) return cudaSuccess;
    decode_pass_kernel<<<(unsigned)((n_codes + 7) / 8), 256, 0, s>>>(
        static_cast<const fic_code*>(codes), n_codes, ds, src, dst, N, changed);
    return cudaGetLastError();
}

}  // namespace fic
