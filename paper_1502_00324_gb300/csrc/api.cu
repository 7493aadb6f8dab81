// api.cu -- C ABI of the range-domain search (include/fic.h): per-device
// workspace, the quadtree step driver and instrumentation.
//
// Step driver for one image (Sec. 2 quadtree, Sec. 3 pool, Sec. 3.2 S):
//   active ranges <- every B_max x B_max block in raster order
//   for each step: [entropy -> scan -> pool list] (threshold >= 0 only)
//                  -> domain gather (operand D', column constants)
//                  -> range prep (operand A' with inverse isometries)
//                  -> contraction + scoring (tensor or CUDA-core engine)
//                  -> split decision -> scan -> records / children
//   -> record ordering (raster of top ranges, then TL, TR, BL, BR).
// Host and device meet at the image upload, one count read per step (pool
// size, number of splits) and the final records.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fic.h"
#include "kernels.h"

namespace fic {
namespace {

// ---------------------------------------------------------------------------
// Instrumentation
// ---------------------------------------------------------------------------
struct StatsState {
    std::mutex mu;
    fic_stats st;
    bool timing = false;
};
StatsState g_stats;

struct PendingTiming {
    int kind;
    cudaEvent_t a, b;
};

class Launcher {
public:
    explicit Launcher(cudaStream_t s) : s_(s)
    {
        std::lock_guard<std::mutex> g(g_stats.mu);
        timing_ = g_stats.timing;
    }
    ~Launcher() { harvest(); }

    // Brackets one or more kernel launches of one kind.
    void begin(int kind)
    {
        kind_ = kind;
        if (!timing_) return;
        cur_.kind = kind;
        cudaEventCreate(&cur_.a);
        cudaEventCreate(&cur_.b);
        cudaEventRecord(cur_.a, s_);
    }
    void end(int launches, double flops = 0.0, double bytes = 0.0, int64_t matches = 0)
    {
        {
            std::lock_guard<std::mutex> g(g_stats.mu);
            g_stats.st.launches[kind_] += launches;
            g_stats.st.flops[kind_] += flops;
            g_stats.st.bytes[kind_] += bytes;
            g_stats.st.matches += matches;
        }
        if (!timing_) return;
        cudaEventRecord(cur_.b, s_);
        pending_.push_back(cur_);
    }
    void harvest()
    {
        for (auto& p : pending_) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.b) == cudaSuccess &&
                cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                std::lock_guard<std::mutex> g(g_stats.mu);
                g_stats.st.ms[p.kind] += ms;
            }
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        pending_.clear();
    }

private:
    cudaStream_t s_;
    bool timing_ = false;
    int kind_ = FIC_K_MISC;
    PendingTiming cur_{};
    std::vector<PendingTiming> pending_;
};

// ---------------------------------------------------------------------------
// Workspace: device buffers grown on demand and kept for the process.
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 8 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        cap = want;
        return cudaSuccess;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Small device scalars.
struct Scalars {
    uint32_t total;
    uint32_t changed;
    unsigned long long near;
    unsigned long long vd_max;
    unsigned long long vd_min_key;
    int err;
    int pad;
};

struct Context {
    std::mutex mu;
    int device = -1;
    bool ready = false;
    int sm_count = 0;
    DevBuf img, entT, flags, pos, scan_tmp, pool, D, cf, ci, A, rc, part, best, split,
        split_pos, act0, act1, codes_tmp, codes_out, cellmap, cellflag, cellrank, H, gbest, box2,
        dec0, dec1, scal;
    Scalars* host_scal = nullptr;  // pinned
    static constexpr int kEntTable = 4097;
};

std::mutex g_ctx_mu;
Context* g_ctx[64] = {};

thread_local char g_last_error[160] = "";

int to_status(cudaError_t e)
{
    if (e == cudaSuccess) return FIC_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FIC_ENOMEM;
    return FIC_ECUDA;
}

#define FIC_TRY(expr)                           \
    do {                                        \
        cudaError_t e__ = (expr);               \
        if (e__ != cudaSuccess) {               \
            return to_status(e__);              \
        }                                       \
    } while (0)

int get_context(Context** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIC_ENODEV;
    if (dev < 0 || dev >= 64) return FIC_ENODEV;
    std::lock_guard<std::mutex> g(g_ctx_mu);
    if (!g_ctx[dev]) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return FIC_ENODEV;
        if (prop.major != 10 || prop.minor != 3) return FIC_ENODEV;
        Context* c = new Context();
        c->device = dev;
        c->sm_count = prop.multiProcessorCount;
        g_ctx[dev] = c;
    }
    *out = g_ctx[dev];
    return FIC_OK;
}

int ensure_ready(Context* c, cudaStream_t s)
{
    if (c->ready) return FIC_OK;
    FIC_TRY(c->entT.ensure(sizeof(double) * Context::kEntTable));
    FIC_TRY(c->scal.ensure(sizeof(Scalars)));
    FIC_TRY(cudaMallocHost((void**)&c->host_scal, sizeof(Scalars)));
    FIC_TRY(launch_entropy_table(c->entT.as<double>(), Context::kEntTable, s));
    FIC_TRY(cudaStreamSynchronize(s));
    c->ready = true;
    return FIC_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
int ilog2i(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

bool valid_side(int b) { return b == 2 || b == 4 || b == 8 || b == 16; }

int validate(const fic_params* p, int* n_levels)
{
    if (!p) return FIC_EINVAL;
    if (p->N <= 0 || p->N > 65535) return FIC_EINVAL;
    if (!valid_side(p->B_max) || !valid_side(p->B_min) || p->B_min > p->B_max) return FIC_EINVAL;
    if (p->N % p->B_max) return FIC_EINVAL;
    if (p->L < 1) return FIC_EINVAL;
    if (!(p->err_tol >= 0.0 && p->err_tol <= 255.0)) return FIC_EINVAL;
    if (p->engine != FIC_ENGINE_TENSOR && p->engine != FIC_ENGINE_PLAIN) return FIC_EINVAL;
    if (p->reserved != 0) return FIC_EINVAL;
    const int nl = ilog2i(p->B_max) - ilog2i(p->B_min) + 1;
    if (nl > FIC_MAX_LEVELS) return FIC_EINVAL;
    for (int l = 0; l < nl; ++l) {
        const fic_sset& s = p->S_sets[l];
        // S = p/q in [0, 1] (Sec. 2); q <= 256 keeps every score term in int64
        if (s.n_s < 1 || s.n_s > FIC_MAX_S || s.q < 1 || s.q > 256) return FIC_EINVAL;
        for (int i = 0; i < s.n_s; ++i)
            if (s.p[i] < 0 || s.p[i] > s.q) return FIC_EINVAL;
    }
    *n_levels = nl;
    return FIC_OK;
}

StepParams make_step(const fic_sset& s, int n)
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

// Pool of one step: entropy flags -> scan -> raster-order list.  Returns DN
// through *dn (host); pool list in c->pool.  When thr < 0 the pool is every
// position and no list is built (*use_list = false).
int build_pool(Context* c, Launcher& L, const uint8_t* dimg, int N, int B, int Lstep, double thr,
               bool filter, cudaStream_t s, int64_t* dn, int64_t* near, bool* use_list,
               bool want_H)
{
    const int per = (N >= 2 * B) ? (N - 2 * B) / Lstep + 1 : 0;
    const int64_t npos = (int64_t)per * per;
    *near = 0;
    if (!filter) {
        *dn = npos;
        *use_list = false;
        return FIC_OK;
    }
    *use_list = true;
    if (npos == 0) {
        *dn = 0;
        return FIC_OK;
    }
    FIC_TRY(c->flags.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(c->pos.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(c->pool.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(c->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(npos)));
    if (want_H) FIC_TRY(c->H.ensure(sizeof(double) * npos));
    Scalars* ds = c->scal.as<Scalars>();
    FIC_TRY(cudaMemsetAsync(&ds->near, 0, sizeof(unsigned long long), s));
    L.begin(FIC_K_ENTROPY);
    FIC_TRY(launch_entropy(dimg, N, B, Lstep, per, thr, c->entT.as<double>(),
                           c->flags.as<uint32_t>(), want_H ? c->H.as<double>() : nullptr,
                           &ds->near, s));
    L.end(1, 0.0, (double)npos * (4.0 * B * B + 4.0));
    L.begin(FIC_K_SCAN);
    int nl = 0;
    FIC_TRY(launch_scan(c->flags.as<uint32_t>(), c->pos.as<uint32_t>(), npos,
                        c->scan_tmp.as<uint32_t>(), &ds->total, s, &nl));
    FIC_TRY(launch_pool_scatter(c->flags.as<uint32_t>(), c->pos.as<uint32_t>(), npos, per,
                                Lstep, c->pool.as<uint32_t>(), s));
    L.end(nl + 1, 0.0, (double)npos * 12.0);
    FIC_TRY(cudaMemcpyAsync(c->host_scal, ds, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    FIC_TRY(cudaStreamSynchronize(s));
    *dn = c->host_scal->total;
    *near = (int64_t)c->host_scal->near;
    return FIC_OK;
}

// Column chunking of the contraction: work items are (128-row M tile,
// chunk of column tiles).  Picks the chunk count that minimises the
// estimated makespan over `slots` concurrent items (waves x tiles per item,
// plus a per-item cost of refilling the pipeline).
void choose_chunks(int sm_count, int64_t n_mtiles, int64_t n_ct, int* n_chunks, int* per_chunk)
{
    const int64_t slots = sm_count;
    const double item_cost = 2.0;  // in tiles
    int64_t best_nc = 1;
    double best = 1e300;
    const int64_t max_nc = n_ct < 4096 ? n_ct : 4096;
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

int encode_impl(const uint8_t* img, const fic_params* p, fic_code* codes_out, int64_t codes_cap,
                fic_result* out, cudaStream_t s)
{
    if (!img || !out) return FIC_EINVAL;
    int n_levels = 0;
    int st = validate(p, &n_levels);
    if (st) return st;
    Context* c = nullptr;
    st = get_context(&c);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    st = ensure_ready(c, s);
    if (st) return st;

    memset(out, 0, sizeof(*out));
    const int N = p->N, Lstep = p->L;
    out->N = N;
    out->B_max = p->B_max;
    out->n_levels = n_levels;
    for (int l = 0; l < n_levels; ++l) out->S_sets[l] = p->S_sets[l];

    Launcher L(s);
    Scalars* ds = c->scal.as<Scalars>();

    // input image
    const uint8_t* dimg = img;
    if (!is_device_ptr(img)) {
        FIC_TRY(c->img.ensure((size_t)N * N));
        FIC_TRY(cudaMemcpyAsync(c->img.p, img, (size_t)N * N, cudaMemcpyHostToDevice, s));
        dimg = c->img.as<uint8_t>();
    }

    // 2x2 box sums, shared by every step's domain gather
    FIC_TRY(c->box2.ensure(sizeof(uint16_t) * (size_t)N * N));
    L.begin(FIC_K_GATHER);
    FIC_TRY(launch_box2(dimg, N, c->box2.as<uint16_t>(), s));
    L.end(1, 0.0, (double)N * N * 3.0);

    // capacity of records and cells: every record covers >= 1 finest cell
    const int64_t cells = (int64_t)(N / p->B_min) * (N / p->B_min);
    FIC_TRY(c->codes_tmp.ensure(sizeof(fic_code) * cells));
    FIC_TRY(c->codes_out.ensure(sizeof(fic_code) * cells));

    // top-level ranges in raster order
    int64_t R = (int64_t)(N / p->B_max) * (N / p->B_max);
    {
        std::vector<uint32_t> top((size_t)R);
        const int tops = N / p->B_max;
        for (int64_t i = 0; i < R; ++i)
            top[(size_t)i] = (uint32_t)((i % tops) * p->B_max) |
                             ((uint32_t)((i / tops) * p->B_max) << 16);
        FIC_TRY(c->act0.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(c->act1.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(cudaMemcpyAsync(c->act0.p, top.data(), sizeof(uint32_t) * R,
                                cudaMemcpyHostToDevice, s));
        FIC_TRY(cudaStreamSynchronize(s));  // 'top' leaves scope
    }
    uint32_t* act = c->act0.as<uint32_t>();
    uint32_t* next = c->act1.as<uint32_t>();
    int64_t n_codes = 0;
    const int e16 = (int)llround(16.0 * p->err_tol);

    for (int lvl = 0; lvl < n_levels && R > 0; ++lvl) {
        const int B = p->B_max >> lvl;
        const int n = B * B;
        const int K = k_pad(n);
        const int per = (N >= 2 * B) ? (N - 2 * B) / Lstep + 1 : 0;
        const int last = (lvl == n_levels - 1);
        out->n_positions[lvl] = (int64_t)per * per;
        out->ranges[lvl] = R;

        int64_t dn = 0, near = 0;
        bool use_list = false;
        st = build_pool(c, L, dimg, N, B, Lstep, p->entropy_thresh, p->entropy_thresh >= 0.0, s,
                        &dn, &near, &use_list, false);
        if (st) return st;
        out->pool_size[lvl] = dn;
        out->near_thresh[lvl] = near;
        const uint32_t* pool_xy = use_list ? c->pool.as<uint32_t>() : nullptr;

        const StepParams sp = make_step(p->S_sets[lvl], n);
        const int64_t cols_pad = round_up(dn > 0 ? dn : 1, kColPad);
        // 2x2 .. 8x8 ranges with up to 3 S values: isometry-in-accumulator
        // kernel (ranges in TMEM lanes, iso-major A); otherwise rows are
        // (range, isometry) pairs
        const bool iso = p->engine == FIC_ENGINE_TENSOR && contract_tc_iso_supports(K, sp.ns);
        const int64_t rows_pad = iso ? 8 * round_up(R, 128) : round_up(8 * R, kMTile);

        FIC_TRY(c->D.ensure(sizeof(__half) * cols_pad * K));
        FIC_TRY(c->cf.ensure(sizeof(float) * cols_pad * sp.cw));
        FIC_TRY(c->ci.ensure(sizeof(ColExact) * cols_pad));
        FIC_TRY(c->A.ensure(sizeof(__half) * rows_pad * K));
        FIC_TRY(c->rc.ensure(sizeof(RowConst) * (rows_pad / 8)));
        FIC_TRY(c->best.ensure(sizeof(Best) * R));
        FIC_TRY(c->split.ensure(sizeof(uint32_t) * R));
        FIC_TRY(c->split_pos.ensure(sizeof(uint32_t) * R));
        FIC_TRY(c->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(R)));

        FIC_TRY(cudaMemsetAsync(&ds->vd_max, 0, sizeof(unsigned long long), s));
        FIC_TRY(cudaMemsetAsync(&ds->vd_min_key, 0xff, sizeof(unsigned long long), s));
        L.begin(FIC_K_GATHER);
        FIC_TRY(launch_gather(c->box2.as<uint16_t>(), N, B, Lstep, per, pool_xy, dn, cols_pad, K, sp,
                              c->D.as<__half>(), c->cf.as<float>(), c->ci.as<ColExact>(),
                              &ds->vd_max, &ds->vd_min_key, s));
        L.end(1, 0.0, (double)cols_pad * (2.0 * K + 4.0 * sp.cw + 8.0) + (double)dn * 4.0 * n);

        L.begin(FIC_K_RANGE_PREP);
        FIC_TRY(launch_range_prep(dimg, N, B, act, (int)R, rows_pad, K, sp, &ds->vd_max, iso ? 1 : 0,
                                  c->A.as<__half>(), c->rc.as<RowConst>(), s));
        L.end(1, 0.0, (double)rows_pad * K * 2.0 + (double)R * (n + 20.0));

        int n_chunks = 0, n_parts = 0;
        if (dn > 0) {
            int per_chunk = 0;
            const int64_t tile_w = iso ? contract_tc_iso_ntile(K)
                                       : (p->engine == FIC_ENGINE_TENSOR ? contract_tc_ntile() : 128);
            const int64_t n_mtiles = iso ? rows_pad / 8 / 128 : rows_pad / kMTile;
            choose_chunks(c->sm_count, n_mtiles, cols_pad / tile_w, &n_chunks, &per_chunk);
            // the tensor kernels write one partial per chunk and column slice
            n_parts = iso ? contract_tc_iso_parts_per_chunk() * n_chunks
                          : (p->engine == FIC_ENGINE_TENSOR ? contract_tc_parts_per_chunk() * n_chunks
                                                            : n_chunks);
            FIC_TRY(c->part.ensure(sizeof(Best) * R * n_parts));
            FIC_TRY(c->gbest.ensure(sizeof(long long) * rows_pad));
            FIC_TRY(cudaMemsetAsync(c->gbest.p, 0x7f, sizeof(long long) * rows_pad, s));
            ContractArgs a;
            a.A = c->A.as<__half>();
            a.rows_pad = rows_pad;
            a.D = c->D.as<__half>();
            a.cols_pad = cols_pad;
            a.K = K;
            a.cf = c->cf.as<float>();
            a.ci = c->ci.as<ColExact>();
            a.rc = c->rc.as<RowConst>();
            a.R = (int)R;
            a.dn = (int)dn;
            a.n_chunks = n_chunks;
            a.ctiles_per_chunk = per_chunk;
            a.part = c->part.as<Best>();
            a.gbest = c->gbest.as<long long>();
            a.sp = sp;
            a.err = &ds->err;
            a.grid_ctas = c->sm_count;
            const double flops = 2.0 * (8.0 * R) * (double)dn * n;
            const int64_t matches = 8 * R * dn;
            const double bytes = (double)rows_pad * K * 2.0 + (double)cols_pad * (2.0 * K + 4.0 * sp.cw);
            if (p->engine == FIC_ENGINE_TENSOR) {
                FIC_TRY(cudaMemsetAsync(&ds->err, 0, sizeof(int), s));
                L.begin(FIC_K_CONTRACT_TC);
                FIC_TRY(iso ? launch_contract_tc_iso(a, s) : launch_contract_tc(a, s));
                L.end(1, flops, bytes, matches);
            } else {
                L.begin(FIC_K_CONTRACT_PLAIN);
                FIC_TRY(launch_contract_plain(a, s));
                L.end(1, flops, bytes, matches);
            }
        }
        out->matches[lvl] = 8 * R * dn;

        L.begin(FIC_K_SPLIT);
        FIC_TRY(launch_split_decide(c->part.as<Best>(), n_parts, c->rc.as<RowConst>(), (int)R, n,
                                    sp, e16, last, (int)dn, &ds->vd_min_key, c->best.as<Best>(),
                                    c->split.as<uint32_t>(), s));
        int nl = 0;
        FIC_TRY(launch_scan(c->split.as<uint32_t>(), c->split_pos.as<uint32_t>(), R,
                            c->scan_tmp.as<uint32_t>(), &ds->total, s, &nl));
        FIC_TRY(launch_split_scatter(act, c->best.as<Best>(), c->split.as<uint32_t>(),
                                     c->split_pos.as<uint32_t>(), c->rc.as<RowConst>(), (int)R, B,
                                     lvl, pool_xy, per, Lstep, (int)dn, next,
                                     c->codes_tmp.p, n_codes, s));
        L.end(2 + nl, 0.0, (double)R * 64.0);
        FIC_TRY(cudaMemcpyAsync(c->host_scal, ds, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        FIC_TRY(cudaStreamSynchronize(s));
        if (p->engine == FIC_ENGINE_TENSOR && c->host_scal->err) return FIC_ETIMEOUT;
        const int64_t splits = c->host_scal->total;
        n_codes += R - splits;
        R = 4 * splits;
        uint32_t* t = act;
        act = next;
        next = t;
    }

    // record order
    FIC_TRY(c->cellmap.ensure(sizeof(uint32_t) * cells));
    FIC_TRY(c->cellflag.ensure(sizeof(uint32_t) * cells));
    FIC_TRY(c->cellrank.ensure(sizeof(uint32_t) * cells));
    FIC_TRY(c->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(cells)));
    L.begin(FIC_K_ORDER);
    FIC_TRY(cudaMemsetAsync(c->cellflag.p, 0, sizeof(uint32_t) * cells, s));
    FIC_TRY(launch_order_mark(c->codes_tmp.p, n_codes, N, p->B_max, p->B_min,
                              c->cellmap.as<uint32_t>(), c->cellflag.as<uint32_t>(), s));
    int nl = 0;
    FIC_TRY(launch_scan(c->cellflag.as<uint32_t>(), c->cellrank.as<uint32_t>(), cells,
                        c->scan_tmp.as<uint32_t>(), &ds->total, s, &nl));
    FIC_TRY(launch_order_gather(c->codes_tmp.p, c->cellmap.as<uint32_t>(),
                                c->cellflag.as<uint32_t>(), c->cellrank.as<uint32_t>(), cells,
                                c->codes_out.p, s));
    L.end(2 + nl, 0.0, (double)cells * 16.0 + (double)n_codes * 32.0);

    out->n_codes = n_codes;
    if (codes_out) {
        out->codes = codes_out;
        out->owns_codes = 0;
        if (n_codes > codes_cap) {
            cudaStreamSynchronize(s);
            return FIC_ECAP;
        }
        FIC_TRY(cudaMemcpyAsync(codes_out, c->codes_out.p, sizeof(fic_code) * n_codes,
                                cudaMemcpyDefault, s));
    } else {
        fic_code* h = (fic_code*)malloc(sizeof(fic_code) * (size_t)(n_codes ? n_codes : 1));
        if (!h) return FIC_ENOMEM;
        out->codes = h;
        out->owns_codes = 1;
        cudaError_t e = cudaMemcpyAsync(h, c->codes_out.p, sizeof(fic_code) * n_codes,
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            free(h);
            out->codes = nullptr;
            out->owns_codes = 0;
            return to_status(e);
        }
    }
    FIC_TRY(cudaStreamSynchronize(s));
    return FIC_OK;
}

}  // namespace
}  // namespace fic

using namespace fic;

extern "C" {

const char* fic_strerror(int status)
{
    switch (status) {
        case FIC_OK: return "ok";
        case FIC_EINVAL: return "invalid argument";
        case FIC_ENOMEM: return "out of memory";
        case FIC_ECUDA: return "CUDA error";
        case FIC_ETIMEOUT: return "device wait timed out";
        case FIC_EBUSY: return "busy: admission refused";
        case FIC_ENODEV: return "no sm_103 CUDA device";
        case FIC_ECAP: return "output buffer too small";
        case FIC_ENOTREADY: return "not finished";
        default: return "unknown status";
    }
}

const char* fic_version(void) { return "fic-gb300 0.1 (sm_103a)"; }

const char* fic_last_error(void) { return g_last_error; }

int fic_encode_ex(const uint8_t* img, const fic_params* p, fic_code* codes_out, int64_t codes_cap,
                  fic_result* out, void* stream)
{
    try {
        return encode_impl(img, p, codes_out, codes_cap, out, (cudaStream_t)stream);
    } catch (...) {
        return FIC_ENOMEM;
    }
}

int fic_encode(const uint8_t* img, int N, int B_max, int B_min, int L, double entropy_thresh,
               const fic_sset* S_sets, double err_tol, fic_result* out, void* stream)
{
    if (!S_sets) return FIC_EINVAL;
    fic_params p;
    memset(&p, 0, sizeof(p));
    p.N = N;
    p.B_max = B_max;
    p.B_min = B_min;
    p.L = L;
    p.entropy_thresh = entropy_thresh;
    p.err_tol = err_tol;
    p.engine = FIC_ENGINE_TENSOR;
    int nl = 0;
    for (int b = B_max; b >= B_min && b >= 1 && nl < FIC_MAX_LEVELS; b /= 2) {
        p.S_sets[nl] = S_sets[nl];
        ++nl;
    }
    return fic_encode_ex(img, &p, nullptr, 0, out, stream);
}

void fic_result_free(fic_result* r)
{
    if (!r) return;
    if (r->owns_codes && r->codes) free(r->codes);
    r->codes = nullptr;
    r->owns_codes = 0;
    r->n_codes = 0;
}

int fic_decode(const fic_result* r, int N, int iters_max, uint8_t* out_img, int* iters_used,
               void* stream)
{
    if (!r || !out_img || N <= 0 || iters_max < 1 || (r->n_codes > 0 && !r->codes))
        return FIC_EINVAL;
    Context* c = nullptr;
    int st = get_context(&c);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_ready(c, s);
    if (st) return st;
    if (!valid_side(r->B_max)) return FIC_EINVAL;
    DecodeS ds;
    memset(&ds, 0, sizeof(ds));
    ds.B_max = r->B_max;
    for (int l = 0; l < FIC_MAX_LEVELS; ++l) {
        ds.q[l] = r->S_sets[l].q > 0 ? r->S_sets[l].q : 1;
        for (int i = 0; i < FIC_MAX_S; ++i) ds.p[l][i] = r->S_sets[l].p[i];
    }
    const void* dcodes = r->codes;
    if (r->n_codes > 0 && !is_device_ptr(r->codes)) {
        FIC_TRY(c->codes_tmp.ensure(sizeof(fic_code) * r->n_codes));
        FIC_TRY(cudaMemcpyAsync(c->codes_tmp.p, r->codes, sizeof(fic_code) * r->n_codes,
                                cudaMemcpyHostToDevice, s));
        dcodes = c->codes_tmp.p;
    }
    const size_t npx = (size_t)N * N;
    FIC_TRY(c->dec0.ensure(npx));
    FIC_TRY(c->dec1.ensure(npx));
    uint8_t* cur = c->dec0.as<uint8_t>();
    uint8_t* nxt = c->dec1.as<uint8_t>();
    FIC_TRY(cudaMemsetAsync(cur, 128, npx, s));
    Scalars* dsc = c->scal.as<Scalars>();
    Launcher L(s);
    int used = 0;
    while (used < iters_max) {
        FIC_TRY(cudaMemsetAsync(&dsc->changed, 0, sizeof(unsigned), s));
        FIC_TRY(cudaMemcpyAsync(nxt, cur, npx, cudaMemcpyDeviceToDevice, s));
        L.begin(FIC_K_DECODE);
        FIC_TRY(launch_decode_pass(dcodes, r->n_codes, ds, cur, nxt, N, &dsc->changed, s));
        L.end(1, 0.0, (double)npx * 2.0);
        FIC_TRY(cudaMemcpyAsync(c->host_scal, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        FIC_TRY(cudaStreamSynchronize(s));
        ++used;
        uint8_t* t = cur;
        cur = nxt;
        nxt = t;
        if (!c->host_scal->changed) break;
    }
    FIC_TRY(cudaMemcpyAsync(out_img, cur, npx, cudaMemcpyDefault, s));
    FIC_TRY(cudaStreamSynchronize(s));
    if (iters_used) *iters_used = used;
    return FIC_OK;
}

int fic_domain_pool(const uint8_t* img, int N, int B, int L, double entropy_thresh,
                    int32_t* pool_xy, int64_t cap, int64_t* dn, double* entropy, int64_t* near,
                    void* stream)
{
    if (!img || !dn || N <= 0 || !valid_side(B) || L < 1) return FIC_EINVAL;
    Context* c = nullptr;
    int st = get_context(&c);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_ready(c, s);
    if (st) return st;
    const uint8_t* dimg = img;
    if (!is_device_ptr(img)) {
        FIC_TRY(c->img.ensure((size_t)N * N));
        FIC_TRY(cudaMemcpyAsync(c->img.p, img, (size_t)N * N, cudaMemcpyHostToDevice, s));
        dimg = c->img.as<uint8_t>();
    }
    const int per = (N >= 2 * B) ? (N - 2 * B) / L + 1 : 0;
    const int64_t npos = (int64_t)per * per;
    // entropy is always evaluated here, so a negative threshold still gives H
    const double thr = entropy_thresh;
    int64_t d = 0, nr = 0;
    bool use_list = false;
    Launcher Lk(s);
    // entropy is evaluated for every position; a negative threshold admits all
    st = build_pool(c, Lk, dimg, N, B, L, thr < 0.0 ? -1.0e300 : thr, true, s, &d, &nr,
                    &use_list, entropy != nullptr);
    if (thr < 0.0) nr = 0;
    if (st) return st;
    *dn = d;
    if (near) *near = nr;
    if (entropy && npos > 0)
        FIC_TRY(cudaMemcpyAsync(entropy, c->H.p, sizeof(double) * npos, cudaMemcpyDeviceToHost, s));
    if (pool_xy && cap >= d && d > 0) {
        std::vector<uint32_t> tmp((size_t)d);
        FIC_TRY(cudaMemcpyAsync(tmp.data(), c->pool.p, sizeof(uint32_t) * d,
                                cudaMemcpyDeviceToHost, s));
        FIC_TRY(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < d; ++i) {
            pool_xy[2 * i] = (int32_t)(tmp[(size_t)i] & 0xffffu);
            pool_xy[2 * i + 1] = (int32_t)(tmp[(size_t)i] >> 16);
        }
    }
    FIC_TRY(cudaStreamSynchronize(s));
    if (pool_xy && cap < d) return FIC_ECAP;
    return FIC_OK;
}

int fic_stats_reset(int timing)
{
    std::lock_guard<std::mutex> g(g_stats.mu);
    memset(&g_stats.st, 0, sizeof(g_stats.st));
    g_stats.timing = timing != 0;
    return FIC_OK;
}

int fic_stats_read(fic_stats* out)
{
    if (!out) return FIC_EINVAL;
    std::lock_guard<std::mutex> g(g_stats.mu);
    *out = g_stats.st;
    return FIC_OK;
}

}  // extern "C"
