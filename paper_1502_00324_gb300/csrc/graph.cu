// graph.cu -- graph-captured encodes: the whole quadtree (every step of every
// image of a call) as one CUDA graph, replayed for later calls with the same
// configuration.
//
// The eager driver (engine.cu) reads the pool sizes and split counts back to
// the host between steps to size the next launches.  Here those counts stay
// in device memory (Scalars of the plan): every kernel is launched with the
// grid of the largest possible count (all (N / B)^2 ranges of a step, every
// domain position) and reads the actual count, the step plan kernel builds
// the contraction's problem table and item count on the device (chunking.cuh,
// the arithmetic of the eager driver), and the persistent contraction reads
// its item count from there.  The host meets the device once per call, after
// the graph, to read the record counts.  Records are identical to the eager
// path's: the same kernels, the same shapes, the same items.
//
// A configuration (image sides, parameters, tuning mode, timing) is first
// encoded eagerly, which tunes the contraction shapes; the shapes the eager
// run used are then captured.  Buffers of a plan are sized for the maxima
// and owned by the plan (nothing is allocated while capturing).
#include <algorithm>
#include <array>
#include <atomic>
#include <cstring>
#include <string>

#include "chunking.cuh"
#include "engine.h"
#include "kernels.h"
#include "shape.h"

namespace fic {

// Static data of one image for one captured step, read by the plan kernels.
struct PlanJob {
    Problem base;        // pointers and layout strides (the captured maxima)
    int slot;            // index into the plan's Scalars
    uint32_t R0;         // top-level ranges
    uint32_t dn_static;  // pool size of full and top-DN pools
    int dn_from_total;   // threshold pool: its size is the pool scan's total
    int use_list;        // a pool list is built (threshold or top-DN rule)
    int pad;
};

struct PlanStep {
    int n_jobs, iso, tile_w, parts_per_chunk, refill, K, sm_count, last;
};

namespace {

__global__ void graph_init_kernel(const PlanJob* __restrict__ jobs, int n, Scalars* __restrict__ ds)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    Scalars& d = ds[jobs[j].slot];
    d.total = 0;
    d.near = 0;
    d.err = 0;
    d.err2 = 0;
    d.R = jobs[j].R0;
    d.dn = 0;
    d.n_codes = 0;
    d.n_parts = 0;
    for (int l = 0; l < FIC_MAX_LEVELS; ++l) {
        d.lvl_R[l] = 0;
        d.lvl_dn[l] = 0;
        d.lvl_near[l] = 0;
    }
}

// After the step's pool: its size, and the step's counters for the result.
__global__ void graph_level_begin_kernel(const PlanJob* __restrict__ jobs, int n,
                                         Scalars* __restrict__ ds, int lvl)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const PlanJob& J = jobs[j];
    Scalars& d = ds[J.slot];
    const uint32_t dn = J.dn_from_total ? d.total : J.dn_static;
    const bool live = d.R > 0;
    d.dn = live ? dn : 0u;
    d.lvl_R[lvl] = d.R;
    d.lvl_dn[lvl] = live ? dn : 0u;
    d.lvl_near[lvl] = live && J.use_list ? d.near : 0ull;
}

// After the split scan: records emitted by this step and the next step's
// active ranges (4 children per split; none after the last step).
__global__ void graph_level_end_kernel(const PlanJob* __restrict__ jobs, int n,
                                       Scalars* __restrict__ ds, int last)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    Scalars& d = ds[jobs[j].slot];
    const uint32_t splits = d.R > 0 ? d.total : 0u;
    d.n_codes += d.R - splits;
    d.R = last ? 0u : 4u * splits;
}

__device__ __forceinline__ void plan_sizes(const PlanStep& ps, uint32_t R, uint32_t dn,
                                           int64_t* n_mtiles, int64_t* n_ct)
{
    const int64_t rows = ps.iso ? 8 * round_up64(R, 128) : round_up64(8 * (int64_t)R, kMTile);
    *n_mtiles = ps.iso ? rows / 8 / 128 : rows / kMTile;
    *n_ct = round_up64(dn > 0 ? dn : 1, kColPad) / ps.tile_w;
}

// The step's problem table and item count from the device counts: the
// eager driver's chunking (alone in the launch: the makespan search,
// evaluated by the whole block; shared: tiles per item).
__global__ void __launch_bounds__(256)
graph_plan_kernel(const PlanJob* __restrict__ jobs, Scalars* __restrict__ ds,
                  Problem* __restrict__ probs, int* __restrict__ n_items, PlanStep ps)
{
    __shared__ int s_single, s_group;
    __shared__ double s_tiles;
    __shared__ long long s_mt, s_ct;
    __shared__ long long s_cost[256];
    __shared__ int s_nc[256];
    if (threadIdx.x == 0) {
        int group = 0, single = -1;
        double tiles = 0.0;
        for (int j = 0; j < ps.n_jobs; ++j) {
            const Scalars& d = ds[jobs[j].slot];
            if (d.R == 0 || d.dn == 0) continue;
            int64_t mt, ct;
            plan_sizes(ps, d.R, d.dn, &mt, &ct);
            tiles += (double)mt * (double)ct;
            ++group;
            single = j;
            s_mt = mt;
            s_ct = ct;
        }
        s_group = group;
        s_single = group == 1 ? single : -1;
        s_tiles = tiles;
    }
    __syncthreads();
    int nc_alone = 1;
    if (s_single >= 0) {
        // smallest chunk count of least estimated makespan (choose_chunks_alone)
        const int64_t mt = s_mt, ct = s_ct, slots = ps.sm_count;
        const int64_t max_nc = max_chunks(ps.sm_count, mt, ct);
        long long best = -1;
        int best_nc = 0;
        for (int64_t nc = 1 + threadIdx.x; nc <= max_nc; nc += blockDim.x) {
            const int64_t per = (ct + nc - 1) / nc;
            if ((ct + per - 1) / per != nc) continue;
            const int64_t waves = (mt * nc + slots - 1) / slots;
            const long long cost = (long long)(waves * (per + ps.refill));
            if (best < 0 || cost < best) {
                best = cost;
                best_nc = (int)nc;
            }
        }
        s_cost[threadIdx.x] = best;
        s_nc[threadIdx.x] = best_nc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long b = -1;
            int bnc = 1;
            for (int t = 0; t < (int)blockDim.x; ++t) {
                if (s_cost[t] < 0) continue;
                if (b < 0 || s_cost[t] < b || (s_cost[t] == b && s_nc[t] < bnc)) {
                    b = s_cost[t];
                    bnc = s_nc[t];
                }
            }
            s_nc[0] = bnc;
        }
        __syncthreads();
        nc_alone = s_nc[0];
    }
    if (threadIdx.x != 0) return;
    const double tiles_per_item = s_tiles / ((16.0 / ps.refill) * ps.sm_count);
    int64_t items = 0;
    for (int j = 0; j < ps.n_jobs; ++j) {
        const PlanJob& J = jobs[j];
        Scalars& d = ds[J.slot];
        Problem pr = J.base;
        pr.R = (int)d.R;
        pr.dn = (int)d.dn;
        pr.item_start = (int)items;
        pr.diag = 0;
        if (d.R == 0 || d.dn == 0) {
            pr.n_mtiles = 1;
            pr.n_ct = 1;
            pr.n_chunks = 0;
            pr.per_chunk = 1;
            d.n_parts = 0;
        } else {
            int64_t mt, ct;
            plan_sizes(ps, d.R, d.dn, &mt, &ct);
            int nc = 1, per = 1;
            if (s_group == 1) {
                nc = nc_alone;
                per = (int)((ct + nc - 1) / nc);
            } else {
                choose_chunks_shared(ps.sm_count, mt, ct, tiles_per_item, &nc, &per);
            }
            pr.n_mtiles = (int)mt;
            pr.n_ct = (int)ct;
            // diagonal chunk order while the pool operand stays in L2
            pr.diag = (double)(ct * ps.tile_w) * ps.K * 2.0 <= kDiagMaxPoolBytes ? 1 : 0;
            pr.n_chunks = nc;
            pr.per_chunk = per;
            d.n_parts = (uint32_t)(ps.parts_per_chunk * nc);
            items += mt * nc;
        }
        probs[j] = pr;
    }
    *n_items = (int)items;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static std::atomic<int> g_graph_mode{1};
int graph_mode() { return g_graph_mode.load(); }
void set_graph_mode(int mode) { g_graph_mode.store(mode); }

struct Engine::GraphPlan {
    std::string key;
    int n = 0, nl = 0;
    fic_params p{};
    std::vector<int> Ns;
    TuneChoice choice[FIC_MAX_LEVELS];
    std::vector<std::unique_ptr<ImageWork>> work;
    DevBuf scal, items, jobs[FIC_MAX_LEVELS], probs[FIC_MAX_LEVELS];
    Scalars* host_scal = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphRec rec;
    std::vector<std::array<int64_t, FIC_MAX_LEVELS>> positions;  // per image and step
    uint64_t last_use = 0;

    ~GraphPlan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (host_scal) cudaFreeHost(host_scal);
        for (auto& w : work) w->release();
        scal.release();
        items.release();
        for (auto& b : jobs) b.release();
        for (auto& b : probs) b.release();
    }
};

namespace {

// The captured configuration: image sides, every parameter, the tuning mode
// and whether stages are timed.
std::string graph_key(int n, const int* Ns, const fic_params& p, bool timed)
{
    std::string k;
    auto put = [&k](const void* v, size_t b) { k.append(static_cast<const char*>(v), b); };
    put(&n, sizeof n);
    put(Ns, sizeof(int) * (size_t)n);
    put(&p.B_max, sizeof p.B_max);
    put(&p.B_min, sizeof p.B_min);
    put(&p.L, sizeof p.L);
    put(&p.entropy_thresh, sizeof p.entropy_thresh);
    put(&p.err_tol, sizeof p.err_tol);
    put(&p.engine, sizeof p.engine);
    put(&p.pool_dn, sizeof p.pool_dn);
    for (int l = 0; l < FIC_MAX_LEVELS; ++l) {
        const fic_sset& s = p.S_sets[l];
        put(&s.n_s, sizeof s.n_s);
        put(&s.q, sizeof s.q);
        put(s.p, sizeof(int) * (size_t)std::max(0, std::min(s.n_s, FIC_MAX_S)));
    }
    const int mode = tune_mode();
    put(&mode, sizeof mode);
    const char t = timed ? 1 : 0;
    put(&t, 1);
    return k;
}

bool stats_timed()
{
    std::lock_guard<std::mutex> g(g_stats.mu);
    return g_stats.timing;
}

}  // namespace

void Engine::note_config(int n, const int* Ns, const fic_params& p)
{
    Seen& sn = seen_[graph_key(n, Ns, p, stats_timed())];
    for (int l = 0; l < FIC_MAX_LEVELS; ++l)
        sn.choice[l] = used_valid_[l] ? used_choice_[l] : default_choice();
}

void Engine::drop_plans()
{
    for (GraphPlan* g : plans_) delete g;
    plans_.clear();
}

void Engine::reset_used()
{
    for (int l = 0; l < FIC_MAX_LEVELS; ++l) used_valid_[l] = false;
}

int Engine::graph_build(GraphPlan& G, cudaStream_t /*s*/)
{
    const fic_params& p = G.p;
    const int n = G.n, nl = G.nl;
    const bool filter = p.entropy_thresh >= 0.0;
    const int64_t top = p.pool_dn;
    const bool use_list = filter || top > 0;
    const int e16 = (int)llround(16.0 * p.err_tol);
    const int sms = sm_count_;

    // ---- buffers at the maxima of every step
    G.work.clear();
    G.positions.assign((size_t)n, {});
    for (int i = 0; i < n; ++i) {
        G.work.emplace_back(new ImageWork());
        ImageWork& w = *G.work.back();
        const int N = G.Ns[(size_t)i];
        const int64_t cells = (int64_t)(N / p.B_min) * (N / p.B_min);
        FIC_TRY(w.img.ensure((size_t)N * N));
        FIC_TRY(w.box2.ensure(sizeof(uint16_t) * (size_t)N * N));
        FIC_TRY(w.act0.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(w.act1.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(w.codes_tmp.ensure(sizeof(fic_code) * cells));
        FIC_TRY(w.codes_out.ensure(sizeof(fic_code) * cells));
        FIC_TRY(w.cellmap.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(w.cellflag.ensure(sizeof(uint32_t) * cells));
        FIC_TRY(w.cellrank.ensure(sizeof(uint32_t) * cells));
        int64_t scan_n = cells;
        for (int lvl = 0; lvl < nl; ++lvl) {
            const StepShape h = step_shape(p, lvl, G.choice[lvl]);
            const int per = positions_per_axis(N, h.B, p.L);
            const int64_t npos = (int64_t)per * per;
            G.positions[(size_t)i][(size_t)lvl] = npos;
            const int64_t R_max = (int64_t)(N / h.B) * (N / h.B);
            const int64_t rows = 8 * round_up(R_max, 128);
            const int64_t cols = round_up(npos > 0 ? npos : 1, kColPad);
            if (use_list && npos > 0) {
                FIC_TRY(w.flags.ensure(sizeof(uint32_t) * npos));
                FIC_TRY(w.pos.ensure(sizeof(uint32_t) * npos));
                FIC_TRY(w.pool.ensure(sizeof(uint32_t) * npos));
                if (top > 0) FIC_TRY(w.keys.ensure(sizeof(unsigned long long) * npos));
                if (top > 0 && top < npos) FIC_TRY(w.sel.ensure(select_state_bytes()));
            }
            FIC_TRY(w.D.ensure(sizeof(__half) * cols * h.K));
            FIC_TRY(w.cf.ensure(sizeof(float) * cols * h.sp.cw));
            FIC_TRY(w.ci.ensure(sizeof(ColExact) * cols));
            FIC_TRY(w.A.ensure(sizeof(__half) * rows * h.K));
            FIC_TRY(w.rc.ensure(sizeof(RowConst) * (rows / 8)));
            FIC_TRY(w.gbest.ensure(sizeof(long long) * rows));
            FIC_TRY(w.best.ensure(sizeof(Best) * R_max));
            FIC_TRY(w.split.ensure(sizeof(uint32_t) * R_max));
            FIC_TRY(w.split_pos.ensure(sizeof(uint32_t) * R_max));
            // partial bests: R x chunks <= 128 M tiles x (16 SMs / M tiles + 1)
            const int64_t n_ct = cols / h.tile_w;
            const int64_t pairs = std::min<int64_t>(R_max * n_ct, 2048LL * sms + R_max + 128);
            FIC_TRY(w.part.ensure(sizeof(Best) * pairs * h.parts_per_chunk));
            scan_n = std::max(scan_n, std::max(npos, R_max));
        }
        FIC_TRY(w.scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(scan_n)));
    }
    FIC_TRY(G.scal.ensure(sizeof(Scalars) * (size_t)n));
    FIC_TRY(G.items.ensure(sizeof(int) * FIC_MAX_LEVELS));
    FIC_TRY(cudaMallocHost((void**)&G.host_scal, sizeof(Scalars) * (size_t)n));
    Scalars* ds = G.scal.as<Scalars>();
    int* items = G.items.as<int>();

    // ---- the static per-step job data
    std::vector<PlanJob> pj((size_t)n);
    for (int lvl = 0; lvl < nl; ++lvl) {
        const StepShape h = step_shape(p, lvl, G.choice[lvl]);
        for (int i = 0; i < n; ++i) {
            ImageWork& w = *G.work[(size_t)i];
            const int N = G.Ns[(size_t)i];
            const int64_t npos = G.positions[(size_t)i][(size_t)lvl];
            const int64_t R_max = (int64_t)(N / h.B) * (N / h.B);
            PlanJob& J = pj[(size_t)i];
            memset(&J, 0, sizeof(J));
            J.base.A = w.A.as<__half>();
            J.base.D = w.D.as<__half>();
            J.base.cf = w.cf.as<float>();
            J.base.ci = w.ci.as<ColExact>();
            J.base.rc = w.rc.as<RowConst>();
            J.base.part = w.part.as<Best>();
            J.base.gbest = w.gbest.as<long long>();
            J.base.rows_pad = 8 * round_up(R_max, 128);
            J.base.cols_pad = round_up(npos > 0 ? npos : 1, kColPad);
            J.slot = i;
            J.R0 = (uint32_t)((N / p.B_max) * (N / p.B_max));
            J.dn_static = (uint32_t)(top > 0 ? std::min<int64_t>(top, npos) : npos);
            J.dn_from_total = use_list && top == 0 ? 1 : 0;
            J.use_list = use_list ? 1 : 0;
        }
        FIC_TRY(G.jobs[lvl].ensure(sizeof(PlanJob) * (size_t)n));
        FIC_TRY(G.probs[lvl].ensure(sizeof(Problem) * (size_t)n));
        FIC_TRY(cudaMemcpy(G.jobs[lvl].p, pj.data(), sizeof(PlanJob) * (size_t)n,
                           cudaMemcpyHostToDevice));
    }
    // the contraction launchers set their shared-memory limits outside capture
    FIC_TRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    const cudaStream_t s = G.cap;

    // ---- capture
    G.rec.timed = stats_timed();
    G.rec.entries.clear();
    FIC_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> int {
        Launcher L(s, &G.rec);
        const unsigned jb = (unsigned)((n + 127) / 128);
        G.rec.level = -1;
        L.begin(FIC_K_MISC);
        graph_init_kernel<<<jb, 128, 0, s>>>(G.jobs[0].as<PlanJob>(), n, ds);
        FIC_TRY(cudaGetLastError());
        L.end(1);
        std::vector<uint32_t*> act((size_t)n), next((size_t)n);
        for (int i = 0; i < n; ++i) {
            ImageWork& w = *G.work[(size_t)i];
            const int N = G.Ns[(size_t)i];
            act[(size_t)i] = w.act0.as<uint32_t>();
            next[(size_t)i] = w.act1.as<uint32_t>();
            G.rec.job = i;
            L.begin(FIC_K_GATHER);
            FIC_TRY(launch_init_ranges(act[(size_t)i], N / p.B_max, p.B_max, s));
            FIC_TRY(launch_box2(w.img.as<uint8_t>(), N, w.box2.as<uint16_t>(), s));
            L.end(2, 0.0, (double)N * N * 3.0);
        }
        for (int lvl = 0; lvl < nl; ++lvl) {
            G.rec.level = lvl;
            const StepShape h = step_shape(p, lvl, G.choice[lvl]);
            const bool last = lvl == nl - 1;
            const PlanJob* jobs = G.jobs[lvl].as<PlanJob>();
            if (use_list)
                for (int i = 0; i < n; ++i) {
                    G.rec.job = i;
                    int st = pool_launches(G.work[(size_t)i].get(), ds + i, entT_.as<long long>(),
                                           G.work[(size_t)i]->img.as<uint8_t>(), G.Ns[(size_t)i],
                                           h.B, p.L, top > 0 ? -1.0 : p.entropy_thresh, top,
                                           false, L, s);
                    if (st) return st;
                }
            G.rec.job = -1;
            L.begin(FIC_K_MISC);
            graph_level_begin_kernel<<<jb, 128, 0, s>>>(jobs, n, ds, lvl);
            FIC_TRY(cudaGetLastError());
            L.end(1);
            int64_t item_bound = 0;
            for (int i = 0; i < n; ++i) {
                ImageWork& w = *G.work[(size_t)i];
                const int N = G.Ns[(size_t)i];
                const int per = positions_per_axis(N, h.B, p.L);
                const int64_t npos = G.positions[(size_t)i][(size_t)lvl];
                const int64_t dn_max = top > 0 ? std::min<int64_t>(top, npos) : npos;
                const int64_t cols = round_up(npos > 0 ? npos : 1, kColPad);
                const int64_t R_max = (int64_t)(N / h.B) * (N / h.B);
                const int64_t rows = 8 * round_up(R_max, 128);
                G.rec.job = i;
                FIC_TRY(cudaMemsetAsync(&ds[i].vd_max, 0, sizeof(unsigned long long), s));
                FIC_TRY(cudaMemsetAsync(&ds[i].vd_min_key, 0xff, sizeof(unsigned long long), s));
                L.begin(FIC_K_GATHER);
                FIC_TRY(launch_gather(w.box2.as<uint16_t>(), N, h.B, p.L, per,
                                      use_list ? w.pool.as<uint32_t>() : nullptr, dn_max, cols,
                                      h.K, h.sp, w.D.as<__half>(), w.cf.as<float>(),
                                      w.ci.as<ColExact>(), &ds[i].vd_max, &ds[i].vd_min_key, s,
                                      &ds[i].dn));
                L.end(2, 0.0, (double)cols * (2.0 * h.K + 4.0 * h.sp.cw + 8.0));
                L.begin(FIC_K_RANGE_PREP);
                FIC_TRY(launch_range_prep(w.img.as<uint8_t>(), N, h.B, act[(size_t)i],
                                          (int)R_max, rows, h.K, h.sp, &ds[i].vd_max,
                                          h.iso ? 1 : 0, w.A.as<__half>(), w.rc.as<RowConst>(), s,
                                          &ds[i].R));
                L.end(1, 0.0, (double)rows * h.K * 2.0);
                FIC_TRY(cudaMemsetAsync(w.gbest.p, 0x7f, sizeof(long long) * rows, s));
                // bound on the items: M tiles x chunks <= 16 SMs + M tiles
                item_bound += 16LL * sms + rows / (h.iso ? 1024 : kMTile);
            }
            G.rec.job = -1;
            PlanStep ps;
            ps.n_jobs = n;
            ps.iso = h.iso ? 1 : 0;
            ps.tile_w = (int)h.tile_w;
            ps.parts_per_chunk = h.parts_per_chunk;
            ps.refill = h.refill;
            ps.K = h.K;
            ps.sm_count = sms;
            ps.last = last ? 1 : 0;
            L.begin(FIC_K_MISC);
            graph_plan_kernel<<<1, 256, 0, s>>>(jobs, ds, G.probs[lvl].as<Problem>(), items + lvl,
                                                ps);
            FIC_TRY(cudaGetLastError());
            L.end(1);
            ContractArgs a;
            a.probs = G.probs[lvl].as<Problem>();
            a.n_probs = n;
            a.n_items = (int)std::min<int64_t>(item_bound, 1 << 30);
            a.n_items_dev = items + lvl;
            a.K = h.K;
            a.sp = h.sp;
            a.err = &ds[0].err;
            a.grid_ctas = sms;
            a.variant = h.epi;
            if (p.engine == FIC_ENGINE_TENSOR) {
                FIC_TRY(cudaMemsetAsync(a.err, 0, 2 * sizeof(int), s));
                L.begin(FIC_K_CONTRACT_TC);
                FIC_TRY(h.red   ? launch_contract_tc_red(a, s)
                        : h.iso ? launch_contract_tc_iso(a, s)
                                : launch_contract_tc(a, s));
                L.end(1);
            } else {
                L.begin(FIC_K_CONTRACT_PLAIN);
                FIC_TRY(launch_contract_plain(a, s));
                L.end(1);
            }
            for (int i = 0; i < n; ++i) {
                ImageWork& w = *G.work[(size_t)i];
                const int N = G.Ns[(size_t)i];
                const int per = positions_per_axis(N, h.B, p.L);
                const int64_t npos = G.positions[(size_t)i][(size_t)lvl];
                const int64_t dn_max = top > 0 ? std::min<int64_t>(top, npos) : npos;
                const int64_t R_max = (int64_t)(N / h.B) * (N / h.B);
                G.rec.job = i;
                StepCounts dc;
                dc.R = &ds[i].R;
                dc.dn = &ds[i].dn;
                dc.n_parts = &ds[i].n_parts;
                L.begin(FIC_K_SPLIT);
                FIC_TRY(launch_split_decide(w.part.as<Best>(), 0, w.rc.as<RowConst>(), (int)R_max,
                                            h.n2, h.sp, e16, last ? 1 : 0, (int)dn_max,
                                            &ds[i].vd_min_key, w.best.as<Best>(),
                                            w.split.as<uint32_t>(), s, dc));
                int nlaunch = 0;
                FIC_TRY(launch_scan(w.split.as<uint32_t>(), w.split_pos.as<uint32_t>(), R_max,
                                    w.scan_tmp.as<uint32_t>(), &ds[i].total, s, &nlaunch,
                                    &ds[i].R));
                StepCounts dc2;
                dc2.R = &ds[i].R;
                dc2.dn = &ds[i].dn;
                dc2.code_base = &ds[i].n_codes;
                FIC_TRY(launch_split_scatter(act[(size_t)i], w.best.as<Best>(),
                                             w.split.as<uint32_t>(), w.split_pos.as<uint32_t>(),
                                             w.rc.as<RowConst>(), (int)R_max, h.B, lvl,
                                             use_list ? w.pool.as<uint32_t>() : nullptr, per, p.L,
                                             (int)dn_max, next[(size_t)i], w.codes_tmp.p, 0, s,
                                             dc2));
                L.end(2 + nlaunch, 0.0, (double)R_max * 64.0);
            }
            G.rec.job = -1;
            L.begin(FIC_K_MISC);
            graph_level_end_kernel<<<jb, 128, 0, s>>>(jobs, n, ds, last ? 1 : 0);
            FIC_TRY(cudaGetLastError());
            L.end(1);
            for (int i = 0; i < n; ++i) std::swap(act[(size_t)i], next[(size_t)i]);
        }
        G.rec.level = -1;
        for (int i = 0; i < n; ++i) {
            ImageWork& w = *G.work[(size_t)i];
            const int N = G.Ns[(size_t)i];
            const int64_t cells = (int64_t)(N / p.B_min) * (N / p.B_min);
            G.rec.job = i;
            L.begin(FIC_K_ORDER);
            FIC_TRY(cudaMemsetAsync(w.cellflag.p, 0, sizeof(uint32_t) * cells, s));
            FIC_TRY(launch_order_mark(w.codes_tmp.p, cells, N, p.B_max, p.B_min,
                                      w.cellmap.as<uint32_t>(), w.cellflag.as<uint32_t>(), s,
                                      &ds[i].n_codes));
            int nlaunch = 0;
            FIC_TRY(launch_scan(w.cellflag.as<uint32_t>(), w.cellrank.as<uint32_t>(), cells,
                                w.scan_tmp.as<uint32_t>(), &ds[i].total, s, &nlaunch));
            FIC_TRY(launch_order_gather(w.codes_tmp.p, w.cellmap.as<uint32_t>(),
                                        w.cellflag.as<uint32_t>(), w.cellrank.as<uint32_t>(),
                                        cells, w.codes_out.p, s));
            L.end(2 + nlaunch, 0.0, (double)cells * 16.0);
        }
        return FIC_OK;
    };
    const int st = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    FIC_TRY(ce);
    G.graph = graph;
    FIC_TRY(cudaGraphInstantiate(&G.exec, G.graph, 0));
    return FIC_OK;
}

int Engine::encode_graph(int n, const uint8_t* const* imgs, const int* Ns, const fic_params& p,
                         fic_code* const* dsts, const int64_t* caps, fic_result* outs,
                         cudaStream_t s, bool* used)
{
    *used = false;
    if (graph_mode() != 1 || n <= 0) return FIC_OK;
    const bool timed = stats_timed();
    const std::string key = graph_key(n, Ns, p, timed);
    auto seen = seen_.find(key);
    if (seen == seen_.end() || seen->second.no_graph) return FIC_OK;  // eager first (tunes)
    GraphPlan* G = nullptr;
    for (GraphPlan* g : plans_)
        if (g->key == key) G = g;
    if (!G) {
        int nl = 0;
        int st = validate_params(&p, Ns[0], &nl);
        if (st) return st;
        // keep a few plans; the least recently used one goes first
        while (plans_.size() >= kMaxPlans) {
            auto lru = std::min_element(
                plans_.begin(), plans_.end(),
                [](const GraphPlan* a, const GraphPlan* b) { return a->last_use < b->last_use; });
            delete *lru;
            plans_.erase(lru);
        }
        std::unique_ptr<GraphPlan> np(new GraphPlan());
        np->key = key;
        np->n = n;
        np->nl = nl;
        np->p = p;
        np->Ns.assign(Ns, Ns + n);
        for (int l = 0; l < FIC_MAX_LEVELS; ++l) np->choice[l] = seen->second.choice[l];
        st = graph_build(*np, s);
        if (st) {
            // not capturable here: this configuration stays eager
            seen->second.no_graph = true;
            cudaGetLastError();
            return FIC_OK;
        }
        ++graph_captures_;
        plans_.push_back(np.release());
        G = plans_.back();
    }
    G->last_use = ++plan_clock_;
    const fic_params& P = G->p;
    // inputs into the plan's image buffers, the graph, then the counts
    for (int i = 0; i < n; ++i)
        FIC_TRY(cudaMemcpyAsync(G->work[(size_t)i]->img.p, imgs[i], (size_t)Ns[i] * Ns[i],
                                cudaMemcpyDefault, s));
    FIC_TRY(cudaGraphLaunch(G->exec, s));
    FIC_TRY(cudaMemcpyAsync(G->host_scal, G->scal.p, sizeof(Scalars) * (size_t)n,
                            cudaMemcpyDeviceToHost, s));
    FIC_TRY(cudaStreamSynchronize(s));
    ++graph_replays_;
    const Scalars* hs = G->host_scal;
    if (P.engine == FIC_ENGINE_TENSOR && (hs[0].err || hs[0].err2)) return FIC_ETIMEOUT;

    // fic_stats: the captured stages, with the contraction's work from the counts
    {
        std::lock_guard<std::mutex> g(g_stats.mu);
        for (const GraphRec::Entry& e : G->rec.entries) {
            g_stats.st.launches[e.kind] += e.launches;
            // stages whose work depends on the counts: the eager driver's
            // algorithmic bytes from this call's counts
            double bytes = e.bytes;
            if (e.job >= 0) {
                const Scalars& c = hs[e.job];
                const int64_t cells = (int64_t)(Ns[e.job] / P.B_min) * (Ns[e.job] / P.B_min);
                if (e.kind == FIC_K_ORDER) bytes = (double)cells * 16.0 + (double)c.n_codes * 32.0;
                if (e.level >= 0) {
                    const StepShape h = step_shape(P, e.level, G->choice[e.level]);
                    const double R = c.lvl_R[e.level], dn = c.lvl_dn[e.level];
                    const double cols = (double)round_up(dn > 0 ? (int64_t)dn : 1, kColPad);
                    if (e.kind == FIC_K_GATHER)
                        bytes = R > 0 ? cols * (2.0 * h.K + 4.0 * h.sp.cw + 8.0) + dn * 2.0 * h.n2
                                      : 0.0;
                    if (e.kind == FIC_K_RANGE_PREP)
                        bytes = (double)rows_pad_for(h, (int64_t)R) * h.K * 2.0 + R * (h.n2 + 20.0);
                    if (e.kind == FIC_K_SPLIT) bytes = R * 64.0;
                    // an image already finished does no pool work (eager skips it)
                    if ((e.kind == FIC_K_ENTROPY || e.kind == FIC_K_SCAN) && R == 0) bytes = 0.0;
                }
            }
            g_stats.st.bytes[e.kind] += bytes;
            if ((e.kind == FIC_K_CONTRACT_TC || e.kind == FIC_K_CONTRACT_PLAIN) && e.level >= 0) {
                const int B = P.B_max >> e.level;
                for (int i = 0; i < n; ++i) {
                    const double R = hs[i].lvl_R[e.level], dn = hs[i].lvl_dn[e.level];
                    g_stats.st.flops[e.kind] += 2.0 * 8.0 * R * dn * B * B;
                    g_stats.st.matches += (int64_t)(8.0 * R * dn);
                }
            }
            float ms = 0.f;
            if (e.a && e.b && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess)
                g_stats.st.ms[e.kind] += ms;
        }
    }

    int cap_status = FIC_OK;
    for (int i = 0; i < n; ++i) {
        fic_result& r = outs[i];
        memset(&r, 0, sizeof(r));
        r.N = Ns[i];
        r.B_max = P.B_max;
        r.n_levels = G->nl;
        for (int l = 0; l < G->nl; ++l) r.S_sets[l] = P.S_sets[l];
        for (int l = 0; l < G->nl; ++l) {
            const int64_t R = hs[i].lvl_R[l];
            if (R == 0) continue;
            r.n_positions[l] = G->positions[(size_t)i][(size_t)l];
            r.ranges[l] = R;
            r.pool_size[l] = hs[i].lvl_dn[l];
            r.matches[l] = 8 * R * (int64_t)hs[i].lvl_dn[l];
            r.near_thresh[l] = (int64_t)hs[i].lvl_near[l];
        }
        r.n_codes = hs[i].n_codes;
        const void* src = G->work[(size_t)i]->codes_out.p;
        if (dsts && dsts[i]) {
            r.codes = dsts[i];
            r.owns_codes = 0;
            if (r.n_codes > caps[i]) {
                cap_status = FIC_ECAP;
                continue;
            }
            FIC_TRY(cudaMemcpyAsync(dsts[i], src, sizeof(fic_code) * r.n_codes, cudaMemcpyDefault,
                                    s));
        } else {
            fic_code* h = (fic_code*)malloc(sizeof(fic_code) * (size_t)(r.n_codes ? r.n_codes : 1));
            if (!h) return FIC_ENOMEM;
            r.codes = h;
            r.owns_codes = 1;
            FIC_TRY(cudaMemcpyAsync(h, src, sizeof(fic_code) * r.n_codes, cudaMemcpyDeviceToHost,
                                    s));
        }
    }
    *used = true;
    return cap_status;
}

}  // namespace fic
