// engine.cu -- the quadtree step driver (Sec. 2 quadtree, Sec. 3 pool, Sec.
// 3.2 S) over any number of images, each at its own step:
//   begin:  active ranges <- every B_max x B_max block in raster order
//   step:   per job [entropy -> scan -> pool list] (threshold >= 0 only)
//           -> per job domain gather (operand D', column constants)
//           -> per job range prep (operand A' with inverse isometries)
//           -> per quadtree step present: ONE contraction + scoring launch
//              over the work items of all jobs at that step
//           -> per job split decision -> scan -> records / children
//   finish: record ordering (raster of top ranges, then TL, TR, BL, BR).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "engine.h"
#include "chunking.cuh"
#include "shape.h"
#include "kernels.h"

namespace fic {

// ---------------------------------------------------------------------------
// Instrumentation
// ---------------------------------------------------------------------------
StatsState g_stats;

Launcher::Launcher(cudaStream_t s, bool allow_timing) : s_(s)
{
    std::lock_guard<std::mutex> g(g_stats.mu);
    timing_ = allow_timing && g_stats.timing;
}

void Launcher::begin(int kind)
{
    kind_ = kind;
    if (rec_) {
        cur_.kind = kind;
        cur_.a = cur_.b = nullptr;
        if (rec_->timed && cudaEventCreate(&cur_.a) == cudaSuccess &&
            cudaEventCreate(&cur_.b) == cudaSuccess)
            cudaEventRecordWithFlags(cur_.a, s_, cudaEventRecordExternal);
        return;
    }
    if (!timing_) return;
    cur_.kind = kind;
    cudaEventCreate(&cur_.a);
    cudaEventCreate(&cur_.b);
    cudaEventRecord(cur_.a, s_);
}

void Launcher::end(int launches, double flops, double bytes, int64_t matches)
{
    if (rec_) {
        if (cur_.b) cudaEventRecordWithFlags(cur_.b, s_, cudaEventRecordExternal);
        rec_->entries.push_back(
            GraphRec::Entry{kind_, launches, rec_->level, rec_->job, bytes, cur_.a, cur_.b});
        cur_.a = cur_.b = nullptr;
        return;
    }
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

GraphRec::~GraphRec()
{
    for (auto& e : entries) {
        if (e.a) cudaEventDestroy(e.a);
        if (e.b) cudaEventDestroy(e.b);
    }
}

void Launcher::harvest()
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

thread_local char g_last_error[160] = "";

int to_status(cudaError_t e)
{
    if (e == cudaSuccess) return FIC_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FIC_ENOMEM;
    return FIC_ECUDA;
}

// ---------------------------------------------------------------------------
// Buffers
// ---------------------------------------------------------------------------
cudaError_t DevBuf::ensure(size_t bytes)
{
    if (bytes <= cap) return cudaSuccess;
    release();
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        return e;
    }
    cap = want;
    return cudaSuccess;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

void ImageWork::release()
{
    DevBuf* all[] = {&img, &box2, &flags, &pos, &scan_tmp, &pool, &D, &cf, &ci, &A, &rc, &part,
                     &gbest, &best, &split, &split_pos, &act0, &act1, &codes_tmp, &codes_out,
                     &cellmap, &cellflag, &cellrank, &H, &keys, &sel};
    for (DevBuf* b : all) b->release();
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

namespace {

int ilog2i(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

bool valid_side(int b) { return b == 2 || b == 4 || b == 8 || b == 16; }

// The shapes the tuner tries for a step (all give identical records).
std::vector<TuneChoice> tune_candidates(const fic_params& p, int lvl)
{
    const int B = p.B_max >> lvl;
    const int K = k_pad(B * B);
    const bool iso_ok =
        p.engine == FIC_ENGINE_TENSOR && contract_tc_iso_supports(K, p.S_sets[lvl].n_s);
    const bool red_ok =
        p.engine == FIC_ENGINE_TENSOR && contract_tc_red_supports(B * B, p.S_sets[lvl].n_s);
    std::vector<TuneChoice> c;
    for (int refill : {1, 2, 4}) c.push_back(TuneChoice{iso_ok ? 1 : 0, refill, 0});
    if (iso_ok) {
        c.push_back(TuneChoice{1, 2, 1});  // 16 epilogue warps, 8-column reads
        c.push_back(TuneChoice{0, 2, 0});  // the row kernel on the same step
    }
    if (red_ok)
        for (int refill : {2, 4}) c.push_back(TuneChoice{2, refill, 0});
    return c;
}

}  // namespace

int positions_per_axis(int N, int B, int L) { return (N >= 2 * B) ? (N - 2 * B) / L + 1 : 0; }

static std::atomic<int> g_tune_mode{1};
// tuned shapes of the process (one device per process)
static std::mutex g_tune_mu;
static std::vector<Engine::TuneEntry> g_tuned;

std::vector<Engine::TuneEntry> Engine::tuned()
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_tuned;
}

int tune_mode() { return g_tune_mode.load(); }
void set_tune_mode(int mode) { g_tune_mode.store(mode); }

int validate_params(const fic_params* p, int N, int* n_levels)
{
    g_last_error[0] = '\0';
    if (!p) return FIC_EINVAL;
    if (N <= 0 || N > 65535) return FIC_EINVAL;
    if (!valid_side(p->B_max) || !valid_side(p->B_min) || p->B_min > p->B_max) return FIC_EINVAL;
    if (N % p->B_max) return FIC_EINVAL;
    if (p->L < 1) return FIC_EINVAL;
    if (!(p->err_tol >= 0.0 && p->err_tol <= 255.0)) return FIC_EINVAL;
    if (p->engine != FIC_ENGINE_TENSOR && p->engine != FIC_ENGINE_PLAIN) return FIC_EINVAL;
    if (p->pool_dn < 0) return FIC_EINVAL;
    const int nl = ilog2i(p->B_max) - ilog2i(p->B_min) + 1;
    if (nl > FIC_MAX_LEVELS) return FIC_EINVAL;
    for (int l = 0; l < nl; ++l) {
        const fic_sset& s = p->S_sets[l];
        // S = p/q in [0, 1] (Sec. 2); q <= 256 keeps every score term in int64
        if (s.n_s < 1 || s.n_s > FIC_MAX_S || s.q < 1 || s.q > 256) return FIC_EINVAL;
        for (int i = 0; i < s.n_s; ++i)
            if (s.p[i] < 0 || s.p[i] > s.q) return FIC_EINVAL;
    }
    const int st = check_size_limits(*p, N, nl);
    if (st) return st;
    *n_levels = nl;
    return FIC_OK;
}

int check_size_limits(const fic_params& p, int N, int nl)
{
    const bool listed = p.entropy_thresh >= 0.0 || p.pool_dn > 0;
    for (int lvl = 0; lvl < nl; ++lvl) {
        const int B = p.B_max >> lvl;
        const int per = positions_per_axis(N, B, p.L);
        const int64_t npos = (int64_t)per * per;
        const int64_t dn = p.pool_dn > 0 && p.pool_dn < npos ? p.pool_dn : npos;
        const int64_t ranges = (int64_t)(N / B) * (N / B);
        if (round_up64(dn > 0 ? dn : 1, kColPad) > kMaxPoolColumns) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "step %d (B=%d): pool of %lld domains exceeds the %lld-column limit of the "
                     "argmin key",
                     lvl, B, (long long)dn, (long long)kMaxPoolColumns);
            return FIC_EINVAL;
        }
        if ((listed && npos > kMaxScanCount) || ranges > kMaxScanCount) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "step %d (B=%d): %lld domain positions or %lld ranges exceed the scan "
                     "limit of %lld",
                     lvl, B, (long long)npos, (long long)ranges, (long long)kMaxScanCount);
            return FIC_EINVAL;
        }
    }
    const int64_t cells = (int64_t)(N / p.B_min) * (N / p.B_min);
    if (cells > kMaxScanCount) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "%lld finest cells exceed the scan limit of %lld", (long long)cells,
                 (long long)kMaxScanCount);
        return FIC_EINVAL;
    }
    return FIC_OK;
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
Engine::~Engine()
{
    drop_plans();
    for (auto& w : work_) w->release();
    entT_.release();
    scal_.release();
    for (auto& b : probs_) b.release();
    if (host_scal_) cudaFreeHost(host_scal_);
}

int Engine::init(cudaStream_t s)
{
    if (ready_) return FIC_OK;
    int dev = 0;
    FIC_TRY(cudaGetDevice(&dev));
    FIC_TRY(cudaDeviceGetAttribute(&sm_count_, cudaDevAttrMultiProcessorCount, dev));
    FIC_TRY(entT_.ensure(sizeof(long long) * kEntTableCount));
    FIC_TRY(launch_entropy_table(entT_.as<long long>(), kEntTableCount, s));
    FIC_TRY(cudaStreamSynchronize(s));
    ready_ = true;
    return FIC_OK;
}

int Engine::ensure_slots(int n)
{
    if (n > scal_cap_) {
        int cap = scal_cap_ ? scal_cap_ : 8;
        while (cap < n) cap *= 2;
        FIC_TRY(scal_.ensure(sizeof(Scalars) * (size_t)cap));
        FIC_TRY(cudaMemset(scal_.p, 0, sizeof(Scalars) * (size_t)cap));
        if (host_scal_) cudaFreeHost(host_scal_);
        host_scal_ = nullptr;
        scal_cap_ = 0;
        FIC_TRY(cudaMallocHost((void**)&host_scal_, sizeof(Scalars) * (size_t)cap));
        scal_cap_ = cap;
    }
    while ((int)work_.size() < n) work_.emplace_back(new ImageWork());
    return FIC_OK;
}

int Engine::read_scalars(int n, cudaStream_t s)
{
    FIC_TRY(cudaMemcpyAsync(host_scal_, scal_.p, sizeof(Scalars) * (size_t)n,
                            cudaMemcpyDeviceToHost, s));
    FIC_TRY(cudaStreamSynchronize(s));
    return FIC_OK;
}

int64_t Engine::slot_bytes(int N, const fic_params& p) const
{
    int nl = 0;
    if (validate_params(&p, N, &nl)) return -1;
    const int64_t cells = (int64_t)(N / p.B_min) * (N / p.B_min);
    int64_t fixed = (int64_t)N * N * 3                    // image copy + 2x2 sums
                    + cells * (2 * 16 + 2 * 4 + 3 * 4);   // records x2, act x2, order maps
    int64_t peak = 0;
    for (int lvl = 0; lvl < nl; ++lvl) {
        const StepShape h = step_shape(p, lvl, default_choice());
        const int per = positions_per_axis(N, h.B, p.L);
        const int64_t npos = (int64_t)per * per;
        const int64_t R = (int64_t)(N / h.B) * (N / h.B);
        const int64_t cols = round_up(npos > 0 ? npos : 1, kColPad);
        const int64_t rows = rows_pad_for(h, R);
        const int64_t n_mtiles = mtiles_for(h, rows);
        const int64_t nc = max_chunks(sm_count_ > 0 ? sm_count_ : 152, n_mtiles, cols / h.tile_w);
        const int64_t b = npos * (4 * 3 + 8 + 8)                        // flags, pos, pool, H, keys
                          + cols * (2 * h.K + 4 * h.sp.cw + 8)          // D, cf, ci
                          + rows * (2 * h.K + 8) + R * (16 + 16 + 8)   // A, gbest, rc, best, split
                          + R * h.parts_per_chunk * nc * 16;            // partial bests
        if (b > peak) peak = b;
    }
    return fixed + peak + (1 << 20);
}

int Engine::begin(Job& job, int slot, const uint8_t* img, int N, const fic_params& p,
                  Launcher& L, cudaStream_t s)
{
    int nl = 0;
    int st = validate_params(&p, N, &nl);
    if (st) return st;
    st = ensure_slots(slot + 1);
    if (st) return st;
    ImageWork* w = work_[(size_t)slot].get();
    job = Job();
    job.slot = slot;
    job.N = N;
    job.res.N = N;
    job.res.B_max = p.B_max;
    job.res.n_levels = nl;
    for (int l = 0; l < nl; ++l) job.res.S_sets[l] = p.S_sets[l];
    job.dimg = img;
    if (!is_device_ptr(img)) {
        FIC_TRY(w->img.ensure((size_t)N * N));
        FIC_TRY(cudaMemcpyAsync(w->img.p, img, (size_t)N * N, cudaMemcpyHostToDevice, s));
        job.dimg = w->img.as<uint8_t>();
    }
    // every record covers >= 1 finest cell
    job.cells = (int64_t)(N / p.B_min) * (N / p.B_min);
    FIC_TRY(w->codes_tmp.ensure(sizeof(fic_code) * job.cells));
    FIC_TRY(w->codes_out.ensure(sizeof(fic_code) * job.cells));
    FIC_TRY(w->act0.ensure(sizeof(uint32_t) * job.cells));
    FIC_TRY(w->act1.ensure(sizeof(uint32_t) * job.cells));
    job.act = w->act0.as<uint32_t>();
    job.next = w->act1.as<uint32_t>();
    const int tops = N / p.B_max;
    job.R = (int64_t)tops * tops;
    // 2x2 box sums, shared by every step's domain gather
    FIC_TRY(w->box2.ensure(sizeof(uint16_t) * (size_t)N * N));
    L.begin(FIC_K_GATHER);
    FIC_TRY(launch_init_ranges(job.act, tops, p.B_max, s));
    FIC_TRY(launch_box2(job.dimg, N, w->box2.as<uint16_t>(), s));
    L.end(2, 0.0, (double)N * N * 3.0);
    return FIC_OK;
}

// Pool of one step: entropy -> flags (threshold rule, or the top-DN keys and
// a radix select) -> scan -> raster-order list into the slot's pool buffer,
// its size into the slot's scalars.
int Engine::launch_pool(Job& j, int B, int L_step, double thr, int64_t top, bool want_H,
                        Launcher& L, cudaStream_t s)
{
    return pool_launches(work_[(size_t)j.slot].get(), scal_.as<Scalars>() + j.slot,
                         entT_.as<long long>(), j.dimg, j.N, B, L_step, thr, top, want_H, L, s);
}

int pool_launches(ImageWork* w, Scalars* ds, const long long* entT, const uint8_t* dimg, int N,
                  int B, int L_step, double thr, int64_t top, bool want_H, Launcher& L,
                  cudaStream_t s)
{
    const int per = positions_per_axis(N, B, L_step);
    const int64_t npos = (int64_t)per * per;
    FIC_TRY(cudaMemsetAsync(&ds->near, 0, sizeof(unsigned long long), s));
    if (npos == 0) {
        FIC_TRY(cudaMemsetAsync(&ds->total, 0, sizeof(uint32_t), s));
        return FIC_OK;
    }
    FIC_TRY(w->flags.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(w->pos.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(w->pool.ensure(sizeof(uint32_t) * npos));
    FIC_TRY(w->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(npos)));
    if (want_H) FIC_TRY(w->H.ensure(sizeof(double) * npos));
    const bool select = top > 0 && top < npos;
    if (top > 0) FIC_TRY(w->keys.ensure(sizeof(unsigned long long) * npos));
    if (select) FIC_TRY(w->sel.ensure(select_state_bytes()));
    L.begin(FIC_K_ENTROPY);
    FIC_TRY(launch_entropy(dimg, N, B, L_step, per, thr, entT,
                           w->flags.as<uint32_t>(), want_H ? w->H.as<double>() : nullptr,
                           top > 0 ? w->keys.as<unsigned long long>() : nullptr, &ds->near, s));
    int nl = 1;
    if (select) {
        FIC_TRY(launch_top_select(w->keys.as<unsigned long long>(), npos, top, w->sel.p,
                                  w->flags.as<uint32_t>(), &ds->near, s, &nl));
    } else if (top > 0) {
        // the pool holds every position
        FIC_TRY(launch_fill_u32(w->flags.as<uint32_t>(), npos, 1u, s));
        ++nl;
    }
    L.end(nl, 0.0, (double)npos * (4.0 * B * B + 4.0));
    L.begin(FIC_K_SCAN);
    nl = 0;
    FIC_TRY(launch_scan(w->flags.as<uint32_t>(), w->pos.as<uint32_t>(), npos,
                        w->scan_tmp.as<uint32_t>(), &ds->total, s, &nl));
    FIC_TRY(launch_pool_scatter(w->flags.as<uint32_t>(), w->pos.as<uint32_t>(), npos, per, L_step,
                                w->pool.as<uint32_t>(), s));
    L.end(nl + 1, 0.0, (double)npos * 12.0);
    return FIC_OK;
}

int Engine::pool_only(int slot, const uint8_t* dimg, int N, int B, int L, double thr,
                      int64_t top, bool want_H, Launcher& Lk, cudaStream_t s, int64_t* dn,
                      int64_t* near)
{
    int st = ensure_slots(slot + 1);
    if (st) return st;
    Job j;
    j.slot = slot;
    j.dimg = dimg;
    j.N = N;
    st = launch_pool(j, B, L, thr, top, want_H, Lk, s);
    if (st) return st;
    st = read_scalars(slot + 1, s);
    if (st) return st;
    const int per = positions_per_axis(N, B, L);
    *dn = per > 0 ? (int64_t)host_scal_[slot].total : 0;
    *near = (int64_t)host_scal_[slot].near;
    return FIC_OK;
}

int Engine::step(const fic_params& p, const std::vector<Job*>& jobs, Launcher& L,
                 cudaStream_t s)
{
    int nl = 0;
    int st = validate_params(&p, jobs.empty() ? p.B_max : jobs[0]->N, &nl);
    if (st) return st;
    const bool filter = p.entropy_thresh >= 0.0;
    const int e16 = (int)llround(16.0 * p.err_tol);
    Scalars* ds = scal_.as<Scalars>();
    int n_slots = 0;
    std::vector<Job*> live;
    for (Job* j : jobs)
        if (!j->done && j->R > 0) {
            live.push_back(j);
            if (j->slot + 1 > n_slots) n_slots = j->slot + 1;
        }
    if (live.empty()) return FIC_OK;

    // pools: the threshold rule needs the pool sizes back before the
    // gathers; the top-DN pool size is known (near counts are read with the
    // split counts)
    const int64_t top = p.pool_dn;
    for (Job* j : live) {
        const int B = p.B_max >> j->lvl;
        j->per = positions_per_axis(j->N, B, p.L);
        const int64_t npos = (int64_t)j->per * j->per;
        j->res.n_positions[j->lvl] = npos;
        j->res.ranges[j->lvl] = j->R;
        j->use_list = filter || top > 0;
        if (j->use_list) {
            st = launch_pool(*j, B, p.L, top > 0 ? -1.0 : p.entropy_thresh, top, false, L, s);
            if (st) return st;
        }
        j->dn = top > 0 ? (top < npos ? top : npos) : npos;
    }
    if (filter && top == 0) {
        st = read_scalars(n_slots, s);
        if (st) return st;
        for (Job* j : live) {
            j->dn = j->per > 0 ? (int64_t)host_scal_[j->slot].total : 0;
            j->res.near_thresh[j->lvl] = (int64_t)host_scal_[j->slot].near;
        }
    }

    // the contraction shape of each quadtree step present: tuned, fixed or
    // forced (a step not seen before in tuning mode is measured below)
    TuneChoice choice[FIC_MAX_LEVELS];
    bool trial[FIC_MAX_LEVELS] = {false, false, false, false};
    int tkey[FIC_MAX_LEVELS][4];
    {
        double work[FIC_MAX_LEVELS] = {0, 0, 0, 0};
        for (Job* j : live) work[j->lvl] += (double)j->R * (double)j->dn;
        const int mode = tune_mode();
        for (int lvl = 0; lvl < nl; ++lvl) {
            choice[lvl] = default_choice();
            const int B = p.B_max >> lvl;
            tkey[lvl][0] = p.engine;
            tkey[lvl][1] = k_pad(B * B);
            tkey[lvl][2] = p.S_sets[lvl].n_s;
            tkey[lvl][3] = (int)std::floor(std::log2(work[lvl] + 1.0));
            if (work[lvl] <= 0.0) continue;
            const std::vector<TuneChoice> cand = tune_candidates(p, lvl);
            if (mode >= 2) {
                choice[lvl] = cand[(size_t)(mode - 2) % cand.size()];
            } else if (mode == 1 && cand.size() > 1) {
                // the class's tuned shape; without one, measure the candidates
                // (synchronous entry points) or take the tuned shape of the
                // nearest size class, else the default (the request server,
                // whose steps must not wait for tuning runs)
                int near_d = 1 << 30;
                bool exact = false;
                for (const TuneEntry& t : tuned())
                    if (t.engine == tkey[lvl][0] && t.K == tkey[lvl][1] && t.ns == tkey[lvl][2]) {
                        const int d = std::abs(t.size_class - tkey[lvl][3]);
                        if (d < near_d) {
                            near_d = d;
                            choice[lvl] = t.choice;
                            exact = d == 0;
                        }
                    }
                trial[lvl] = !exact && allow_trials_;
                if (!exact && allow_trials_) choice[lvl] = default_choice();
            }
        }
    }

    // operand A' and the range constants in the layout of a shape
    auto prep = [&](Job* j, const StepShape& h) -> int {
        ImageWork* w = work_[(size_t)j->slot].get();
        j->rows_pad = rows_pad_for(h, j->R);
        const int64_t rows_max = 8 * round_up(j->R, 128);  // either layout
        FIC_TRY(w->A.ensure(sizeof(__half) * rows_max * h.K));
        FIC_TRY(w->rc.ensure(sizeof(RowConst) * (rows_max / 8)));
        L.begin(FIC_K_RANGE_PREP);
        FIC_TRY(launch_range_prep(j->dimg, j->N, h.B, j->act, (int)j->R, j->rows_pad, h.K, h.sp,
                                  &ds[j->slot].vd_max, h.iso ? 1 : 0, w->A.as<__half>(),
                                  w->rc.as<RowConst>(), s));
        L.end(1, 0.0, (double)j->rows_pad * h.K * 2.0 + (double)j->R * (h.n2 + 20.0));
        return FIC_OK;
    };

    // domain gathers and range preps
    for (Job* j : live) {
        const StepShape h = step_shape(p, j->lvl, choice[j->lvl]);
        ImageWork* w = work_[(size_t)j->slot].get();
        Scalars* d = ds + j->slot;
        j->res.pool_size[j->lvl] = j->dn;
        j->res.matches[j->lvl] = 8 * j->R * j->dn;
        j->cols_pad = round_up(j->dn > 0 ? j->dn : 1, kColPad);
        FIC_TRY(w->D.ensure(sizeof(__half) * j->cols_pad * h.K));
        FIC_TRY(w->cf.ensure(sizeof(float) * j->cols_pad * h.sp.cw));
        FIC_TRY(w->ci.ensure(sizeof(ColExact) * j->cols_pad));
        FIC_TRY(w->best.ensure(sizeof(Best) * j->R));
        FIC_TRY(w->split.ensure(sizeof(uint32_t) * j->R));
        FIC_TRY(w->split_pos.ensure(sizeof(uint32_t) * j->R));
        FIC_TRY(w->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(j->R)));
        const uint32_t* pool_xy = j->use_list ? w->pool.as<uint32_t>() : nullptr;
        FIC_TRY(cudaMemsetAsync(&d->vd_max, 0, sizeof(unsigned long long), s));
        FIC_TRY(cudaMemsetAsync(&d->vd_min_key, 0xff, sizeof(unsigned long long), s));
        L.begin(FIC_K_GATHER);
        FIC_TRY(launch_gather(w->box2.as<uint16_t>(), j->N, h.B, p.L, j->per, pool_xy, j->dn,
                              j->cols_pad, h.K, h.sp, w->D.as<__half>(), w->cf.as<float>(),
                              w->ci.as<ColExact>(), &d->vd_max, &d->vd_min_key, s));
        L.end(2, 0.0,
              (double)j->cols_pad * (2.0 * h.K + 4.0 * h.sp.cw + 8.0) +
                  (double)j->dn * 2.0 * h.n2);
        st = prep(j, h);
        if (st) return st;
        j->n_chunks = 0;
        j->n_parts = 0;
    }

    // one contraction launch per quadtree step present (over every job at
    // that step); timed with events when the tuner measures a shape
    int leaders[FIC_MAX_LEVELS] = {-1, -1, -1, -1};
    auto run_group = [&](int lvl, const StepShape& h, float* ms) -> int {
        double group_tiles = 0.0;
        int group_jobs = 0;
        for (Job* j : live)
            if (j->lvl == lvl && j->dn > 0) {
                group_tiles += (double)mtiles_for(h, j->rows_pad) * (double)(j->cols_pad / h.tile_w);
                ++group_jobs;
            }
        table_.clear();
        int64_t items = 0;
        double flops = 0.0, bytes = 0.0;
        int64_t matches = 0;
        for (Job* j : live) {
            if (j->lvl != lvl || j->dn == 0) continue;
            ImageWork* w = work_[(size_t)j->slot].get();
            const int64_t n_mtiles = mtiles_for(h, j->rows_pad);
            const int64_t n_ct = j->cols_pad / h.tile_w;
            if (group_jobs == 1)
                choose_chunks_alone(sm_count_, n_mtiles, n_ct, h.refill, &j->n_chunks,
                                    &j->per_chunk);
            else
                choose_chunks_shared(sm_count_, n_mtiles, n_ct,
                                     group_tiles / ((16.0 / h.refill) * sm_count_), &j->n_chunks,
                                     &j->per_chunk);
            j->n_parts = h.parts_per_chunk * j->n_chunks;
            FIC_TRY(w->part.ensure(sizeof(Best) * j->R * j->n_parts));
            FIC_TRY(w->gbest.ensure(sizeof(long long) * j->rows_pad));
            FIC_TRY(cudaMemsetAsync(w->gbest.p, 0x7f, sizeof(long long) * j->rows_pad, s));
            Problem pr;
            memset(&pr, 0, sizeof(pr));
            pr.A = w->A.as<__half>();
            pr.D = w->D.as<__half>();
            pr.cf = w->cf.as<float>();
            pr.ci = w->ci.as<ColExact>();
            pr.rc = w->rc.as<RowConst>();
            pr.part = w->part.as<Best>();
            pr.gbest = w->gbest.as<long long>();
            pr.rows_pad = j->rows_pad;
            pr.cols_pad = j->cols_pad;
            pr.R = (int)j->R;
            pr.dn = (int)j->dn;
            pr.n_mtiles = (int)n_mtiles;
            pr.n_ct = (int)n_ct;
            pr.n_chunks = j->n_chunks;
            pr.per_chunk = j->per_chunk;
            pr.item_start = (int)items;
            // diagonal chunk order while the pool operand stays in L2
            pr.diag = (double)j->cols_pad * h.K * 2.0 <= kDiagMaxPoolBytes ? 1 : 0;
            table_.push_back(pr);
            items += n_mtiles * j->n_chunks;
            flops += 2.0 * (8.0 * j->R) * (double)j->dn * h.n2;
            matches += 8 * j->R * j->dn;
            bytes += (double)j->rows_pad * h.K * 2.0 +
                     (double)j->cols_pad * (2.0 * h.K + 4.0 * h.sp.cw);
            if (leaders[lvl] < 0) leaders[lvl] = j->slot;
        }
        FIC_TRY(probs_[lvl].ensure(sizeof(Problem) * table_.size()));
        FIC_TRY(cudaMemcpyAsync(probs_[lvl].p, table_.data(), sizeof(Problem) * table_.size(),
                                cudaMemcpyHostToDevice, s));
        ContractArgs a;
        a.probs = probs_[lvl].as<Problem>();
        a.n_probs = (int)table_.size();
        a.n_items = (int)items;
        a.K = h.K;
        a.sp = h.sp;
        a.err = &ds[leaders[lvl]].err;
        a.grid_ctas = sm_count_;
        a.variant = h.epi;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ms) {
            FIC_TRY(cudaEventCreate(&e0));
            FIC_TRY(cudaEventCreate(&e1));
            FIC_TRY(cudaEventRecord(e0, s));
        }
        if (p.engine == FIC_ENGINE_TENSOR) {
            FIC_TRY(cudaMemsetAsync(a.err, 0, 2 * sizeof(int), s));
            L.begin(FIC_K_CONTRACT_TC);
            FIC_TRY(h.red   ? launch_contract_tc_red(a, s)
                    : h.iso ? launch_contract_tc_iso(a, s)
                            : launch_contract_tc(a, s));
            L.end(1, flops, bytes, matches);
        } else {
            L.begin(FIC_K_CONTRACT_PLAIN);
            FIC_TRY(launch_contract_plain(a, s));
            L.end(1, flops, bytes, matches);
        }
        if (ms) {
            FIC_TRY(cudaEventRecord(e1, s));
            FIC_TRY(cudaEventSynchronize(e1));
            FIC_TRY(cudaEventElapsedTime(ms, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            // a tuning run that gave up waiting must not be mistaken for a fast one
            Scalars chk;
            FIC_TRY(cudaMemcpy(&chk, &ds[leaders[lvl]], sizeof(chk), cudaMemcpyDeviceToHost));
            if (p.engine == FIC_ENGINE_TENSOR && (chk.err || chk.err2)) return FIC_ETIMEOUT;
        }
        return FIC_OK;
    };

    for (int lvl = 0; lvl < nl; ++lvl) {
        bool present = false;
        for (Job* j : live) present |= (j->lvl == lvl && j->dn > 0);
        if (!present) continue;
        if (trial[lvl]) {
            // measure every candidate on this step's operands, keep the fastest
            const std::vector<TuneChoice> cand = tune_candidates(p, lvl);
            float best_ms = 3.4e38f;
            TuneChoice best = choice[lvl];
            bool layout_iso = step_shape(p, lvl, choice[lvl]).iso;
            for (const TuneChoice& c : cand) {
                const StepShape h = step_shape(p, lvl, c);
                if (h.iso != layout_iso) {
                    for (Job* j : live)
                        if (j->lvl == lvl) {
                            st = prep(j, h);
                            if (st) return st;
                        }
                    layout_iso = h.iso;
                }
                // two runs, the faster one counts: the first run of a shape
                // also pays for its cold start (instruction cache, L2)
                float ms = 3.4e38f;
                for (int rep = 0; rep < 2; ++rep) {
                    float m = 0.0f;
                    st = run_group(lvl, h, &m);
                    if (st) return st;
                    ms = std::min(ms, m);
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            TuneEntry t;
            t.engine = tkey[lvl][0];
            t.K = tkey[lvl][1];
            t.ns = tkey[lvl][2];
            t.size_class = tkey[lvl][3];
            t.choice = best;
            t.ms = best_ms;
            t.candidates = (int)cand.size();
            {
                std::lock_guard<std::mutex> g(g_tune_mu);
                g_tuned.push_back(t);
            }
            choice[lvl] = best;
            const StepShape h = step_shape(p, lvl, best);
            if (h.iso != layout_iso)
                for (Job* j : live)
                    if (j->lvl == lvl) {
                        st = prep(j, h);
                        if (st) return st;
                    }
            st = run_group(lvl, h, nullptr);
            if (st) return st;
        } else {
            st = run_group(lvl, step_shape(p, lvl, choice[lvl]), nullptr);
            if (st) return st;
        }
        used_choice_[lvl] = choice[lvl];
        used_valid_[lvl] = true;
    }

    // split / requeue
    for (Job* j : live) {
        const StepShape h = step_shape(p, j->lvl, choice[j->lvl]);
        ImageWork* w = work_[(size_t)j->slot].get();
        const uint32_t* pool_xy = j->use_list ? w->pool.as<uint32_t>() : nullptr;
        const int last = (j->lvl == nl - 1);
        L.begin(FIC_K_SPLIT);
        FIC_TRY(launch_split_decide(w->part.as<Best>(), j->n_parts, w->rc.as<RowConst>(),
                                    (int)j->R, h.n2, h.sp, e16, last, (int)j->dn,
                                    &ds[j->slot].vd_min_key, w->best.as<Best>(),
                                    w->split.as<uint32_t>(), s));
        int nlaunch = 0;
        FIC_TRY(launch_scan(w->split.as<uint32_t>(), w->split_pos.as<uint32_t>(), j->R,
                            w->scan_tmp.as<uint32_t>(), &ds[j->slot].total, s, &nlaunch));
        FIC_TRY(launch_split_scatter(j->act, w->best.as<Best>(), w->split.as<uint32_t>(),
                                     w->split_pos.as<uint32_t>(), w->rc.as<RowConst>(),
                                     (int)j->R, h.B, j->lvl, pool_xy, j->per, p.L, (int)j->dn,
                                     j->next, w->codes_tmp.p, j->n_codes, s));
        L.end(2 + nlaunch, 0.0, (double)j->R * 64.0);
    }
    st = read_scalars(n_slots, s);
    if (st) return st;
    if (p.engine == FIC_ENGINE_TENSOR)
        for (int lvl = 0; lvl < nl; ++lvl)
            if (leaders[lvl] >= 0 && (host_scal_[leaders[lvl]].err || host_scal_[leaders[lvl]].err2))
                return FIC_ETIMEOUT;
    for (Job* j : live) {
        if (top > 0) j->res.near_thresh[j->lvl] = (int64_t)host_scal_[j->slot].near;
        const int64_t splits = host_scal_[j->slot].total;
        j->n_codes += j->R - splits;
        j->R = 4 * splits;
        std::swap(j->act, j->next);
        j->lvl += 1;
        if (j->R == 0 || j->lvl >= nl) j->done = true;
    }
    return FIC_OK;
}

int Engine::finish(Job& j, const fic_params& p, fic_code* dst, int64_t cap, Launcher& L,
                   cudaStream_t s)
{
    ImageWork* w = work_[(size_t)j.slot].get();
    Scalars* ds = scal_.as<Scalars>() + j.slot;
    FIC_TRY(w->cellmap.ensure(sizeof(uint32_t) * j.cells));
    FIC_TRY(w->cellflag.ensure(sizeof(uint32_t) * j.cells));
    FIC_TRY(w->cellrank.ensure(sizeof(uint32_t) * j.cells));
    FIC_TRY(w->scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(j.cells)));
    L.begin(FIC_K_ORDER);
    FIC_TRY(cudaMemsetAsync(w->cellflag.p, 0, sizeof(uint32_t) * j.cells, s));
    FIC_TRY(launch_order_mark(w->codes_tmp.p, j.n_codes, j.N, p.B_max, p.B_min,
                              w->cellmap.as<uint32_t>(), w->cellflag.as<uint32_t>(), s));
    int nl = 0;
    FIC_TRY(launch_scan(w->cellflag.as<uint32_t>(), w->cellrank.as<uint32_t>(), j.cells,
                        w->scan_tmp.as<uint32_t>(), &ds->total, s, &nl));
    FIC_TRY(launch_order_gather(w->codes_tmp.p, w->cellmap.as<uint32_t>(),
                                w->cellflag.as<uint32_t>(), w->cellrank.as<uint32_t>(), j.cells,
                                w->codes_out.p, s));
    L.end(2 + nl, 0.0, (double)j.cells * 16.0 + (double)j.n_codes * 32.0);
    j.res.n_codes = j.n_codes;
    if (dst) {
        j.res.codes = dst;
        j.res.owns_codes = 0;
        if (j.n_codes > cap) return FIC_ECAP;
        FIC_TRY(cudaMemcpyAsync(dst, w->codes_out.p, sizeof(fic_code) * j.n_codes,
                                cudaMemcpyDefault, s));
    } else {
        fic_code* h = (fic_code*)malloc(sizeof(fic_code) * (size_t)(j.n_codes ? j.n_codes : 1));
        if (!h) return FIC_ENOMEM;
        j.res.codes = h;
        j.res.owns_codes = 1;
        FIC_TRY(cudaMemcpyAsync(h, w->codes_out.p, sizeof(fic_code) * j.n_codes,
                                cudaMemcpyDeviceToHost, s));
    }
    return FIC_OK;
}

}  // namespace fic
