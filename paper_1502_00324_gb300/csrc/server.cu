// server.cu -- the request server of include/fic.h (fic_server_*):
// continuous batching of image encodes on one device.
//
// Worker iteration (one host thread per server, one CUDA stream):
//   1. admission: queue (FIFO, or smallest image first with aging) -> free
//      slot, while the estimated device bytes
//      of all slots stay within the budget (slots keep their buffers between
//      images; idle slots are emptied when room is needed);
//   2. begin() for the images admitted now (upload, 2x2 sums, top ranges);
//   3. Engine::step() over the admitted images of side <= 512, then over
//      the larger ones: each image advances one quadtree step, with one
//      grouped contraction launch per step present in the class;
//   4. after each class, its finished images: records ordered and copied to
//      the host, the slot freed, pollers woken (a small image does not wait
//      for the large images' step of the same iteration).
// Images are independent: the engine gives each the same records it would
// get alone (its own pool, its own partial bests, its own split decisions).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "engine.h"
#include "fic.h"

using namespace fic;

namespace {

// Side classes of an iteration: images up to this side step (and finish)
// before the larger ones.
constexpr int kSmallSide = 512;

struct Request {
    int64_t ticket = 0;
    int N = 0;
    std::vector<uint8_t> host;     // copy of a host image
    const uint8_t* dptr = nullptr; // caller's device image (not copied)
    double submit_ms = 0.0;
    int64_t est = 0;
};

struct Finished {
    int status = FIC_OK;
    fic_result res{};
    fic_timing t{};
};

struct InFlight {
    Request req;
    Job job;
    bool begun = false;
    double admit_ms = 0.0;
    int steps = 0, shared = 0;
};

}  // namespace

struct fic_server {
    fic_params p{};
    fic_server_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    Engine eng;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<int64_t, Finished> done;
    std::unordered_set<int64_t> pending;  // queued or in flight
    std::vector<std::unique_ptr<InFlight>> inflight;
    std::vector<int64_t> slot_cap;        // estimated bytes held per slot
    std::vector<char> slot_busy;
    std::vector<int> to_release;
    int64_t next_ticket = 1;
    bool stop = false;
    fic_server_stats st{};
    double inflight_sum = 0.0;
    std::chrono::steady_clock::time_point t0;
    std::thread worker;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    }

    // Under mu: record a result; has_slot: f holds a workspace slot.
    void finish_one(std::unique_ptr<InFlight>& f, int status, bool has_slot = true)
    {
        Finished d;
        d.status = status;
        d.res = f->job.res;
        if (status != FIC_OK) {
            fic_result_free(&d.res);
            memset(&d.res, 0, sizeof(d.res));
        }
        d.t.submit_ms = f->req.submit_ms;
        d.t.admit_ms = f->admit_ms;
        d.t.done_ms = now_ms();
        d.t.steps = f->steps;
        d.t.shared_steps = f->shared;
        if (status == FIC_OK) {
            st.completed += 1;
            for (int l = 0; l < FIC_MAX_LEVELS; ++l) st.matches += d.res.matches[l];
        } else {
            st.failed += 1;
        }
        if (has_slot) slot_busy[(size_t)f->job.slot] = 0;
        done[f->req.ticket] = d;
        pending.erase(f->req.ticket);
    }

    // Under mu: move queued requests into free slots within the budget.
    void admit(std::vector<InFlight*>& fresh)
    {
        while (!queue.empty() && (int)inflight.size() < cfg.max_inflight) {
            // policy 1: the oldest request once it has waited age_ms, else the
            // smallest image (earliest among equals); policy 0: the oldest
            size_t pick = 0;
            if (cfg.policy == 1 && now_ms() - queue.front().submit_ms < (double)cfg.age_ms)
                for (size_t q = 1; q < queue.size(); ++q)
                    if (queue[q].N < queue[pick].N) pick = q;
            Request& r = queue[pick];
            int slot = -1;
            for (int k = 0; k < cfg.max_inflight; ++k) {
                if (slot_busy[(size_t)k]) continue;
                if (slot < 0) slot = k;
                const bool fits_k = slot_cap[(size_t)k] >= r.est;
                const bool fits_s = slot_cap[(size_t)slot] >= r.est;
                // prefer the smallest slot that already fits, else the largest
                if ((fits_k && (!fits_s || slot_cap[(size_t)k] < slot_cap[(size_t)slot])) ||
                    (!fits_k && !fits_s && slot_cap[(size_t)k] > slot_cap[(size_t)slot]))
                    slot = k;
            }
            if (slot < 0) break;
            int64_t grow = r.est > slot_cap[(size_t)slot] ? r.est - slot_cap[(size_t)slot] : 0;
            for (int k = 0; k < cfg.max_inflight && st.hbm_in_use + grow > cfg.hbm_budget; ++k) {
                if (k == slot || slot_busy[(size_t)k] || slot_cap[(size_t)k] == 0) continue;
                st.hbm_in_use -= slot_cap[(size_t)k];
                slot_cap[(size_t)k] = 0;
                to_release.push_back(k);
            }
            if (st.hbm_in_use + grow > cfg.hbm_budget) {
                if (!inflight.empty()) break;  // wait for memory to free up
                // larger than the whole budget: refuse this one
                std::unique_ptr<InFlight> f(new InFlight());
                f->req = std::move(r);
                queue.erase(queue.begin() + (std::ptrdiff_t)pick);
                f->admit_ms = now_ms();
                finish_one(f, FIC_ENOMEM, false);
                continue;
            }
            slot_cap[(size_t)slot] += grow;
            st.hbm_in_use += grow;
            if (st.hbm_in_use > st.hbm_peak) st.hbm_peak = st.hbm_in_use;
            std::unique_ptr<InFlight> f(new InFlight());
            f->req = std::move(r);
            queue.erase(queue.begin() + (std::ptrdiff_t)pick);
            f->job.slot = slot;
            f->admit_ms = now_ms();
            slot_busy[(size_t)slot] = 1;
            fresh.push_back(f.get());
            inflight.push_back(std::move(f));
        }
        st.queued = (int64_t)queue.size();
        st.inflight = (int64_t)inflight.size();
        if (st.inflight > st.peak_inflight) st.peak_inflight = st.inflight;
    }

    void fail_all_inflight(int status)
    {
        std::lock_guard<std::mutex> g(mu);
        for (auto& f : inflight) finish_one(f, status);
        inflight.clear();
        st.inflight = 0;
        cv_done.notify_all();
    }

    // The worker's last act when its loop ends on an exception: every
    // request it holds or has queued fails with `status`, waiting polls wake,
    // and later submits are refused (the server takes no more work).
    void fail_all_and_stop(int status)
    {
        std::lock_guard<std::mutex> g(mu);
        stop = true;
        for (auto& f : inflight) finish_one(f, status);
        inflight.clear();
        while (!queue.empty()) {
            std::unique_ptr<InFlight> f(new InFlight());
            f->req = std::move(queue.front());
            queue.pop_front();
            finish_one(f, status, false);
        }
        st.inflight = 0;
        st.queued = 0;
        cv_done.notify_all();
    }

    void run()
    {
        cudaSetDevice(device);
        Launcher L(stream, false);
        for (;;) {
            std::vector<InFlight*> fresh;
            std::vector<int> release;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !queue.empty() || !inflight.empty(); });
                if (stop) {
                    // queued requests are not started; in-flight ones finish
                    while (!queue.empty()) {
                        std::unique_ptr<InFlight> f(new InFlight());
                        f->req = std::move(queue.front());
                        queue.pop_front();
                        finish_one(f, FIC_EBUSY, false);
                    }
                    st.queued = 0;
                    cv_done.notify_all();
                    if (inflight.empty()) break;
                } else {
                    admit(fresh);
                    cv_done.notify_all();  // refused requests
                }
                release.swap(to_release);
            }
            for (int k : release) eng.work(k).release();
            if (inflight.empty()) continue;
            const double t_iter = now_ms();

            // 2. start the images admitted now
            for (InFlight* f : fresh) {
                const uint8_t* src = f->req.dptr ? f->req.dptr : f->req.host.data();
                const int slot = f->job.slot;
                const int s2 = eng.begin(f->job, slot, src, f->req.N, p, L, stream);
                if (s2) {
                    fail_all_inflight(s2);
                    break;
                }
                f->begun = true;
            }
            if (inflight.empty()) continue;

            // 3-4. one quadtree step of every image in flight, smaller images
            // first: each side class steps in its own grouped launches and
            // its finished images are released before the next class steps,
            // so a small image does not wait for a large image's step
            const double n_start = (double)inflight.size();
            bool failed = false;
            for (int cls = 0; cls < 2 && !failed; ++cls) {
                std::vector<Job*> jobs;
                bool levels[FIC_MAX_LEVELS] = {false, false, false, false};
                for (auto& f : inflight)
                    if ((f->req.N > kSmallSide) == (cls == 1)) jobs.push_back(&f->job);
                if (jobs.empty()) continue;
                for (auto& f : inflight)
                    if ((f->req.N > kSmallSide) == (cls == 1)) {
                        f->steps += 1;
                        if (jobs.size() > 1) f->shared += 1;
                        if (f->job.lvl < FIC_MAX_LEVELS) levels[f->job.lvl] = true;
                    }
                int status = eng.step(p, jobs, L, stream);
                bool any_done = false;
                if (!status)
                    for (Job* j : jobs)
                        if (j->done) {
                            any_done = true;
                            status = eng.finish(*j, p, nullptr, 0, L, stream);
                            if (status) break;
                        }
                if (!status && any_done) status = to_status(cudaStreamSynchronize(stream));
                if (status) {
                    fail_all_inflight(status);
                    failed = true;
                    break;
                }
                std::lock_guard<std::mutex> g(mu);
                for (bool b : levels) st.contraction_launches += b ? 1 : 0;
                std::vector<std::unique_ptr<InFlight>> keep;
                for (auto& f : inflight) {
                    if (f->job.done)
                        finish_one(f, FIC_OK);
                    else
                        keep.push_back(std::move(f));
                }
                inflight.swap(keep);
                st.inflight = (int64_t)inflight.size();
                if (any_done) cv_done.notify_all();
            }
            if (failed) continue;
            {
                std::lock_guard<std::mutex> g(mu);
                st.iterations += 1;
                inflight_sum += n_start;
                st.mean_inflight = inflight_sum / (double)st.iterations;
                st.busy_ms += now_ms() - t_iter;
            }
        }
    }
};

extern "C" {

int fic_server_create(const fic_params* p, const fic_server_config* cfg, fic_server** out)
{
    if (!p || !out) return FIC_EINVAL;
    *out = nullptr;
    int nl = 0;
    if (validate_params(p, p->B_max, &nl)) return FIC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIC_ENODEV;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return FIC_ENODEV;
    if (major != 10 || minor != 3) return FIC_ENODEV;
    try {
        std::unique_ptr<fic_server> s(new fic_server());
        s->p = *p;
        s->device = dev;
        if (cfg) s->cfg = *cfg;
        if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 64;
        if (s->cfg.max_queue <= 0) s->cfg.max_queue = 65536;
        if (s->cfg.policy != 0 && s->cfg.policy != 1) return FIC_EINVAL;
        if (s->cfg.age_ms <= 0) s->cfg.age_ms = 2000;
        if (s->cfg.hbm_budget <= 0) {
            size_t fr = 0, tot = 0;
            FIC_TRY(cudaMemGetInfo(&fr, &tot));
            s->cfg.hbm_budget = (int64_t)(fr / 2);
        }
        FIC_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->eng.set_trials(false);
        int st = s->eng.init(s->stream);
        if (st == FIC_OK) st = s->eng.ensure_slots(s->cfg.max_inflight);
        if (st) {
            cudaStreamDestroy(s->stream);
            return st;
        }
        s->slot_cap.assign((size_t)s->cfg.max_inflight, 0);
        s->slot_busy.assign((size_t)s->cfg.max_inflight, 0);
        s->st.hbm_budget = s->cfg.hbm_budget;
        s->t0 = std::chrono::steady_clock::now();
        fic_server* raw = s.get();
        s->worker = std::thread([raw] {
            try {
                raw->run();
            } catch (...) {
                try {
                    raw->fail_all_and_stop(FIC_ENOMEM);
                } catch (...) {
                }
            }
        });
        *out = s.release();
        return FIC_OK;
    } catch (...) {
        return FIC_ENOMEM;
    }
}

int fic_server_submit(fic_server* s, const uint8_t* img, int N, int64_t* ticket)
{
    if (!s || !img || !ticket) return FIC_EINVAL;
    int nl = 0;
    if (validate_params(&s->p, N, &nl)) return FIC_EINVAL;
    try {
        Request r;
        r.N = N;
        if (is_device_ptr(img)) {
            r.dptr = img;
        } else {
            r.host.assign(img, img + (size_t)N * N);
        }
        r.est = s->eng.slot_bytes(N, s->p);
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return FIC_EBUSY;
        if ((int64_t)s->queue.size() >= s->cfg.max_queue) return FIC_EBUSY;
        r.ticket = s->next_ticket++;
        r.submit_ms = s->now_ms();
        *ticket = r.ticket;
        s->pending.insert(r.ticket);
        s->queue.push_back(std::move(r));
        s->st.submitted += 1;
        s->st.queued = (int64_t)s->queue.size();
        s->cv_work.notify_one();
        return FIC_OK;
    } catch (...) {
        return FIC_ENOMEM;
    }
}

int fic_server_poll(fic_server* s, int64_t ticket, int wait_ms, fic_result* out,
                    fic_timing* timing)
{
    if (!s || !out) return FIC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (!ready() && !s->pending.count(ticket)) return FIC_EINVAL;
    if (wait_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    if (!ready()) return FIC_ENOTREADY;
    Finished d = s->done[ticket];
    s->done.erase(ticket);
    *out = d.res;
    if (timing) *timing = d.t;
    return d.status;
}

int fic_server_stats_read(fic_server* s, fic_server_stats* out)
{
    if (!s || !out) return FIC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    return FIC_OK;
}

int fic_server_destroy(fic_server* s)
{
    if (!s) return FIC_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->done) fic_result_free(&kv.second.res);
    s->done.clear();
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
    delete s;
    return FIC_OK;
}

}  // extern "C"
