// engine.h -- the quadtree step driver shared by the synchronous entry points
// (fic_encode*, one engine per device) and the request server (one engine per
// server).  Internal to libfic.so.
//
// An Engine holds device workspaces in slots; a Job is one image in flight,
// bound to one slot.  step() advances every job it is given by one quadtree
// step (Sec. 2), each job at its own step: per job the pool (Sec. 3), the
// domain gather and the range prep; per quadtree step present, ONE grouped
// contraction + scoring launch over the work items of all its jobs; per job
// the split decision and requeue.  Host and device meet twice per step()
// (pool sizes, numbers of splits) whatever the number of jobs.
#pragma once

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"
#include "fic.h"

namespace fic {

// ---------------------------------------------------------------------------
// Instrumentation (fic_stats): per-kind launch counts, algorithmic flops and
// bytes, and (when enabled) device time from events around each stage.
// ---------------------------------------------------------------------------
struct StatsState {
    std::mutex mu;
    fic_stats st;
    bool timing = false;
};
extern StatsState g_stats;

// The stages recorded while a graph is captured: launches, bytes and (when
// timed) the external events around each stage, replayed into fic_stats
// after every launch of the graph (graph.cu).
struct GraphRec {
    struct Entry {
        int kind, launches, level, job;
        double bytes;
        cudaEvent_t a, b;
    };
    bool timed = false;
    int level = -1;  // quadtree step being captured
    int job = -1;    // image of the stage being captured (-1: all)
    std::vector<Entry> entries;
    ~GraphRec();
};

class Launcher {
public:
    explicit Launcher(cudaStream_t s, bool allow_timing = true);
    // capture mode: stages go to rec instead of fic_stats
    Launcher(cudaStream_t s, GraphRec* rec) : s_(s), rec_(rec) {}
    ~Launcher() { harvest(); }
    void begin(int kind);
    void end(int launches, double flops = 0.0, double bytes = 0.0, int64_t matches = 0);
    void harvest();

private:
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    cudaStream_t s_;
    bool timing_ = false;
    int kind_ = FIC_K_MISC;
    Pending cur_{};
    std::vector<Pending> pending_;
    GraphRec* rec_ = nullptr;
};

// Last CUDA error text of this thread (fic_last_error).
extern thread_local char g_last_error[160];
int to_status(cudaError_t e);

#define FIC_TRY(expr)                           \
    do {                                        \
        cudaError_t e__ = (expr);               \
        if (e__ != cudaSuccess) {               \
            return ::fic::to_status(e__);       \
        }                                       \
    } while (0)

// Device buffer grown on demand (contents are not kept when it grows).
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes);
    void release();
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Small device scalars of one slot.
struct Scalars {
    uint32_t total;                 // scan total (pool size, splits, records)
    uint32_t changed;               // decoder: pixels changed in a pass
    unsigned long long near;        // positions within 1e-9 of the threshold
    unsigned long long vd_max;      // pool's largest Vd
    unsigned long long vd_min_key;  // pool's smallest (Vd, index) key
    int err;                        // contraction error words (err, err + 1)
    int err2;
    // device-side step state of a graph-captured encode (graph.cu)
    uint32_t R;                     // active ranges at the current step
    uint32_t dn;                    // pool size of the current step
    uint32_t n_codes;               // records emitted so far
    uint32_t n_parts;               // partial bests per range of the current step
    uint32_t lvl_R[FIC_MAX_LEVELS];
    uint32_t lvl_dn[FIC_MAX_LEVELS];
    unsigned long long lvl_near[FIC_MAX_LEVELS];
};

// Device workspaces of one slot (kept and grown across jobs).
struct ImageWork {
    DevBuf img, box2, flags, pos, scan_tmp, pool, D, cf, ci, A, rc, part, gbest, best, split,
        split_pos, act0, act1, codes_tmp, codes_out, cellmap, cellflag, cellrank, H, keys, sel;
    void release();
};

// One image in flight.
struct Job {
    const uint8_t* dimg = nullptr;  // device image (caller's or the slot's copy)
    int N = 0;
    int slot = 0;
    int lvl = 0;                    // next quadtree step to run
    bool done = false;
    int64_t R = 0;                  // active ranges at step lvl
    int64_t n_codes = 0;            // records emitted so far
    int64_t cells = 0;              // (N / B_min)^2
    uint32_t* act = nullptr;        // active ranges (x | y << 16)
    uint32_t* next = nullptr;
    // per-step values
    int per = 0;
    int64_t dn = 0, cols_pad = 0, rows_pad = 0;
    bool use_list = false;
    int n_chunks = 0, per_chunk = 0, n_parts = 0;
    fic_result res{};               // counters; codes set by finish()
};

// A contraction shape choice of the tuner: kernel family where it applies
// (0: row tiles, 1: isometry-in-accumulator tiles, 2: domain-side
// isometries with the maximum taken by the TMEM load), the chunking's
// per-item refill cost in tiles, and the isometry kernel's epilogue (0: 8
// warps x 16-column TMEM reads, 1: 16 warps x 8-column reads).
struct TuneChoice {
    int iso;
    int refill;
    int epi;
};

// Tuning mode (process-wide): 0 fixed default shape, 1 measure on first use
// (default), 2 + i force candidate i (tests).
int tune_mode();
void set_tune_mode(int mode);
// Graph mode (process-wide): 0 eager only; 1 (default) a configuration's
// first encode runs eagerly, later ones replay its captured graph.
int graph_mode();
void set_graph_mode(int mode);

int validate_params(const fic_params* p, int N, int* n_levels);
// Pool, range and record counts within the device code's limits
// (kMaxPoolColumns, kMaxScanCount); FIC_EINVAL with fic_last_error set.
int check_size_limits(const fic_params& p, int N, int n_levels);
int positions_per_axis(int N, int B, int L);

class Engine {
public:
    Engine() = default;
    ~Engine();
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    // Device properties and the entropy table (once, on the current device).
    int init(cudaStream_t s);
    int sm_count() const { return sm_count_; }
    // Slots 0 .. n-1 exist afterwards.
    int ensure_slots(int n);

    // Binds job to slot, uploads a host image, starts the quadtree: every
    // B_max block in raster order.  No host synchronisation.
    int begin(Job& job, int slot, const uint8_t* img, int N, const fic_params& p, Launcher& L,
              cudaStream_t s);
    // One quadtree step of every job in jobs (not done); jobs may be at
    // different steps.  Marks finished jobs done.
    int step(const fic_params& p, const std::vector<Job*>& jobs, Launcher& L, cudaStream_t s);
    // Orders a done job's records (raster of top ranges, then TL, TR, BL, BR)
    // and copies them to dst (host or device, cap records) or, with dst NULL,
    // to a new host array owned by job.res.  Asynchronous: synchronise s
    // before reading.
    int finish(Job& job, const fic_params& p, fic_code* dst, int64_t cap, Launcher& L,
               cudaStream_t s);

    // Device bytes one slot needs for an N x N image (admission estimate).
    int64_t slot_bytes(int N, const fic_params& p) const;

    // Pool of one step of one image into slot's work (used by fic_domain_pool):
    // top > 0 selects the top-DN rule, else the threshold rule.
    int pool_only(int slot, const uint8_t* dimg, int N, int B, int L, double thr, int64_t top,
                  bool want_H, Launcher& Lk, cudaStream_t s, int64_t* dn, int64_t* near);
    ImageWork& work(int slot) { return *work_[(size_t)slot]; }
    Scalars* dev_scalars() { return scal_.as<Scalars>(); }
    const Scalars& host_scalars(int slot) const { return host_scal_[slot]; }
    int read_scalars(int n, cudaStream_t s);
    // The tuned shapes so far: (engine, K, |S|, size class) -> choice, ms.
    struct TuneEntry {
        int engine, K, ns, size_class;
        TuneChoice choice;
        float ms;
        int candidates;
    };
    // process-wide (every engine of the process shares the table)
    static std::vector<TuneEntry> tuned();
    // false: never run tuning trials inside step() (request server)
    void set_trials(bool allow) { allow_trials_ = allow; }

    // Graph-captured encodes (graph.cu).  encode_graph sets *used when it
    // encoded the images (the configuration was encoded eagerly before:
    // note_config after that eager encode records the shapes it used).
    int encode_graph(int n, const uint8_t* const* imgs, const int* Ns, const fic_params& p,
                     fic_code* const* dsts, const int64_t* caps, fic_result* outs,
                     cudaStream_t s, bool* used);
    void reset_used();
    void note_config(int n, const int* Ns, const fic_params& p);
    int64_t graph_captures() const { return graph_captures_; }
    int64_t graph_replays() const { return graph_replays_; }

private:
    int launch_pool(Job& j, int B, int L_step, double thr, int64_t top, bool want_H,
                    Launcher& L, cudaStream_t s);
    int sm_count_ = 0;
    bool ready_ = false;
    DevBuf entT_, scal_, probs_[FIC_MAX_LEVELS];
    Scalars* host_scal_ = nullptr;
    int scal_cap_ = 0;
    std::vector<std::unique_ptr<ImageWork>> work_;
    std::vector<Problem> table_;
    bool allow_trials_ = true;
    // shapes the last eager encode used per step
    TuneChoice used_choice_[FIC_MAX_LEVELS] = {};
    bool used_valid_[FIC_MAX_LEVELS] = {};
    struct Seen {
        TuneChoice choice[FIC_MAX_LEVELS];
        bool no_graph = false;  // capture failed: this configuration stays eager
    };
    struct GraphPlan;
    static constexpr size_t kMaxPlans = 4;
    std::map<std::string, Seen> seen_;
    std::vector<GraphPlan*> plans_;
    uint64_t plan_clock_ = 0;
    int64_t graph_captures_ = 0, graph_replays_ = 0;
    int graph_build(GraphPlan& G, cudaStream_t s);
    void drop_plans();
};

bool is_device_ptr(const void* p);

// Pool of one step: entropy -> flags (threshold rule, or the top-DN keys and
// a radix select) -> scan (size into ds->total) -> raster-order list in
// w->pool.  Buffers of w grow as needed.
int pool_launches(ImageWork* w, Scalars* ds, const long long* entT, const uint8_t* dimg, int N,
                  int B, int L_step, double thr, int64_t top, bool want_H, Launcher& L,
                  cudaStream_t s);

}  // namespace fic
