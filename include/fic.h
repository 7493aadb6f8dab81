/*
 * fic.h -- C ABI of the GB300 (sm_103a) range-domain block search of the
 * modified fast fractal image encoder (Salarian & Miar Naimi, arXiv
 * 1502.00324).
 *
 * What one encode computes (paper section in brackets):
 *   - ranges: non-overlapping B x B blocks of the N x N grey image, stored
 *     left to right, top to bottom [Sec. 2, Sec. 3.3];
 *   - domains: every 2B x 2B block at integer step L in x and y, decimated
 *     2x2 before comparison [Sec. 2]; the pool keeps the domains whose
 *     grey-level entropy is greater than a threshold [Abstract, Sec. 3,
 *     eq. 5-6];
 *   - for every range: every pool domain in each of the 8 isometries (0, 90,
 *     180, 270 degrees clockwise, and each mirrored) [Sec. 2], at each
 *     predefined contrast factor S of the step [Sec. 3.2], with the
 *     least-squares optimal offset O [eq. 3], scored by eq. 1; the best
 *     mapping is kept;
 *   - quadtree steps: a range whose RMS error exceeds the tolerance splits
 *     into four children for the next, smaller step; the last step stores
 *     its best mapping regardless [Sec. 2].
 *
 * Exactness: decimated domains are carried as 2x2 SUMS d' (0..1020) and
 * S = p/q, so 16 q^2 n E(S, O*) = 16 q^2 Vr - 8 p q Crd + p^2 Vd is an
 * exact integer (n = B*B, Vr = n sum r^2 - (sum r)^2,
 * Crd = n sum r d' - sum r sum d', Vd = n sum d'^2 - (sum d')^2).  Selection
 * is the lexicographic minimum of (score, pool index, isometry, S index);
 * the codes are therefore bit-exact across engines and against a CPU
 * reference.
 *
 * Memory and threads: every entry point is host-callable and synchronous
 * with respect to the host (it returns when its results are written).  GPU
 * work runs on the given CUDA stream (NULL = legacy default stream) of the
 * current device.  Pointers documented "host or device" are classified with
 * cudaPointerGetAttributes.  The library keeps one workspace per device and
 * context; calls that share a context must not overlap in time.
 *
 * Errors: every int-returning call returns FIC_OK (0) or a negative FIC_E*
 * code; fic_strerror() names it.  No call aborts the process.
 */
#ifndef FIC_H
#define FIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes                                                        */
/* ------------------------------------------------------------------ */
#define FIC_OK 0
#define FIC_EINVAL (-1)   /* bad argument: N % B_max != 0, B_min > B_max,
                             B not a power of two in {2,4,8,16}, L < 1,
                             err_tol outside [0, 255], bad S set (n_s < 1
                             or > FIC_MAX_S, q < 1 or > 256, p < 0 or
                             p > q), NULL pointer                         */
#define FIC_ENOMEM (-2)   /* device or host allocation failed            */
#define FIC_ECUDA (-3)    /* a CUDA runtime call or kernel failed        */
#define FIC_ETIMEOUT (-4) /* a bounded device-side wait gave up; the
                             kernel returned early and the context is
                             still usable                                */
#define FIC_EBUSY (-5)    /* server admission refused (no slot / memory) */
#define FIC_ENODEV (-6)   /* no CUDA device, or not compute capability
                             10.3 (sm_103a)                              */
#define FIC_ECAP (-7)     /* caller-provided output buffer too small;
                             the needed count is still reported           */
#define FIC_ENOTREADY (-8)/* server ticket not finished yet              */

#define FIC_MAX_LEVELS 4  /* quadtree steps: 16 -> 8 -> 4 -> 2 (Sec. 2)  */
#define FIC_MAX_S 16      /* contrast factors per step                   */

/* Contraction engine for the sum r d' term.                           */
#define FIC_ENGINE_TENSOR 0 /* tcgen05.mma kind::f16 (FP16 in, FP32 accum),
                               operands centred so every partial sum is an
                               integer below 2^24 (exact)                 */
#define FIC_ENGINE_PLAIN 1  /* CUDA-core int32 multiply-add              */

/* One step's contrast factors S_i = p[i] / q (Sec. 3.2: 16x16 {0.1},
 * 8x8 {0.2, 0.4}, 4x4 {0.3, 0.8}, 2x2 {0.5, 0.9}, i.e. q = 10). */
typedef struct {
    int32_t n_s;
    int32_t q;
    int32_t p[FIC_MAX_S];
} fic_sset;

/* One stored record per coded range (Sec. 3.3, Fig. 7).  16 bytes.
 * Positions are explicit for checking; pool_idx is the domain address (the
 * index in the step's domain list, Sec. 3.3, eq. 8).  The range side is
 * B_max >> level.  s_idx == 0xFF and pool_idx == 0xFFFFFFFF mark a
 * mean-only record (empty pool at the last step).  The decoded range mean
 * is 2 * o_q + 1. */
typedef struct {
    uint16_t rx, ry;     /* range top-left, pixels                       */
    uint16_t dx, dy;     /* domain top-left, pixels                      */
    uint32_t pool_idx;   /* domain address                                */
    uint8_t level;       /* quadtree step, 0 = B_max                      */
    uint8_t iso;         /* isometry 0..7: rot^k (k<4), mirror(rot^(k-4)) */
    uint8_t s_idx;       /* index into the step's S set                   */
    uint8_t o_q;         /* 7-bit range mean, min(127, floor(sum r/(2n))) */
} fic_code;

/* Encode result.  Codes are ordered by top-level range in raster order,
 * then depth-first in TL, TR, BL, BR order (the order of Sec. 3.3). */
typedef struct {
    fic_code* codes;                    /* host array unless the caller gave
                                           its own buffer                    */
    int64_t n_codes;
    int32_t n_levels;
    int32_t N;
    int32_t B_max;
    int32_t owns_codes;                 /* 1: free with fic_result_free      */
    fic_sset S_sets[FIC_MAX_LEVELS];    /* the S sets used, for decoding     */
    int64_t n_positions[FIC_MAX_LEVELS];/* domain positions per step         */
    int64_t pool_size[FIC_MAX_LEVELS];  /* admitted pool size DN per step    */
    int64_t ranges[FIC_MAX_LEVELS];     /* ranges searched per step          */
    int64_t matches[FIC_MAX_LEVELS];    /* ranges * DN * 8 per step          */
    int64_t near_thresh[FIC_MAX_LEVELS];/* positions with |H - thr| < 1e-9   */
} fic_result;

/* Full parameter set. */
typedef struct {
    int32_t N;               /* image side; N % B_max == 0                 */
    int32_t B_max, B_min;    /* range sides, powers of two in {2,4,8,16}   */
    int32_t L;               /* domain step >= 1                            */
    double entropy_thresh;   /* bits; < 0 admits every domain               */
    double err_tol;          /* RMS grey levels, quantised to 1/16          */
    fic_sset S_sets[FIC_MAX_LEVELS]; /* one per step, B_max first          */
    int32_t engine;          /* FIC_ENGINE_*                                */
    int32_t pool_dn;         /* 0: threshold pool (entropy > entropy_thresh);
                                > 0: top-DN pool, the pool_dn positions of
                                highest entropy [Sec. 3.2.1, Sec. 4], with
                                entropies rounded to 2^-20 bit and equal
                                ones taken in raster order (entropy_thresh
                                ignored); near_thresh then counts positions
                                whose rounding is ambiguous near the cut   */
} fic_params;

/* fic_encode -- encode one N x N uint8 image (row-major, pitch N).
 *   img      host or device pointer, caller-owned, read only.
 *   S_sets   host array, one fic_sset per quadtree step, B_max first.
 *   err_tol  split when RMS error > err_tol (ignored when B_max == B_min).
 *   out      host struct; out->codes is a host array allocated by the
 *            library (free with fic_result_free).
 *   stream   cudaStream_t or NULL.
 * Uses the tensor-core engine.  Returns FIC_OK or FIC_E*. */
int fic_encode(const uint8_t* img, int N, int B_max, int B_min, int L,
               double entropy_thresh, const fic_sset* S_sets, double err_tol,
               fic_result* out, void* stream);

/* fic_encode_ex -- as fic_encode with a full parameter set and an optional
 * caller-owned output buffer.
 *   codes_out  NULL: the library allocates a host array (out->owns_codes=1);
 *              else a host or device buffer of codes_cap records that
 *              receives the codes (out->codes = codes_out).  If it is too
 *              small the call returns FIC_ECAP with out->n_codes set. */
int fic_encode_ex(const uint8_t* img, const fic_params* p, fic_code* codes_out,
                  int64_t codes_cap, fic_result* out, void* stream);

/* fic_encode_batch -- encode n_img images of (possibly different) sides
 * Ns[i] with one parameter set (p->N is ignored; every Ns[i] must satisfy
 * the rules of p->N).  The images share each quadtree step: pools, gathers
 * and split decisions run per image, the range-domain contraction of a step
 * runs as ONE launch over the work of every image.  Each image's records
 * are identical to those of fic_encode_ex on that image alone.
 *   imgs   host array of n_img pointers, each host or device, N_i*N_i bytes.
 *   Ns     host array of n_img sides.
 *   outs   host array of n_img results; each outs[i].codes is a host array
 *          allocated by the library (free each with fic_result_free).
 * On error every outs[i] is left without codes.  The paper encodes one
 * image at a time (Sec. 3); batching is this library's serving form. */
int fic_encode_batch(int n_img, const uint8_t* const* imgs, const int* Ns,
                     const fic_params* p, fic_result* outs, void* stream);

/* fic_decode -- rebuild the image from a result on the GPU (Sec. 2): start
 * from a constant 128 image; each pass rebuilds every range from its domain
 * in the previous pass, pixel = clamp(round_half_up((2 o_q + 1) +
 * S (d - mean d)), 0, 255) with d = T_iso(d')/4; stop at a fixed point or
 * after iters_max passes.
 *   r          host struct from fic_encode*; r->codes host or device.
 *   out_img    host or device, N*N bytes, caller-owned.
 *   iters_used host, may be NULL. */
int fic_decode(const fic_result* r, int N, int iters_max, uint8_t* out_img,
               int* iters_used, void* stream);

/* fic_domain_pool -- kernels (a) and (b) alone: entropy of every 2B x 2B
 * domain position at step L (eq. 5-6, bits, FP64 from integer counts) and
 * the stable raster-order list of admitted positions (Sec. 3).
 *   pool_dn   0: admit entropy > entropy_thresh (< 0 admits all); > 0: the
 *             top-DN rule of fic_params.pool_dn.
 *   pool_xy   host, 2 * cap int32 (x, y pairs); may be NULL with cap 0.
 *   entropy   host, n_positions doubles, may be NULL.
 *   dn, near  host outputs (near: positions with |H - thr| < 1e-9, or with
 *             an ambiguous rounding near the top-DN cut).
 * Returns FIC_ECAP (with *dn set) when cap < DN. */
int fic_domain_pool(const uint8_t* img, int N, int B, int L, double entropy_thresh,
                    int64_t pool_dn, int32_t* pool_xy, int64_t cap, int64_t* dn,
                    double* entropy, int64_t* near, void* stream);

/* fic_domain_pool_noalloc -- fic_domain_pool for callers that cannot
 * allocate device memory.  The paper has no counterpart: this entry point
 * exists for deployment.  Some callers must not call cudaMalloc: code that
 * runs in a host callback, a plugin handed device buffers by its host
 * application, or a process that reserved all device memory up front.  This
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine); the caller passes device buffers for the input and the outputs,
 * and the intermediates live in one static device array of the library
 * (8,398,592 bytes = 8.0 MiB per GPU, held until the process exits).
 *   d_img      device, N*N bytes, read only.
 *   d_pool_xy  device, cap uint32 entries: admitted positions in raster
 *              order, packed x | (y << 16).  May be NULL with cap 0.
 *   dn, near   host outputs: pool size; positions with |H - thr| < 1e-9.
 *   d_entropy  device, n_positions doubles (eq. 5-6, bits), or NULL.
 * Returns FIC_EINVAL when N > 65535, when n_positions = ((N-2B)/L+1)^2
 * exceeds FIC_NOALLOC_MAX_POSITIONS or a buffer is not device memory,
 * FIC_ECAP (with *dn set) when cap < DN.  Every call looks the scratch's
 * device address up; the first call on each device (and the first after a
 * device reset) also fills a table with one kernel and waits for it: make
 * that call before any stream capture.  Calls share the scratch: calls that
 * overlap on the GPU race. */
#define FIC_NOALLOC_MAX_POSITIONS (1 << 20)
int fic_domain_pool_noalloc(const uint8_t* d_img, int N, int B, int L,
                            double entropy_thresh, uint32_t* d_pool_xy, int64_t cap,
                            int64_t* dn, double* d_entropy, int64_t* near, void* stream);

/* fic_pack -- the stored stream of an encode [Sec. 3.3, Fig. 7, eq. 8].
 * Records in their stored order (ranges implicit), each: step (2 bits),
 * range mean o_q (7 bits), and when the step's pool is not empty the
 * isometry (3 bits), the domain address (X = ceil(log2 DN) bits, eq. 8) and
 * the S index (ceil(log2 |S|) bits: none for a one-valued set).  Before the
 * records, a byte-aligned header carries what a decoder needs: "FIC1", u16
 * N, u8 B_max, u8 steps, u16 L, u8 pool rule (0 threshold, 1 top-DN), u32
 * records; per step u8 |S|, u16 q, |S| x u16 p, u32 DN (0 when no range
 * reached the step), u8 list form and the step's domain list (form 0: none
 * needed, empty pool or every position; 1: DN positions (x/L, y/L) of
 * ceil(log2 per) bits each; 2: a bitmap of the per^2 positions, whichever
 * is shorter, 1 on ties), padded to a byte.  Integers big-endian, fields
 * most significant bit first, the records padded to a byte at the end.
 *   img    the encoded image (host or device), to rebuild the domain lists
 *          with the encode's pool rule; p the encode's parameters (p->N is
 *          taken from r->N); r the result (codes host or device).
 *   out    host buffer of cap bytes, or NULL with cap 0 for the size only.
 *   n_bytes, payload_bits  host outputs (stream bytes; record bits alone).
 * Returns FIC_ECAP (with *n_bytes set) when cap < *n_bytes. */
int fic_pack(const uint8_t* img, const fic_params* p, const fic_result* r, uint8_t* out,
             int64_t cap, int64_t* n_bytes, int64_t* payload_bits, void* stream);

/* ------------------------------------------------------------------ */
/* Request server (continuous batching)                                */
/* ------------------------------------------------------------------ */
/* A server owns a worker thread, a CUDA stream and device workspaces on
 * the device current at creation.  Requests (images of any valid side,
 * one parameter set per server) wait in a FIFO queue; between quadtree
 * steps the worker admits queued images while a workspace slot is free
 * and the device bytes of the admitted images (an estimate per image from
 * N, B_max..B_min, L and the engine) stay within the HBM budget.  Each
 * worker iteration advances EVERY admitted image by one quadtree step,
 * whatever step it is at, with one grouped contraction launch per step
 * present (fic_encode_batch's engine), so images that arrive while others
 * are on the GPU join the next launch.  Pools, active ranges and partial
 * records stay on the device until an image's last step; then its records
 * are ordered and copied to a host array.  Each image's records are
 * identical to those of fic_encode_ex on that image alone.  The paper
 * encodes one image at a time (Sec. 3); the server is this library's
 * serving form. */
typedef struct fic_server fic_server;

typedef struct {
    int64_t hbm_budget;    /* device bytes for admitted images; 0 = half of
                              the free device memory at creation          */
    int32_t max_inflight;  /* admitted images at once (slots); 0 = 64      */
    int32_t max_queue;     /* waiting requests; 0 = 65536.  A submit
                              beyond it returns FIC_EBUSY                 */
    int32_t policy;        /* admission order: 0 FIFO; 1 smallest image
                              first, except that a request waiting longer
                              than age_ms goes first (oldest first)        */
    int32_t age_ms;        /* policy 1 aging limit; 0 = 2000 ms           */
} fic_server_config;

typedef struct {
    double submit_ms;      /* host steady clock, ms since server creation */
    double admit_ms;       /* taken from the queue onto the device         */
    double done_ms;        /* records on the host                          */
    int32_t steps;         /* worker iterations the image took part in     */
    int32_t shared_steps;  /* ... of which with other images in flight     */
} fic_timing;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t queued, inflight;          /* now                              */
    int64_t iterations;                /* worker iterations (steps)        */
    int64_t contraction_launches;
    double mean_inflight;              /* images per iteration, mean       */
    int64_t peak_inflight;
    int64_t hbm_in_use, hbm_peak;      /* estimated bytes held by slots    */
    int64_t hbm_budget;
    int64_t matches;                   /* (range, domain, isometry) total  */
    double busy_ms;                    /* worker time with images in flight*/
} fic_server_stats;

/* fic_server_create -- p: host, copied (p->N is ignored); cfg: host, may be
 * NULL.  *out receives the server.  Returns FIC_EINVAL for a bad parameter
 * set, FIC_ENODEV without an sm_103 device current. */
int fic_server_create(const fic_params* p, const fic_server_config* cfg, fic_server** out);
/* fic_server_submit -- queue one N x N image.  img: host pointer (copied
 * before return) or device pointer (NOT copied: its contents must be
 * complete on the device before the call, e.g. its producing stream
 * synchronised, and stay valid and unchanged until the ticket completes;
 * the server reads it from its own stream).  *ticket receives an id > 0.
 * FIC_EINVAL: N invalid for the parameter set; FIC_EBUSY: queue full, or
 * the server stopped (destroyed, or its worker failed: then every queued and
 * running request completes with FIC_ENOMEM). */
int fic_server_submit(fic_server* s, const uint8_t* img, int N, int64_t* ticket);
/* fic_server_poll -- wait up to wait_ms (0: do not wait, < 0: forever) for
 * a ticket.  FIC_OK: *out receives the result (host codes owned by the
 * caller: fic_result_free) and *timing (may be NULL) its times; the ticket
 * is then forgotten.  FIC_ENOTREADY: still queued or running.  A failed
 * encode returns its status once.  FIC_EINVAL: unknown ticket. */
int fic_server_poll(fic_server* s, int64_t ticket, int wait_ms, fic_result* out,
                    fic_timing* timing);
/* fic_server_stats_read -- counters since creation. */
int fic_server_stats_read(fic_server* s, fic_server_stats* out);
/* fic_server_destroy -- finish the images in flight, fail the queued ones,
 * stop the worker and free every resource (unpolled results included). */
int fic_server_destroy(fic_server* s);

/* Frees the library-owned parts of a result (the code array when
 * owns_codes).  Safe on a zeroed struct. */
void fic_result_free(fic_result* r);

/* Human-readable name of a status code (static string). */
const char* fic_strerror(int status);

/* ------------------------------------------------------------------ */
/* Contraction shape tuning                                            */
/* ------------------------------------------------------------------ */
/* The contraction of a quadtree step can run with several tile shapes that
 * give identical records: domain-side isometry tiles (128 ranges x 32 pool
 * domains x 8 isometries, the maximum over the isometries taken by the
 * tensor-memory load; 2x2 to 8x8 ranges with at most 3 S values),
 * isometry-in-accumulator tiles (128 ranges x 64 domains x 8 isometries,
 * same steps) or row tiles (128 (range, isometry) rows x 256 domains), each
 * with a work chunking tuned for a per-item refill cost of 1, 2 or 4 tiles,
 * and for isometry-in-accumulator tiles 8 or 16 epilogue warps.  In mode 1
 * (the default) the first step of each (engine, K = B*B padded, |S|, size
 * class = floor(log2(ranges x pool domains))) runs every candidate twice on
 * its own operands, timed with CUDA events, and keeps the fastest for that
 * class (one table per process, shared by the synchronous entry points and
 * the servers; a server never runs the candidates itself: a class without
 * an entry takes the nearest tuned class of the same (engine, K, |S|), else
 * the default).  Mode 0: the fixed default (domain-side isometry tiles
 * where they apply, refill 2); mode 2 + i: candidate i
 * for every step
 * (i taken modulo the step's candidate count).  The paper has no
 * counterpart; this is the GPU design's tile-shape choice. */
typedef struct {
    int32_t engine, K, n_s, size_class;  /* the class                      */
    int32_t iso_tiles;                   /* 0: row tiles; 1: isometry tiles; 2: domain-side
                                            isometries, maximum by the TMEM load */
    int32_t refill;                      /* chunking refill cost, tiles     */
    int32_t epi_warps;                   /* epilogue warps (isometry-in-
                                            accumulator tiles: 8 with 16-column
                                            TMEM reads, or 16 with 8-column
                                            reads; domain-side tiles: 8)   */
    float ms;                            /* measured contraction time       */
    int32_t candidates;                  /* shapes measured                 */
} fic_tune_entry;

/* fic_tune_mode -- set the mode (mode >= 0) and/or read the previous one
 * (previous may be NULL; mode < 0 only reads).  Process-wide. */
int fic_tune_mode(int mode, int* previous);
/* fic_tune_read -- the tuned classes so far: up to cap entries into out
 * (host), *n the total. */
int fic_tune_read(fic_tune_entry* out, int cap, int* n);

/* ------------------------------------------------------------------ */
/* Graph-captured encodes                                              */
/* ------------------------------------------------------------------ */
/* fic_encode, fic_encode_ex and fic_encode_batch run the whole quadtree of
 * a call (every step of every image, Sec. 2) as one CUDA graph once the same
 * configuration -- image sides, every parameter, the tuning mode, stage
 * timing on or off -- has been encoded before: the first call runs the
 * steps one by one (and tunes the contraction shapes), the next captures
 * the steps with the shapes that call used, later ones replay the graph.
 * Pool sizes, split counts and the contraction's work items stay in device
 * memory (kernels are launched for the largest possible counts and read the
 * actual ones), so the host waits once per call instead of once per step.
 * Records are identical either way.  The library keeps the graphs of the 4
 * most recently used configurations, each with its own device buffers.
 *
 * fic_graph_mode -- mode 1 (default): as above; mode 0: steps one by one
 * always.  mode < 0 only reads; previous may be NULL.  Process-wide. */
int fic_graph_mode(int mode, int* previous);
/* fic_graph_counts -- graphs captured and replayed by the synchronous entry
 * points on the current device (either pointer may be NULL). */
int fic_graph_counts(int64_t* captures, int64_t* replays);

/* ------------------------------------------------------------------ */
/* Instrumentation                                                     */
/* ------------------------------------------------------------------ */
#define FIC_K_ENTROPY 0
#define FIC_K_SCAN 1
#define FIC_K_GATHER 2
#define FIC_K_RANGE_PREP 3
#define FIC_K_CONTRACT_TC 4
#define FIC_K_CONTRACT_PLAIN 5
#define FIC_K_SPLIT 6
#define FIC_K_ORDER 7
#define FIC_K_DECODE 8
#define FIC_K_MISC 9
#define FIC_K_COUNT 10

typedef struct {
    int64_t launches[FIC_K_COUNT];  /* kernel launches per kind            */
    double ms[FIC_K_COUNT];         /* summed CUDA-event time per kind
                                       (only while timing is enabled)      */
    double flops[FIC_K_COUNT];      /* algorithmic flops: 2 * M * N * K of
                                       the contraction (M = 8 ranges,
                                       N = DN, K = B*B), summed            */
    double bytes[FIC_K_COUNT];      /* algorithmic DRAM bytes, summed      */
    int64_t matches;                /* (range, pool domain, isometry)      */
} fic_stats;

/* Zero the counters; enable (1) or disable (0) per-kernel CUDA-event
 * timing.  Events are recorded on the stream each kernel runs on. */
int fic_stats_reset(int timing);
/* Copy the counters accumulated since the last reset. */
int fic_stats_read(fic_stats* out);

/* Library build string (compiled architectures and version). */
const char* fic_version(void);

/* Name and text of the last CUDA error behind a FIC_ECUDA / FIC_ENOMEM
 * returned on this thread ("" if none).  Static per-thread storage. */
const char* fic_last_error(void);

/* fic_wait_selftest -- a check of the library's failure handling; the paper
 * has no counterpart.  Runs the bounded mbarrier wait that every tensor-core
 * kernel uses, in a one-warp kernel on the current device:
 *   complete      nonzero: the barrier's phase completes before the wait
 *                 (the wait succeeds); 0: nothing ever arrives, so the wait
 *                 runs until its limit and gives up.
 *   limit_cycles  the wait's limit in SM clock cycles, 1 ..
 *                 FIC_SELFTEST_MAX_CYCLES (about 2 s at 2 GHz); the clock is
 *                 read every 16 polls of at most 1 ms each.
 *   stream        CUDA stream (NULL = default); the call synchronises it.
 * Returns FIC_OK when the wait saw the phase, FIC_ETIMEOUT when it gave up
 * (the kernel returned early and the context stays usable, as after an
 * encode's timeout), FIC_EINVAL for a limit out of range, FIC_ENODEV without
 * an sm_103 device, FIC_ECUDA on a CUDA error.  The error word is shared by
 * all calls: calls that overlap on the GPU race. */
#define FIC_SELFTEST_MAX_CYCLES 4000000000LL
int fic_wait_selftest(int complete, int64_t limit_cycles, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FIC_H */
