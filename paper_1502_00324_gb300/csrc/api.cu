// api.cu -- C ABI of the range-domain search (include/fic.h): the per-device
// engine of the synchronous entry points, the encoders (one image, a batch),
// the decoder, the domain pool and instrumentation.  The quadtree step driver
// itself is engine.cu; the request server is server.cu.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "fic.h"
#include "kernels.h"

namespace fic {
namespace {

// Per-device state of the synchronous entry points (one call at a time per
// device; concurrent callers serialise on the mutex).
struct Context {
    std::mutex mu;
    Engine eng;
    DevBuf dec0, dec1, dcodes, pack_sizes, pack_offs, pack_words;
};

// Most-significant-bit-first writer of the stored stream's header.
struct BitWriter {
    std::vector<uint8_t> buf;
    int64_t bit = 0;
    void put(uint64_t v, int nb)
    {
        for (int i = nb - 1; i >= 0; --i) {
            if ((bit >> 3) >= (int64_t)buf.size()) buf.push_back(0);
            if ((v >> i) & 1u) buf[(size_t)(bit >> 3)] |= (uint8_t)(0x80u >> (bit & 7));
            ++bit;
        }
    }
    void align()
    {
        while (bit & 7) put(0, 1);
    }
};

int ceil_log2(int64_t v)
{
    int x = 0;
    while (((int64_t)1 << x) < v) ++x;
    return x;
}

std::mutex g_ctx_mu;
Context* g_ctx[64] = {};

int get_context(Context** out, cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIC_ENODEV;
    if (dev < 0 || dev >= 64) return FIC_ENODEV;
    std::lock_guard<std::mutex> g(g_ctx_mu);
    if (!g_ctx[dev]) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return FIC_ENODEV;
        if (major != 10 || minor != 3) return FIC_ENODEV;
        std::unique_ptr<Context> c(new Context());
        const int st = c->eng.init(s);
        if (st) return st;
        g_ctx[dev] = c.release();
    }
    *out = g_ctx[dev];
    return FIC_OK;
}

bool valid_side(int b) { return b == 2 || b == 4 || b == 8 || b == 16; }

// Encode n images with one parameter set: jobs in slots 0 .. n-1, stepped
// together until every quadtree is finished, then ordered and copied out.
int encode_jobs(Context* c, int n, const uint8_t* const* imgs, const int* Ns,
                const fic_params& p, fic_code* const* dsts, const int64_t* caps, fic_result* outs,
                cudaStream_t s)
{
    Engine& E = c->eng;
    // a configuration encoded before replays its captured graph
    bool used = false;
    int st = E.encode_graph(n, imgs, Ns, p, dsts, caps, outs, s, &used);
    if (used) {
        if (st && st != FIC_ECAP) return st;
        FIC_TRY(cudaStreamSynchronize(s));
        return st;
    }
    if (st) return st;
    E.reset_used();
    st = E.ensure_slots(n);
    if (st) return st;
    Launcher L(s);
    std::vector<Job> jobs((size_t)n);
    std::vector<Job*> ptrs;
    for (int i = 0; i < n; ++i) {
        st = E.begin(jobs[(size_t)i], i, imgs[i], Ns[i], p, L, s);
        if (st) return st;
        ptrs.push_back(&jobs[(size_t)i]);
    }
    for (;;) {
        bool any = false;
        for (const Job& j : jobs) any |= !j.done;
        if (!any) break;
        st = E.step(p, ptrs, L, s);
        if (st) return st;
    }
    int cap_status = FIC_OK;
    for (int i = 0; i < n; ++i) {
        Job& j = jobs[(size_t)i];
        st = E.finish(j, p, dsts ? dsts[i] : nullptr, caps ? caps[i] : 0, L, s);
        outs[i] = j.res;
        if (st == FIC_ECAP) {
            cap_status = FIC_ECAP;
            continue;
        }
        if (st) return st;
    }
    FIC_TRY(cudaStreamSynchronize(s));
    E.note_config(n, Ns, p);
    return cap_status;
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
    if (!img || !p || !out) return FIC_EINVAL;
    int nl = 0;
    if (validate_params(p, p->N, &nl)) return FIC_EINVAL;
    memset(out, 0, sizeof(*out));
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Context* c = nullptr;
        int st = get_context(&c, s);
        if (st) return st;
        std::lock_guard<std::mutex> guard(c->mu);
        const uint8_t* imgs[1] = {img};
        const int Ns[1] = {p->N};
        fic_code* dsts[1] = {codes_out};
        const int64_t caps[1] = {codes_cap};
        st = encode_jobs(c, 1, imgs, Ns, *p, codes_out ? dsts : nullptr, caps, out, s);
        if (st && st != FIC_ECAP) fic_result_free(out);
        return st;
    } catch (...) {
        return FIC_ENOMEM;
    }
}

int fic_encode_batch(int n_img, const uint8_t* const* imgs, const int* Ns, const fic_params* p,
                     fic_result* outs, void* stream)
{
    if (n_img < 0 || (n_img > 0 && (!imgs || !Ns || !p || !outs))) return FIC_EINVAL;
    if (n_img == 0) return FIC_OK;
    for (int i = 0; i < n_img; ++i) {
        int nl = 0;
        if (!imgs[i] || validate_params(p, Ns[i], &nl)) return FIC_EINVAL;
    }
    memset(outs, 0, sizeof(fic_result) * (size_t)n_img);
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Context* c = nullptr;
        int st = get_context(&c, s);
        if (st) return st;
        std::lock_guard<std::mutex> guard(c->mu);
        st = encode_jobs(c, n_img, imgs, Ns, *p, nullptr, nullptr, outs, s);
        if (st) {
            for (int i = 0; i < n_img; ++i) fic_result_free(&outs[i]);
        }
        return st;
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
    if (!valid_side(r->B_max)) return FIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Context* c = nullptr;
    int st = get_context(&c, s);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    DecodeS ds;
    memset(&ds, 0, sizeof(ds));
    ds.B_max = r->B_max;
    for (int l = 0; l < FIC_MAX_LEVELS; ++l) {
        ds.q[l] = r->S_sets[l].q > 0 ? r->S_sets[l].q : 1;
        for (int i = 0; i < FIC_MAX_S; ++i) ds.p[l][i] = r->S_sets[l].p[i];
    }
    st = c->eng.ensure_slots(1);
    if (st) return st;
    const void* dcodes = r->codes;
    if (r->n_codes > 0 && !is_device_ptr(r->codes)) {
        FIC_TRY(c->dcodes.ensure(sizeof(fic_code) * r->n_codes));
        FIC_TRY(cudaMemcpyAsync(c->dcodes.p, r->codes, sizeof(fic_code) * r->n_codes,
                                cudaMemcpyHostToDevice, s));
        dcodes = c->dcodes.p;
    }
    const size_t npx = (size_t)N * N;
    FIC_TRY(c->dec0.ensure(npx));
    FIC_TRY(c->dec1.ensure(npx));
    uint8_t* cur = c->dec0.as<uint8_t>();
    uint8_t* nxt = c->dec1.as<uint8_t>();
    FIC_TRY(cudaMemsetAsync(cur, 128, npx, s));
    Scalars* dsc = c->eng.dev_scalars();
    Launcher L(s);
    int used = 0;
    while (used < iters_max) {
        FIC_TRY(cudaMemsetAsync(&dsc->changed, 0, sizeof(unsigned), s));
        FIC_TRY(cudaMemcpyAsync(nxt, cur, npx, cudaMemcpyDeviceToDevice, s));
        L.begin(FIC_K_DECODE);
        FIC_TRY(launch_decode_pass(dcodes, r->n_codes, ds, cur, nxt, N, &dsc->changed, s));
        L.end(1, 0.0, (double)npx * 2.0);
        st = c->eng.read_scalars(1, s);
        if (st) return st;
        ++used;
        uint8_t* t = cur;
        cur = nxt;
        nxt = t;
        if (!c->eng.host_scalars(0).changed) break;
    }
    FIC_TRY(cudaMemcpyAsync(out_img, cur, npx, cudaMemcpyDefault, s));
    FIC_TRY(cudaStreamSynchronize(s));
    if (iters_used) *iters_used = used;
    return FIC_OK;
}

int fic_domain_pool(const uint8_t* img, int N, int B, int L, double entropy_thresh,
                    int64_t pool_dn, int32_t* pool_xy, int64_t cap, int64_t* dn,
                    double* entropy, int64_t* near, void* stream)
{
    g_last_error[0] = '\0';
    if (!img || !dn || N <= 0 || N > 65535 || !valid_side(B) || L < 1 || pool_dn < 0)
        return FIC_EINVAL;
    const int64_t per_axis = positions_per_axis(N, B, L);
    if (per_axis * per_axis > kMaxScanCount) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "%lld domain positions exceed the scan limit of %lld",
                 (long long)(per_axis * per_axis), (long long)kMaxScanCount);
        return FIC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Context* c = nullptr;
    int st = get_context(&c, s);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    st = c->eng.ensure_slots(1);
    if (st) return st;
    ImageWork& w = c->eng.work(0);
    const uint8_t* dimg = img;
    if (!is_device_ptr(img)) {
        FIC_TRY(w.img.ensure((size_t)N * N));
        FIC_TRY(cudaMemcpyAsync(w.img.p, img, (size_t)N * N, cudaMemcpyHostToDevice, s));
        dimg = w.img.as<uint8_t>();
    }
    const int per = positions_per_axis(N, B, L);
    const int64_t npos = (int64_t)per * per;
    Launcher Lk(s);
    // entropy is evaluated for every position; a negative threshold admits all
    int64_t d = 0, nr = 0;
    st = c->eng.pool_only(0, dimg, N, B, L, entropy_thresh < 0.0 ? -1.0e300 : entropy_thresh,
                          pool_dn, entropy != nullptr, Lk, s, &d, &nr);
    if (st) return st;
    *dn = d;
    if (near) *near = (entropy_thresh < 0.0 && pool_dn == 0) ? 0 : nr;
    if (entropy && npos > 0)
        FIC_TRY(cudaMemcpyAsync(entropy, w.H.p, sizeof(double) * npos, cudaMemcpyDeviceToHost, s));
    if (pool_xy && cap >= d && d > 0) {
        std::vector<uint32_t> tmp((size_t)d);
        FIC_TRY(cudaMemcpyAsync(tmp.data(), w.pool.p, sizeof(uint32_t) * d,
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

int fic_pack(const uint8_t* img, const fic_params* p, const fic_result* r, uint8_t* out,
             int64_t cap, int64_t* n_bytes, int64_t* payload_bits, void* stream)
{
    if (!img || !p || !r || !n_bytes || cap < 0 || (cap > 0 && !out)) return FIC_EINVAL;
    fic_params prm = *p;
    prm.N = r->N;
    int nl = 0;
    if (validate_params(&prm, prm.N, &nl) || nl != r->n_levels || prm.L > 65535) return FIC_EINVAL;
    if (r->n_codes < 0 || (r->n_codes > 0 && !r->codes)) return FIC_EINVAL;
    // record bits stay below 2^32 (at most 48 bits per record)
    if (r->n_codes > ((int64_t)1 << 32) / 48) return FIC_EINVAL;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Context* c = nullptr;
        int st = get_context(&c, s);
        if (st) return st;
        std::lock_guard<std::mutex> guard(c->mu);
        Engine& E = c->eng;
        st = E.ensure_slots(1);
        if (st) return st;
        ImageWork& w = E.work(0);
        const int N = prm.N;
        const uint8_t* dimg = img;
        if (!is_device_ptr(img)) {
            FIC_TRY(w.img.ensure((size_t)N * N));
            FIC_TRY(cudaMemcpyAsync(w.img.p, img, (size_t)N * N, cudaMemcpyHostToDevice, s));
            dimg = w.img.as<uint8_t>();
        }
        Launcher Lk(s);
        BitWriter bw;
        for (const char ch : {'F', 'I', 'C', '1'}) bw.put((uint64_t)ch, 8);
        bw.put((uint64_t)N, 16);
        bw.put((uint64_t)prm.B_max, 8);
        bw.put((uint64_t)nl, 8);
        bw.put((uint64_t)prm.L, 16);
        bw.put(prm.pool_dn > 0 ? 1u : 0u, 8);
        bw.put((uint64_t)r->n_codes, 32);
        PackLevels pl;
        memset(&pl, 0, sizeof(pl));
        const bool listed = prm.pool_dn > 0 || prm.entropy_thresh >= 0.0;
        std::vector<uint32_t> list;
        for (int l = 0; l < nl; ++l) {
            const fic_sset& ss = prm.S_sets[l];
            bw.put((uint64_t)ss.n_s, 8);
            bw.put((uint64_t)ss.q, 16);
            for (int i = 0; i < ss.n_s; ++i) bw.put((uint64_t)ss.p[i], 16);
            const int B = prm.B_max >> l;
            const int per = positions_per_axis(N, B, prm.L);
            const int64_t npos = (int64_t)per * per;
            int64_t dn = 0;
            list.clear();
            if (r->ranges[l] > 0) {
                if (listed) {
                    int64_t near = 0;
                    st = E.pool_only(0, dimg, N, B, prm.L,
                                     prm.pool_dn > 0 ? -1.0 : prm.entropy_thresh, prm.pool_dn,
                                     false, Lk, s, &dn, &near);
                    if (st) return st;
                    list.resize((size_t)dn);
                    if (dn > 0) {
                        FIC_TRY(cudaMemcpyAsync(list.data(), w.pool.p, sizeof(uint32_t) * dn,
                                                cudaMemcpyDeviceToHost, s));
                        FIC_TRY(cudaStreamSynchronize(s));
                    }
                } else {
                    dn = npos;
                }
            }
            // the result must come from this image and these parameters
            if (dn != (r->ranges[l] > 0 ? r->pool_size[l] : 0)) return FIC_EINVAL;
            bw.put((uint64_t)dn, 32);
            const int pw = ceil_log2(per);
            int form = 0;
            if (dn > 0 && dn < npos) form = (dn * 2 * pw <= npos) ? 1 : 2;
            bw.put((uint64_t)form, 8);
            if (form == 1) {
                for (int64_t i = 0; i < dn; ++i) {
                    bw.put((list[(size_t)i] & 0xffffu) / (uint32_t)prm.L, pw);
                    bw.put((list[(size_t)i] >> 16) / (uint32_t)prm.L, pw);
                }
            } else if (form == 2) {
                int64_t k = 0;
                for (int64_t i = 0; i < npos; ++i) {
                    const uint32_t xy = (uint32_t)((i % per) * prm.L) |
                                        ((uint32_t)((i / per) * prm.L) << 16);
                    const bool in = k < dn && list[(size_t)k] == xy;
                    if (in) ++k;
                    bw.put(in ? 1u : 0u, 1);
                }
            }
            bw.align();
            pl.has_pool[l] = dn > 0;
            pl.addr_bits[l] = ceil_log2(dn);
            pl.s_bits[l] = ceil_log2(ss.n_s);
        }
        // the records, on the GPU
        const int64_t n = r->n_codes;
        const void* dcodes = r->codes;
        if (n > 0 && !is_device_ptr(r->codes)) {
            FIC_TRY(c->dcodes.ensure(sizeof(fic_code) * n));
            FIC_TRY(cudaMemcpyAsync(c->dcodes.p, r->codes, sizeof(fic_code) * n,
                                    cudaMemcpyHostToDevice, s));
            dcodes = c->dcodes.p;
        }
        const int64_t n_words = (n * 48 + 31) / 32 + 1;
        FIC_TRY(c->pack_sizes.ensure(sizeof(uint32_t) * (n ? n : 1)));
        FIC_TRY(c->pack_offs.ensure(sizeof(uint32_t) * (n ? n : 1)));
        FIC_TRY(c->pack_words.ensure(sizeof(uint32_t) * n_words));
        FIC_TRY(w.scan_tmp.ensure(sizeof(uint32_t) * scan_tmp_words(n ? n : 1)));
        Scalars* ds = E.dev_scalars();
        Lk.begin(FIC_K_MISC);
        FIC_TRY(launch_pack_records(dcodes, n, pl, c->pack_sizes.as<uint32_t>(),
                                    c->pack_offs.as<uint32_t>(), w.scan_tmp.as<uint32_t>(),
                                    &ds->total, c->pack_words.as<uint32_t>(), n_words, s));
        Lk.end(4, 0.0, (double)n * 24.0);
        st = E.read_scalars(1, s);
        if (st) return st;
        const int64_t bits = E.host_scalars(0).total;
        const int64_t head = (int64_t)bw.buf.size();
        const int64_t total = head + (bits + 7) / 8;
        *n_bytes = total;
        if (payload_bits) *payload_bits = bits;
        if (!out) return FIC_OK;
        if (cap < total) return FIC_ECAP;
        std::vector<uint32_t> words((size_t)((bits + 31) / 32));
        if (!words.empty()) {
            FIC_TRY(cudaMemcpyAsync(words.data(), c->pack_words.p, sizeof(uint32_t) * words.size(),
                                    cudaMemcpyDeviceToHost, s));
            FIC_TRY(cudaStreamSynchronize(s));
        }
        memcpy(out, bw.buf.data(), (size_t)head);
        for (int64_t k = 0; k < (bits + 7) / 8; ++k)
            out[head + k] = (uint8_t)(words[(size_t)(k >> 2)] >> (24 - 8 * (k & 3)));
        return FIC_OK;
    } catch (...) {
        return FIC_ENOMEM;
    }
}

int fic_tune_mode(int mode, int* previous)
{
    if (previous) *previous = tune_mode();
    if (mode >= 0) set_tune_mode(mode);
    return FIC_OK;
}

int fic_graph_mode(int mode, int* previous)
{
    if (mode > 1) return FIC_EINVAL;
    if (previous) *previous = graph_mode();
    if (mode >= 0) set_graph_mode(mode);
    return FIC_OK;
}

int fic_graph_counts(int64_t* captures, int64_t* replays)
{
    Context* c = nullptr;
    int st = get_context(&c, nullptr);
    if (st) return st;
    std::lock_guard<std::mutex> guard(c->mu);
    if (captures) *captures = c->eng.graph_captures();
    if (replays) *replays = c->eng.graph_replays();
    return FIC_OK;
}

int fic_tune_read(fic_tune_entry* out, int cap, int* n)
{
    if (!n || cap < 0 || (cap > 0 && !out)) return FIC_EINVAL;
    Context* c = nullptr;
    int st = get_context(&c, nullptr);
    if (st) return st;
    const auto t = Engine::tuned();
    *n = (int)t.size();
    for (int i = 0; i < cap && i < (int)t.size(); ++i) {
        out[i].engine = t[(size_t)i].engine;
        out[i].K = t[(size_t)i].K;
        out[i].n_s = t[(size_t)i].ns;
        out[i].size_class = t[(size_t)i].size_class;
        out[i].iso_tiles = t[(size_t)i].choice.iso;
        out[i].refill = t[(size_t)i].choice.refill;
        out[i].epi_warps = t[(size_t)i].choice.iso ? (t[(size_t)i].choice.epi ? 16 : 8) : 8;
        out[i].ms = t[(size_t)i].ms;
        out[i].candidates = t[(size_t)i].candidates;
    }
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
