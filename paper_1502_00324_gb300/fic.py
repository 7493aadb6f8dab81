"""Thin ctypes binding of libfic.so (include/fic.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  If the library is missing the import of a function raises;
there is no fallback path.  PyTorch is used only to hand over device memory
and streams (``data_ptr()``, ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfic.so")

FIC_OK = 0
FIC_EINVAL = -1
FIC_ENOMEM = -2
FIC_ECUDA = -3
FIC_ETIMEOUT = -4
FIC_EBUSY = -5
FIC_ENODEV = -6
FIC_ECAP = -7
FIC_ENOTREADY = -8
MAX_LEVELS = 4
MAX_S = 16
ENGINE_TENSOR = 0
ENGINE_PLAIN = 1
KERNEL_KINDS = ["entropy", "scan", "gather", "range_prep", "contract_tc", "contract_plain",
                "split", "order", "decode", "misc"]


class FicSset(C.Structure):
    _fields_ = [("n_s", C.c_int32), ("q", C.c_int32), ("p", C.c_int32 * MAX_S)]


class FicCode(C.Structure):
    _fields_ = [("rx", C.c_uint16), ("ry", C.c_uint16), ("dx", C.c_uint16), ("dy", C.c_uint16),
                ("pool_idx", C.c_uint32), ("level", C.c_uint8), ("iso", C.c_uint8),
                ("s_idx", C.c_uint8), ("o_q", C.c_uint8)]


class FicResult(C.Structure):
    _fields_ = [("codes", C.POINTER(FicCode)), ("n_codes", C.c_int64), ("n_levels", C.c_int32),
                ("N", C.c_int32), ("B_max", C.c_int32), ("owns_codes", C.c_int32),
                ("S_sets", FicSset * MAX_LEVELS), ("n_positions", C.c_int64 * MAX_LEVELS),
                ("pool_size", C.c_int64 * MAX_LEVELS), ("ranges", C.c_int64 * MAX_LEVELS),
                ("matches", C.c_int64 * MAX_LEVELS), ("near_thresh", C.c_int64 * MAX_LEVELS)]


class FicParams(C.Structure):
    _fields_ = [("N", C.c_int32), ("B_max", C.c_int32), ("B_min", C.c_int32), ("L", C.c_int32),
                ("entropy_thresh", C.c_double), ("err_tol", C.c_double),
                ("S_sets", FicSset * MAX_LEVELS), ("engine", C.c_int32),
                ("pool_dn", C.c_int32)]


class FicServerConfig(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("max_inflight", C.c_int32), ("max_queue", C.c_int32),
                ("policy", C.c_int32), ("age_ms", C.c_int32)]


class FicTiming(C.Structure):
    _fields_ = [("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double),
                ("steps", C.c_int32), ("shared_steps", C.c_int32)]


class FicServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int64), ("inflight", C.c_int64), ("iterations", C.c_int64),
                ("contraction_launches", C.c_int64), ("mean_inflight", C.c_double),
                ("peak_inflight", C.c_int64), ("hbm_in_use", C.c_int64), ("hbm_peak", C.c_int64),
                ("hbm_budget", C.c_int64), ("matches", C.c_int64), ("busy_ms", C.c_double)]


class FicTuneEntry(C.Structure):
    _fields_ = [("engine", C.c_int32), ("K", C.c_int32), ("n_s", C.c_int32),
                ("size_class", C.c_int32), ("iso_tiles", C.c_int32), ("refill", C.c_int32),
                ("epi_warps", C.c_int32), ("ms", C.c_float), ("candidates", C.c_int32)]


class FicStats(C.Structure):
    _fields_ = [("launches", C.c_int64 * 10), ("ms", C.c_double * 10),
                ("flops", C.c_double * 10), ("bytes", C.c_double * 10), ("matches", C.c_int64)]


CODE_DTYPE = np.dtype([("rx", np.uint16), ("ry", np.uint16), ("dx", np.uint16),
                       ("dy", np.uint16), ("pool_idx", np.uint32), ("level", np.uint8),
                       ("iso", np.uint8), ("s_idx", np.uint8), ("o_q", np.uint8)])
assert CODE_DTYPE.itemsize == C.sizeof(FicCode) == 16

EXPORTS = ["fic_encode", "fic_encode_ex", "fic_encode_batch", "fic_decode", "fic_domain_pool", "fic_result_free",
           "fic_strerror", "fic_stats_reset", "fic_stats_read", "fic_version",
           "fic_domain_pool_noalloc", "fic_last_error", "fic_pack", "fic_tune_mode",
           "fic_tune_read", "fic_graph_mode", "fic_graph_counts", "fic_server_create", "fic_server_submit",
           "fic_server_poll", "fic_server_stats_read", "fic_server_destroy", "fic_wait_selftest"]


class FicError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        detail = ""
        if status in (FIC_ECUDA, FIC_ENOMEM, FIC_EINVAL):
            text = lib().fic_last_error().decode()
            detail = " [" + text + "]" if text else ""
        super().__init__(f"{what}: {strerror(status)} ({status}){detail}")


_lib = None


def lib():
    """Load libfic.so (built by paper_1502_00324_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libfic.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.fic_encode.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                             C.POINTER(FicSset), C.c_double, C.POINTER(FicResult), vp]
    L.fic_encode_ex.argtypes = [vp, C.POINTER(FicParams), vp, C.c_int64, C.POINTER(FicResult), vp]
    L.fic_encode_batch.argtypes = [C.c_int, vp, vp, C.POINTER(FicParams), C.POINTER(FicResult),
                                   vp]
    L.fic_decode.argtypes = [C.POINTER(FicResult), C.c_int, C.c_int, vp, C.POINTER(C.c_int), vp]
    L.fic_domain_pool.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64,
                                  C.POINTER(C.c_int32), C.c_int64, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int64), vp]
    L.fic_result_free.argtypes = [C.POINTER(FicResult)]
    L.fic_result_free.restype = None
    L.fic_strerror.argtypes = [C.c_int]
    L.fic_strerror.restype = C.c_char_p
    L.fic_stats_reset.argtypes = [C.c_int]
    L.fic_stats_read.argtypes = [C.POINTER(FicStats)]
    L.fic_version.restype = C.c_char_p
    L.fic_last_error.restype = C.c_char_p
    L.fic_domain_pool_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, vp,
                                          C.c_int64, C.POINTER(C.c_int64), vp,
                                          C.POINTER(C.c_int64), vp]
    L.fic_pack.argtypes = [vp, C.POINTER(FicParams), C.POINTER(FicResult), vp, C.c_int64,
                           C.POINTER(C.c_int64), C.POINTER(C.c_int64), vp]
    L.fic_tune_mode.argtypes = [C.c_int, C.POINTER(C.c_int)]
    L.fic_tune_read.argtypes = [C.POINTER(FicTuneEntry), C.c_int, C.POINTER(C.c_int)]
    L.fic_graph_mode.argtypes = [C.c_int, C.POINTER(C.c_int)]
    L.fic_graph_counts.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.fic_server_create.argtypes = [C.POINTER(FicParams), C.POINTER(FicServerConfig),
                                    C.POINTER(vp)]
    L.fic_server_submit.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int64)]
    L.fic_server_poll.argtypes = [vp, C.c_int64, C.c_int, C.POINTER(FicResult),
                                  C.POINTER(FicTiming)]
    L.fic_server_stats_read.argtypes = [vp, C.POINTER(FicServerStats)]
    L.fic_server_destroy.argtypes = [vp]
    L.fic_wait_selftest.argtypes = [C.c_int, C.c_int64, vp]
    _lib = L
    return L


def strerror(status: int) -> str:
    return lib().fic_strerror(status).decode()


def _check(st, what):
    if st != FIC_OK:
        raise FicError(st, what)


def _buf(x, what, min_bytes=0, u8=False, itemsize=None):
    """(address, keepalive, bytes) of a C-contiguous numpy array or torch
    tensor.  The library reads and writes these buffers by the sizes passed
    beside them, so a strided view, an image of another element type or a
    buffer shorter than ``min_bytes`` is refused here: it would otherwise be
    read or written past its end, on the host or on the device."""
    if isinstance(x, np.ndarray):
        contig, nbytes, isz = x.flags.c_contiguous, x.nbytes, x.itemsize
        is_u8 = x.dtype == np.uint8
        addr = x.ctypes.data
    elif hasattr(x, "data_ptr"):
        contig, isz = x.is_contiguous(), x.element_size()
        nbytes = x.numel() * isz
        is_u8 = str(x.dtype) == "torch.uint8"
        addr = x.data_ptr()
    else:
        raise TypeError(f"{what}: expected a numpy array or torch tensor, got {type(x)}")
    if not contig:
        raise ValueError(f"{what}: the buffer must be C-contiguous")
    if u8 and not is_u8:
        raise TypeError(f"{what}: expected uint8 elements, got {x.dtype}")
    if itemsize is not None and isz != itemsize:
        raise TypeError(f"{what}: expected {itemsize}-byte elements, got {x.dtype}")
    if nbytes < min_bytes:
        raise ValueError(f"{what}: {nbytes} bytes, at least {min_bytes} needed")
    return addr, x, nbytes


def _square_side(img, what):
    """Side of a square 2-D image (batch and server take N from the shape)."""
    if len(img.shape) != 2 or img.shape[0] != img.shape[1]:
        raise ValueError(f"{what}: expected a square 2-D image, got shape {tuple(img.shape)}")
    return int(img.shape[0])


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def make_ssets(ssets):
    """[(q, [p...]), ...] (one per quadtree step) -> FicSset array."""
    arr = (FicSset * MAX_LEVELS)()
    if len(ssets) > MAX_LEVELS:
        raise ValueError(f"{len(ssets)} S sets, at most {MAX_LEVELS} quadtree steps")
    for i, (q, ps) in enumerate(ssets):
        if len(ps) > MAX_S:
            raise ValueError(f"S set {i}: {len(ps)} values, at most {MAX_S}")
        arr[i].n_s = len(ps)
        arr[i].q = q
        for j, p in enumerate(ps):
            arr[i].p[j] = p
    return arr


class Encoded:
    """Result of an encode: codes (numpy structured array on the host, or the
    caller's device buffer) plus per-step counters."""

    def __init__(self, res: FicResult, codes):
        self._res = res
        self.codes = codes
        nl = res.n_levels
        self.N = res.N
        self.n_codes = int(res.n_codes)
        self.n_levels = nl
        self.n_positions = [int(res.n_positions[i]) for i in range(nl)]
        self.pool_size = [int(res.pool_size[i]) for i in range(nl)]
        self.ranges = [int(res.ranges[i]) for i in range(nl)]
        self.matches = [int(res.matches[i]) for i in range(nl)]
        self.near_thresh = [int(res.near_thresh[i]) for i in range(nl)]

    @property
    def total_matches(self):
        return sum(self.matches)


def make_params(N, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine=ENGINE_TENSOR,
                pool_dn=0):
    """fic_params; pool_dn > 0 selects the top-DN pool instead of the
    entropy threshold."""
    p = FicParams()
    p.N, p.B_max, p.B_min, p.L = N, B_max, B_min, L
    p.entropy_thresh = float(entropy_thresh)
    p.err_tol = float(err_tol)
    p.S_sets = make_ssets(ssets)
    p.engine = engine
    p.pool_dn = int(pool_dn)
    return p


def fic_encode_ex(img, N, B_max, B_min, L, entropy_thresh, ssets, err_tol,
                  engine=ENGINE_TENSOR, stream=None, codes_out=None, pool_dn=0):
    """Encode one N x N uint8 image (numpy array, or torch tensor on the host
    or the GPU).  ``codes_out``: optional torch/numpy buffer of 16-byte
    records receiving the codes (host or device); otherwise a host array is
    returned."""
    p = make_params(N, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine, pool_dn)
    ip, keep, _ = _buf(img, "img", N * N, u8=True)
    res = FicResult()
    if codes_out is not None:
        cp, keep2, nb = _buf(codes_out, "codes_out")
        cap = nb // 16
        st = lib().fic_encode_ex(ip, C.byref(p), cp, cap, C.byref(res), _stream(stream))
        _check(st, "fic_encode_ex")
        return Encoded(res, codes_out)
    st = lib().fic_encode_ex(ip, C.byref(p), None, 0, C.byref(res), _stream(stream))
    _check(st, "fic_encode_ex")
    return _adopt(res)


def fic_encode_batch(imgs, B_max, B_min, L, entropy_thresh, ssets, err_tol,
                     engine=ENGINE_TENSOR, stream=None, pool_dn=0):
    """Encode a list of square uint8 images (numpy arrays or torch tensors,
    host or GPU, sides may differ) in one batched call; returns one Encoded
    per image."""
    n = len(imgs)
    if n == 0:
        return []
    p = make_params(0, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine, pool_dn)
    ptrs = (C.c_void_p * n)()
    Ns = (C.c_int * n)()
    keep = []
    for i, im in enumerate(imgs):
        side = _square_side(im, f"imgs[{i}]")
        ip, k, _ = _buf(im, f"imgs[{i}]", side * side, u8=True)
        keep.append(k)
        ptrs[i] = ip
        Ns[i] = side
    outs = (FicResult * n)()
    st = lib().fic_encode_batch(n, C.cast(ptrs, C.c_void_p), C.cast(Ns, C.c_void_p), C.byref(p),
                                outs, _stream(stream))
    _check(st, "fic_encode_batch")
    res = []
    for i in range(n):
        res.append(_adopt(FicResult.from_buffer_copy(outs[i])))
    return res


def _adopt(res: FicResult) -> Encoded:
    """Copy library-owned host codes into numpy and free the library array;
    the result then points at the numpy copy (for fic_decode)."""
    n = int(res.n_codes)
    codes = np.empty(n, CODE_DTYPE)
    if n:
        C.memmove(codes.ctypes.data, res.codes, n * 16)
    lib().fic_result_free(C.byref(res))
    res.codes = C.cast(C.c_void_p(codes.ctypes.data), C.POINTER(FicCode))
    res.owns_codes = 0
    res.n_codes = n
    out = Encoded(res, codes)
    out._keep = codes
    return out


def fic_encode(img, N, B_max, B_min, L, entropy_thresh, ssets, err_tol, stream=None):
    """fic_encode of include/fic.h (tensor-core engine, host codes)."""
    ip, keep, _ = _buf(img, "img", N * N, u8=True)
    res = FicResult()
    ss = make_ssets(ssets)
    st = lib().fic_encode(ip, N, B_max, B_min, L, float(entropy_thresh), ss, float(err_tol),
                          C.byref(res), _stream(stream))
    _check(st, "fic_encode")
    return _adopt(res)


def fic_pack(img, enc: Encoded, B_max, B_min, L, entropy_thresh, ssets, err_tol,
             engine=ENGINE_TENSOR, pool_dn=0, stream=None):
    """The stored stream of an encode (bytes) and its record bits alone; the
    arguments after ``enc`` are the encode's parameters."""
    p = make_params(enc.N, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine, pool_dn)
    ip, keep, _ = _buf(img, "img", enc.N * enc.N, u8=True)
    nb = C.c_int64(0)
    pb = C.c_int64(0)
    _check(lib().fic_pack(ip, C.byref(p), C.byref(enc._res), None, 0, C.byref(nb), C.byref(pb),
                          _stream(stream)), "fic_pack")
    out = np.zeros(max(int(nb.value), 1), np.uint8)
    _check(lib().fic_pack(ip, C.byref(p), C.byref(enc._res), out.ctypes.data, out.size,
                          C.byref(nb), C.byref(pb), _stream(stream)), "fic_pack")
    return out[: int(nb.value)].tobytes(), int(pb.value)


def fic_decode(enc: Encoded, iters_max=64, out=None, stream=None):
    """GPU decode of an Encoded result; returns (image, passes used)."""
    N = enc.N
    if out is None:
        out = np.empty((N, N), np.uint8)
    op, keep, _ = _buf(out, "out", N * N, u8=True)
    used = C.c_int(0)
    st = lib().fic_decode(C.byref(enc._res), N, iters_max, op, C.byref(used), _stream(stream))
    _check(st, "fic_decode")
    return out, int(used.value)


def fic_domain_pool(img, N, B, L, entropy_thresh, stream=None, pool_dn=0):
    """Kernels (a)+(b) alone: (pool positions (DN, 2), entropy per position,
    near-threshold count); pool_dn > 0: the top-DN rule."""
    ip, keep, _ = _buf(img, "img", N * N, u8=True)
    per = (N - 2 * B) // L + 1 if N >= 2 * B else 0
    npos = per * per
    ent = np.empty(max(npos, 1), np.float64)
    xy = np.empty((max(npos, 1), 2), np.int32)
    dn = C.c_int64(0)
    near = C.c_int64(0)
    st = lib().fic_domain_pool(ip, N, B, L, float(entropy_thresh), int(pool_dn),
                               xy.ctypes.data_as(C.POINTER(C.c_int32)), npos, C.byref(dn),
                               ent.ctypes.data_as(C.POINTER(C.c_double)), C.byref(near),
                               _stream(stream))
    _check(st, "fic_domain_pool")
    return xy[: dn.value].copy(), ent[:npos].copy(), int(near.value)


def fic_tune_mode(mode=-1):
    """Set the contraction-shape tuning mode (0 fixed, 1 measure on first
    use, 2 + i force candidate i); returns the previous mode."""
    prev = C.c_int(0)
    _check(lib().fic_tune_mode(int(mode), C.byref(prev)), "fic_tune_mode")
    return prev.value


def fic_graph_mode(mode=-1):
    """Set the graph mode (1: a configuration encoded before replays its
    captured graph; 0: steps one by one); returns the previous mode."""
    prev = C.c_int(0)
    _check(lib().fic_graph_mode(int(mode), C.byref(prev)), "fic_graph_mode")
    return prev.value


def fic_graph_counts():
    """(graphs captured, graph replays) of the synchronous entry points."""
    cap, rep = C.c_int64(0), C.c_int64(0)
    _check(lib().fic_graph_counts(C.byref(cap), C.byref(rep)), "fic_graph_counts")
    return cap.value, rep.value


def fic_tune_read():
    """The tuned classes so far (list of dicts)."""
    n = C.c_int(0)
    _check(lib().fic_tune_read(None, 0, C.byref(n)), "fic_tune_read")
    arr = (FicTuneEntry * max(n.value, 1))()
    _check(lib().fic_tune_read(arr, n.value, C.byref(n)), "fic_tune_read")
    return [{k: getattr(arr[i], k) for k, _ in FicTuneEntry._fields_} for i in range(n.value)]


def fic_stats_reset(timing=False):
    _check(lib().fic_stats_reset(1 if timing else 0), "fic_stats_reset")


def fic_stats_read():
    s = FicStats()
    _check(lib().fic_stats_read(C.byref(s)), "fic_stats_read")
    return {k: dict(launches=int(s.launches[i]), ms=float(s.ms[i]), flops=float(s.flops[i]),
                    bytes=float(s.bytes[i])) for i, k in enumerate(KERNEL_KINDS)} | {
        "matches": int(s.matches)}


def fic_wait_selftest(complete, limit_cycles, stream=None):
    """The tensor kernels' bounded mbarrier wait on its own (include/fic.h):
    returns the library status, FIC_OK when the phase completed, FIC_ETIMEOUT
    when the wait gave up at its limit."""
    return lib().fic_wait_selftest(1 if complete else 0, int(limit_cycles), _stream(stream))


def fic_version():
    return lib().fic_version().decode()


def fic_domain_pool_noalloc(d_img, N, B, L, entropy_thresh, d_pool_xy, d_entropy=None,
                            stream=None):
    """fic_domain_pool for callers that cannot allocate device memory: all
    buffers are the caller's device tensors (``d_pool_xy``: int32/uint32
    tensor receiving packed x | y << 16; ``d_entropy``: float64 tensor or
    None).  Returns (pool size, near-threshold count)."""
    ip, keep, _ = _buf(d_img, "d_img", N * N, u8=True)
    pp, keep2, nb = _buf(d_pool_xy, "d_pool_xy", itemsize=4)
    cap = nb // 4
    ep = None
    if d_entropy is not None:
        per = (N - 2 * B) // L + 1 if N >= 2 * B and L > 0 else 0
        ep, keep3, _ = _buf(d_entropy, "d_entropy", 8 * per * per, itemsize=8)
    dn = C.c_int64(0)
    near = C.c_int64(0)
    st = lib().fic_domain_pool_noalloc(ip, N, B, L, float(entropy_thresh), pp, cap, C.byref(dn),
                                       ep, C.byref(near), _stream(stream))
    _check(st, "fic_domain_pool_noalloc")
    return int(dn.value), int(near.value)


class Server:
    """Request server of include/fic.h (continuous batching on the current
    device).  ``submit`` takes a square uint8 image (numpy: copied by the
    library; torch CUDA tensor: kept referenced here until its ticket is
    polled) and returns a ticket; ``poll`` returns (Encoded, timing dict),
    or None while the image is queued or running."""

    def __init__(self, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine=ENGINE_TENSOR,
                 hbm_budget=0, max_inflight=0, max_queue=0, pool_dn=0, policy=0, age_ms=0):
        self._p = make_params(B_max, B_max, B_min, L, entropy_thresh, ssets, err_tol, engine,
                              pool_dn)
        cfg = FicServerConfig(int(hbm_budget), int(max_inflight), int(max_queue), int(policy),
                              int(age_ms))
        h = C.c_void_p()
        _check(lib().fic_server_create(C.byref(self._p), C.byref(cfg), C.byref(h)),
               "fic_server_create")
        self._h = h
        self._keep = {}

    def submit(self, img):
        side = _square_side(img, "img")
        ip, keep, _ = _buf(img, "img", side * side, u8=True)
        t = C.c_int64(0)
        st = lib().fic_server_submit(self._h, ip, side, C.byref(t))
        _check(st, "fic_server_submit")
        if not isinstance(img, np.ndarray):
            self._keep[t.value] = keep
        return t.value

    def poll(self, ticket, wait_ms=-1):
        res = FicResult()
        tm = FicTiming()
        st = lib().fic_server_poll(self._h, int(ticket), int(wait_ms), C.byref(res), C.byref(tm))
        if st == FIC_ENOTREADY:
            return None
        self._keep.pop(ticket, None)
        _check(st, "fic_server_poll")
        timing = {k: getattr(tm, k) for k, _ in FicTiming._fields_}
        return _adopt(res), timing

    def stats(self):
        s = FicServerStats()
        _check(lib().fic_server_stats_read(self._h, C.byref(s)), "fic_server_stats_read")
        return {k: getattr(s, k) for k, _ in FicServerStats._fields_}

    def close(self):
        if self._h:
            lib().fic_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
