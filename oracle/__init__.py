"""ctypes front end of the CPU oracle (oracle/fic_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product package.  The
oracle follows the paper's algorithm step by step in plain loops (see the C
file's header for the steps and the readings of open points).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

MAX_S = 16
MAX_LEVELS = 5


class OrCode(C.Structure):
    _fields_ = [("rx", C.c_int32), ("ry", C.c_int32), ("level", C.c_int32),
                ("B", C.c_int32), ("iso", C.c_int32), ("s_idx", C.c_int32),
                ("o_q", C.c_int32), ("dx", C.c_int32), ("dy", C.c_int32),
                ("pool_idx", C.c_uint32), ("score", C.c_int64)]


class OrSset(C.Structure):
    _fields_ = [("n_s", C.c_int), ("q", C.c_int), ("p", C.c_int * MAX_S)]


class OrPool(C.Structure):
    _fields_ = [("B", C.c_int), ("L", C.c_int), ("n_pos", C.c_int), ("dn", C.c_int64),
                ("x", C.POINTER(C.c_int32)), ("y", C.POINTER(C.c_int32)),
                ("dsum", C.POINTER(C.c_int32)), ("sum_d", C.POINTER(C.c_int64)),
                ("sum_d2", C.POINTER(C.c_int64)), ("near_thresh", C.c_int64)]


class OrStats(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("pool_size", C.c_int64 * MAX_LEVELS),
                ("ranges", C.c_int64 * MAX_LEVELS), ("near_thresh", C.c_int64 * MAX_LEVELS)]


CODE_DTYPE = np.dtype([("rx", np.int32), ("ry", np.int32), ("level", np.int32),
                       ("B", np.int32), ("iso", np.int32), ("s_idx", np.int32),
                       ("o_q", np.int32), ("dx", np.int32), ("dy", np.int32),
                       ("pool_idx", np.uint32), ("score", np.int64)])
assert CODE_DTYPE.itemsize == C.sizeof(OrCode)

_lib = None
_path = None


def use_library(path):
    """Load the build of the oracle at ``path`` instead of the default one.
    Only the pins' mutation test does this, passing a copy with a planted
    mistake explicitly (pytest's --oracle-lib option); it must come before
    the first call into the oracle."""
    global _path
    if _lib is not None:
        raise RuntimeError("the oracle library is already loaded")
    _path = os.path.abspath(path)


def lib():
    """The compiled oracle (built from oracle/fic_oracle.c on first use)."""
    global _lib
    if _lib is None:
        path = _path or _build()
        L = C.CDLL(path)
        u8p = C.POINTER(C.c_uint8)
        i32p = C.POINTER(C.c_int32)
        i64p = C.POINTER(C.c_int64)
        L.or_isometry.argtypes = [i32p, C.c_int, C.c_int, i32p]
        L.or_decimate.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int, i32p]
        L.or_entropy_bits.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_entropy_bits.restype = C.c_double
        L.or_score.argtypes = [i32p, i32p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_score.restype = C.c_int64
        L.or_positions_per_axis.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_pool_build.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(OrPool)]
        L.or_pool_build_ex.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64,
                                       C.POINTER(OrPool)]
        L.or_pool_free.argtypes = [C.POINTER(OrPool)]
        L.or_search_range.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.POINTER(OrPool),
                                      C.POINTER(OrSset), i64p, i64p, i32p, i32p]
        L.or_search_ranges.argtypes = [u8p, C.c_int, C.c_int64, i32p, i32p, C.POINTER(OrPool),
                                       C.POINTER(OrSset), C.c_int, i64p, i64p, i32p, i32p]
        L.or_encode.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64,
                                C.POINTER(OrSset), C.c_double, C.c_int, C.POINTER(OrCode),
                                C.c_int64, i64p, C.POINTER(OrStats)]
        L.or_decode.argtypes = [C.POINTER(OrCode), C.c_int64, C.POINTER(OrSset), C.c_int,
                                C.c_int, u8p, C.POINTER(C.c_int)]
        L.or_psnr.argtypes = [u8p, u8p, C.c_int64]
        L.or_psnr.restype = C.c_double
        L.or_address_bits.argtypes = [C.c_int64]
        L.or_max_threads.restype = C.c_int
        L.or_pack.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64,
                              C.POINTER(OrSset), i64p, C.POINTER(OrCode), C.c_int64, u8p,
                              C.c_int64, i64p]
        L.or_pack.restype = C.c_int64
        L.or_unpack.argtypes = [u8p, C.c_int64, C.POINTER(OrCode), C.c_int64, i64p,
                                C.POINTER(OrSset), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int)]
        _lib = L
    return _lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint8))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def make_ssets(ssets):
    """ssets: list of (q, [p...]) per level -> ctypes array of OrSset."""
    arr = (OrSset * MAX_LEVELS)()
    for i, (q, ps) in enumerate(ssets):
        arr[i].n_s = len(ps)
        arr[i].q = q
        for j, p in enumerate(ps):
            arr[i].p[j] = p
    return arr


def isometry(block, k):
    b, bp = _i32(block)
    B = b.shape[0]
    out = np.empty_like(b)
    lib().or_isometry(bp, B, k, out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def decimate(img, x, y, B):
    a, ap = _u8(img)
    out = np.empty((B, B), np.int32)
    lib().or_decimate(ap, a.shape[0], x, y, B, out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def entropy_bits(img, x, y, size):
    a, ap = _u8(img)
    return lib().or_entropy_bits(ap, a.shape[0], x, y, size)


def score(r, dsum, k, p, q):
    rr, rp = _i32(r)
    dd, dp = _i32(dsum)
    return int(lib().or_score(rp, dp, rr.shape[0], k, p, q))


def positions_per_axis(N, B, L):
    return int(lib().or_positions_per_axis(N, B, L))


class Pool:
    """A step's domain pool (positions in raster order and decimated blocks).
    ``dn_top`` > 0: the dn_top highest-entropy positions (ties in raster
    order) instead of the threshold rule."""

    def __init__(self, img, B, L, thr, dn_top=0):
        self._img, ap = _u8(img)
        self.N = self._img.shape[0]
        self._p = OrPool()
        rc = lib().or_pool_build_ex(ap, self.N, B, L, thr, int(dn_top), C.byref(self._p))
        if rc:
            raise MemoryError("oracle pool build failed")
        self.B, self.L = B, L

    @property
    def dn(self):
        return int(self._p.dn)

    @property
    def near_thresh(self):
        return int(self._p.near_thresh)

    def positions(self):
        n = self.dn
        if n == 0:
            return np.zeros((0, 2), np.int32)
        x = np.ctypeslib.as_array(self._p.x, shape=(n,)).copy()
        y = np.ctypeslib.as_array(self._p.y, shape=(n,)).copy()
        return np.stack([x, y], axis=1)

    def search(self, rx, ry, sset, nthreads=0):
        """Best (score, pool_idx, iso, s_idx) for each range top-left (rx, ry)."""
        rx = np.atleast_1d(np.asarray(rx, np.int32))
        ry = np.atleast_1d(np.asarray(ry, np.int32))
        n = rx.shape[0]
        sc = np.empty(n, np.int64)
        pi = np.empty(n, np.int64)
        iso = np.empty(n, np.int32)
        si = np.empty(n, np.int32)
        ss = make_ssets([sset])
        _, ap = _u8(self._img)
        lib().or_search_ranges(ap, self.N, n, rx.ctypes.data_as(C.POINTER(C.c_int32)),
                               ry.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(self._p),
                               C.byref(ss[0]), nthreads,
                               sc.ctypes.data_as(C.POINTER(C.c_int64)),
                               pi.ctypes.data_as(C.POINTER(C.c_int64)),
                               iso.ctypes.data_as(C.POINTER(C.c_int32)),
                               si.ctypes.data_as(C.POINTER(C.c_int32)))
        return sc, pi, iso, si

    def __del__(self):
        try:
            lib().or_pool_free(C.byref(self._p))
        except Exception:
            pass


def encode(img, B_max, B_min, L, entropy_thresh, ssets, err_tol, nthreads=0, pool_dn=0):
    """Full oracle encode.  Returns (codes structured array, stats dict).
    ``pool_dn`` > 0 selects the top-DN pool rule at every step."""
    a, ap = _u8(img)
    N = a.shape[0]
    ss = make_ssets(ssets)
    st = OrStats()
    n_out = C.c_int64(0)
    cap = 1024
    while True:
        buf = (OrCode * cap)()
        rc = lib().or_encode(ap, N, B_max, B_min, L, entropy_thresh, int(pool_dn), ss, err_tol,
                             nthreads,
                             buf, cap, C.byref(n_out), C.byref(st))
        if rc == -2:
            cap = int(n_out.value)
            continue
        if rc:
            raise ValueError(f"oracle encode rejected the arguments (rc={rc})")
        break
    n = int(n_out.value)
    codes = np.frombuffer(bytearray(buf)[: n * CODE_DTYPE.itemsize], dtype=CODE_DTYPE).copy()
    stats = dict(n_levels=st.n_levels,
                 pool_size=[st.pool_size[i] for i in range(st.n_levels)],
                 ranges=[st.ranges[i] for i in range(st.n_levels)],
                 near_thresh=[st.near_thresh[i] for i in range(st.n_levels)])
    return codes, stats


def decode(codes, ssets, N, iters_max=64):
    codes = np.ascontiguousarray(codes, dtype=CODE_DTYPE)
    ss = make_ssets(ssets)
    out = np.empty((N, N), np.uint8)
    used = C.c_int(0)
    rc = lib().or_decode(codes.ctypes.data_as(C.POINTER(OrCode)), codes.shape[0], ss, N,
                         iters_max, out.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(used))
    if rc:
        raise MemoryError("oracle decode failed")
    return out, int(used.value)


def psnr(a, b):
    a, ap = _u8(a)
    b, bp = _u8(b)
    return float(lib().or_psnr(ap, bp, a.size))


def address_bits(dn):
    return int(lib().or_address_bits(dn))


def max_threads():
    return int(lib().or_max_threads())


def pack(img, codes, B_max, n_levels, L, entropy_thresh, ssets, searched, pool_dn=0):
    """The stored stream (Sec. 3.3, Fig. 7, eq. 8) of oracle records:
    (bytes, payload bits).  searched[l]: ranges searched at step l (steps no
    range reached carry DN = 0)."""
    a, ap = _u8(img)
    codes = np.ascontiguousarray(codes, dtype=CODE_DTYPE)
    ss = make_ssets(ssets)
    sr = (C.c_int64 * 4)(*[int(v) for v in list(searched) + [0] * (4 - len(searched))])
    pb = C.c_int64(0)
    need = lib().or_pack(ap, a.shape[0], B_max, n_levels, L, float(entropy_thresh), int(pool_dn),
                         ss, sr, codes.ctypes.data_as(C.POINTER(OrCode)), codes.shape[0], None,
                         0, C.byref(pb))
    if need < 0:
        raise ValueError("oracle pack rejected the arguments")
    out = np.zeros(need, np.uint8)
    lib().or_pack(ap, a.shape[0], B_max, n_levels, L, float(entropy_thresh), int(pool_dn), ss, sr,
                  codes.ctypes.data_as(C.POINTER(OrCode)), codes.shape[0],
                  out.ctypes.data_as(C.POINTER(C.c_uint8)), need, C.byref(pb))
    return out.tobytes(), int(pb.value)


def unpack(stream):
    """Records, S sets and geometry from a stream written by pack()."""
    buf = np.frombuffer(stream, np.uint8).copy()
    n = C.c_int64(0)
    ss = (OrSset * MAX_LEVELS)()
    N, Bm, nl = C.c_int(0), C.c_int(0), C.c_int(0)
    cap = 1024
    while True:
        out = (OrCode * cap)()
        rc = lib().or_unpack(buf.ctypes.data_as(C.POINTER(C.c_uint8)), buf.size, out, cap,
                             C.byref(n), ss, C.byref(N), C.byref(Bm), C.byref(nl))
        if rc == -2:
            cap = int(n.value)
            continue
        if rc:
            raise ValueError("malformed stream")
        break
    k = int(n.value)
    codes = np.frombuffer(bytearray(out)[: k * CODE_DTYPE.itemsize], dtype=CODE_DTYPE).copy()
    ssets = [(ss[i].q, [ss[i].p[j] for j in range(ss[i].n_s)]) for i in range(nl.value)]
    return codes, ssets, int(N.value), int(Bm.value)
