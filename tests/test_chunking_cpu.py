"""Host checks of the contraction's work chunking (csrc/chunking.cuh): the
eager step driver runs it on the host, the graph-captured plan kernel runs
the alone case as a parallel search on the device.  Both must pick the
same chunk count, the smallest one of least estimated makespan (waves x
(tiles per item + refill)), so that a replayed graph launches the same work
items as the eager steps."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r"""
#define __host__
#define __device__
#include "chunking.cuh"
extern "C" {
long long mc(int sm, long long mt, long long ct) { return fic::max_chunks(sm, mt, ct); }
void alone(int sm, long long mt, long long ct, int refill, int* nc, int* per)
{ fic::choose_chunks_alone(sm, mt, ct, refill, nc, per); }
void shared(int sm, long long mt, long long ct, double tpi, int* nc, int* per)
{ fic::choose_chunks_shared(sm, mt, ct, tpi, nc, per); }
}
"""


@pytest.fixture(scope="module")
def chunking():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    lib = os.path.join(d, "libshim.so")
    with open(src, "w") as f:
        f.write(SHIM)
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-std=c++17",
                    "-I" + os.path.join(ROOT, "paper_1502_00324_gb300", "csrc"), src, "-o", lib],
                   check=True)
    L = C.CDLL(lib)
    L.mc.restype = C.c_longlong
    L.mc.argtypes = [C.c_int, C.c_longlong, C.c_longlong]
    L.alone.argtypes = [C.c_int, C.c_longlong, C.c_longlong, C.c_int, C.POINTER(C.c_int),
                        C.POINTER(C.c_int)]
    L.shared.argtypes = [C.c_int, C.c_longlong, C.c_longlong, C.c_double, C.POINTER(C.c_int),
                         C.POINTER(C.c_int)]
    return L


def device_rule(sm, mt, ct, refill, max_nc):
    """The plan kernel's search restated: integer cost, smallest count on ties."""
    best, best_nc = None, None
    for nc in range(1, max_nc + 1):
        per = -(-ct // nc)
        if -(-ct // per) != nc:
            continue
        waves = -(-(mt * nc) // sm)
        cost = waves * (per + refill)
        if best is None or cost < best:
            best, best_nc = cost, nc
    return best_nc, -(-ct // best_nc)


def test_alone_matches_the_device_search(chunking):
    rng = np.random.default_rng(3)
    cases = [(152, 1, 1, 1), (152, 1, 3985, 2), (152, 117, 3985, 4), (152, 31, 3864, 2),
             (152, 64, 904, 4), (148, 2000, 5000, 1)]
    cases += [(int(rng.choice([148, 152])), int(rng.integers(1, 3000)),
               int(rng.integers(1, 6000)), int(rng.choice([1, 2, 4]))) for _ in range(300)]
    for sm, mt, ct, refill in cases:
        nc, per = C.c_int(0), C.c_int(0)
        chunking.alone(sm, mt, ct, refill, C.byref(nc), C.byref(per))
        max_nc = chunking.mc(sm, mt, ct)
        assert (nc.value, per.value) == device_rule(sm, mt, ct, refill, max_nc), (sm, mt, ct)
        # every chunk holds at least one column tile, together all of them
        assert 1 <= nc.value <= max_nc
        assert nc.value * per.value >= ct and (nc.value - 1) * per.value < ct


def test_shared_chunks_cover_the_tiles(chunking):
    rng = np.random.default_rng(4)
    for _ in range(300):
        sm = int(rng.choice([148, 152]))
        mt, ct = int(rng.integers(1, 3000)), int(rng.integers(1, 6000))
        tpi = float(rng.uniform(0.1, 400.0))
        nc, per = C.c_int(0), C.c_int(0)
        chunking.shared(sm, mt, ct, tpi, C.byref(nc), C.byref(per))
        assert 1 <= nc.value <= chunking.mc(sm, mt, ct)
        assert nc.value * per.value >= ct and (nc.value - 1) * per.value < ct


def test_partial_best_bound(chunking):
    """Ranges x chunks stays within 2048 SMs + R + 128 (the partial-best
    buffers of a captured plan are sized by it), for both M-tile layouts."""
    for sm in (148, 152):
        for R in list(range(1, 300)) + [1024, 3912, 14896, 16384, 65536, 262144]:
            for ranges_per_mtile in (16, 128):
                mt = -(-R // ranges_per_mtile)
                for ct in (1, 7, 768, 5000):
                    assert R * chunking.mc(sm, mt, ct) <= 2048 * sm + R + 128
