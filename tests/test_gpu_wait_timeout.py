"""Failure handling of the tensor kernels' bounded waits, made to expire
without a fault.  fic_wait_selftest runs the same bounded mbarrier wait as
the contraction kernels, on a barrier whose phase never completes (nothing
arrives).  The wait must give up at its limit, the call must return
FIC_ETIMEOUT promptly, and the context must stay usable: the same wait on a
completing barrier succeeds afterwards and an encode still gives the oracle's
records."""
from __future__ import annotations

import time

import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes

pytestmark = pytest.mark.gpu

LIMIT = 2_000_000   # SM cycles: about 1 ms at 2 GHz


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


def test_bounded_wait_expires_and_the_context_survives(pkg):
    import torch
    f = pkg.fic
    s = torch.cuda.current_stream()
    assert f.fic_wait_selftest(True, LIMIT, s) == f.FIC_OK
    t0 = time.perf_counter()
    st = f.fic_wait_selftest(False, LIMIT, s)
    waited = time.perf_counter() - t0
    assert st == f.FIC_ETIMEOUT
    assert waited < 5.0, waited
    assert f.fic_wait_selftest(True, LIMIT, s) == f.FIC_OK
    img = fic_synth.one_over_f(64, 0)
    ss = pkg.paper_ssets(16, 4)
    want, _ = oracle.encode(img, 16, 4, 2, 3.0, ss, 6.0)
    enc = pkg.fic_encode_ex(torch.from_numpy(img).cuda(), 64, 16, 4, 2, 3.0, ss, 6.0, stream=s)
    assert_same_codes(enc.codes, want, 16, "encode after a wait timeout")


def test_wait_limit_out_of_range_is_rejected(pkg):
    f = pkg.fic
    assert f.fic_wait_selftest(False, 0) == f.FIC_EINVAL
    assert f.fic_wait_selftest(False, 4_000_000_001) == f.FIC_EINVAL
