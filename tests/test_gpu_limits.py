"""The largest sizes the device code accepts (the limits themselves are
checked on the host in tests/test_lib_cpu.py).

The device-wide scan takes at most 4096 tiles of 4096 elements; a 4096 x
4096 image at B = 4, L = 1 has 4089^2 = 16,719,921 domain positions, 4082
tiles of the scan, the largest threshold pool below the limit.  Its pool
list, entropies and near-threshold count must equal the oracle's."""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


def test_largest_threshold_pool_below_the_scan_limit(pkg):
    N, B, L, thr = 4096, 4, 1, 5.0
    img = fic_synth.one_over_f(N, 77, 2.0)
    xy, H, near = pkg.fic_domain_pool(img, N, B, L, thr)
    per = N - 2 * B + 1
    assert H.shape == (per * per,)
    pool = oracle.Pool(img, B, L, thr)
    want = pool.positions()
    assert 0 < len(want) < per * per            # a mixed pool, not all or nothing
    assert len(xy) == len(want)
    np.testing.assert_array_equal(xy, want)
    assert near == pool.near_thresh
    rng = np.random.default_rng(3)
    for i in rng.choice(per * per, 4000, replace=False):
        y, x = divmod(int(i), per)
        assert abs(H[i] - oracle.entropy_bits(img, x * L, y * L, 2 * B)) < 1e-12, (x, y)
