"""The contraction-shape tuner: every candidate shape gives the same records,
and tuning keeps one of the measured candidates per class."""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes

pytestmark = pytest.mark.gpu

PAPER_S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    prev = p.fic_tune_mode(-1)
    yield p
    p.fic_tune_mode(prev)


CASES = [
    dict(N=128, B_max=16, B_min=4, L=1, thr=-1.0, dn=0, tol=8.0, seed=2),
    dict(N=96, B_max=8, B_min=2, L=2, thr=4.0, dn=0, tol=10.0, seed=3),
    dict(N=128, B_max=16, B_min=2, L=2, thr=-1.0, dn=64, tol=12.0, seed=4),
]


@pytest.mark.parametrize("case", CASES, ids=["16-4_full", "8-2_thr", "16-2_top64"])
def test_every_shape_gives_the_oracle_records(pkg, case):
    img = fic_synth.with_step_edges(case["N"], case["seed"], alpha=2.5)
    sides = []
    b = case["B_max"]
    while b >= case["B_min"]:
        sides.append(b)
        b //= 2
    ss = [PAPER_S[s] for s in sides]
    want, _ = oracle.encode(img, case["B_max"], case["B_min"], case["L"], case["thr"], ss,
                            case["tol"], pool_dn=case["dn"])
    outs = []
    for mode in (0, 2, 3, 4, 5, 6, 7, 8):
        pkg.fic_tune_mode(mode)
        enc = pkg.fic_encode_ex(img, case["N"], case["B_max"], case["B_min"], case["L"],
                                case["thr"], ss, case["tol"], pool_dn=case["dn"])
        assert_same_codes(enc.codes, want, case["B_max"], f"mode {mode}")
        outs.append(enc.codes)
    pkg.fic_tune_mode(1)
    for e in (pkg.ENGINE_TENSOR, pkg.ENGINE_PLAIN):
        enc = pkg.fic_encode_ex(img, case["N"], case["B_max"], case["B_min"], case["L"],
                                case["thr"], ss, case["tol"], engine=e, pool_dn=case["dn"])
        np.testing.assert_array_equal(enc.codes, outs[0])


def test_tuned_classes_are_recorded(pkg):
    pkg.fic_tune_mode(1)
    img = fic_synth.with_step_edges(160, 11, alpha=2.0)
    ss = [PAPER_S[s] for s in (16, 8, 4)]
    a = pkg.fic_encode_ex(img, 160, 16, 4, 1, -1.0, ss, 8.0)
    table = pkg.fic_tune_read()
    assert table, "no tuned class recorded"
    for t in table:
        assert t["candidates"] >= 3 and t["refill"] in (1, 2, 4) and t["iso_tiles"] in (0, 1, 2)
        assert t["epi_warps"] in (8, 16)
        assert t["ms"] > 0
    # a second encode of the same classes reuses the choices (no new entries)
    n = len(table)
    b = pkg.fic_encode_ex(img, 160, 16, 4, 1, -1.0, ss, 8.0)
    assert len(pkg.fic_tune_read()) == n
    np.testing.assert_array_equal(a.codes, b.codes)


@pytest.mark.parametrize("kind", ["black", "binary_noise", "checker"])
def test_forced_shapes_on_extreme_images(pkg, kind):
    """The domain-side kernel (mode 7) and the isometry-in-accumulator kernel
    (mode 2) on the extremes of the centred operands, with 2x2 ranges: the
    all-black image gives the largest partial sums and all-equal filter values
    (every tie broken by the index), noise and checkerboards mix signs and
    isometries that map a block onto itself."""
    N = 64
    rng = np.random.default_rng(11)
    if kind == "black":
        img = np.zeros((N, N), np.uint8)
    elif kind == "binary_noise":
        img = (rng.integers(0, 2, (N, N)) * 255).astype(np.uint8)
    else:
        img = (((np.indices((N, N)).sum(0)) % 2) * 255).astype(np.uint8)
    ss = [PAPER_S[s] for s in (16, 8, 4, 2)]
    want, _ = oracle.encode(img, 16, 2, 1, -1.0, ss, 4.0)
    for mode in (2, 7):
        pkg.fic_tune_mode(mode)
        enc = pkg.fic_encode_ex(img, N, 16, 2, 1, -1.0, ss, 4.0)
        assert_same_codes(enc.codes, want, 16, f"{kind} mode {mode}")
    pkg.fic_tune_mode(1)
