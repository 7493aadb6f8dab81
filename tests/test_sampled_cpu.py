"""The stratified sampled oracle check (tests/sampled.py) used on images too
large for a whole oracle encode must itself catch wrong records: it passes on
the oracle's own records and fails on records with one planted mistake."""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle
from tests.sampled import check_sampled

PAPER_S = [(10, [1]), (10, [2, 4]), (10, [3, 8])]
ARGS = dict(B_max=16, B_min=4, L=2, thr=4.0, tol=8.0)


def oracle_as_gpu(img):
    """The oracle's encode in the GPU record layout the check reads."""
    want, st = oracle.encode(img, ARGS["B_max"], ARGS["B_min"], ARGS["L"], ARGS["thr"], PAPER_S,
                             ARGS["tol"])
    dt = np.dtype([("rx", "<u2"), ("ry", "<u2"), ("dx", "<u2"), ("dy", "<u2"),
                   ("pool_idx", "<u4"), ("level", "u1"), ("iso", "u1"), ("s_idx", "u1"),
                   ("o_q", "u1")])
    c = np.zeros(len(want), dt)
    for f in ("rx", "ry", "dx", "dy", "pool_idx", "level", "iso", "o_q"):
        c[f] = want[f]
    c["s_idx"] = np.where(want["s_idx"] < 0, 0xFF, want["s_idx"])
    return c, st["pool_size"]


@pytest.fixture(scope="module")
def case():
    img = fic_synth.one_over_f(128, 31, 2.0)
    codes, pools = oracle_as_gpu(img)
    return img, codes, pools


def run(img, codes, pools):
    return check_sampled(img, codes, pools, ARGS["B_max"], ARGS["B_min"], ARGS["L"], ARGS["thr"],
                         PAPER_S, ARGS["tol"], "cpu self-check", per_step=1000, parents=1000)


def test_passes_on_the_oracles_own_records(case):
    img, codes, pools = case
    assert run(img, codes, pools) >= len(codes)


@pytest.mark.parametrize("mistake", ["pool_idx", "iso", "s_idx", "order", "tiling", "pool size"])
def test_fails_on_a_planted_mistake(case, mistake):
    img, codes, pools = case
    c = codes.copy()
    pools = list(pools)
    leaf = int(np.nonzero(c["s_idx"] != 0xFF)[0][len(c) // 2])
    if mistake == "pool_idx":
        c["pool_idx"][leaf] += 1
    elif mistake == "iso":
        c["iso"][leaf] ^= 1
    elif mistake == "s_idx":
        # a leaf of a step with two S values
        leaf = int(np.nonzero((c["s_idx"] != 0xFF) & (c["level"] > 0))[0][0])
        c["s_idx"][leaf] ^= 1
    elif mistake == "order":
        c[[0, 1]] = c[[1, 0]]
    elif mistake == "tiling":
        c = c[1:]
    else:
        pools[1] += 1
    with pytest.raises(AssertionError):
        run(img, c, pools)
