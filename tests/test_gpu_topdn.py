"""GPU parity of the top-DN domain pool (Sec. 3.2.1, Sec. 4: the DN domains
of highest entropy; entropies rounded to 2^-20 bit, equal ones in raster
order) and of full encodes that use it, down to 2x2 ranges."""
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
    return p


@pytest.mark.parametrize("B,L,dn", [(16, 2, 32), (8, 1, 64), (4, 2, 144), (2, 1, 256),
                                    (8, 3, 10 ** 6), (4, 1, 1)])
def test_top_dn_pool_matches_oracle(pkg, B, L, dn):
    img = fic_synth.one_over_f(192, 31, 2.0)
    xy, ent, near = pkg.fic_domain_pool(img, 192, B, L, -1.0, pool_dn=dn)
    pl = oracle.Pool(img, B, L, -1.0, dn_top=dn)
    assert near == pl.near_thresh == 0
    np.testing.assert_array_equal(xy, pl.positions())
    # entropies: GPU fixed-point sums against the oracle's FP64 sums
    per = oracle.positions_per_axis(192, B, L)
    idx = np.random.default_rng(B * 10 + L).choice(per * per, 200)
    want = [oracle.entropy_bits(img, int(i % per) * L, int(i // per) * L, 2 * B) for i in idx]
    np.testing.assert_allclose(ent[idx], want, rtol=0, atol=1e-12)


def test_top_dn_ties_take_raster_order(pkg):
    """Periodic image: every window at step 2 holds one full period (all
    positions tie); with a noisy patch the higher-entropy windows come
    first, then tied ones in raster order."""
    rng = np.random.default_rng(5)
    tile = rng.integers(0, 6, (8, 8)).astype(np.uint8) * 40
    img = np.tile(tile, (12, 12))
    img2 = img.copy()
    img2[40:72, 40:72] = rng.integers(0, 256, (32, 32))
    for im in (img, img2):
        for dn in (5, 40, 300):
            xy, _, near = pkg.fic_domain_pool(im, 96, 4, 2, -1.0, pool_dn=dn)
            pl = oracle.Pool(im, 4, 2, -1.0, dn_top=dn)
            assert near == pl.near_thresh
            np.testing.assert_array_equal(xy, pl.positions())


@pytest.mark.parametrize("dn", [32, 64, 144, 256])
def test_top_dn_encode_16_to_2_matches_oracle(pkg, dn):
    """Quadtree 16 -> 8 -> 4 -> 2 (all four steps of the paper, S {0.1},
    {0.2, 0.4}, {0.3, 0.8}, {0.5, 0.9}), L = 2, top-DN pool, 128 x 128
    texture with step edges (records at every step); both engines."""
    import torch
    img = fic_synth.with_step_edges(128, 40 + dn, alpha=3.0)
    ss = [PAPER_S[b] for b in (16, 8, 4, 2)]
    want, st = oracle.encode(img, 16, 2, 2, -1.0, ss, 12.0, pool_dn=dn)
    assert sum(st["near_thresh"]) == 0
    got = {}
    for e in (pkg.ENGINE_TENSOR, pkg.ENGINE_PLAIN):
        enc = pkg.fic_encode_ex(torch.from_numpy(img).cuda(), 128, 16, 2, 2, -1.0, ss, 12.0,
                                engine=e, pool_dn=dn)
        assert_same_codes(enc.codes, want, 16, f"top-{dn} engine {e}")
        for l in range(enc.n_levels):
            if enc.ranges[l]:
                assert enc.pool_size[l] == st["pool_size"][l] == dn
        got[e] = enc.codes
    np.testing.assert_array_equal(got[pkg.ENGINE_TENSOR], got[pkg.ENGINE_PLAIN])
    assert len(set(int(v) for v in want["level"])) == 4  # records at all four steps


def test_top_dn_batch_and_server_match_single(pkg):
    imgs = [fic_synth.one_over_f(n, 70 + i, 2.0) for i, n in enumerate((64, 128, 96, 160))]
    ss = [PAPER_S[b] for b in (16, 8, 4)]
    alone = [pkg.fic_encode_ex(im, im.shape[0], 16, 4, 2, -1.0, ss, 8.0, pool_dn=64).codes
             for im in imgs]
    for enc, want in zip(pkg.fic_encode_batch(imgs, 16, 4, 2, -1.0, ss, 8.0, pool_dn=64), alone):
        np.testing.assert_array_equal(enc.codes, want)
    with pkg.Server(16, 4, 2, -1.0, ss, 8.0, pool_dn=64) as srv:
        ts = [srv.submit(im) for im in imgs]
        for t, want in zip(ts, alone):
            enc, _ = srv.poll(t)
            np.testing.assert_array_equal(enc.codes, want)


def test_ten_value_S_baseline_matches_oracle(pkg):
    """The entropy-based baseline's search space: S = k/10, k = 1..10, at
    every step (16 -> 2, top-64 pool); both engines against the oracle."""
    img = fic_synth.with_step_edges(64, 77, alpha=3.0)
    ss = [(10, list(range(1, 11)))] * 4
    want, st = oracle.encode(img, 16, 2, 2, -1.0, ss, 12.0, pool_dn=64)
    assert sum(st["near_thresh"]) == 0
    for e in (pkg.ENGINE_TENSOR, pkg.ENGINE_PLAIN):
        enc = pkg.fic_encode_ex(img, 64, 16, 2, 2, -1.0, ss, 12.0, engine=e, pool_dn=64)
        assert_same_codes(enc.codes, want, 16, f"k/10 engine {e}")
    assert (want["s_idx"] >= 2).any()  # S values beyond the paper's pairs are chosen
