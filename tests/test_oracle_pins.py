"""Pins for the CPU oracle against the paper and against independent maths.

Each test fixes a part of the oracle by something other than the oracle
itself: values printed in the paper (tests/golden/paper_pins.json), closed
forms (eq. 2, eq. 3), library routines (numpy rot90/fliplr, lstsq, scipy
entropy), exact rational evaluation of eq. 1, and brute force on tiny inputs.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import fic_synth
from tests import brute

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
SIDES = [2, 4, 8, 16]


# ---------------------------------------------------------------- isometries

@pytest.mark.parametrize("B", SIDES + [3, 5])
def test_isometries_match_numpy_rot90_fliplr(B):
    rng = np.random.default_rng(B)
    a = rng.integers(0, 1000, size=(B, B)).astype(np.int32)
    for k in range(GOLD["isometries"]["count"]):
        np.testing.assert_array_equal(oracle.isometry(a, k), brute.iso_numpy(a, k))


def test_rotation_is_clockwise_and_mirror_is_left_right():
    a = np.array([[1, 2], [3, 4]], np.int32)
    # 90 degrees clockwise: the left column (1 over 3) becomes the top row (3, 1).
    np.testing.assert_array_equal(oracle.isometry(a, 1), [[3, 1], [4, 2]])
    np.testing.assert_array_equal(oracle.isometry(a, 4), [[2, 1], [4, 3]])


@pytest.mark.parametrize("B", [4, 8])
def test_isometries_form_dihedral_group(B):
    rng = np.random.default_rng(7)
    a = rng.permutation(B * B).reshape(B, B).astype(np.int32)  # all distinct
    imgs = [oracle.isometry(a, k) for k in range(8)]
    keys = {im.tobytes() for im in imgs}
    assert len(keys) == 8
    # closure: T_j(T_k(a)) is again one of the 8
    for j in range(8):
        for k in range(8):
            assert oracle.isometry(imgs[k], j).tobytes() in keys
    # inverses: rot^k undone by rot^(4-k); mirrored maps are involutions
    for k in range(4):
        np.testing.assert_array_equal(oracle.isometry(imgs[k], (4 - k) % 4), a)
    for k in range(4, 8):
        np.testing.assert_array_equal(oracle.isometry(imgs[k], k), a)


# ---------------------------------------------------------------- decimation, sums

@pytest.mark.parametrize("B", SIDES)
def test_decimation_is_2x2_sum(B):
    img = fic_synth.one_over_f(64, 3)
    for (x, y) in [(0, 0), (5, 9), (64 - 2 * B, 64 - 2 * B)]:
        np.testing.assert_array_equal(oracle.decimate(img, x, y, B),
                                      brute.decimate_numpy(img, x, y, B))


@pytest.mark.parametrize("B", SIDES)
def test_domain_sums_invariant_under_isometries(B):
    rng = np.random.default_rng(B + 11)
    d = rng.integers(0, 1021, size=(B, B)).astype(np.int32)
    s, s2 = int(d.sum()), int((d.astype(np.int64) ** 2).sum())
    for k in range(8):
        t = oracle.isometry(d, k).astype(np.int64)
        assert int(t.sum()) == s and int((t ** 2).sum()) == s2


# ---------------------------------------------------------------- eq. 1-3

@pytest.mark.parametrize("B", [2, 4, 8])
def test_score_equals_literal_eq1_at_eq3_offset(B):
    """16 q^2 n E(S, O*) from the oracle equals eq. 1 evaluated in exact
    rationals with O* from eq. 3, for random blocks, extremes, all 8 maps."""
    rng = np.random.default_rng(100 + B)
    n = B * B
    cases = []
    for _ in range(6):
        cases.append((rng.integers(0, 256, (B, B)), rng.integers(0, 1021, (B, B))))
    cases.append((np.zeros((B, B), int), np.full((B, B), 1020)))
    cases.append((np.full((B, B), 255), np.zeros((B, B), int)))
    cases.append((np.full((B, B), 255), np.full((B, B), 1020)))
    for r, d in cases:
        r = r.astype(np.int32)
        d = d.astype(np.int32)
        for k in range(8):
            t = brute.iso_numpy(d, k)
            for (p, q) in [(1, 10), (4, 10), (9, 10), (5, 16), (16, 16)]:
                S = Fraction(p, q)
                O = brute.optimal_offset_eq3(r, t, S)
                E = brute.error_eq1_fraction(r, t, S, O)
                want = E * 16 * q * q * n
                assert want.denominator == 1
                assert oracle.score(r, d, k, p, q) == int(want)


def test_score_equals_integer_eq1_on_16x16():
    rng = np.random.default_rng(5)
    for _ in range(10):
        r = rng.integers(0, 256, (16, 16)).astype(np.int32)
        d = rng.integers(0, 1021, (16, 16)).astype(np.int32)
        k = int(rng.integers(0, 8))
        got = oracle.score(r, d, k, 1, 10)
        assert got == brute.scaled_error_int(r, brute.iso_numpy(d, k), 1, 10)


def test_eq3_offset_is_the_minimiser():
    rng = np.random.default_rng(9)
    r = rng.integers(0, 256, (4, 4))
    t = rng.integers(0, 1021, (4, 4))
    for S in [Fraction(3, 10), Fraction(8, 10)]:
        O = brute.optimal_offset_eq3(r, t, S)
        E0 = brute.error_eq1_fraction(r, t, S, O)
        for eps in [Fraction(1, 1000), Fraction(1, 3), Fraction(5)]:
            assert brute.error_eq1_fraction(r, t, S, O + eps) > E0
            assert brute.error_eq1_fraction(r, t, S, O - eps) > E0
        # the same offset from a least-squares fit of r - S d on a constant
        lsq = np.linalg.lstsq(np.ones((16, 1)), (r - float(S) * t / 4.0).ravel(), rcond=None)[0]
        assert abs(float(O) - lsq[0]) < 1e-9


def test_best_grid_S_bounded_by_eq2_optimum_and_exact_when_on_grid():
    """Eq. 2's unconstrained optimum (here via lstsq on [d, 1]) is a lower bound
    for the best grid S; a range built as S d + O with S on the grid scores 0."""
    rng = np.random.default_rng(21)
    grid = list(range(1, 17))
    for _ in range(20):
        r = rng.integers(0, 256, (4, 4)).astype(np.int32)
        d = rng.integers(0, 1021, (4, 4)).astype(np.int32)
        A = np.stack([d.ravel() / 4.0, np.ones(16)], axis=1)
        coef, res, *_ = np.linalg.lstsq(A, r.ravel().astype(float), rcond=None)
        e_star = float(((A @ coef - r.ravel()) ** 2).sum())
        best = min(oracle.score(r, d, 0, p, 16) for p in grid) / (16 * 16 * 16 * 16)
        assert best >= e_star - 1e-6
        # eq. 2 closed form agrees with lstsq
        dd = d.ravel() / 4.0
        s2 = ((r.ravel() - r.mean()) @ (dd - dd.mean())) / ((dd - dd.mean()) @ (dd - dd.mean()))
        assert abs(s2 - coef[0]) < 1e-9
    # exact map: d multiple of 64 -> d/4 multiple of 16 -> (5/16) d/4 integral
    d = (rng.integers(0, 16, (4, 4)) * 64).astype(np.int32)
    r = (5 * (d // 4) // 16 + 37).astype(np.int32)
    scores = [oracle.score(r, d, 0, p, 16) for p in grid]
    assert scores[4] == 0 and min(scores) == 0


# ---------------------------------------------------------------- entropy (eq. 5-6)

def test_entropy_special_cases():
    z = np.zeros((16, 16), np.uint8)
    assert oracle.entropy_bits(z, 0, 0, 16) == 0.0
    # 4n distinct grey levels: log2(4n) bits (256 pixels of a 16x16 block)
    a = np.arange(256, dtype=np.uint8).reshape(16, 16)
    assert oracle.entropy_bits(a, 0, 0, 16) == 8.0
    # two equal halves: 1 bit
    h = np.zeros((8, 8), np.uint8)
    h[:, 4:] = 200
    assert oracle.entropy_bits(h, 0, 0, 8) == 1.0
    # 16 levels x 4 pixels in an 8x8 block: exactly 4 bits, not > 4.0
    b = np.repeat(np.arange(16, dtype=np.uint8) * 9, 4).reshape(8, 8)
    assert oracle.entropy_bits(b, 0, 0, 8) == 4.0


def test_entropy_matches_scipy():
    img = fic_synth.one_over_f(64, 4)
    rng = np.random.default_rng(3)
    for _ in range(30):
        s = int(rng.choice([4, 8, 16, 32]))
        x, y = (int(v) for v in rng.integers(0, 64 - s + 1, 2))
        got = oracle.entropy_bits(img, x, y, s)
        assert abs(got - brute.entropy_bits_scipy(img[y:y + s, x:x + s])) < 1e-12


def test_entropy_depends_only_on_the_count_multiset():
    """Relabelling the grey levels of a block (a bijection) permutes its
    histogram; eq. 5-6 is unchanged and the oracle's value is bit-identical
    (the tie rule of the top-DN pool relies on it)."""
    rng = np.random.default_rng(12)
    for s in (4, 8, 16, 32):
        blk = (rng.integers(0, 7, (s, s)) * 31 + rng.integers(0, 2, (s, s))).astype(np.uint8)
        perm = rng.permutation(256).astype(np.uint8)
        h0 = oracle.entropy_bits(blk, 0, 0, s)
        h1 = oracle.entropy_bits(perm[blk], 0, 0, s)
        assert h0 == h1
        assert abs(h0 - brute.entropy_bits_scipy(blk)) < 1e-12


# ---------------------------------------------------------------- counts (Sec. 1-3)

def test_worked_example_domain_count():
    g = GOLD["domain_count_worked_example"]
    B = g["domain_side"] // 2
    assert oracle.positions_per_axis(g["N"], B, g["L"]) ** 2 == g["count"]
    img = fic_synth.one_over_f(g["N"], 0)
    assert oracle.Pool(img, B, g["L"], -1.0).dn == g["count"]
    red = GOLD["pool_reduction_worked_example"]
    assert round(g["count"] / red["pool"]) in range(red["factor_about"] - 2, red["factor_about"] + 3)


def test_range_and_full_domain_counts():
    for N, n in GOLD["range_count"]["cases"]:
        img = fic_synth.one_over_f(N, 1)
        assert oracle.Pool(img, n, 1, -1.0).dn == (N - 2 * n + 1) ** 2
    # (N/n)^2 ranges: one record each when nothing splits
    img = fic_synth.one_over_f(64, 1)
    codes, _ = oracle.encode(img, 8, 8, 16, -1.0, [(10, [1])], 8.0)
    assert len(codes) == (64 // 8) ** 2
    # the tiny workload: 64x64, 8x8 ranges, 16x16 domains at step 4 -> 13^2 = 169
    assert oracle.positions_per_axis(64, 8, 4) ** 2 == 169


def test_address_bits_eq8():
    for dn, bits in GOLD["address_bits"]["cases"]:
        assert oracle.address_bits(dn) == bits
    assert [oracle.address_bits(v) for v in (32, 144, 256, 257)] == [5, 8, 8, 9]


# ---------------------------------------------------------------- pool and search

@pytest.mark.parametrize("thr", [-1.0, 3.5, 4.0])
def test_pool_matches_brute_force(thr):
    img = fic_synth.one_over_f(40, 6)
    for B, L in [(4, 2), (2, 1), (8, 3)]:
        want = brute.brute_pool(img, B, L, thr)
        pl = oracle.Pool(img, B, L, thr)
        assert [tuple(p) for p in pl.positions().tolist()] == want


@pytest.mark.parametrize("dn", [1, 32, 64, 144, 256, 10 ** 6])
def test_top_dn_pool_matches_brute_force(dn):
    """Top-DN pool (Sec. 4: the DN highest-entropy domains), ties in raster
    order, listed in raster order; DN above the position count keeps all."""
    img = fic_synth.one_over_f(48, 9, 1.5)
    for B, L in [(4, 1), (8, 2), (2, 1)]:
        pl = oracle.Pool(img, B, L, -1.0, dn_top=dn)
        assert [tuple(p) for p in pl.positions().tolist()] == brute.brute_top_pool(img, B, L, dn)
        assert pl.near_thresh == 0


def test_top_dn_pool_ties_in_raster_order():
    """A periodic image (period 8): every 8x8 window at step 2 holds one full
    period, so all positions tie; the pool is the first DN in raster order.
    With a noisy patch, higher-entropy windows come first, then the tied
    periodic ones in raster order."""
    rng = np.random.default_rng(5)
    tile = rng.integers(0, 6, (8, 8)).astype(np.uint8) * 40
    img = np.tile(tile, (6, 6))
    pl = oracle.Pool(img, 4, 2, -1.0, dn_top=10)
    per = oracle.positions_per_axis(48, 4, 2)
    want = [((i % per) * 2, (i // per) * 2) for i in range(10)]
    assert [tuple(p) for p in pl.positions().tolist()] == want
    img2 = img.copy()
    img2[30:46, 30:46] = rng.integers(0, 256, (16, 16))
    for dn in (5, 40, 100):
        pl = oracle.Pool(img2, 4, 2, -1.0, dn_top=dn)
        assert [tuple(p) for p in pl.positions().tolist()] == brute.brute_top_pool(img2, 4, 2, dn)


def test_top_dn_encode_matches_brute_force():
    """Quadtree 8 -> 4 -> 2 with a 32-domain top-entropy pool at every step
    and the paper's S sets per side (2x2 step: {0.5, 0.9})."""
    img = fic_synth.one_over_f(32, 21, 1.8)
    ss = [(10, [2, 4]), (10, [3, 8]), (10, [5, 9])]
    got, st = oracle.encode(img, 8, 2, 2, -1.0, ss, 24.0, pool_dn=32)
    assert st["pool_size"] == [32, 32, 32]
    want = brute.brute_encode(img, 8, 2, 2, -1.0, ss, 24.0,
                              pool_fn=lambda B: brute.brute_top_pool(img, B, 2, 32))
    assert len(got) == len(want)
    for g, w in zip(got, want):
        for f in ("rx", "ry", "level", "B", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx"):
            assert int(g[f]) == int(w[f]), (f, g, w)
    assert len(set(int(v) for v in got["B"])) == 3  # records at all three steps


def test_search_matches_brute_force():
    img = fic_synth.one_over_f(24, 8)
    B, L = 4, 2
    pool = brute.brute_pool(img, B, L, -1.0)
    pl = oracle.Pool(img, B, L, -1.0)
    xs, ys = np.meshgrid(np.arange(0, 24, B), np.arange(0, 24, B))
    for sset in [(10, [3, 8]), (16, list(range(1, 17)))]:
        sc, pi, iso, si = pl.search(xs.ravel(), ys.ravel(), sset)
        for i, (x, y) in enumerate(zip(xs.ravel(), ys.ravel())):
            want = brute.brute_search(img, int(x), int(y), B, pool, sset)
            assert (int(sc[i]), int(pi[i]), int(iso[i]), int(si[i])) == want


def test_search_tie_break_lowest_index():
    # flat image: every candidate ties at score 0 -> pool 0, isometry 0, S index 0
    img = np.full((32, 32), 77, np.uint8)
    pl = oracle.Pool(img, 4, 2, -1.0)
    sc, pi, iso, si = pl.search([8], [8], (10, [3, 8]))
    assert (sc[0], pi[0], iso[0], si[0]) == (0, 0, 0, 0)
    # symmetric domain: rot180 equals identity -> the identity (lower index) wins
    img = fic_synth.one_over_f(32, 2)
    sym = img.copy()
    blk = sym[0:8, 0:8]
    sym[0:8, 0:8] = np.maximum(blk, np.rot90(blk, 2))
    pl = oracle.Pool(sym, 4, 32, -1.0)  # one domain at (0, 0)
    sc, pi, iso, si = pl.search([16], [16], (10, [3, 8]))
    assert iso[0] not in (2, 6)


@pytest.mark.parametrize("params", [
    dict(N=32, B_max=8, B_min=4, L=2, thr=-1.0, tol=8.0, seed=1),
    dict(N=32, B_max=8, B_min=2, L=3, thr=4.0, tol=6.0, seed=2),
    dict(N=32, B_max=16, B_min=4, L=4, thr=3.0, tol=10.0, seed=3),
])
def test_quadtree_encode_matches_brute_force(params):
    img = fic_synth.one_over_f(params["N"], params["seed"])
    sides = []
    b = params["B_max"]
    while b >= params["B_min"]:
        sides.append(b)
        b //= 2
    S_BY_SIDE = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}
    ssets = [S_BY_SIDE[s] for s in sides]
    want = brute.brute_encode(img, params["B_max"], params["B_min"], params["L"],
                              params["thr"], ssets, params["tol"])
    got, st = oracle.encode(img, params["B_max"], params["B_min"], params["L"],
                            params["thr"], ssets, params["tol"])
    assert len(got) == len(want)
    for g, w in zip(got, want):
        for f in ("rx", "ry", "level", "B", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx"):
            assert int(g[f]) == int(w[f]), (f, g, w)
        if "score" in w:
            assert int(g["score"]) == w["score"]
    # leaves tile the image exactly once
    cover = np.zeros((params["N"],) * 2, int)
    for g in got:
        cover[g["ry"]:g["ry"] + g["B"], g["rx"]:g["rx"] + g["B"]] += 1
    assert (cover == 1).all()


def test_empty_pool_rules():
    """2x2 ranges use 4x4 domains: 16 pixels carry at most 4 bits, so an
    entropy threshold of 4.0 admits nothing; the last step then stores the
    range mean only, and earlier steps split every range."""
    img = fic_synth.one_over_f(16, 5)
    codes, st = oracle.encode(img, 4, 2, 2, 4.0, [(10, [3, 8]), (10, [5, 9])], 0.0)
    assert st["pool_size"][1] == 0
    assert all(c["s_idx"] == -1 and c["pool_idx"] == 0xFFFFFFFF for c in codes if c["B"] == 2)


# ---------------------------------------------------------------- split rule

def test_split_threshold_is_rms_greater_than_tol():
    img = fic_synth.one_over_f(32, 4)
    ss = [(10, [2, 4]), (10, [3, 8])]
    codes, _ = oracle.encode(img, 8, 4, 2, -1.0, ss, 8.0)
    pl = oracle.Pool(img, 8, 2, -1.0)
    for ty in range(0, 32, 8):
        for tx in range(0, 32, 8):
            sc, *_ = pl.search([tx], [ty], ss[0])
            E = Fraction(int(sc[0]), 16 * 100 * 64)
            split = E / 64 > 64  # RMS > 8  <=>  E/n > 8^2
            top = [c for c in codes if c["rx"] == tx and c["ry"] == ty and c["level"] == 0]
            assert (len(top) == 0) == split


def test_split_tolerance_is_quantised_to_sixteenths():
    """tol enters the split test as e16 / 16 with e16 = round(16 tol), halves
    up.  For a range whose RMS error e lies in [k/16, (k+1)/16): tol just
    above k/16 + 1/32 (or exactly there) rounds up to (k+1)/16 > e, so the
    range is kept; tol at k/16 + 1/64 rounds to k/16, so it splits unless
    e = k/16 exactly.  Errors from an exhaustive search (tests/brute.py)."""
    img = fic_synth.one_over_f(32, 4)
    ss = [(10, [2, 4]), (10, [3, 8])]
    pool = brute.brute_pool(img, 8, 2, -1.0)
    for tx, ty in [(0, 0), (8, 0), (16, 8), (24, 24)]:
        score, *_ = brute.brute_search(img, tx, ty, 8, pool, ss[0])
        ms = Fraction(score, 16 * 100 * 64) / 64       # E / n = RMS^2
        k = math.isqrt(math.floor(256 * ms))            # k/16 <= RMS < (k+1)/16
        assert Fraction(k * k, 256) <= ms < Fraction((k + 1) ** 2, 256)
        for frac, keep in [(0.75, True), (0.5, True), (0.25, ms == Fraction(k * k, 256))]:
            tol = (k + frac) / 16
            codes, _ = oracle.encode(img, 8, 4, 2, -1.0, ss, tol)
            top = [c for c in codes if c["rx"] == tx and c["ry"] == ty and c["level"] == 0]
            assert (len(top) == 1) == keep, (tx, ty, k, frac)


# ---------------------------------------------------------------- decoder, eq. 4

def test_decoder_one_iteration_matches_literal():
    img = fic_synth.one_over_f(32, 7)
    ss = [(10, [2, 4]), (10, [3, 8])]
    codes, _ = oracle.encode(img, 8, 4, 2, -1.0, ss, 8.0)
    got, it = oracle.decode(codes, ss, 32, iters_max=1)
    want = brute.decode_one_iteration(codes, ss, np.full((32, 32), 128, np.uint8))
    np.testing.assert_array_equal(got, want)
    # a second pass from the first
    got2, _ = oracle.decode(codes, ss, 32, iters_max=2)
    np.testing.assert_array_equal(got2, brute.decode_one_iteration(codes, ss, want))


def test_decoder_constant_image_and_psnr_closed_form():
    for v in (0, 77, 200, 255):
        img = np.full((32, 32), v, np.uint8)
        ss = [(10, [2, 4])]
        codes, _ = oracle.encode(img, 8, 8, 4, -1.0, ss, 8.0)
        dec, it = oracle.decode(codes, ss, 32)
        want = min(255, 2 * (v // 2) + 1)
        assert (dec == want).all()
        p = oracle.psnr(img, dec)
        if want == v:
            assert p == math.inf
        else:  # MSE = 1 -> 10 log10(255^2)
            assert abs(p - 10 * math.log10(255.0 ** 2)) < 1e-12


def test_decoder_reaches_fixed_point():
    img = fic_synth.one_over_f(64, 0)
    ss = [(10, [2, 4]), (10, [3, 8])]
    codes, _ = oracle.encode(img, 8, 4, 2, -1.0, ss, 4.0)
    dec, it = oracle.decode(codes, ss, 64, iters_max=64)
    if it < 64:
        once, _ = oracle.decode(codes, ss, 64, iters_max=it + 1)
        np.testing.assert_array_equal(once, dec)
    assert oracle.psnr(img, dec) > 20.0


def test_psnr_eq4():
    a = np.zeros((4, 4), np.uint8)
    b = a.copy()
    b[0, 0] = 4  # MSE = 16/16 = 1
    assert abs(oracle.psnr(a, b) - 10 * math.log10(255 ** 2)) < 1e-12
    b[0, 1] = 4  # MSE = 2
    assert abs(oracle.psnr(a, b) - 10 * math.log10(255 ** 2 / 2)) < 1e-12


def test_predefined_S_and_steps_golden():
    g = GOLD["predefined_S"]["by_side"]
    assert fic_synth.images.PAPER_S[16] == (10, [1])
    for side, vals in g.items():
        q, ps = fic_synth.images.PAPER_S[int(side)]
        assert [Fraction(p, q) for p in ps] == [Fraction(v).limit_denominator(100) for v in vals]
    assert GOLD["steps"]["sides"] == [16, 8, 4, 2]


# ---------------------------------------------------------------- stored stream (Sec. 3.3, Fig. 7, eq. 8)

def _bits_writer():
    bits = []

    def put(v, n):
        for i in range(n - 1, -1, -1):
            bits.append((int(v) >> i) & 1)

    def align():
        while len(bits) % 8:
            bits.append(0)

    def tobytes():
        align()
        return bytes(int("".join(map(str, bits[i:i + 8])), 2) for i in range(0, len(bits), 8))

    return bits, put, align, tobytes


def _ceil_log2(v):
    return 0 if v <= 1 else int(math.ceil(math.log2(v)))


def _stream_python(img, codes, B_max, n_levels, L, ssets, pools, rule):
    """The stream written from the format statement alone (independent of
    the C writer): header, per-step S set and domain list, then records of
    step 2 bits, mean 7 bits, isometry 3 bits, address ceil(log2 DN) bits,
    S index ceil(log2 |S|) bits."""
    bits, put, align, tobytes = _bits_writer()
    N = img.shape[0]
    for ch in b"FIC1":
        put(ch, 8)
    put(N, 16); put(B_max, 8); put(n_levels, 8); put(L, 16); put(rule, 8); put(len(codes), 32)
    for l in range(n_levels):
        q, ps = ssets[l]
        put(len(ps), 8); put(q, 16)
        for p in ps:
            put(p, 16)
        pool = pools[l]
        put(len(pool), 32)
        per = (N - 2 * (B_max >> l)) // L + 1
        pw = _ceil_log2(per)
        npos = per * per
        form = 0 if len(pool) in (0, npos) else (1 if len(pool) * 2 * pw <= npos else 2)
        put(form, 8)
        if form == 1:
            for x, y in pool:
                put(x // L, pw); put(y // L, pw)
        elif form == 2:
            s = set(pool)
            for i in range(npos):
                put(1 if ((i % per) * L, (i // per) * L) in s else 0, 1)
        align()
    for c in codes:
        l = int(c["level"])
        put(l, 2); put(int(c["o_q"]), 7)
        if pools[l]:
            put(int(c["iso"]), 3)
            put(int(c["pool_idx"]), _ceil_log2(len(pools[l])))
            put(int(c["s_idx"]), _ceil_log2(len(ssets[l][1])))
    return tobytes()


@pytest.mark.parametrize("case", [
    dict(N=64, B_max=16, n=3, L=2, thr=4.0, dn=0, tol=8.0, seed=5),      # threshold pools
    dict(N=64, B_max=16, n=3, L=2, thr=-1.0, dn=32, tol=8.0, seed=6),    # top-32 pools
    dict(N=48, B_max=8, n=3, L=1, thr=-1.0, dn=0, tol=12.0, seed=7),     # full pools
    dict(N=32, B_max=8, n=3, L=1, thr=4.0, dn=0, tol=2.0, seed=8),       # empty last pool
])
def test_stream_roundtrip_and_independent_writer(case):
    img = fic_synth.with_step_edges(case["N"], case["seed"], alpha=2.5)
    sides = [case["B_max"] >> l for l in range(case["n"])]
    S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}
    ss = [S[b] for b in sides]
    codes, st = oracle.encode(img, case["B_max"], sides[-1], case["L"], case["thr"], ss,
                              case["tol"], pool_dn=case["dn"])
    stream, pbits = oracle.pack(img, codes, case["B_max"], case["n"], case["L"], case["thr"], ss,
                                st["ranges"], pool_dn=case["dn"])
    back, ss2, N2, Bm2 = oracle.unpack(stream)
    assert (N2, Bm2) == (case["N"], case["B_max"]) and ss2 == ss
    for f in ("rx", "ry", "level", "B", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx"):
        np.testing.assert_array_equal(back[f], codes[f], err_msg=f)
    pools = []
    for l, B in enumerate(sides):
        if st["ranges"][l] == 0:
            pools.append([])
        elif case["dn"]:
            pools.append(brute.brute_top_pool(img, B, case["L"], case["dn"]))
        else:
            pools.append(brute.brute_pool(img, B, case["L"], case["thr"]))
    assert stream == _stream_python(img, codes, case["B_max"], case["n"], case["L"], ss, pools,
                                    1 if case["dn"] else 0)
    # record bits (Fig. 7, eq. 8): step 2 + mean 7 + [pool] (isometry 3 + address + S index)
    want = sum(9 + ((3 + _ceil_log2(len(pools[int(c["level"])])) +
                     _ceil_log2(len(ss[int(c["level"])][1]))) if pools[int(c["level"])] else 0)
               for c in codes)
    assert pbits == want


def test_stream_field_widths_follow_fig7():
    g = GOLD["record_fields_bits"]
    # S field: none for the one-valued step-1 set, one bit for the two-valued sets
    by_side = GOLD["predefined_S"]["by_side"]
    assert [_ceil_log2(len(by_side[str(b)])) for b in (16, 8, 4, 2)] == g["s_bits_by_step"]
    assert _ceil_log2(4) == g["step"] and _ceil_log2(8) == g["isometry"]
    # the address field is eq. 8's X = ceil(log2 DN)
    for dn, bits in GOLD["address_bits"]["cases"]:
        assert _ceil_log2(dn) == bits
