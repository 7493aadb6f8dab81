"""GPU parity: the CUDA search (both engines) against the CPU oracle.

Records must match the oracle bit-exactly (pool index, isometry, S index,
7-bit mean, quadtree shape); the two engines must match each other.  Small
cases run the oracle in full; the 512 x 512 workload is checked on sampled
ranges that the oracle searches one by one.
"""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes, to_oracle_records

pytestmark = pytest.mark.gpu

ENGINES = ("tensor", "plain")


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


def encode(pkg, img, B_max, B_min, L, thr, ssets, tol, engine, device=True):
    import torch
    e = pkg.ENGINE_TENSOR if engine == "tensor" else pkg.ENGINE_PLAIN
    src = torch.from_numpy(np.ascontiguousarray(img)).cuda() if device else img
    return pkg.fic_encode_ex(src, img.shape[0], B_max, B_min, L, thr, ssets, tol, engine=e,
                             stream=torch.cuda.current_stream())


def check_against_oracle(pkg, img, B_max, B_min, L, thr, ssets, tol, what):
    want, st = oracle.encode(img, B_max, B_min, L, thr, ssets, tol)
    outs = {}
    for eng in ENGINES:
        enc = encode(pkg, img, B_max, B_min, L, thr, ssets, tol, eng)
        # steps that no range reached are not built on the GPU
        for l in range(enc.n_levels):
            if enc.ranges[l] > 0:
                assert enc.pool_size[l] == st["pool_size"][l], (what, eng, l)
                assert enc.ranges[l] == st["ranges"][l] or st["pool_size"][l] == 0, (what, eng, l)
        assert_same_codes(enc.codes, want, B_max, f"{what}/{eng}")
        outs[eng] = enc
    np.testing.assert_array_equal(outs["tensor"].codes, outs["plain"].codes)
    return outs, want


# ---------------------------------------------------------------- named workloads

def test_tiny64_paper_S_and_k16_grid(pkg):
    """64x64, seed 0: fixed 8x8 ranges, 16x16 domains at step 4 (169 x 8),
    no filter, no split; the paper's S set and the k/16 grid."""
    img = fic_synth.workload_image("tiny64")
    for ss in ([(10, [2, 4])], [(16, list(range(1, 17)))], [(10, [1])], [(10, [3, 8])]):
        outs, _ = check_against_oracle(pkg, img, 8, 8, 4, -1.0, ss, 8.0, f"tiny64 {ss}")
        assert outs["tensor"].matches == [64 * 169 * 8]


def test_plain256_entropy_pool_quadtree(pkg):
    """256x256, seed 1: quadtree 8 -> 4, L = 2, entropy > 4.0 bits, RMS 8."""
    w = fic_synth.WORKLOADS["plain256"]
    img = fic_synth.workload_image("plain256")
    ss = pkg.paper_ssets(w["B_max"], w["B_min"])
    outs, _ = check_against_oracle(pkg, img, w["B_max"], w["B_min"], w["L"],
                                   w["entropy_thresh"], ss, w["err_tol"], "plain256")
    assert outs["tensor"].n_positions == [14641, 15625]


@pytest.mark.parametrize("case", [
    dict(N=48, B_max=16, B_min=4, L=1, thr=-1.0, tol=8.0, seed=11),
    dict(N=96, B_max=16, B_min=4, L=3, thr=-1.0, tol=5.0, seed=12),
    dict(N=80, B_max=8, B_min=2, L=2, thr=3.5, tol=4.0, seed=13),
    dict(N=64, B_max=16, B_min=2, L=2, thr=4.0, tol=6.0, seed=14),
    dict(N=40, B_max=4, B_min=2, L=1, thr=2.0, tol=3.0, seed=15),
    dict(N=112, B_max=16, B_min=8, L=5, thr=5.5, tol=10.0, seed=16),
])
def test_ragged_quadtree_cases(pkg, case):
    """Several tiles with ragged tails in rows (ranges) and columns (pool)."""
    img = fic_synth.one_over_f(case["N"], case["seed"], 1.8)
    ss = pkg.paper_ssets(case["B_max"], case["B_min"])
    check_against_oracle(pkg, img, case["B_max"], case["B_min"], case["L"], case["thr"], ss,
                         case["tol"], f"ragged {case}")


@pytest.mark.parametrize("kind", ["black", "white", "checker", "binary_noise", "ramp"])
def test_extreme_values_exact(pkg, kind):
    """Extremes of the centred FP16 operands: all-black ranges and domains give
    the largest partial sums (16,711,680 at 16x16); checkerboards and 0/255
    noise mix signs."""
    N = 64
    rng = np.random.default_rng(5)
    if kind == "black":
        img = np.zeros((N, N), np.uint8)
    elif kind == "white":
        img = np.full((N, N), 255, np.uint8)
    elif kind == "checker":
        img = (((np.indices((N, N)).sum(0)) % 2) * 255).astype(np.uint8)
    elif kind == "binary_noise":
        img = (rng.integers(0, 2, (N, N)) * 255).astype(np.uint8)
    else:
        img = (np.add.outer(np.arange(N), np.arange(N)) * 2).clip(0, 255).astype(np.uint8)
    ss = [(10, [1]), (10, [2, 4]), (10, [3, 8])]
    check_against_oracle(pkg, img, 16, 4, 1, -1.0, ss, 8.0, f"extreme {kind}")


def test_host_and_device_inputs_agree(pkg):
    img = fic_synth.one_over_f(64, 21)
    ss = pkg.paper_ssets(16, 4)
    a = encode(pkg, img, 16, 4, 2, -1.0, ss, 6.0, "tensor", device=True)
    b = encode(pkg, img, 16, 4, 2, -1.0, ss, 6.0, "tensor", device=False)
    np.testing.assert_array_equal(a.codes, b.codes)
    c = pkg.fic_encode(img, 64, 16, 4, 2, -1.0, ss, 6.0)
    np.testing.assert_array_equal(a.codes, c.codes)


def test_device_codes_output(pkg):
    import torch
    img = fic_synth.one_over_f(64, 22)
    ss = pkg.paper_ssets(16, 4)
    ref = encode(pkg, img, 16, 4, 2, -1.0, ss, 6.0, "tensor")
    buf = torch.zeros(ref.n_codes * 16, dtype=torch.uint8, device="cuda")
    enc = pkg.fic_encode_ex(torch.from_numpy(img).cuda(), 64, 16, 4, 2, -1.0, ss, 6.0,
                            codes_out=buf, stream=torch.cuda.current_stream())
    got = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=pkg.CODE_DTYPE)
    np.testing.assert_array_equal(got, ref.codes)
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.FicError) as e:
        pkg.fic_encode_ex(torch.from_numpy(img).cuda(), 64, 16, 4, 2, -1.0, ss, 6.0,
                          codes_out=small)
    assert e.value.status == pkg.fic.FIC_ECAP


def test_repeatable(pkg):
    img = fic_synth.one_over_f(128, 23)
    ss = pkg.paper_ssets(16, 4)
    a = encode(pkg, img, 16, 4, 1, -1.0, ss, 8.0, "tensor")
    b = encode(pkg, img, 16, 4, 1, -1.0, ss, 8.0, "tensor")
    np.testing.assert_array_equal(a.codes, b.codes)


# ---------------------------------------------------------------- pool (kernels a, b)

@pytest.mark.parametrize("B,L,thr", [(8, 2, 4.0), (4, 2, 4.0), (16, 3, 6.5), (2, 1, 1.5)])
def test_domain_pool_and_entropy(pkg, B, L, thr):
    img = fic_synth.workload_image("plain256")
    xy, ent, near = pkg.fic_domain_pool(img, 256, B, L, thr)
    pl = oracle.Pool(img, B, L, thr)
    np.testing.assert_array_equal(xy, pl.positions())
    assert near == pl.near_thresh
    per = (256 - 2 * B) // L + 1
    idx = np.random.default_rng(0).choice(per * per, 300, replace=False)
    for i in idx:
        x, y = (i % per) * L, (i // per) * L
        assert abs(ent[i] - oracle.entropy_bits(img, int(x), int(y), 2 * B)) < 1e-12


# ---------------------------------------------------------------- decoder

def test_gpu_decoder_matches_oracle_decoder(pkg):
    w = fic_synth.WORKLOADS["plain256"]
    img = fic_synth.workload_image("plain256")
    ss = pkg.paper_ssets(w["B_max"], w["B_min"])
    enc = encode(pkg, img, w["B_max"], w["B_min"], w["L"], w["entropy_thresh"], ss, w["err_tol"],
                 "tensor")
    for iters in (1, 3, 64):
        got, used = pkg.fic_decode(enc, iters_max=iters)
        want, wused = oracle.decode(to_oracle_records(enc.codes, w["B_max"]), ss, 256, iters)
        np.testing.assert_array_equal(got, want)
        assert used == wused


def test_decoder_mean_only_records(pkg):
    img = fic_synth.one_over_f(32, 5)
    ss = [(10, [3, 8]), (10, [5, 9])]
    enc = encode(pkg, img, 4, 2, 2, 4.0, ss, 0.0, "tensor")
    assert enc.pool_size[1] == 0
    assert (enc.codes["s_idx"][enc.codes["level"] == 1] == 0xFF).all()
    got, used = pkg.fic_decode(enc, iters_max=8)
    want, _ = oracle.decode(to_oracle_records(enc.codes, 4), ss, 32, 8)
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- full-size workload

def test_precision512_engines_agree_and_sampled_oracle(pkg):
    """512x512 texture + edges, quadtree 16 -> 8 -> 4, L = 1, full pool.
    Tensor and CUDA-core engines must agree on every record; sampled ranges
    at every step are re-searched by the oracle one by one."""
    w = fic_synth.WORKLOADS["precision512"]
    img = fic_synth.workload_image("precision512")
    ss = pkg.paper_ssets(w["B_max"], w["B_min"])
    t = encode(pkg, img, w["B_max"], w["B_min"], w["L"], -1.0, ss, w["err_tol"], "tensor")
    p = encode(pkg, img, w["B_max"], w["B_min"], w["L"], -1.0, ss, w["err_tol"], "plain")
    np.testing.assert_array_equal(t.codes, p.codes)
    assert t.n_positions == [481 ** 2, 497 ** 2, 505 ** 2]
    assert t.pool_size == t.n_positions
    codes = t.codes
    rng = np.random.default_rng(0)
    e16 = round(16 * w["err_tol"])
    for lvl in range(3):
        B = 16 >> lvl
        n = B * B
        q, ps = ss[lvl]
        pool = oracle.Pool(img, B, 1, -1.0)
        leaves = np.nonzero(codes["level"] == lvl)[0]
        pick = rng.choice(leaves, min(12, leaves.size), replace=False) if leaves.size else []
        if len(pick):
            sc, pi, iso, si = pool.search(codes["rx"][pick], codes["ry"][pick], ss[lvl])
            np.testing.assert_array_equal(pi, codes["pool_idx"][pick].astype(np.int64))
            np.testing.assert_array_equal(iso, codes["iso"][pick])
            np.testing.assert_array_equal(si, codes["s_idx"][pick])
            if lvl < 2:  # kept at a non-final step: RMS error within the tolerance
                assert (256 * sc <= 16 * q * q * n * n * e16 * e16).all()
        # parents of deeper leaves were split: their best exceeds the tolerance
        deeper = np.nonzero(codes["level"] > lvl)[0]
        if deeper.size:
            par = rng.choice(deeper, min(8, deeper.size), replace=False)
            px = (codes["rx"][par] // B) * B
            py = (codes["ry"][par] // B) * B
            sc, *_ = pool.search(px, py, ss[lvl])
            assert (256 * sc > 16 * q * q * n * n * e16 * e16).all()
