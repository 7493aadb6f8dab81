"""Graph-captured encodes: a configuration encoded before replays one CUDA
graph of the whole quadtree with the counts kept in device memory.  Records
and counters must equal the step-by-step (eager) encode's and the oracle's,
for images whose quadtrees differ (the graph is captured once per
configuration, not per image)."""
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
    yield p
    p.fic_graph_mode(1)


def _counters(enc):
    return (enc.n_codes, enc.n_positions, enc.pool_size, enc.ranges, enc.matches,
            enc.near_thresh)


def _eager(pkg, fn):
    prev = pkg.fic_graph_mode(0)
    try:
        return fn()
    finally:
        pkg.fic_graph_mode(prev)


CONFIGS = [
    # (N, B_max, B_min, L, thr, pool_dn, tol, engine)
    (96, 16, 4, 2, 4.0, 0, 8.0, 0),     # entropy-threshold pool (pool size on the device)
    (64, 16, 4, 1, -1.0, 0, 8.0, 0),    # full pool, L = 1
    (64, 16, 2, 2, -1.0, 64, 12.0, 0),  # top-DN pool, all four steps
    (64, 8, 4, 2, 4.0, 0, 8.0, 1),      # CUDA-core engine
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_graph_replays_match_eager_and_oracle(pkg, cfg):
    N, bmax, bmin, L, thr, dn, tol, engine = cfg
    ss = [PAPER_S[b] for b in (16, 8, 4, 2) if bmin <= b <= bmax]
    imgs = [fic_synth.with_step_edges(N, 300 + 7 * k, alpha=1.5 + 0.25 * k) for k in range(4)]

    def enc(im):
        return pkg.fic_encode_ex(im, N, bmax, bmin, L, thr, ss, tol, engine=engine, pool_dn=dn)

    eager = [_eager(pkg, lambda im=im: enc(im)) for im in imgs]
    c0, r0 = pkg.fic_graph_counts()
    graph = [enc(im) for im in imgs]  # first: eager + noted; then capture, replays
    c1, r1 = pkg.fic_graph_counts()
    assert c1 - c0 <= 1 and r1 - r0 >= len(imgs) - 1
    for e, g in zip(eager, graph):
        np.testing.assert_array_equal(g.codes, e.codes)
        assert _counters(g) == _counters(e)
    # the quadtrees differ from image to image
    assert len({tuple(e.ranges) for e in eager}) > 1
    # one replayed image against the oracle
    want, _ = oracle.encode(imgs[-1], bmax, bmin, L, thr, ss, tol, pool_dn=dn)
    assert_same_codes(graph[-1].codes, want, bmax, f"graph replay {cfg}")


def test_graph_batch_replay_matches_single_encodes(pkg):
    sides = (64, 128, 96, 64)
    ss = [PAPER_S[b] for b in (16, 8, 4)]
    sets = [[fic_synth.one_over_f(n, 500 + 10 * r + i, 2.0) for i, n in enumerate(sides)]
            for r in range(3)]
    for imgs in sets:
        alone = _eager(pkg, lambda imgs=imgs: [
            pkg.fic_encode_ex(im, im.shape[0], 16, 4, 2, 4.0, ss, 8.0).codes for im in imgs])
        got = pkg.fic_encode_batch(imgs, 16, 4, 2, 4.0, ss, 8.0)
        for enc, want in zip(got, alone):
            np.testing.assert_array_equal(enc.codes, want)
    cap, rep = pkg.fic_graph_counts()
    assert cap >= 1 and rep >= 1


def test_graph_device_output_and_capacity(pkg):
    import torch
    N = 64
    ss = [PAPER_S[b] for b in (16, 8, 4)]
    img = fic_synth.with_step_edges(N, 901, alpha=2.0)
    dimg = torch.from_numpy(img).cuda()
    want = _eager(pkg, lambda: pkg.fic_encode_ex(img, N, 16, 4, 1, -1.0, ss, 8.0))
    out = torch.empty((N // 4) ** 2 * 16, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        enc = pkg.fic_encode_ex(dimg, N, 16, 4, 1, -1.0, ss, 8.0, codes_out=out)
        assert enc.n_codes == want.n_codes
        got = out[: enc.n_codes * 16].cpu().numpy().view(pkg.CODE_DTYPE)
        np.testing.assert_array_equal(got, want.codes)
    small = torch.empty(16 * (want.n_codes - 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.FicError) as ei:
        pkg.fic_encode_ex(dimg, N, 16, 4, 1, -1.0, ss, 8.0, codes_out=small)
    assert ei.value.status == -7  # FIC_ECAP


def test_graph_stats_count_the_same_work(pkg):
    N = 64
    ss = [PAPER_S[b] for b in (16, 8, 4)]
    img = fic_synth.with_step_edges(N, 77, alpha=2.0)

    def run():
        pkg.fic_stats_reset(timing=True)
        enc = pkg.fic_encode_ex(img, N, 16, 4, 1, -1.0, ss, 8.0)
        return enc, pkg.fic_stats_read()

    _eager(pkg, run)  # tunes the shapes (no tuning launches in the counted call)
    e_enc, e_st = _eager(pkg, run)
    for _ in range(3):
        g_enc, g_st = run()
    np.testing.assert_array_equal(g_enc.codes, e_enc.codes)
    assert g_st["matches"] == e_st["matches"] == e_enc.total_matches
    assert g_st["contract_tc"]["flops"] == pytest.approx(e_st["contract_tc"]["flops"])
    assert g_st["contract_tc"]["launches"] == e_st["contract_tc"]["launches"]
    assert g_st["contract_tc"]["ms"] > 0.0
    # the memory-bound stages count the same algorithmic bytes
    for k in ("gather", "range_prep", "split", "order"):
        assert g_st[k]["bytes"] == pytest.approx(e_st[k]["bytes"]), k
