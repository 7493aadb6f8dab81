"""GPU tests of the request server (fic_server_*): continuous batching.

Each request's records must be the same whether the image is encoded alone
(fic_encode_ex) or inside the server's mix, where images of different sizes
arrive while others are in flight and share contraction launches.
"""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes

pytestmark = pytest.mark.gpu

ARGS = dict(B_max=16, B_min=4, L=2, entropy_thresh=4.0, err_tol=8.0)


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


def stream_images(count, seed=7, sides=(64, 128, 256, 512)):
    """Poisson-stream shaped mix (sides cycled through a seeded draw)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(np.asarray(sides)))
        out.append(fic_synth.one_over_f(n, seed * 100000 + i, float(rng.uniform(1.5, 2.5))))
    return out


def make_server(pkg, **cfg):
    ss = pkg.paper_ssets(ARGS["B_max"], ARGS["B_min"])
    return pkg.Server(ARGS["B_max"], ARGS["B_min"], ARGS["L"], ARGS["entropy_thresh"], ss,
                      ARGS["err_tol"], **cfg)


def alone(pkg, img):
    ss = pkg.paper_ssets(ARGS["B_max"], ARGS["B_min"])
    return pkg.fic_encode_ex(img, img.shape[0], ARGS["B_max"], ARGS["B_min"], ARGS["L"],
                             ARGS["entropy_thresh"], ss, ARGS["err_tol"])


def test_mix_equals_alone_with_staggered_arrivals(pkg):
    """Requests arrive from a feeder thread at staggered times while others
    are on the GPU; every result equals the image's encode alone, and some
    images shared their steps with others."""
    import torch
    imgs = stream_images(24)
    want_enc = [alone(pkg, im) for im in imgs]
    want = [e.codes for e in want_enc]
    srv = make_server(pkg)
    tickets = [None] * len(imgs)

    def feed():
        for i, im in enumerate(imgs):
            src = torch.from_numpy(im).cuda() if i % 3 == 0 else im
            tickets[i] = srv.submit(src)
            time.sleep(0.002 * (i % 4))

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    shared = 0
    for i, t in enumerate(tickets):
        enc, tm = srv.poll(t, wait_ms=-1)
        np.testing.assert_array_equal(enc.codes, want[i], err_msg=f"request {i}")
        assert enc.N == imgs[i].shape[0]
        assert tm["submit_ms"] <= tm["admit_ms"] <= tm["done_ms"]
        assert 1 <= tm["steps"] <= 3
        shared += tm["shared_steps"]
        if imgs[i].shape[0] <= 128:  # small enough for the oracle in about a second
            ss = pkg.paper_ssets(ARGS["B_max"], ARGS["B_min"])
            ref, _ = oracle.encode(imgs[i], ARGS["B_max"], ARGS["B_min"], ARGS["L"],
                                   ARGS["entropy_thresh"], ss, ARGS["err_tol"])
            assert_same_codes(enc.codes, ref, ARGS["B_max"], f"served request {i}")
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(imgs) and st["failed"] == 0
    assert shared > 0 and st["mean_inflight"] > 1.0
    assert st["matches"] == sum(e.total_matches for e in want_enc)


def test_admission_bounded_by_hbm_budget(pkg):
    """A budget that holds one 256 x 256 image at a time: every request still
    completes, one in flight at a time, results unchanged; an image larger
    than the whole budget is refused with FIC_ENOMEM."""
    imgs = [fic_synth.one_over_f(256, 60 + i, 2.0) for i in range(5)]
    want = [alone(pkg, im).codes for im in imgs]
    with make_server(pkg) as probe:  # the estimate of one 256 x 256 slot
        probe.poll(probe.submit(imgs[0]))
        est = probe.stats()["hbm_in_use"]
    assert est > 0
    budget = est + est // 2
    srv = make_server(pkg, hbm_budget=budget)
    ts = [srv.submit(im) for im in imgs]
    big = srv.submit(fic_synth.one_over_f(1024, 5, 2.0))
    for i, t in enumerate(ts):
        enc, _ = srv.poll(t)
        np.testing.assert_array_equal(enc.codes, want[i])
    with pytest.raises(pkg.FicError) as e:
        srv.poll(big)
    assert e.value.status == pkg.fic.FIC_ENOMEM
    st = srv.stats()
    srv.close()
    assert st["hbm_peak"] <= budget
    assert st["completed"] == len(imgs) and st["failed"] == 1
    assert st["peak_inflight"] == 1


def test_slot_limit_and_ticket_errors(pkg):
    """max_inflight = 2: at most two images in flight; unknown tickets and
    invalid sides are rejected; a ticket is forgotten once polled."""
    imgs = stream_images(5, seed=13, sides=(64, 128))
    srv = make_server(pkg, max_inflight=2)
    ts = [srv.submit(im) for im in imgs]
    with pytest.raises(pkg.FicError) as e:
        srv.submit(np.zeros((40, 40), np.uint8))
    assert e.value.status == pkg.fic.FIC_EINVAL
    for t, im in zip(ts, imgs):
        enc, _ = srv.poll(t)
        np.testing.assert_array_equal(enc.codes, alone(pkg, im).codes)
    with pytest.raises(pkg.FicError) as e:
        srv.poll(ts[0])
    assert e.value.status == pkg.fic.FIC_EINVAL
    with pytest.raises(pkg.FicError):
        srv.poll(123456789)
    st = srv.stats()
    srv.close()
    assert st["peak_inflight"] <= 2 and st["completed"] == 5


def test_destroy_with_work_pending(pkg):
    """Destroying a server with queued and running requests returns cleanly
    (running images finish, queued ones are dropped)."""
    srv = make_server(pkg, max_inflight=1)
    for i in range(6):
        srv.submit(fic_synth.one_over_f(256, 40 + i, 2.0))
    srv.close()
    # the library is still usable afterwards
    img = fic_synth.one_over_f(64, 1, 2.0)
    assert alone(pkg, img).n_codes > 0


def test_smallest_first_policy_with_aging(pkg):
    """Policy 1 admits the smallest queued image first (one slot here), so
    small requests queued behind a large one finish before it; results are
    unchanged.  An unknown policy is rejected."""
    big = [fic_synth.one_over_f(384, 80 + i, 2.0) for i in range(2)]
    small = [fic_synth.one_over_f(64, 90 + i, 2.0) for i in range(3)]
    srv = make_server(pkg, max_inflight=1, policy=1, age_ms=60000)
    t_big0 = srv.submit(big[0])
    t_big1 = srv.submit(big[1])
    t_small = [srv.submit(im) for im in small]
    res = {t: srv.poll(t) for t in [t_big0, t_big1] + t_small}
    srv.close()
    done = {t: tm["done_ms"] for t, (_, tm) in res.items()}
    assert max(done[t] for t in t_small) < done[t_big1]
    for t, im in zip([t_big0, t_big1] + t_small, big + small):
        np.testing.assert_array_equal(res[t][0].codes, alone(pkg, im).codes)
    with pytest.raises(pkg.FicError) as e:
        make_server(pkg, policy=7)
    assert e.value.status == pkg.fic.FIC_EINVAL


def test_mix_with_1024_and_2048_images_equals_alone(pkg):
    """The serving workload's large sides: a 1024 x 1024 and a 2048 x 2048
    request arrive among smaller ones while others are on the GPU.  Each
    result equals the image's encode alone; the 2048 x 2048 result is also
    checked against the oracle by a stratified sample of its leaves and
    split parents at every step (the whole oracle encode of that image is
    too slow for a test)."""
    import torch
    from tests.sampled import check_sampled
    sides = (256, 1024, 64, 2048, 512, 128, 256, 64)
    imgs = [fic_synth.one_over_f(n, 7100 + i, 2.0) for i, n in enumerate(sides)]
    want = [alone(pkg, im) for im in imgs]
    srv = make_server(pkg)
    tickets = [None] * len(imgs)

    def feed():
        for i, im in enumerate(imgs):
            src = torch.from_numpy(im).cuda() if i % 2 else im
            tickets[i] = srv.submit(src)
            time.sleep(0.003)

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    got = {}
    for i, t in enumerate(tickets):
        enc, tm = srv.poll(t, wait_ms=-1)
        np.testing.assert_array_equal(enc.codes, want[i].codes, err_msg=f"request {i}")
        assert enc.pool_size == want[i].pool_size and enc.ranges == want[i].ranges
        got[i] = enc
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(imgs) and st["failed"] == 0
    i = sides.index(2048)
    ss = pkg.paper_ssets(ARGS["B_max"], ARGS["B_min"])
    n = check_sampled(imgs[i], got[i].codes, got[i].pool_size, ARGS["B_max"], ARGS["B_min"],
                      ARGS["L"], ARGS["entropy_thresh"], ss, ARGS["err_tol"], "2048 request")
    assert n >= 64 * 2
