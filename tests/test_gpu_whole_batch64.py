"""The 64-image batching workload in the launch configuration the benchmark
times (all 64 images in one fic_encode_batch call), against the oracle's own
full encodes of its images of side <= 384 and four of side 512 (38 of the 64).

Those encodes are stored as per-field SHA-256 digests with per-step counts in
tests/golden/batch64_oracle.json, written by tests/golden/make_batch64.py
from the oracle alone.  Every stored image's records must match field for
field, with both engines.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import fic_synth
from tests.codes import field_digests, gpu_to_common

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch64_oracle.json")


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


@pytest.mark.parametrize("engine", ["tensor", "plain"])
def test_batch64_images_match_the_oracle_encodes(pkg, engine):
    import torch
    gold = json.load(open(GOLD))
    gw = gold["workload"]
    imgs = fic_synth.batch_images(gw["count"], gw["seed0"])
    ss = pkg.paper_ssets(gw["B_max"], gw["B_min"])
    assert [[q, list(p)] for q, p in ss] == gw["S"]
    e = pkg.ENGINE_TENSOR if engine == "tensor" else pkg.ENGINE_PLAIN
    dimgs = [torch.from_numpy(im).cuda() for im in imgs]
    got = pkg.fic_encode_batch(dimgs, gw["B_max"], gw["B_min"], gw["L"], gw["entropy_thresh"],
                               ss, gw["err_tol"], engine=e, stream=torch.cuda.current_stream())
    assert len(got) == len(imgs)
    assert len(gold["images"]) > 0
    for g in gold["images"]:
        i = g["index"]
        img, enc = imgs[i], got[i]
        what = f"{engine} image {i} (N={g['N']})"
        assert hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest() == \
            g["image_sha256"], what
        assert enc.N == g["N"], what
        # steps that no range reached are not built on the GPU
        for lvl in range(enc.n_levels):
            if enc.ranges[lvl] > 0:
                assert enc.pool_size[lvl] == g["pool_size"][lvl], (what, lvl)
                assert enc.ranges[lvl] == g["ranges"][lvl] or g["pool_size"][lvl] == 0, \
                    (what, lvl)
        assert len(enc.codes) == g["n_records"], what
        dg = field_digests(gpu_to_common(enc.codes, gw["B_max"]))
        bad = [f for f in dg if dg[f] != g["field_sha256"][f]]
        assert not bad, f"{what}: record fields differ from the oracle's encode: {bad}"


def test_batch64_remaining_images_sampled_oracle(pkg):
    """The images of the 64-image workload whose whole oracle encode is not
    stored (the larger sides, which reach the large-pool and many-chunk
    paths), from the same one-call batch the benchmark times: every image's
    records tile it in the stored order, every step's pool equals the
    oracle's, and a stratified sample of at least 64 leaves per step (image
    border, the end of the pool, the rest at random) plus 16 split parents
    per step are re-searched by the oracle one by one."""
    import torch
    from tests.sampled import check_sampled
    gold = json.load(open(GOLD))
    gw = gold["workload"]
    stored = {g["index"] for g in gold["images"]}
    imgs = fic_synth.batch_images(gw["count"], gw["seed0"])
    ss = pkg.paper_ssets(gw["B_max"], gw["B_min"])
    dimgs = [torch.from_numpy(im).cuda() for im in imgs]
    got = pkg.fic_encode_batch(dimgs, gw["B_max"], gw["B_min"], gw["L"], gw["entropy_thresh"],
                               ss, gw["err_tol"], stream=torch.cuda.current_stream())
    rest = [i for i in range(len(imgs)) if i not in stored]
    assert rest, "every image has a stored encode"
    total = 0
    for i in rest:
        enc = got[i]
        total += check_sampled(imgs[i], enc.codes, enc.pool_size, gw["B_max"], gw["B_min"],
                               gw["L"], gw["entropy_thresh"], ss, gw["err_tol"],
                               f"image {i} (N={imgs[i].shape[0]})", seed=i)
    assert total >= 64 * len(rest)
