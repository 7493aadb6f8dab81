"""Every record of the full-size 512 x 512 encode against the oracle's own
full encode of the same image.

The oracle's encode (about 4e10 matches, tens of minutes on host cores) is
stored as per-field SHA-256 digests with its per-step counts and decoded PSNR
in tests/golden/precision512_oracle.json, written by
tests/golden/make_precision512.py from the oracle alone.  Both engines must
give the same records field for field; the GPU decode's PSNR (eq. 4) must be
within 0.01 dB of the oracle's.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import field_digests, gpu_to_common

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "precision512_oracle.json")


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


@pytest.mark.parametrize("engine", ["tensor", "plain"])
def test_precision512_every_record_matches_the_oracle_encode(pkg, engine):
    import torch
    gold = json.load(open(GOLD))
    gw = gold["workload"]
    w = fic_synth.WORKLOADS["precision512"]
    img = fic_synth.workload_image("precision512")
    assert hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest() == gw["image_sha256"]
    ss = pkg.paper_ssets(w["B_max"], w["B_min"])
    assert [[q, list(p)] for q, p in ss] == gw["S"]
    e = pkg.ENGINE_TENSOR if engine == "tensor" else pkg.ENGINE_PLAIN
    enc = pkg.fic_encode_ex(torch.from_numpy(img).cuda(), img.shape[0], w["B_max"], w["B_min"],
                            w["L"], -1.0, ss, w["err_tol"], engine=e,
                            stream=torch.cuda.current_stream())
    assert list(enc.ranges) == gold["ranges"]
    assert list(enc.pool_size) == gold["pool_size"]
    assert len(enc.codes) == gold["n_records"]
    got = field_digests(gpu_to_common(enc.codes, w["B_max"]))
    bad = [f for f in got if got[f] != gold["field_sha256"][f]]
    assert not bad, f"{engine}: record fields differ from the oracle's encode: {bad}"
    dec, _ = pkg.fic_decode(enc)
    assert abs(oracle.psnr(img, dec) - gold["psnr_db"]) <= 0.01
