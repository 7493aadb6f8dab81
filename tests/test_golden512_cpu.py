"""Host checks of the stored full-size oracle encode (tests/golden/
precision512_oracle.json) and of the path by which GPU records are compared
with it: the input image is still the one that was encoded, the stored counts
obey the quadtree's arithmetic, and records in the GPU's 16-byte format give
the oracle's digests once converted."""
from __future__ import annotations

import hashlib
import importlib.util
import json
import os

import numpy as np

import fic_synth
import oracle
from tests.codes import field_digests, gpu_to_common, oracle_to_common

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "precision512_oracle.json")


def _gpu_format(codes: np.ndarray, B_max: int) -> np.ndarray:
    """Oracle records rewritten in the library's record layout (as the GPU
    writes them), so the comparison path can be run without a GPU."""
    from paper_1502_00324_gb300.fic import CODE_DTYPE
    out = np.zeros(len(codes), CODE_DTYPE)
    for f in ("rx", "ry", "dx", "dy", "pool_idx", "iso", "o_q"):
        out[f] = codes[f]
    out["level"] = codes["level"]
    assert (codes["B"] == B_max >> codes["level"]).all()
    out["s_idx"] = np.where(codes["s_idx"] < 0, 0xFF, codes["s_idx"])
    return out


def test_stored_encode_is_of_the_current_image():
    gold = json.load(open(GOLD))
    img = fic_synth.workload_image("precision512")
    assert hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest() == \
        gold["workload"]["image_sha256"]


def test_stored_counts_follow_the_quadtree():
    gold = json.load(open(GOLD))
    N, L = gold["workload"]["N"], gold["workload"]["L"]
    sides = [16, 8, 4]
    assert gold["pool_size"] == [((N - 2 * B) // L + 1) ** 2 for B in sides]
    assert gold["ranges"][0] == (N // 16) ** 2
    for l in range(2):  # every range not kept at a step has four children
        assert gold["ranges"][l + 1] == 4 * (gold["ranges"][l] - gold["records_per_level"][l])
    assert gold["records_per_level"][2] == gold["ranges"][2]  # last step keeps all
    assert sum(gold["records_per_level"]) == gold["n_records"]
    assert gold["matches"] == [r * p * 8 for r, p in zip(gold["ranges"], gold["pool_size"])]
    assert 0 < gold["psnr_db"] < 99 and 1 <= gold["decode_iters"] <= 64


def test_gpu_record_format_gives_the_oracle_digests():
    """A quadtree encode with mean-only records (empty pool at the last step):
    the digests of GPU-format records equal those of the oracle's records, and
    the writer script's own digest function agrees with the tests'."""
    img = fic_synth.workload_image("plain256")[:64, :64].copy()
    ss = [(10, [2, 4]), (10, [3, 8]), (10, [5, 9])]
    codes, _ = oracle.encode(img, 8, 2, 2, 4.0, ss, 8.0)
    assert (codes["s_idx"] < 0).any() and (codes["s_idx"] >= 0).any()
    want = field_digests(oracle_to_common(codes))
    assert field_digests(gpu_to_common(_gpu_format(codes, 8), 8)) == want
    spec = importlib.util.spec_from_file_location(
        "make_precision512", os.path.join(HERE, "golden", "make_precision512.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert mk.field_digests(mk.oracle_fields(codes)) == want
    # a change in any one field changes its digest only
    bad = codes.copy()
    bad["iso"][len(bad) // 2] ^= 1
    got = field_digests(oracle_to_common(bad))
    assert [f for f in got if got[f] != want[f]] == ["iso"]


GOLD_B64 = os.path.join(HERE, "golden", "batch64_oracle.json")


def test_stored_batch_encodes_cover_the_small_images_of_the_workload():
    gold = json.load(open(GOLD_B64))
    gw = gold["workload"]
    imgs = fic_synth.batch_images(gw["count"], gw["seed0"])
    want = [i for i, im in enumerate(imgs) if im.shape[0] <= gw["max_side"]]
    want = sorted(set(want) | set(gold.get("extra_indices", [])))
    assert [g["index"] for g in gold["images"]] == want and len(want) > 0
    for g in gold["images"]:
        img = imgs[g["index"]]
        assert g["N"] == img.shape[0] and g["seed"] == gw["seed0"] + g["index"]
        assert hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest() == \
            g["image_sha256"]
        N, L = g["N"], gw["L"]
        sides = [gw["B_max"] >> l for l in range(len(g["ranges"]))]
        assert sides[-1] == gw["B_min"]
        assert g["ranges"][0] == (N // gw["B_max"]) ** 2
        for l, B in enumerate(sides):   # entropy-filtered pools within the positions
            assert 0 <= g["pool_size"][l] <= ((N - 2 * B) // L + 1) ** 2
        for l in range(len(sides) - 1):  # split ranges have four children each
            assert g["ranges"][l + 1] % 4 == 0 and g["ranges"][l + 1] <= 4 * g["ranges"][l]
        # every range of the last step is kept; the steps before keep the rest
        kept = sum(g["ranges"][l] - g["ranges"][l + 1] // 4 for l in range(len(sides) - 1))
        assert g["n_records"] == kept + g["ranges"][-1]
