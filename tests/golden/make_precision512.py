"""Write precision512_oracle.json: the oracle's full encode of the 512 x 512
precision workload (1/f texture, alpha 2, seed 2, 16 step edges; quadtree
16 -> 8 -> 4, domains at step L = 1, full pool, the paper's predefined S per
step, RMS tolerance 8).

Every value in the file comes from the oracle (oracle/) on the seeded input
image (fic_synth); nothing is taken from the CUDA path.  The records are stored
as one SHA-256 per record field (int64 little-endian, in record order, a
mean-only record's S index as -1), beside the per-step counts and the decoded
PSNR (eq. 4), so that a GPU test can check every record of the full-size encode
and name the field that differs.

    python tests/golden/make_precision512.py [--threads T]

The encode runs about 4e10 matches through the plain C oracle: tens of minutes
on a few host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import fic_synth  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "precision512_oracle.json")
FIELDS = ("rx", "ry", "level", "B", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx")
# the paper's predefined S per step, keyed by block side (Sec. 3.2)
PAPER_S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8])}


def field_digests(rec: dict) -> dict:
    """SHA-256 of each field as int64 little-endian, in record order."""
    return {f: hashlib.sha256(np.ascontiguousarray(rec[f], dtype="<i8").tobytes()).hexdigest()
            for f in FIELDS}


def oracle_fields(codes: np.ndarray) -> dict:
    return {f: codes[f].astype(np.int64) for f in FIELDS}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    w = fic_synth.WORKLOADS["precision512"]
    img = fic_synth.workload_image("precision512")
    sides = [w["B_max"] >> l for l in range(3)]
    ss = [PAPER_S[b] for b in sides]
    t0 = time.time()
    codes, st = oracle.encode(img, w["B_max"], w["B_min"], w["L"], -1.0, ss, w["err_tol"],
                              nthreads=args.threads)
    secs = time.time() - t0
    dec, iters = oracle.decode(codes, ss, img.shape[0])
    rec = oracle_fields(codes)
    out = {
        "_about": ("Oracle full encode of the 512x512 precision workload; written by "
                   "tests/golden/make_precision512.py from oracle/ alone (no CUDA-path value)."),
        "workload": {"name": "precision512", "N": int(img.shape[0]), "B_max": w["B_max"],
                     "B_min": w["B_min"], "L": w["L"], "entropy_thresh": None,
                     "err_tol": w["err_tol"], "S": ss,
                     "image_sha256": hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest()},
        "ranges": [int(x) for x in st["ranges"]],
        "pool_size": [int(x) for x in st["pool_size"]],
        "matches": [int(r) * int(p) * 8 for r, p in zip(st["ranges"], st["pool_size"])],
        "n_records": int(len(codes)),
        "records_per_level": [int((codes["level"] == l).sum()) for l in range(3)],
        "field_sha256": field_digests(rec),
        "decode_iters": int(iters),
        "psnr_db": float(oracle.psnr(img, dec)),
        "oracle_seconds": round(secs, 1),
        "oracle_threads": int(args.threads or oracle.max_threads()),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({k: out[k] for k in ("ranges", "n_records", "psnr_db", "oracle_seconds")}))


if __name__ == "__main__":
    main()
