"""Write batch64_oracle.json: the oracle's full encodes of the images of the
64-image batching workload (seeds 100..163, sides drawn from {128, 256, 384,
512, 768, 1024}, alpha in [1.5, 2.5]; quadtree 16 -> 4, domains at step
L = 2, entropy > 4.0 bits, the paper's predefined S per step, RMS tolerance
8) whose side is at most --max-side.

Every value in the file comes from the oracle (oracle/) on the seeded input
images (fic_synth); nothing is taken from the CUDA path.  Per image: seed,
side, SHA-256 of the pixels, per-step counts and one SHA-256 per record field
(int64 little-endian, in record order, a mean-only record's S index as -1).

    python tests/golden/make_batch64.py [--max-side 256] [--threads T]
    python tests/golden/make_batch64.py --add 3,4   # append images 3 and 4

``--add`` keeps the stored images and appends the oracle's encodes of the
listed image indices (of any side); ``extra_indices`` in the file lists them.
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
sys.path.insert(0, HERE)

import fic_synth  # noqa: E402
import oracle  # noqa: E402
from make_precision512 import PAPER_S, field_digests, oracle_fields  # noqa: E402

OUT = os.path.join(HERE, "batch64_oracle.json")
B_MAX, B_MIN, L, THR, TOL = 16, 4, 2, 4.0, 8.0
SEED0, COUNT = 100, 64


def encode_one(imgs, i, ss, threads):
    """The oracle's full encode of image i, as stored."""
    img = imgs[i]
    n = int(img.shape[0])
    t0 = time.time()
    codes, st = oracle.encode(img, B_MAX, B_MIN, L, THR, ss, TOL, nthreads=threads)
    rec = {
        "index": i, "seed": SEED0 + i, "N": n,
        "image_sha256": hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest(),
        "ranges": [int(x) for x in st["ranges"]],
        "pool_size": [int(x) for x in st["pool_size"]],
        "n_records": int(len(codes)),
        "field_sha256": field_digests(oracle_fields(codes)),
        "oracle_seconds": round(time.time() - t0, 2),
    }
    print(i, n, len(codes), round(time.time() - t0, 1), flush=True)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-side", type=int, default=256)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--add", default="")
    args = ap.parse_args()
    ss = [PAPER_S[b] for b in (16, 8, 4)]
    imgs = fic_synth.batch_images(COUNT, SEED0)
    if args.add:
        add = [int(x) for x in args.add.split(",")]
        out = json.load(open(OUT))
        have = {g["index"] for g in out["images"]}
        for i in add:
            if i not in have:
                out["images"].append(encode_one(imgs, i, ss, args.threads))
        out["images"].sort(key=lambda g: g["index"])
        out["extra_indices"] = sorted(set(out.get("extra_indices", [])) | set(add))
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        return
    out = {
        "_about": ("Oracle full encodes of the 64-image batching workload's images of side "
                   f"<= {args.max_side}; written by tests/golden/make_batch64.py from oracle/ "
                   "alone (no CUDA-path value)."),
        "workload": {"name": "batch64", "count": COUNT, "seed0": SEED0, "B_max": B_MAX,
                     "B_min": B_MIN, "L": L, "entropy_thresh": THR, "err_tol": TOL, "S": ss,
                     "max_side": args.max_side},
        "images": [],
    }
    t_all = time.time()
    for i, img in enumerate(imgs):
        if int(img.shape[0]) <= args.max_side:
            out["images"].append(encode_one(imgs, i, ss, args.threads))
    out["oracle_seconds_total"] = round(time.time() - t_all, 1)
    out["oracle_threads"] = int(args.threads or oracle.max_threads())
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
