"""Stratified sampled comparison of one image's GPU records with the oracle,
for images too large for a whole oracle encode in a test.

What it checks (paper Sec. 2 quadtree search, Sec. 3 pool, Sec. 3.3 records):
  * the records tile the image exactly once and come in the stored order
    (top-level ranges in raster order, then depth first TL, TR, BL, BR);
  * every step's pool size equals the oracle's pool of that step;
  * sampled leaves of every step are re-searched by the oracle one by one:
    the same (pool index, isometry, S index), and at a non-final step an
    error within the tolerance;
  * sampled split parents of every non-final step exceed the tolerance.
Leaves are drawn by strata: ranges on the image border, ranges whose winning
domain lies at the end of the pool (the last column chunk and its ragged
tail), and ranges drawn at random from the rest.
"""
from __future__ import annotations

import numpy as np

import oracle


def morton(x, y, bits):
    """Interleave the bits of x (low) and y (high): TL, TR, BL, BR order."""
    k = np.zeros_like(x, dtype=np.int64)
    for b in range(bits):
        k |= ((x >> b) & 1).astype(np.int64) << (2 * b)
        k |= ((y >> b) & 1).astype(np.int64) << (2 * b + 1)
    return k


def check_tiling_and_order(codes, N, B_max, B_min, what):
    rx = codes["rx"].astype(np.int64)
    ry = codes["ry"].astype(np.int64)
    B = (B_max >> codes["level"].astype(np.int64))
    cells = N // B_min
    cover = np.zeros((cells, cells), np.int32)
    for x, y, b in zip(rx // B_min, ry // B_min, B // B_min):
        cover[y:y + b, x:x + b] += 1
    assert (cover == 1).all(), f"{what}: records do not tile the image exactly once"
    tops = N // B_max
    top = (ry // B_max) * tops + (rx // B_max)
    bits = int(np.log2(B_max // B_min))
    key = top * (1 << (2 * bits)) + morton((rx % B_max) // B_min, (ry % B_max) // B_min, bits)
    assert (np.diff(key) > 0).all(), f"{what}: records not in the stored order"


def check_sampled(img, codes, pool_sizes, B_max, B_min, L, thr, ssets, tol, what,
                  per_step=64, parents=16, seed=0):
    """Stratified sampled comparison (module docstring).  pool_sizes[l] is
    the GPU's pool size at step l (steps no range reached are skipped)."""
    N = img.shape[0]
    check_tiling_and_order(codes, N, B_max, B_min, what)
    rng = np.random.default_rng(seed)
    e16 = int(np.floor(16.0 * tol + 0.5))
    n_steps = len(ssets)
    checked = 0
    for lvl in range(n_steps):
        B = B_max >> lvl
        n = B * B
        q, _ = ssets[lvl]
        here = codes["level"] == lvl
        deeper = np.nonzero(codes["level"] > lvl)[0]
        if not here.any() and not deeper.size:
            continue
        pool = oracle.Pool(img, B, L, thr)
        assert pool.dn == pool_sizes[lvl], (what, lvl, pool.dn, pool_sizes[lvl])
        leaves = np.nonzero(here & (codes["s_idx"] != 0xFF))[0]
        if leaves.size:
            border = leaves[(codes["rx"][leaves] == 0) | (codes["ry"][leaves] == 0) |
                            (codes["rx"][leaves].astype(np.int64) + B == N) |
                            (codes["ry"][leaves].astype(np.int64) + B == N)]
            tail = leaves[np.argsort(codes["pool_idx"][leaves].astype(np.int64))[-per_step // 4:]]
            pick = set(rng.choice(border, min(per_step // 4, border.size), replace=False)
                       .tolist()) if border.size else set()
            pick |= set(tail.tolist())
            rest = np.setdiff1d(leaves, np.fromiter(pick, np.int64, len(pick)))
            k = max(0, min(per_step - len(pick), rest.size))
            pick |= set(rng.choice(rest, k, replace=False).tolist()) if k else set()
            pick = np.array(sorted(pick), np.int64)
            sc, pi, iso, si = pool.search(codes["rx"][pick], codes["ry"][pick], ssets[lvl])
            np.testing.assert_array_equal(pi, codes["pool_idx"][pick].astype(np.int64),
                                          err_msg=f"{what} step {lvl} pool index")
            np.testing.assert_array_equal(iso, codes["iso"][pick], err_msg=f"{what} step {lvl}")
            np.testing.assert_array_equal(si, codes["s_idx"][pick], err_msg=f"{what} step {lvl}")
            if lvl < n_steps - 1:
                assert (256 * sc <= 16 * q * q * n * n * e16 * e16).all(), (what, lvl)
            checked += pick.size
        if deeper.size and lvl < n_steps - 1:
            par = np.unique(np.stack([(codes["rx"][deeper] // B) * B,
                                      (codes["ry"][deeper] // B) * B], axis=1), axis=0)
            sel = par[rng.choice(par.shape[0], min(parents, par.shape[0]), replace=False)]
            sc, *_ = pool.search(sel[:, 0], sel[:, 1], ssets[lvl])
            assert (256 * sc > 16 * q * q * n * n * e16 * e16).all(), (what, lvl, "parent")
            checked += sel.shape[0]
    return checked
