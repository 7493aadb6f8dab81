"""Brute-force restatements used to pin the oracle.

Written directly from the paper's definitions with numpy primitives (rot90,
fliplr, block sums) and exact Python integers / fractions; it shares nothing
with oracle/fic_oracle.c, so a mistake in one is not repeated in the other.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def iso_numpy(block: np.ndarray, k: int) -> np.ndarray:
    """Sec. 2 isometries: rotations by 0/90/180/270 degrees clockwise (k < 4),
    and each of them mirrored left-right (k >= 4)."""
    r = np.rot90(block, -(k % 4))  # negative k: clockwise
    return np.fliplr(r) if k >= 4 else r


def decimate_numpy(img: np.ndarray, x: int, y: int, B: int) -> np.ndarray:
    """2B x 2B block -> B x B sums of 2x2 pixels (the decimated domain, times 4)."""
    blk = img[y:y + 2 * B, x:x + 2 * B].astype(np.int64)
    return blk.reshape(B, 2, B, 2).sum(axis=(1, 3))


def entropy_bits_scipy(block: np.ndarray) -> float:
    from scipy.stats import entropy
    counts = np.bincount(block.ravel().astype(np.int64), minlength=256)
    return float(entropy(counts[counts > 0], base=2))


def error_eq1_fraction(r: np.ndarray, t: np.ndarray, S: Fraction, O: Fraction) -> Fraction:
    """Eq. 1 with d_i = t_i / 4 (decimated = 2x2 mean)."""
    e = Fraction(0)
    for ri, ti in zip(r.ravel().tolist(), t.ravel().tolist()):
        v = S * Fraction(ti, 4) + O - ri
        e += v * v
    return e


def optimal_offset_eq3(r: np.ndarray, t: np.ndarray, S: Fraction) -> Fraction:
    """Eq. 3: O = mean(R) - S mean(D)."""
    n = r.size
    return Fraction(int(r.sum()), n) - S * Fraction(int(t.sum()), 4 * n)


def scaled_error_int(r: np.ndarray, t: np.ndarray, p: int, q: int) -> int:
    """16 q^2 n E(S, O*) from eq. 1 and eq. 3, computed exactly in integers.

    4 q n (S d_i + O* - r_i) = p n t_i + 4 q sum(r) - p sum(t) - 4 q n r_i =: e_i,
    so E = sum e_i^2 / (16 q^2 n^2) and 16 q^2 n E = sum e_i^2 / n (an integer).
    """
    n = r.size
    rr = [int(v) for v in r.ravel()]
    tt = [int(v) for v in t.ravel()]
    sr, st = sum(rr), sum(tt)
    tot = 0
    for ri, ti in zip(rr, tt):
        e = p * n * ti + 4 * q * sr - p * st - 4 * q * n * ri
        tot += e * e
    assert tot % n == 0
    return tot // n


def scaled_error_vec(r: np.ndarray, T: np.ndarray, p: int, q: int) -> np.ndarray:
    """Vectorised scaled_error_int: r is (n,), T is (..., n) int64."""
    n = r.size
    r = r.astype(np.int64).ravel()
    sr = int(r.sum())
    st = T.sum(axis=-1, keepdims=True)
    e = p * n * T + 4 * q * sr - p * st - 4 * q * n * r
    tot = (e * e).sum(axis=-1)
    assert np.all(tot % n == 0)
    return tot // n


def brute_pool(img: np.ndarray, B: int, L: int, thr: float):
    N = img.shape[0]
    pos = []
    for y in range(0, N - 2 * B + 1, L):
        for x in range(0, N - 2 * B + 1, L):
            if thr < 0 or entropy_bits_scipy(img[y:y + 2 * B, x:x + 2 * B]) > thr:
                pos.append((x, y))
    return pos


def entropy_quantised(block: np.ndarray, bits: int = 20) -> int:
    """floor(H 2^bits + 1/2) with H (eq. 5-6, bits) evaluated to 50 digits."""
    import mpmath
    mpmath.mp.dps = 50
    c = np.bincount(block.ravel().astype(np.int64), minlength=256)
    M = int(block.size)
    t = mpmath.fsum(int(q) * mpmath.log(int(q), 2) for q in c if q > 1)
    h = mpmath.log(M, 2) - t / M
    return int(mpmath.floor(h * 2 ** bits + mpmath.mpf(1) / 2))


def brute_top_pool(img: np.ndarray, B: int, L: int, dn: int):
    """The dn highest-entropy positions (entropy rounded to 2^-20 bit from a
    50-digit evaluation; equal values in raster order), listed in raster
    order."""
    N = img.shape[0]
    cand = []
    for y in range(0, N - 2 * B + 1, L):
        for x in range(0, N - 2 * B + 1, L):
            cand.append((entropy_quantised(img[y:y + 2 * B, x:x + 2 * B]), len(cand), (x, y)))
    order = sorted(cand, key=lambda c: (-c[0], c[1]))
    chosen = sorted(order[:dn], key=lambda c: c[1])
    return [c[2] for c in chosen]


def brute_search(img: np.ndarray, rx: int, ry: int, B: int, pool, sset):
    """Exhaustive search of one range: lexicographic min of
    (16 q^2 n E, pool index, isometry, S index)."""
    q, ps = sset
    r = img[ry:ry + B, rx:rx + B].astype(np.int64)
    if not pool:
        return None
    T = np.stack([np.stack([iso_numpy(decimate_numpy(img, x, y, B), k).ravel()
                            for k in range(8)]) for (x, y) in pool])  # (DN, 8, n)
    best = None
    for si, p in enumerate(ps):
        sc = scaled_error_vec(r, T, p, q)  # (DN, 8)
        for c in range(sc.shape[0]):
            for k in range(8):
                key = (int(sc[c, k]), c, k, si)
                if best is None or key < best:
                    best = key
    return best


def brute_encode(img: np.ndarray, B_max: int, B_min: int, L: int, thr: float, ssets, tol,
                 pool_fn=None):
    """Quadtree encoder written from Sec. 2: split while RMS error > tol and the
    step is not the last; children in TL, TR, BL, BR order.  pool_fn(B), if
    given, replaces the threshold pool of side B."""
    N = img.shape[0]
    sides = []
    b = B_max
    while b >= B_min:
        sides.append(b)
        b //= 2
    pools = [pool_fn(s) if pool_fn else brute_pool(img, s, L, thr) for s in sides]
    tol_f = Fraction(math.floor(16 * tol + 0.5), 16)  # e16 / 16, halves up
    out = []

    def rec(x, y, lvl):
        B = sides[lvl]
        n = B * B
        last = lvl == len(sides) - 1
        sr = int(img[y:y + B, x:x + B].astype(np.int64).sum())
        oq = min(127, sr // (2 * n))
        pool = pools[lvl]
        if not pool:
            if last:
                out.append(dict(rx=x, ry=y, level=lvl, B=B, iso=0, s_idx=-1, o_q=oq,
                                dx=0, dy=0, pool_idx=0xFFFFFFFF))
                return
        else:
            q, ps = ssets[lvl]
            score, c, k, si = brute_search(img, x, y, B, pool, ssets[lvl])
            E = Fraction(score, 16 * q * q * n)
            if last or not (E / n > tol_f * tol_f):
                out.append(dict(rx=x, ry=y, level=lvl, B=B, iso=k, s_idx=si, o_q=oq,
                                dx=pool[c][0], dy=pool[c][1], pool_idx=c, score=score))
                return
        h = B // 2
        rec(x, y, lvl + 1)
        rec(x + h, y, lvl + 1)
        rec(x, y + h, lvl + 1)
        rec(x + h, y + h, lvl + 1)

    for ty in range(0, N, B_max):
        for tx in range(0, N, B_max):
            rec(tx, ty, 0)
    return out


def decode_one_iteration(codes, ssets, src: np.ndarray) -> np.ndarray:
    """One decoder pass from Sec. 2 (each range rebuilt from its domain and
    mapping) with r^ = (2 o_q + 1) + S (d - mean d), d = T(d')/4, rounded half
    up and clamped to [0, 255]; exact rational arithmetic."""
    N = src.shape[0]
    dst = src.copy()
    for c in codes:
        B = int(c["B"])
        rx, ry = int(c["rx"]), int(c["ry"])
        if int(c["s_idx"]) < 0:
            dst[ry:ry + B, rx:rx + B] = 2 * int(c["o_q"]) + 1
            continue
        q, ps = ssets[int(c["level"])]
        S = Fraction(ps[int(c["s_idx"])], q)
        t = iso_numpy(decimate_numpy(src, int(c["dx"]), int(c["dy"]), B), int(c["iso"]))
        n = B * B
        mean_d = Fraction(int(t.sum()), 4 * n)
        for i in range(B):
            for j in range(B):
                v = 2 * int(c["o_q"]) + 1 + S * (Fraction(int(t[i, j]), 4) - mean_d)
                iv = (v + Fraction(1, 2)).__floor__()
                dst[ry + i, rx + j] = min(255, max(0, iv))
    return dst
