"""Seeded 1/f-spectrum grey-level images standing in for the paper's test images.

The paper evaluates on Lena, F16, Baboon and Boat (Sec. 4, Tables 2-6), which
are not available here.  These generators make natural-image-like stand-ins
with the same pixel format (8-bit grey levels) and a power-law spectrum.

Recipe (all randomness from ``numpy.random.default_rng(seed)``):
  1. ``z = rng.standard_normal((N, N))``, ``Z = fft2(z)``.
  2. Multiply ``Z`` by ``|f|**(-alpha/2)`` with ``|f| = hypot(fx, fy)`` from
     ``fftfreq(N)``; the DC term is set to 0.  ``alpha = 2`` means amplitude 1/f,
     power 1/f^2.
  3. ``x = real(ifft2(Z))``; min-max rescale to [0, 255].
  4. Optional step edges (see ``with_step_edges``), then clip to [0, 255].
  5. ``np.rint`` (round half to even) and cast to uint8.
"""
from __future__ import annotations

import numpy as np


def _one_over_f_float(n: int, rng: np.random.Generator, alpha: float) -> np.ndarray:
    z = rng.standard_normal((n, n))
    fz = np.fft.fft2(z)
    fx = np.fft.fftfreq(n)[None, :]
    fy = np.fft.fftfreq(n)[:, None]
    f = np.hypot(fx, fy)
    f[0, 0] = 1.0
    fz = fz * f ** (-alpha / 2.0)
    fz[0, 0] = 0.0
    x = np.real(np.fft.ifft2(fz))
    lo, hi = x.min(), x.max()
    if hi > lo:
        x = (x - lo) * (255.0 / (hi - lo))
    else:
        x = np.zeros_like(x)
    return x


def one_over_f(n: int, seed: int, alpha: float = 2.0) -> np.ndarray:
    """N x N uint8 image with a 1/f^alpha power spectrum (steps 1-3, 5)."""
    rng = np.random.default_rng(seed)
    x = _one_over_f_float(n, rng, alpha)
    return np.rint(np.clip(x, 0.0, 255.0)).astype(np.uint8)


def with_step_edges(n: int, seed: int, n_edges: int = 16, alpha: float = 2.0,
                    contrast=(40.0, 120.0)) -> np.ndarray:
    """1/f texture plus ``n_edges`` random axis-aligned step edges.

    Each edge draws, from the same generator after the noise: an orientation
    (vertical or horizontal line), the line coordinate ``c`` in [N/8, 7N/8), a
    span ``[s0, s0 + len)`` along the line (start in [0, N/2), length in
    [N/4, N/2]), a depth in [N/16, N/4], a sign and a contrast U[40, 120].
    The signed contrast is added to the rectangle that starts at the line and
    extends ``depth`` pixels to its far side (coordinates c .. c+depth-1)
    inside the span.  The sum is clipped to [0, 255] before rounding.
    """
    rng = np.random.default_rng(seed)
    x = _one_over_f_float(n, rng, alpha)
    for _ in range(n_edges):
        vertical = bool(rng.integers(0, 2))
        c = int(rng.integers(n // 8, n - n // 8))
        s0 = int(rng.integers(0, n // 2))
        ln = int(rng.integers(n // 4, n // 2 + 1))
        depth = int(rng.integers(n // 16, n // 4 + 1))
        sign = 1.0 if rng.integers(0, 2) else -1.0
        amp = float(rng.uniform(contrast[0], contrast[1]))
        s1 = min(n, s0 + ln)
        c1 = min(n, c + depth)
        if vertical:
            x[s0:s1, c:c1] += sign * amp
        else:
            x[c:c1, s0:s1] += sign * amp
    return np.rint(np.clip(x, 0.0, 255.0)).astype(np.uint8)


# Named workloads: image recipe + encoder parameters.  S sets are given as
# (q, [p...]) so that S = p/q; they follow the paper's predefined contrast
# factors keyed by range size (Sec. 3.2): 16x16 {0.1}, 8x8 {0.2, 0.4},
# 4x4 {0.3, 0.8}, 2x2 {0.5, 0.9}.
PAPER_S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}
GRID16_S = (16, list(range(1, 17)))

WORKLOADS = {
    # 64x64, fixed 8x8 ranges, 16x16 domains at step 4, no entropy filter, no split.
    "tiny64": dict(image=("one_over_f", 64, 0, 2.0), B_max=8, B_min=8, L=4,
                   entropy_thresh=-1.0, err_tol=8.0),
    # 256x256, quadtree 8 -> 4, L=2, entropy > 4.0 bits, RMS tolerance 8.
    "plain256": dict(image=("one_over_f", 256, 1, 2.0), B_max=8, B_min=4, L=2,
                     entropy_thresh=4.0, err_tol=8.0),
    # 512x512 texture + 16 step edges, quadtree 16 -> 8 -> 4, L=1, full pool.
    "precision512": dict(image=("with_step_edges", 512, 2, 2.0), B_max=16, B_min=4, L=1,
                         entropy_thresh=-1.0, err_tol=8.0),
}


def workload_image(name: str) -> np.ndarray:
    kind, n, seed, alpha = WORKLOADS[name]["image"]
    if kind == "one_over_f":
        return one_over_f(n, seed, alpha)
    return with_step_edges(n, seed, alpha=alpha)


def batch_images(count: int = 64, seed0: int = 100,
                 sides=(128, 256, 384, 512, 768, 1024), alpha_range=(1.5, 2.5)):
    """``count`` images with seeds seed0+i; side and spectral exponent drawn
    from a generator seeded with the image's own seed."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.choice(np.asarray(sides)))
        alpha = float(rng.uniform(*alpha_range))
        out.append(one_over_f(n, seed0 + i, alpha))
    return out


def poisson_requests(count: int, seed: int = 7, mean_rate_hz: float = 200.0,
                     sides=(256, 512, 1024, 2048), alpha: float = 2.0):
    """Arrival times (s, exponential inter-arrival gaps) and image sides for a
    Poisson request stream.  Images are generated lazily by the caller with
    ``one_over_f(side, seed * 100000 + i, alpha)``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / mean_rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sz = rng.choice(np.asarray(sides), size=count)
    return t, sz.astype(int)
