"""GB300 (sm_103a) range-domain block search of the modified fast fractal
image encoder (Salarian & Miar Naimi, arXiv 1502.00324).

The search runs in hand-written CUDA kernels behind the C ABI of
include/fic.h (libfic.so); ``fic`` is its thin ctypes binding.
"""
from .fic import (  # noqa: F401
    ENGINE_PLAIN,
    ENGINE_TENSOR,
    CODE_DTYPE,
    Encoded,
    FicError,
    Server,
    fic_decode,
    fic_domain_pool,
    fic_encode,
    fic_encode_batch,
    fic_encode_ex,
    fic_pack,
    fic_graph_counts,
    fic_graph_mode,
    fic_tune_mode,
    fic_tune_read,
    fic_stats_read,
    fic_stats_reset,
    fic_version,
    lib,
)

# The paper's predefined contrast factors (Sec. 3.2), keyed by range side:
# step 1 (16x16) S = 0.1, step 2 (8x8) {0.2, 0.4}, step 3 (4x4) {0.3, 0.8},
# step 4 (2x2) {0.5, 0.9}; as (q, [p...]) with S = p / q.
PAPER_S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}


def paper_ssets(B_max, B_min):
    """S sets for the quadtree steps B_max, B_max/2, ..., B_min."""
    out = []
    b = B_max
    while b >= B_min:
        out.append(PAPER_S[b])
        b //= 2
    return out
