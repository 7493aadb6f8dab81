"""Field-by-field comparison of GPU records with oracle records."""
from __future__ import annotations

import numpy as np

FIELDS = ("rx", "ry", "level", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx")


def gpu_to_common(codes: np.ndarray, B_max: int) -> dict:
    out = {f: codes[f].astype(np.int64) for f in FIELDS}
    s = out["s_idx"].copy()
    s[s == 0xFF] = -1
    out["s_idx"] = s
    out["B"] = (B_max >> out["level"]).astype(np.int64)
    return out


def oracle_to_common(codes: np.ndarray) -> dict:
    out = {f: codes[f].astype(np.int64) for f in FIELDS}
    out["B"] = codes["B"].astype(np.int64)
    return out


def assert_same_codes(gpu: np.ndarray, ora: np.ndarray, B_max: int, what: str = ""):
    g = gpu_to_common(gpu, B_max)
    o = oracle_to_common(ora)
    assert len(gpu) == len(ora), f"{what}: {len(gpu)} GPU records vs {len(ora)} oracle records"
    for f in FIELDS + ("B",):
        bad = np.nonzero(g[f] != o[f])[0]
        assert bad.size == 0, (f"{what}: field {f} differs at {bad.size} records, first {bad[0]}: "
                               f"gpu={ {k: int(g[k][bad[0]]) for k in g} } "
                               f"oracle={ {k: int(o[k][bad[0]]) for k in o} }")


def to_oracle_records(codes: np.ndarray, B_max: int):
    """GPU records -> oracle record array (for decoding with the oracle)."""
    import oracle
    g = gpu_to_common(codes, B_max)
    out = np.zeros(len(codes), oracle.CODE_DTYPE)
    for f in FIELDS + ("B",):
        out[f] = g[f]
    return out


DIGEST_FIELDS = ("rx", "ry", "level", "B", "iso", "s_idx", "o_q", "dx", "dy", "pool_idx")


def field_digests(common: dict) -> dict:
    """SHA-256 of each record field as int64 little-endian, in record order
    (a mean-only record's S index as -1): the form in which the oracle's
    full-size encodes are stored under tests/golden/."""
    import hashlib
    return {f: hashlib.sha256(np.ascontiguousarray(common[f], dtype="<i8").tobytes()).hexdigest()
            for f in DIGEST_FIELDS}
