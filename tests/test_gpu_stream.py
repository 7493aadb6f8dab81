"""GPU parity of the stored stream (fic_pack, Sec. 3.3, Fig. 7, eq. 8): the
library's bytes equal the oracle's for the same records, and the oracle's
reader gets the records back."""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes, to_oracle_records

pytestmark = pytest.mark.gpu

PAPER_S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8]), 2: (10, [5, 9])}


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


@pytest.mark.parametrize("case", [
    dict(N=128, B_max=16, B_min=4, L=2, thr=4.0, dn=0, tol=8.0, seed=5),     # threshold pools
    dict(N=128, B_max=16, B_min=2, L=2, thr=-1.0, dn=64, tol=12.0, seed=6),  # top-64, 4 steps
    dict(N=96, B_max=8, B_min=4, L=1, thr=-1.0, dn=0, tol=8.0, seed=7),      # full pools
    dict(N=64, B_max=8, B_min=2, L=1, thr=4.0, dn=0, tol=2.0, seed=8),       # empty last pool
    dict(N=256, B_max=16, B_min=4, L=3, thr=5.5, dn=0, tol=10.0, seed=9),    # bitmap lists
])
def test_stream_matches_oracle(pkg, case):
    img = fic_synth.with_step_edges(case["N"], case["seed"], alpha=2.5)
    sides = []
    b = case["B_max"]
    while b >= case["B_min"]:
        sides.append(b)
        b //= 2
    ss = [PAPER_S[s] for s in sides]
    enc = pkg.fic_encode_ex(img, case["N"], case["B_max"], case["B_min"], case["L"], case["thr"],
                            ss, case["tol"], pool_dn=case["dn"])
    got, pbits = pkg.fic_pack(img, enc, case["B_max"], case["B_min"], case["L"], case["thr"], ss,
                              case["tol"], pool_dn=case["dn"])
    want_codes, st = oracle.encode(img, case["B_max"], case["B_min"], case["L"], case["thr"], ss,
                                   case["tol"], pool_dn=case["dn"])
    assert_same_codes(enc.codes, want_codes, case["B_max"])
    want, wbits = oracle.pack(img, want_codes, case["B_max"], len(sides), case["L"], case["thr"],
                              ss, st["ranges"], pool_dn=case["dn"])
    assert pbits == wbits
    assert got == want
    back, ss2, N2, _ = oracle.unpack(got)
    assert N2 == case["N"] and ss2 == ss
    np.testing.assert_array_equal(back["pool_idx"], want_codes["pool_idx"])
    np.testing.assert_array_equal(back["dx"], want_codes["dx"])


def test_stream_of_device_records_and_size_query(pkg):
    import torch
    img = fic_synth.with_step_edges(128, 3, alpha=2.5)
    ss = [PAPER_S[s] for s in (16, 8, 4)]
    cap = (128 // 4) ** 2
    dcodes = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
    dimg = torch.from_numpy(img).cuda()
    enc_d = pkg.fic_encode_ex(dimg, 128, 16, 4, 2, 4.0, ss, 8.0, codes_out=dcodes)
    enc_h = pkg.fic_encode_ex(img, 128, 16, 4, 2, 4.0, ss, 8.0)
    a, _ = pkg.fic_pack(dimg, enc_d, 16, 4, 2, 4.0, ss, 8.0)
    b, _ = pkg.fic_pack(img, enc_h, 16, 4, 2, 4.0, ss, 8.0)
    assert a == b
    # a result from another image is rejected (its pool sizes do not match)
    other = fic_synth.with_step_edges(128, 4, alpha=1.5)
    with pytest.raises(pkg.FicError):
        pkg.fic_pack(other, enc_h, 16, 4, 2, 4.0, ss, 8.0)


@pytest.mark.parametrize("tol", [2.0, 16.0])
def test_ratedist_stream_matches_oracle_at_two_tolerances(pkg, tol):
    """The rate-distortion sweep's configuration (the 512 x 512 precision
    image, 16 -> 2, L = 2, top-64 pools, the paper's S per step) at both ends
    of the swept tolerance: the records, the stream bytes and the record
    bits equal the oracle's writer on the oracle's own encode."""
    img = fic_synth.workload_image("precision512")
    ss = [PAPER_S[s] for s in (16, 8, 4, 2)]
    enc = pkg.fic_encode_ex(img, 512, 16, 2, 2, -1.0, ss, tol, pool_dn=64)
    got, pbits = pkg.fic_pack(img, enc, 16, 2, 2, -1.0, ss, tol, pool_dn=64)
    want_codes, st = oracle.encode(img, 16, 2, 2, -1.0, ss, tol, pool_dn=64)
    assert_same_codes(enc.codes, want_codes, 16)
    want, wbits = oracle.pack(img, want_codes, 16, 4, 2, -1.0, ss, st["ranges"], pool_dn=64)
    assert pbits == wbits and got == want
