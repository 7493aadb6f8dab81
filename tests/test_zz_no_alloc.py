"""fic_domain_pool_noalloc: the allocation-free domain-pool entry point.

Callers that cannot allocate device memory (host callbacks, plugins handed
device buffers, processes that reserve all device memory up front) pass
their own device buffers; the library keeps its intermediates in a static
device array.  This test calls the entry point through the C ABI and checks
its output against the allocating fic_domain_pool, on two calls in a row.
It lives in a file of its own that collects last.
"""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth

pytestmark = pytest.mark.gpu

CASES = [(8, 2, 4.0), (4, 1, 3.0), (16, 3, -1.0), (2, 1, 1.5)]


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


def test_noalloc_pool_matches_allocating_entry_point_twice(pkg):
    import torch
    img = fic_synth.workload_image("plain256")
    N = img.shape[0]
    d_img = torch.from_numpy(img).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        for B, L, thr in CASES:
            want_xy, want_h, want_near = pkg.fic_domain_pool(img, N, B, L, thr)
            per = (N - 2 * B) // L + 1
            d_xy = torch.full((per * per,), -1, dtype=torch.int32, device="cuda")
            d_h = torch.empty(per * per, dtype=torch.float64, device="cuda")
            dn, near = pkg.fic.fic_domain_pool_noalloc(d_img, N, B, L, thr, d_xy, d_h,
                                                       stream=stream)
            torch.cuda.synchronize()
            assert dn == len(want_xy), (call, B, L, thr)
            assert near == want_near
            packed = d_xy[:dn].cpu().numpy().view(np.uint32)
            got_xy = np.stack([packed & 0xFFFF, packed >> 16], axis=1).astype(np.int32)
            np.testing.assert_array_equal(got_xy, want_xy)
            np.testing.assert_allclose(d_h.cpu().numpy(), want_h, rtol=0, atol=1e-12)


def test_noalloc_rejects_oversize_and_small_output(pkg):
    import torch
    f = pkg.fic
    big = torch.zeros((2048, 2048), dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    # (2048 - 4 + 1)^2 positions exceed the static scratch
    with pytest.raises(f.FicError) as e:
        f.fic_domain_pool_noalloc(big, 2048, 2, 1, -1.0, out)
    assert e.value.status == f.FIC_EINVAL
    img = torch.from_numpy(fic_synth.workload_image("plain256")).cuda()
    with pytest.raises(f.FicError) as e:
        f.fic_domain_pool_noalloc(img, 256, 8, 2, -1.0, out)
    assert e.value.status == f.FIC_ECAP
    # pool positions are packed x | y << 16: a side above 65535 is refused
    # even when its position count fits the scratch
    del big
    huge = torch.zeros((65536, 65536), dtype=torch.uint8, device="cuda")
    with pytest.raises(f.FicError) as e:
        f.fic_domain_pool_noalloc(huge, 65536, 16, 128, -1.0, out)
    assert e.value.status == f.FIC_EINVAL
    del huge
    torch.cuda.empty_cache()
