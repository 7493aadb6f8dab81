"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function include/fic.h declares, and rejects
bad arguments before touching a device."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def fic():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as pkg
    return pkg


def header_functions():
    src = open(os.path.join(ROOT, "include", "fic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fic_[a-z_]+)\s*\(", src)))


def test_library_exports_every_header_function(fic):
    names = header_functions()
    assert "fic_encode" in names and "fic_decode" in names
    lib = fic.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(fic.fic.EXPORTS) <= set(names)


def test_library_targets_sm103a(fic):
    assert "sm_103a" in fic.fic_version()


def test_strerror(fic):
    for st in range(0, -9, -1):
        assert fic.fic.strerror(st) not in ("", "unknown status")
    assert fic.fic.strerror(-99) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(N=100, B_max=16),          # N % B_max != 0
    dict(B_max=4, B_min=8),          # B_min > B_max
    dict(B_max=12),                  # not a power of two
    dict(B_max=32, N=512),           # side above 16
    dict(L=0),
    dict(err_tol=-1.0),
    dict(err_tol=300.0),
    dict(ssets=[(10, [11]), (10, [2, 4]), (10, [3, 8])]),   # S > 1
    dict(ssets=[(0, [1]), (10, [2, 4]), (10, [3, 8])]),     # q < 1
    dict(ssets=[(10, []), (10, [2, 4]), (10, [3, 8])]),     # empty set
    dict(engine=7),
])
def test_bad_arguments_rejected_on_host(fic, bad):
    args = dict(N=64, B_max=16, B_min=4, L=1, thr=-1.0, err_tol=8.0,
                ssets=[(10, [1]), (10, [2, 4]), (10, [3, 8])], engine=0, pool_dn=0)
    args.update(bad)
    img = np.zeros((args["N"], args["N"]), np.uint8)
    with pytest.raises(fic.FicError) as e:
        fic.fic_encode_ex(img, args["N"], args["B_max"], args["B_min"], args["L"], args["thr"],
                          args["ssets"], args["err_tol"], engine=args["engine"],
                          pool_dn=args["pool_dn"])
    assert e.value.status == fic.fic.FIC_EINVAL


def test_struct_layouts(fic):
    f = fic.fic
    assert C.sizeof(f.FicCode) == 16
    assert C.sizeof(f.FicSset) == 72
    # fic_result / fic_params are plain C layouts of int32/int64/double fields
    assert C.sizeof(f.FicParams) == 4 * 4 + 2 * 8 + 4 * 72 + 2 * 4


def test_process_modes_set_and_read_on_host(fic):
    # tuning and graph modes are process-wide settings: no device needed
    prev = fic.fic_graph_mode(0)
    assert prev in (0, 1)
    assert fic.fic_graph_mode(prev) == 0
    assert fic.fic_graph_mode() == prev
    with pytest.raises(fic.FicError) as e:
        fic.fic_graph_mode(2)
    assert e.value.status == fic.fic.FIC_EINVAL
    t = fic.fic_tune_mode(0)
    assert fic.fic_tune_mode(t) == 0


SS3 = [(10, [1]), (10, [2, 4]), (10, [3, 8])]


def test_binding_refuses_buffers_the_library_would_overrun(fic):
    """The library reads an N x N image and writes records, pool entries and
    entropies by the sizes passed beside the pointers; the binding refuses a
    buffer that is shorter, strided or of another element type before any
    call, so no such pointer reaches the host code or a kernel."""
    import torch
    f = fic.fic
    img = np.zeros((64, 64), np.uint8)
    with pytest.raises(ValueError, match="at least 16384"):
        f.fic_encode_ex(img, 128, 16, 4, 1, -1.0, SS3, 8.0)          # N larger than the buffer
    wide = np.zeros((64, 128), np.uint8)
    with pytest.raises(ValueError, match="contiguous"):
        f.fic_encode_ex(wide[:, ::2], 64, 16, 4, 1, -1.0, SS3, 8.0)   # strided view
    with pytest.raises(TypeError, match="uint8"):
        f.fic_encode_ex(img.astype(np.int16), 64, 16, 4, 1, -1.0, SS3, 8.0)
    with pytest.raises(ValueError, match="contiguous"):
        f.fic_encode(torch.zeros(64, 64, dtype=torch.uint8).t()[:, :32], 64, 16, 4, 1, -1.0, SS3,
                     8.0)
    with pytest.raises(ValueError, match="square"):
        f.fic_encode_batch([img, np.zeros((64, 32), np.uint8)], 16, 4, 1, -1.0, SS3, 8.0)
    with pytest.raises(ValueError, match="at least"):
        f.fic_domain_pool(img[:32], 64, 8, 2, -1.0)
    # allocation-free pool: entries are 4 bytes, entropies 8 bytes per position
    with pytest.raises(TypeError, match="4-byte"):
        f.fic_domain_pool_noalloc(img, 64, 8, 2, -1.0, np.zeros(1024, np.uint8))
    xy = np.zeros(1024, np.int32)
    with pytest.raises(TypeError, match="8-byte"):
        f.fic_domain_pool_noalloc(img, 64, 8, 2, -1.0, xy, np.zeros(625, np.float32))
    with pytest.raises(ValueError, match="at least 5000"):                # (64-16)/2+1 = 25
        f.fic_domain_pool_noalloc(img, 64, 8, 2, -1.0, xy, np.zeros(624, np.float64))


def test_binding_refuses_oversize_S_sets(fic):
    f = fic.fic
    with pytest.raises(ValueError, match="at most 16"):
        f.make_ssets([(64, list(range(17)))])
    with pytest.raises(ValueError, match="at most 4"):
        f.make_ssets([(10, [1])] * 5)
    assert f.make_ssets([(10, list(range(16)))])[0].n_s == 16


def test_wait_selftest_host_checks(fic):
    """The limit is checked before the device: out of range is FIC_EINVAL; in
    range, a machine without an sm_103 device gets FIC_ENODEV."""
    f = fic.fic
    assert f.fic_wait_selftest(False, 0) == f.FIC_EINVAL
    assert f.fic_wait_selftest(False, 4_000_000_001) == f.FIC_EINVAL
    try:
        import torch
        has_dev = torch.cuda.is_available()
    except Exception:
        has_dev = False
    if not has_dev:
        assert f.fic_wait_selftest(False, 1000) == f.FIC_ENODEV


SS4 = SS3 + [(10, [5, 9])]


def _no_device():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.parametrize("case", [
    # full pool at L = 1: (8192 - 8 + 1)^2 = 66,977,025 domains at the 4x4 step
    dict(N=8192, B_min=4, thr=-1.0, pool_dn=0, ssets=SS3, what="argmin key"),
    # just past the key's 2^25 columns: (5808 - 7)^2 = 33,651,601 domains
    dict(N=5808, B_min=4, thr=-1.0, pool_dn=0, ssets=SS3, what="argmin key"),
    # threshold pool: (4112 - 7)^2 = 16,851,025 positions to compact > 4096 x 4096
    dict(N=4112, B_min=4, thr=4.0, pool_dn=0, ssets=SS3, what="scan limit"),
    # top-DN pool lists its positions through the same scan
    dict(N=4112, B_min=4, thr=-1.0, pool_dn=64, ssets=SS3, what="scan limit"),
])
def test_pool_sizes_beyond_the_device_limits_rejected_on_host(fic, case):
    """Pool indices occupy 25 bits of the packed argmin key and the
    device-wide scan takes at most 4096 tiles of 4096 elements: a step whose
    pool or position count exceeds either is refused before any device
    work, with the limit named, instead of a wrapped key or a failed scan."""
    N = case["N"]
    img = np.zeros((N, N), np.uint8)
    with pytest.raises(fic.FicError) as e:
        fic.fic_encode_ex(img, N, 16, case["B_min"], 1, case["thr"], case["ssets"], 8.0,
                          pool_dn=case["pool_dn"])
    assert e.value.status == fic.fic.FIC_EINVAL
    assert case["what"] in str(e.value)


def test_record_count_beyond_the_scan_limit_rejected_on_host(fic):
    # 16 -> 2 at N = 8208: (8208 / 2)^2 = 16,842,816 finest cells > 4096 x 4096
    N = 8208
    img = np.zeros((N, N), np.uint8)
    with pytest.raises(fic.FicError) as e:
        fic.fic_encode_ex(img, N, 16, 2, 64, -1.0, SS4, 8.0)
    assert e.value.status == fic.fic.FIC_EINVAL and "scan limit" in str(e.value)


def test_domain_pool_beyond_the_scan_limit_rejected_on_host(fic):
    img = np.zeros((4112, 4112), np.uint8)
    with pytest.raises(fic.FicError) as e:
        fic.fic_domain_pool(img, 4112, 4, 1, 4.0)
    assert e.value.status == fic.fic.FIC_EINVAL and "scan limit" in str(e.value)


@pytest.mark.skipif(not _no_device(), reason="would run the encode on the device")
def test_largest_sizes_within_the_limits_pass_validation(fic):
    """At the limits themselves validation passes; without an sm_103 device
    the call then ends with FIC_ENODEV, not FIC_EINVAL."""
    for N, thr in ((5792, -1.0), (4096, 4.0)):   # (5792-7)^2 full pool; (4096-7)^2 positions
        img = np.zeros((N, N), np.uint8)
        with pytest.raises(fic.FicError) as e:
            fic.fic_encode_ex(img, N, 16, 4, 1, thr, SS3, 8.0)
        assert e.value.status == fic.fic.FIC_ENODEV, N


def test_noalloc_side_above_65535_rejected_on_host(fic):
    # pool coordinates are packed x | y << 16: a side of 65536 is refused
    # before the buffers are looked at (the array's pages are never touched)
    N = 65536
    img = np.zeros((N, N), np.uint8)
    xy = np.zeros(16, np.int32)
    with pytest.raises(fic.FicError) as e:
        fic.fic.fic_domain_pool_noalloc(img, N, 16, 128, -1.0, xy)
    assert e.value.status == fic.fic.FIC_EINVAL
