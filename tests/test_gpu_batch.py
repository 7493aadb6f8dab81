"""GPU parity of the batched encoder (fic_encode_batch).

A batch runs every image's quadtree step together, with one contraction
launch over the work items of all images.  Each image's records must be
identical to the oracle's and to a single-image encode of the same image,
whatever else is in the batch.
"""
from __future__ import annotations

import numpy as np
import pytest

import fic_synth
import oracle
from tests.codes import assert_same_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_00324_gb300 as p
    torch.cuda.set_device(0)
    return p


# sides and spectral exponents of a small mixed batch; the 16 x 16 image has
# no 32 x 32 domain at all (empty pool at the first step -> every range splits)
SMALL = [(64, 1.5), (96, 2.5), (128, 2.0), (48, 1.8), (32, 2.2), (16, 2.0), (80, 1.6)]


def small_batch(seed0=500):
    return [fic_synth.one_over_f(n, seed0 + i, a) for i, (n, a) in enumerate(SMALL)]


PARAMS = [
    dict(B_max=16, B_min=4, L=2, thr=4.0, tol=8.0),
    dict(B_max=8, B_min=2, L=1, thr=-1.0, tol=12.0),
    dict(B_max=16, B_min=4, L=3, thr=5.5, tol=16.0),
]


@pytest.mark.parametrize("prm", PARAMS, ids=["16-4_L2_thr4", "8-2_L1_all", "16-4_L3_thr5.5"])
@pytest.mark.parametrize("engine", ["tensor", "plain"])
def test_batch_matches_oracle_and_single(pkg, prm, engine):
    imgs = small_batch()
    ss = pkg.paper_ssets(prm["B_max"], prm["B_min"])
    e = pkg.ENGINE_TENSOR if engine == "tensor" else pkg.ENGINE_PLAIN
    got = pkg.fic_encode_batch(imgs, prm["B_max"], prm["B_min"], prm["L"], prm["thr"], ss,
                               prm["tol"], engine=e)
    assert len(got) == len(imgs)
    for i, (img, enc) in enumerate(zip(imgs, got)):
        assert enc.N == img.shape[0]
        want, st = oracle.encode(img, prm["B_max"], prm["B_min"], prm["L"], prm["thr"], ss,
                                 prm["tol"])
        assert_same_codes(enc.codes, want, prm["B_max"], f"batch[{i}] N={img.shape[0]}")
        for lvl in range(enc.n_levels):
            if enc.ranges[lvl] > 0:
                assert enc.pool_size[lvl] == st["pool_size"][lvl]
        one = pkg.fic_encode_ex(img, img.shape[0], prm["B_max"], prm["B_min"], prm["L"],
                                prm["thr"], ss, prm["tol"], engine=e)
        np.testing.assert_array_equal(enc.codes, one.codes)
        assert enc.pool_size == one.pool_size and enc.ranges == one.ranges
        assert enc.matches == one.matches


def test_batch_order_and_company_do_not_matter(pkg):
    """The same image gives the same records alone, first, last, duplicated,
    or next to larger images; host and device inputs mix freely."""
    import torch
    imgs = small_batch(seed0=900)
    ss = pkg.paper_ssets(16, 4)
    args = (16, 4, 2, 4.0, ss, 8.0)
    alone = [pkg.fic_encode_ex(im, im.shape[0], *args).codes for im in imgs]
    rev = pkg.fic_encode_batch(imgs[::-1], *args)
    for i, enc in enumerate(rev[::-1]):
        np.testing.assert_array_equal(enc.codes, alone[i])
    mixed = [torch.from_numpy(im).cuda() if i % 2 else im for i, im in enumerate(imgs)]
    dup = pkg.fic_encode_batch(mixed + mixed, *args, stream=torch.cuda.current_stream())
    for i, enc in enumerate(dup):
        np.testing.assert_array_equal(enc.codes, alone[i % len(imgs)])


def test_batch_edge_cases(pkg):
    """Empty batch, a batch of one, and invalid members (rejected before any
    work, with no results left behind)."""
    ss = pkg.paper_ssets(16, 4)
    assert pkg.fic_encode_batch([], 16, 4, 2, 4.0, ss, 8.0) == []
    img = fic_synth.one_over_f(64, 3, 2.0)
    (one,) = pkg.fic_encode_batch([img], 16, 4, 2, 4.0, ss, 8.0)
    np.testing.assert_array_equal(one.codes, pkg.fic_encode_ex(img, 64, 16, 4, 2, 4.0, ss, 8.0).codes)
    with pytest.raises(pkg.FicError) as e:
        pkg.fic_encode_batch([img, np.zeros((40, 40), np.uint8)], 16, 4, 2, 4.0, ss, 8.0)
    assert e.value.status == pkg.fic.FIC_EINVAL


def test_batch_workload_sample_sampled_oracle(pkg):
    """The first 8 images of the 64-image batching workload (seeds 100..107,
    sides from {128, ..., 1024}, alpha in [1.5, 2.5]; quadtree 16 -> 4, L = 2,
    entropy > 4.0 bits): batch == single-image encodes; sampled leaves of the
    largest image are re-searched by the oracle one by one."""
    imgs = fic_synth.batch_images(8)
    ss = pkg.paper_ssets(16, 4)
    args = (16, 4, 2, 4.0, ss, 8.0)
    got = pkg.fic_encode_batch(imgs, *args)
    for img, enc in zip(imgs, got):
        one = pkg.fic_encode_ex(img, img.shape[0], *args)
        np.testing.assert_array_equal(enc.codes, one.codes)
    big = int(np.argmax([im.shape[0] for im in imgs]))
    img, codes = imgs[big], got[big].codes
    rng = np.random.default_rng(1)
    for lvl in range(3):
        B = 16 >> lvl
        leaves = np.nonzero((codes["level"] == lvl) & (codes["s_idx"] != 0xFF))[0]
        if not leaves.size:
            continue
        pick = rng.choice(leaves, min(6, leaves.size), replace=False)
        pool = oracle.Pool(img, B, 2, 4.0)
        sc, pi, iso, si = pool.search(codes["rx"][pick], codes["ry"][pick], ss[lvl])
        np.testing.assert_array_equal(pi, codes["pool_idx"][pick].astype(np.int64))
        np.testing.assert_array_equal(iso, codes["iso"][pick])
        np.testing.assert_array_equal(si, codes["s_idx"][pick])
