"""Pins of the oracle's connected-component labelling of the pothole mask (Sec. II-E) and of the
fake-pothole rule (Sec. III-B): the partition against scipy.ndimage.label, labels equal to each
component's smallest raster index, statistics against numpy, and hand-made corner and
single-superpixel cases."""
import numpy as np
import pytest

ndimage = pytest.importorskip("scipy.ndimage")


def _structure(conn):
    return np.ones((3, 3), int) if conn == 8 else np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]])


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("seed,density,shape", [(1, 0.3, (37, 53)), (2, 0.55, (64, 64)),
                                                 (3, 0.45, (17, 200)), (4, 0.6, (120, 90))])
def test_partition_matches_scipy(orc, conn, seed, density, shape):
    rng = np.random.default_rng(seed)
    mask = (rng.random(shape) < density).astype(np.uint8)
    labels, n = orc.ccl(mask, conn)
    ref, n_ref = ndimage.label(mask, structure=_structure(conn))
    assert n == n_ref
    assert ((labels >= 0) == (mask > 0)).all()
    flat = np.arange(mask.size).reshape(shape)
    for k in range(1, n_ref + 1):
        comp = ref == k
        vals = np.unique(labels[comp])
        assert vals.size == 1 and vals[0] == flat[comp].min()


def test_hand_cases(orc):
    m = np.zeros((6, 6), np.uint8)
    m[1, 1] = m[2, 2] = 1                    # diagonal neighbours
    m[4, 4] = 1
    lab8, n8 = orc.ccl(m, 8)
    lab4, n4 = orc.ccl(m, 4)
    assert n8 == 2 and n4 == 3
    assert lab8[2, 2] == 7 and lab4[2, 2] == 14 and lab8[4, 4] == 28
    assert orc.ccl(np.zeros((5, 7), np.uint8))[1] == 0
    full, n = orc.ccl(np.ones((5, 7), np.uint8))
    assert n == 1 and (full == 0).all()


def test_component_statistics(orc):
    rng = np.random.default_rng(5)
    H, W = 48, 64
    mask = (rng.random((H, W)) < 0.4).astype(np.uint8)
    sp = (np.arange(H)[:, None] // 12) * 10 + (np.arange(W)[None, :] // 16)
    labels, n = orc.ccl(mask, 8)
    comps = orc.components(labels, sp, n)
    roots = np.sort(np.unique(labels[labels >= 0]))
    assert np.array_equal(comps[:, 0], roots)
    for row in comps:
        vs, us = np.nonzero(labels == row[0])
        assert row[1] == us.size
        assert (row[2], row[3], row[4], row[5]) == (us.min(), vs.min(), us.max(), vs.max())
        assert (row[6], row[7]) == (us.sum(), vs.sum())
        single = np.unique(sp[vs, us]).size == 1
        assert row[8] == (1 if single else 2) and row[10] == single
        cu, cv = us.mean(), vs.mean()
        corner = (cu < W / 8 or cu >= 7 * W / 8) and (cv < H / 8 or cv >= 7 * H / 8)
        assert row[9] == corner and row[11] == (corner or single)


def test_fake_rule_hand_cases(orc):
    """A blob in the top-left corner cell is fake; a blob in the middle spanning two superpixels
    is kept; a blob in the middle inside one superpixel is fake; a blob along the top edge (not in
    a corner cell) spanning two superpixels is kept."""
    H, W = 80, 80
    mask = np.zeros((H, W), np.uint8)
    mask[1:5, 1:5] = 1                       # corner
    mask[30:50, 30:50] = 1                   # middle, two superpixels
    mask[60:66, 20:26] = 1                   # one superpixel
    mask[0:4, 36:46] = 1                     # top edge, two superpixels
    sp = np.where(np.arange(W)[None, :] < 40, 0, 1) * np.ones((H, 1), np.int64)
    sp[55:, :] = 7                           # rows 55.. are one superpixel
    labels, n = orc.ccl(mask, 8)
    comps = orc.components(labels, sp, n)
    byroot = {int(r[0]): r for r in comps}
    assert n == 4
    assert byroot[1 * W + 1][11] == 1 and byroot[1 * W + 1][9] == 1
    assert byroot[30 * W + 30][11] == 0
    assert byroot[60 * W + 20][11] == 1 and byroot[60 * W + 20][10] == 1
    assert byroot[0 * W + 36][11] == 0 and byroot[0 * W + 36][9] == 0
