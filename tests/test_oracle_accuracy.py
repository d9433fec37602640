"""Pins of the oracle's accuracy report (Sec. III): e_p and e_r on hand-made disparity maps, and
the pothole pixel metrics on hand-made masks."""
import math

import numpy as np


def test_disparity_errors_hand_case(orc):
    D4 = np.zeros((4, 5), np.float32) + 10.0
    D1 = D4.copy()
    D1[0, :] += 0.5              # |err| 0.5
    D1[1, :] += 1.5              # 1.5
    D1[2, :] -= 2.5              # 2.5
    D1[3, :2] += 4.0             # 4.0
    D1[3, 2:] = -1.0             # no disparity: not counted
    r = orc.accuracy(D1, D4, np.zeros((4, 5)), np.zeros((4, 5)))
    assert r["q"] == 17
    assert math.isclose(r["e_p1"], 100 * 12 / 17)
    assert math.isclose(r["e_p2"], 100 * 7 / 17)
    assert math.isclose(r["e_p3"], 100 * 2 / 17)
    assert math.isclose(r["e_r"], math.sqrt((5 * 0.25 + 5 * 2.25 + 5 * 6.25 + 2 * 16) / 17))


def test_constant_offset_gives_the_offset_as_rmse(orc):
    rng = np.random.default_rng(1)
    D4 = rng.uniform(5, 50, size=(30, 40))
    r = orc.accuracy(D4 + 0.75, D4, np.zeros((30, 40)), np.zeros((30, 40)))
    assert math.isclose(r["e_r"], 0.75, rel_tol=1e-12)
    assert r["e_p1"] == 0.0 and r["q"] == 1200


def test_mask_metrics_hand_case(orc):
    g = np.zeros((10, 10), np.uint8)
    g[2:6, 2:6] = 1              # 16 pothole pixels
    m = np.zeros((10, 10), np.uint8)
    m[3:7, 3:7] = 1              # 16 detected, 9 of them inside
    r = orc.accuracy(np.zeros((10, 10)), np.zeros((10, 10)), m, g)
    assert (r["tp"], r["fp"], r["fn"], r["tn"]) == (9, 7, 7, 77)
    assert math.isclose(r["precision"], 9 / 16) and math.isclose(r["recall"], 9 / 16)
    assert math.isclose(r["accuracy"], 86 / 100) and math.isclose(r["fscore"], 9 / 16)
