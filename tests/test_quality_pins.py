"""Pins of the evaluation oracle (oracle/quality.py) against facts fixed by the
definitions: hand-computed ESIM crossings of exactly representable ramps,
identical sets, polarity separation, hand-placed distances, and brute force on
tiny random event sets."""
import itertools

import numpy as np
import pytest

from oracle import quality as Q


def test_esim_ramp_crossings():
    # y = 0.375 t, C = 0.25 (all exact in binary): crossings 1, 2, 1, 2, ...
    y = np.stack([np.full((2, 3), 0.375 * t) for t in range(6)])
    c = Q.esim_counts(y, 0.25)
    assert c[0].sum() == 0
    assert [int(c[t, 0, 0]) for t in range(1, 6)] == [1, 2, 1, 2, 1]
    # a falling ramp gives the same counts with negative polarity
    c2 = Q.esim_counts(-y, 0.25)
    assert np.array_equal(c2, -c)


def test_esim_step_threshold_and_level():
    # |dL| = C fires once; just below C fires nothing; the level keeps the remainder
    y0 = np.zeros((1, 3))
    y1 = np.array([[0.5, 0.4999, -1.25]])
    counts, level = Q.esim_step(y1, y0, 0.5)
    assert counts.tolist() == [[1, 0, -2]]
    assert level.tolist() == [[0.5, 0.0, -1.0]]


def test_log_brightness_rec709():
    r = np.stack([np.full((1, 1), 1.0), np.full((1, 1), 2.0), np.full((1, 1), 3.0)])
    Y = 0.2126 * 1 + 0.7152 * 2 + 0.0722 * 3
    assert Q.log_brightness(r, 1e-3)[0, 0] == pytest.approx(np.log(Y + 1e-3), abs=1e-15)


def test_identical_sets_are_perfect():
    rng = np.random.default_rng(1)
    c = rng.integers(-2, 3, size=(4, 5, 6)) * (rng.random((4, 5, 6)) < 0.3)
    q = Q.quality(c, c, [1e-9, 0.1])
    assert q["precision"] == [1.0, 1.0] and q["recall"] == [1.0, 1.0] and q["chamfer"] == 0.0
    assert q["fscore"] == [1.0, 1.0]


def test_fscore_is_the_harmonic_mean():
    """F = 2 P R / (P + R): three generated ON events of which one lies on the
    only reference event gives P = 1/3, R = 1, F = 1/2."""
    F, H, W = 6, 8, 8
    gen = np.zeros((F, H, W), np.int64)
    ref = np.zeros((F, H, W), np.int64)
    gen[1, 2, 2] = 1
    gen[4, 7, 7] = 2          # far from the reference event, counted twice
    ref[1, 2, 2] = 1
    q = Q.quality(gen, ref, [1e-6])
    assert q["precision"] == [pytest.approx(1 / 3)] and q["recall"] == [1.0]
    assert q["fscore"] == [pytest.approx(0.5)]


def test_polarity_is_respected_and_distances_are_normalised():
    F, H, W = 10, 8, 16
    gen = np.zeros((F, H, W), np.int64)
    ref = np.zeros((F, H, W), np.int64)
    gen[2, 3, 5] = 2          # two ON events at (5, 3, 2)
    ref[2, 3, 5] = -1         # an OFF event at the same place does not match
    ref[2, 3, 8] = 1          # the nearest ON event: 3 pixels along x
    ref[4, 0, 0] = -3         # OFF events far away
    d_on = 3 / W
    q = Q.quality(gen, ref, [d_on - 1e-9, d_on + 1e-9])
    assert q["precision"] == [0.0, 1.0]
    dg, wg = q["d_gen"], q["w_gen"]
    assert dg.tolist() == pytest.approx([d_on]) and wg.tolist() == [2]
    # recall: the ON reference event's nearest ON generated event is the same pair;
    # the OFF reference events have no OFF generated event at all (infinite distance)
    assert q["recall"] == [0.0, 0.2]   # 1 of 5 reference events within reach
    assert np.isinf(q["chamfer"])


def test_time_axis_scaling():
    F, H, W = 20, 4, 4
    gen = np.zeros((F, H, W), np.int64)
    ref = np.zeros((F, H, W), np.int64)
    gen[5, 1, 1] = 1
    ref[8, 1, 1] = 1
    ref[5, 1, 3] = 1   # 2 px along x at the same time: 2/4 = 0.5 > 3/20 = 0.15
    q = Q.quality(gen, ref, [1.0])
    assert q["d_gen"].tolist() == pytest.approx([3 / F])
    assert q["chamfer"] == pytest.approx((3 / F) ** 2 + ((3 / F) ** 2 + (2 / W) ** 2) / 2)


def _brute(query_counts, ref_counts):
    F, H, W = query_counts.shape
    d, w = [], []
    for p in (1, -1):
        refs = [(x / W, y / H, t / F) for t, y, x in itertools.product(range(F), range(H), range(W))
                if ref_counts[t, y, x] * p > 0]
        for t, y, x in itertools.product(range(F), range(H), range(W)):
            if query_counts[t, y, x] * p > 0:
                q = np.array([x / W, y / H, t / F])
                d.append(min((np.linalg.norm(q - np.array(r)) for r in refs), default=np.inf))
                w.append(abs(int(query_counts[t, y, x])))
    return np.array(d), np.array(w)


def test_kdtree_matches_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(5):
        g = rng.integers(-3, 4, size=(4, 5, 7)) * (rng.random((4, 5, 7)) < 0.2)
        r = rng.integers(-3, 4, size=(4, 5, 7)) * (rng.random((4, 5, 7)) < 0.2)
        d, w = Q.directed(g, r)
        bd, bw = _brute(g, r)
        assert np.array_equal(w, bw)
        assert np.array_equal(np.isinf(d), np.isinf(bd))
        fin = np.isfinite(bd)
        assert np.allclose(d[fin], bd[fin], rtol=0, atol=1e-15)
