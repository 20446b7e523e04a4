"""Pins of the pre-filter oracle (Sec. III, in vivo reference: frames below 0.8
neighbour correlation excluded, 20-frame moving average) against closed forms
and a library routine.  No GPU."""
import numpy as np
import pytest

from oracle import prefilter_oracle as P


def smooth_frames(seed, T, m, drift=0.05):
    """Frames that change slowly: a fixed random image plus a small drift per frame."""
    rng = np.random.default_rng(seed)
    base = rng.standard_normal(m)
    step = rng.standard_normal((T, m))
    return base[None, :] + drift * np.cumsum(step, axis=0)


def test_correlation_matches_numpy_corrcoef():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(500)
    b = 0.7 * a + 0.3 * rng.standard_normal(500)
    assert P.frame_correlation(a, b) == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-14)


def test_correlation_closed_forms():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(300)
    assert P.frame_correlation(a, a) == pytest.approx(1.0, abs=1e-14)
    assert P.frame_correlation(a, -a) == pytest.approx(-1.0, abs=1e-14)
    assert P.frame_correlation(a, 3.0 * a + 7.0) == pytest.approx(1.0, abs=1e-14)   # affine, positive scale
    # two centred orthogonal frames
    x = np.array([1.0, -1.0, 1.0, -1.0])
    y = np.array([1.0, 1.0, -1.0, -1.0])
    assert P.frame_correlation(x, y) == pytest.approx(0.0, abs=1e-15)
    # a constant frame has no variance: correlation 0 by the stated reading
    assert P.frame_correlation(np.full(10, 2.0), a[:10]) == 0.0


def test_neighbour_correlations_are_adjacent_pairs():
    F = smooth_frames(3, 6, 200)
    c = P.neighbour_correlations(F)
    assert c.shape == (5,)
    for t in range(5):
        assert c[t] == pytest.approx(np.corrcoef(F[t], F[t + 1])[0, 1], abs=1e-13)


def test_planted_bad_frame_is_excluded_alone():
    F = smooth_frames(4, 12, 400)
    rng = np.random.default_rng(5)
    F[5] = rng.standard_normal(400)          # uncorrelated with both neighbours
    kept = P.kept_frames(F, 0.8)
    assert list(kept) == [t for t in range(12) if t != 5]


def test_bad_first_and_last_frames_are_excluded():
    F = smooth_frames(6, 8, 300)
    rng = np.random.default_rng(7)
    F[0] = rng.standard_normal(300)
    F[7] = rng.standard_normal(300)
    assert list(P.kept_frames(F, 0.8)) == [1, 2, 3, 4, 5, 6]


def test_all_uncorrelated_keeps_none_and_single_frame_keeps_it():
    rng = np.random.default_rng(8)
    F = rng.standard_normal((6, 1000))
    assert len(P.kept_frames(F, 0.8)) == 0
    assert list(P.kept_frames(F[:1], 0.8)) == [0]


def test_moving_average_closed_forms():
    m, T, w = 7, 30, 20
    v = np.arange(1, m + 1, dtype=np.float64)
    ramp = np.arange(T, dtype=np.float64)[:, None] * v[None, :]     # frame t = t * v
    kept = np.arange(T)
    out = P.moving_average(ramp, kept, w)
    assert out.shape == (T - w + 1, m)
    for j in range(T - w + 1):
        np.testing.assert_allclose(out[j], (j + (w - 1) / 2.0) * v, rtol=1e-14)
    const = np.full((T, m), 3.5)
    np.testing.assert_allclose(P.moving_average(const, kept, w), 3.5, rtol=1e-15)
    # window 1 is the kept frames themselves; fewer kept frames than the window gives none
    np.testing.assert_array_equal(P.moving_average(ramp, np.array([2, 5, 9]), 1), ramp[[2, 5, 9]])
    assert P.moving_average(ramp, np.arange(5), 6).shape == (0, m)


def test_moving_average_skips_excluded_frames():
    T, m = 10, 3
    F = np.arange(T, dtype=np.float64)[:, None] * np.ones((1, m))
    kept = np.array([0, 1, 2, 4, 5, 6, 7, 8, 9])                        # frame 3 excluded
    out = P.moving_average(F, kept, 3)
    want = [np.mean([F[kept[j + i]] for i in range(3)], axis=0) for j in range(len(kept) - 2)]
    np.testing.assert_allclose(out, np.array(want), rtol=1e-15)
    assert out[2, 0] == pytest.approx((2 + 4 + 5) / 3.0)
