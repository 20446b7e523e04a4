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


def test_frame_exactly_at_the_limit_is_kept():
    # "below 0.8 is excluded": a neighbour correlation equal to the limit keeps
    # the frame.  Frames with exactly representable coefficients: a and a have
    # correlation 4 / (2 * 2) = 1, a and b (orthogonal, zero mean) 0 / 4 = 0.
    a = np.array([1.0, -1.0, 1.0, -1.0])
    b = np.array([1.0, 1.0, -1.0, -1.0])
    assert P.frame_correlation(a, a) == 1.0 and P.frame_correlation(a, b) == 0.0
    assert list(P.kept_frames(np.stack([a, a]), 1.0)) == [0, 1]
    assert list(P.kept_frames(np.stack([a, b]), 0.0)) == [0, 1]
    assert list(P.kept_frames(np.stack([a, b]), 1e-12)) == []


def test_prefilter_outputs_by_hand():
    # three frames: one pixel pattern plus the offsets 0, 3, 6 (neighbours
    # correlate exactly 1, so all are kept); window of 2 frames
    pat = np.array([1.0, -1.0, 1.0, -1.0])
    F = np.stack([0.0 + pat, 3.0 + pat, 6.0 + pat])
    avg, kept, c = P.prefilter(F, 0.8, 2)
    assert list(kept) == [0, 1, 2] and np.all(c == 1.0)
    np.testing.assert_array_equal(avg, np.stack([1.5 + pat, 4.5 + pat]))        # moving average of 2
    hp, _, _ = P.prefilter(F, 0.8, 2, high_pass=True)
    np.testing.assert_array_equal(hp, np.full((2, 4), -1.5))                       # frame j minus the mean


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


def test_highpass_removes_constant_and_linear_trends():
    # centred window (odd w): the mean of a linear sequence is its centre value
    m, T, w = 5, 25, 7
    v = np.linspace(-2.0, 3.0, m)
    kept = np.arange(T)
    trend = 4.0 + np.arange(T, dtype=np.float64)[:, None] * v[None, :]
    out = P.highpass(trend, kept, w)
    assert out.shape == (T - w + 1, m)
    np.testing.assert_allclose(out, 0.0, atol=1e-12)
    # even window: centre half a frame early, so a unit ramp leaves -1/2
    np.testing.assert_allclose(P.highpass(np.arange(T, dtype=np.float64)[:, None], kept, 6), -0.5, atol=1e-12)


def test_highpass_frequency_response_of_a_temporal_sinusoid():
    # a centred w-frame mean scales cos(2 pi f t + phi) by sin(pi f w) / (w sin(pi f))
    T, w = 60, 9
    t = np.arange(T, dtype=np.float64)
    kept = np.arange(T)
    h = (w - 1) // 2
    for f, phi in [(0.05, 0.3), (0.21, -1.1), (1.0 / w, 0.7), (3.0 / w, 2.0), (0.5, 0.0)]:
        x = np.cos(2 * np.pi * f * t + phi)[:, None] * np.array([[1.0, -0.5]])
        H = np.sin(np.pi * f * w) / (w * np.sin(np.pi * f))
        want = (1.0 - H) * x[h:h + T - w + 1]
        np.testing.assert_allclose(P.highpass(x, kept, w), want, atol=1e-12)
    # at multiples of 1/w the window mean is zero: the sinusoid passes unchanged
    x = np.sin(2 * np.pi * (2.0 / w) * t)[:, None]
    np.testing.assert_allclose(P.highpass(x, kept, w), x[h:h + T - w + 1], atol=1e-12)


def test_highpass_brute_force_with_excluded_frames():
    rng = np.random.default_rng(11)
    T, m, w = 11, 4, 4
    F = rng.standard_normal((T, m))
    kept = np.array([0, 2, 3, 4, 6, 7, 8, 10])
    out = P.highpass(F, kept, w)
    assert out.shape == (len(kept) - w + 1, m)
    for j in range(out.shape[0]):
        for p in range(m):
            s = 0.0
            for i in range(w):
                s += F[kept[j + i], p]
            assert out[j, p] == pytest.approx(F[kept[j + 1], p] - s / w, abs=1e-14)
    assert P.highpass(F, np.arange(3), 4).shape == (0, m)
    np.testing.assert_array_equal(P.highpass(F, kept, 1), 0.0)   # a one-frame window removes everything


def test_prefilter_high_pass_is_frames_minus_average():
    F = smooth_frames(12, 30, 200)
    avg, kept, c = P.prefilter(F, 0.8, 5)
    hp, kept2, c2 = P.prefilter(F, 0.8, 5, high_pass=True)
    np.testing.assert_array_equal(kept, kept2)
    np.testing.assert_array_equal(c, c2)
    np.testing.assert_allclose(hp + avg, F[kept[2:2 + avg.shape[0]]], atol=1e-13)
