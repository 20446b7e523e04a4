"""The seeded input generator (no method arithmetic): recipe properties."""
import numpy as np

from paper_2506_10257_gb300 import synth


def test_curved_tracks_bend_and_reduce_to_straight():
    # the generator's curved-track option (Sec. II-C motion model): with zero
    # acceleration the free-bubble ground truth equals the straight tracks';
    # with acceleration the centroid path of a lone bubble leaves its line
    kw = dict(seed=5, ny=48, nx=48, T=12, n_bound=0, n_free=1, speed=(1.5, 1.5))
    straight = synth.make_window(**kw)
    zero = synth.make_window(**kw, accel=(0.0, 0.0))
    assert np.allclose(zero.S_gt, straight.S_gt, atol=1e-9)
    bent = synth.make_window(**kw, accel=(0.8, 0.8))
    img = np.abs(bent.S_gt).reshape(12, 48, 48)
    yy, xx = np.mgrid[0:48, 0:48]
    pts = [((img[t] * yy).sum() / img[t].sum(), (img[t] * xx).sum() / img[t].sum())
           for t in range(12) if img[t].sum() > 0]
    P = np.array(pts)
    assert len(P) >= 4
    # distance of the middle points from the chord through the first and last visible points
    d = P[-1] - P[0]
    n = np.array([-d[1], d[0]]) / np.linalg.norm(d)
    assert np.abs((P[1:-1] - P[0]) @ n).max() > 0.5
