"""CPU FP64 oracle for the frame pre-filter applied before RPCA (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only the test-suite and the benchmark's CPU legs
may import this module; the product path never does.  It shares no code with
the CUDA path.

Sec. III (in vivo reference, "Applying the RPCA method"): before the 132-frame
reference solve, frames whose correlation with their neighbouring frames is
below 0.8 are excluded, and a temporal moving average over 20 frames is
applied to the data.  The paper gives no formula; the readings taken here
(each listed in the repository's design notes) are:

* correlation of two frames = Pearson's coefficient over all pixels of the
  two frames (real frames);
* frame t is excluded when it correlates below the limit with every
  neighbour it has (frames t-1 and t+1; the first and last frames have one),
  so a single corrupted frame goes and its neighbours, which still match
  their other neighbour, stay; a window of one frame keeps it;
* the moving average runs over the kept frames in their order, over whole
  windows only: output frame j is the mean of kept frames j .. j+w-1, for
  j = 0 .. K-w (K kept frames; none when K < w);
* a frame with zero variance has correlation 0 with every frame.

Sec. IV names a temporal high-pass filter before RPCA (to take out slowly
varying background motion) as an option, without defining one.  The reading
taken here is the complement of the same moving average: output frame j is
the kept frame at the centre of window j minus the window's mean,
kept[j + h] - mean(kept[j] .. kept[j+w-1]) with h = (w - 1) // 2 (exactly
centred for odd w), so a signal that is constant or linear in time over a
window (odd w) gives 0, and a temporal sinusoid of frequency f (cycles per
frame) is scaled by 1 - sin(pi f w) / (w sin(pi f)).

Frames are rows of a (T, m) array (frame t = row t), the layout of the
solver's frame-major Casorati matrix.
"""
from __future__ import annotations

import numpy as np


def frame_correlation(a: np.ndarray, b: np.ndarray) -> float:
    """Pearson correlation of two frames (1-D arrays over the same pixels)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ac = a - a.mean()
    bc = b - b.mean()
    na = np.sqrt(np.sum(ac * ac))
    nb = np.sqrt(np.sum(bc * bc))
    if na == 0.0 or nb == 0.0:
        return 0.0
    return float(np.sum(ac * bc) / (na * nb))


def neighbour_correlations(frames: np.ndarray) -> np.ndarray:
    """c[t] = correlation of frames t and t+1, t = 0 .. T-2."""
    T = frames.shape[0]
    return np.array([frame_correlation(frames[t], frames[t + 1]) for t in range(T - 1)], dtype=np.float64)


def kept_frames(frames: np.ndarray, corr_min: float) -> np.ndarray:
    """Indices of the frames that correlate at or above corr_min with at least
    one neighbour (all of them when T == 1)."""
    T = frames.shape[0]
    if T == 1:
        return np.array([0], dtype=np.int64)
    c = neighbour_correlations(frames)
    keep = []
    for t in range(T):
        best = -np.inf
        if t > 0:
            best = max(best, c[t - 1])
        if t < T - 1:
            best = max(best, c[t])
        if best >= corr_min:
            keep.append(t)
    return np.array(keep, dtype=np.int64)


def moving_average(frames: np.ndarray, kept: np.ndarray, window: int) -> np.ndarray:
    """Whole-window temporal moving average over the kept frames: row j is the
    mean of frames kept[j] .. kept[j+window-1]."""
    K = len(kept)
    n = K - window + 1
    if n <= 0:
        return np.zeros((0, frames.shape[1]), dtype=np.float64)
    sel = frames[kept].astype(np.float64)
    out = np.empty((n, frames.shape[1]), dtype=np.float64)
    for j in range(n):
        out[j] = sel[j:j + window].sum(axis=0) / window
    return out


def highpass(frames: np.ndarray, kept: np.ndarray, window: int) -> np.ndarray:
    """Temporal high-pass over the kept frames: row j is frame kept[j + h]
    minus the mean of frames kept[j] .. kept[j+window-1], h = (window-1)//2."""
    avg = moving_average(frames, kept, window)
    h = (window - 1) // 2
    out = np.empty_like(avg)
    for j in range(avg.shape[0]):
        out[j] = frames[kept[j + h]].astype(np.float64) - avg[j]
    return out


def prefilter(frames: np.ndarray, corr_min: float = 0.8, window: int = 20, high_pass: bool = False):
    """The reference pre-filter: (filtered frames, kept indices, neighbour
    correlations); the moving average, or with high_pass its complement."""
    c = neighbour_correlations(frames) if frames.shape[0] > 1 else np.zeros(0)
    kept = kept_frames(frames, corr_min)
    filt = highpass if high_pass else moving_average
    return filt(frames, kept, window), kept, c
