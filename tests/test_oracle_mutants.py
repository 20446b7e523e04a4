"""Planted mistakes in the oracles, on the CPU: every one must fail a pin.

The pins of tests/test_oracle.py (the solver's oracle) and of
tests/test_prefilter_oracle.py (the pre-filter's) check the oracles against
closed forms, hand derivations, certificates and brute force.  Here each test
plants one plausible mistake in one oracle function (a dropped term, a wrong
sign, a wrong threshold, a transposed operand, a misplaced step), swaps the
mutated function into the oracle module for the duration of the test, runs
that oracle's pins and requires at least one of them to fail.  A mistake that
no pin notices would mean the pins leave that part of Sec. II-A (or of the
pre-filter of Sec. III-IV) unchecked.
"""
import __future__
import inspect
import textwrap

import numpy as np
import pytest

import test_oracle as pins
import test_prefilter_oracle as pf_pins
from oracle import prefilter_oracle as PF
from oracle import rpca_oracle as O

# (oracle function, text in its source, replacement, what the mistake is)
MUTANTS = [
    # Eq. 4-6 and the loop around them
    ("rpca", "svt(X - S + Y / mu, 1.0 / mu)", "svt(X - S, 1.0 / mu)", "Eq. 4 without Y/mu"),
    ("rpca", "svt(X - S + Y / mu, 1.0 / mu)", "svt(X - S + Y / mu, mu)", "Eq. 4 threshold mu for 1/mu"),
    ("rpca", "svt(X - S + Y / mu, 1.0 / mu)", "svt(X + S + Y / mu, 1.0 / mu)", "Eq. 4 sign of S"),
    ("rpca", "shrink(X - L + Y / mu, lam / mu)", "shrink(X - L - Y / mu, lam / mu)", "Eq. 5 sign of Y/mu"),
    ("rpca", "shrink(X - L + Y / mu, lam / mu)", "shrink(X - L + Y / mu, lam * mu)", "Eq. 5 threshold lam*mu"),
    ("rpca", "shrink(X - L + Y / mu, lam / mu)", "shrink(X - L + Y / mu, 1.0 / mu)", "Eq. 5 without lambda"),
    ("rpca", "Y = Y + mu * E", "Y = Y - mu * E", "Eq. 6 sign"),
    ("rpca", "Y = Y + mu * E", "Y = Y + E", "Eq. 6 without mu"),
    ("rpca", "if k > 1 and schedule", "if k >= 1 and schedule", "penalty grown before the first iteration"),
    ("rpca", "mu = min(rho * mu, mu_max)", "mu = rho * mu", "penalty cap dropped"),
    ("rpca", "resid = float(np.linalg.norm(E)) / normX", "resid = float(np.linalg.norm(E))",
     "absolute instead of relative stopping residual"),
    ("rpca", "if resid <= tol:", "if resid <= tol and k > 1:", "stopping test skipped at the first iteration"),
    ("rpca", "\n    mu_max = mu_max_factor * mu0\n", "\n    mu_max = mu_max_factor * mu\n", "cap taken from the warm mu"),
    # singular value thresholding (Eq. 4)
    ("svt", "(U[:, :r] * kept[:r])", "(U[:, :r] * sig[:r])", "hard instead of soft singular value threshold"),
    ("svt", "@ Vh[:r, :]", "@ Vh[:, :r].T", "transposed right factor"),
    ("svt", "kept = np.maximum(sig - tau, 0.0)", "kept = np.maximum(sig - tau * tau, 0.0)", "threshold squared"),
    ("svt", "np.count_nonzero(kept > 0)", "np.count_nonzero(kept >= 0)", "rank counts the dropped values"),
    # soft thresholding (Eq. 5)
    ("shrink", "return np.sign(x) * keep", "return x * (mag > gamma)", "hard instead of soft threshold"),
    ("shrink", "return np.sign(x) * keep", "return keep", "sign dropped"),
    ("shrink", "out[nz] = x[nz] / mag[nz] * keep[nz]", "out[nz] = keep[nz]", "complex phase dropped"),
    ("shrink", "keep = np.maximum(mag - gamma, 0.0)", "keep = np.maximum(mag - 0.5 * gamma, 0.0)", "half threshold"),
    # parameters
    ("initial_mu", "m * T / (4.0 * float(np.sum(np.abs(X))))", "m * T / (2.0 * float(np.sum(np.abs(X))))",
     "fixed schedule's mu off by two"),
    ("initial_mu", "m * T / (4.0 * float(np.sum(np.abs(X))))", "m * T / (4.0 * float(np.sum(X)))",
     "l1 norm without the absolute value"),
    ("initial_mu", "return mu0_scale / spectral_norm(X)", "return mu0_scale / float(np.linalg.norm(X))",
     "Frobenius for the spectral norm"),
    ("default_lambda", "np.sqrt(max(m, T))", "np.sqrt(min(m, T))", "lambda from the smaller dimension"),
    ("spectral_norm", "[0])", "[-1])", "smallest singular value"),
    # layout and evaluation (Sec. II-F)
    ("rpca_frames", "r.L, r.S, r.Y = r.L.T, r.S.T, r.Y.T", "r.L, r.S, r.Y = r.S.T, r.L.T, r.Y.T", "L and S swapped"),
    ("temporal_mean_abs", "axis=0", "axis=1", "mean over pixels instead of frames"),
    ("temporal_mean_abs", "np.mean(np.abs(", "np.mean((", "mean without the absolute value"),
    ("dice", "2.0 * int(", "1.0 * int(", "Dice without the factor 2"),
    ("dice", "np.logical_and(a, b)", "np.logical_or(a, b)", "union for intersection"),
    ("rmse", "np.sqrt(np.mean(", "(np.mean(", "mean square without the root"),
    ("mask_threshold", "0.5 * float(", "1.0 * float(", "threshold at the full mean"),
    ("bound_mask", ">= theta", "> theta", "strict threshold"),
]


# the pre-filter's oracle (Sec. III frame exclusion and moving average, the
# Sec. IV high-pass): (function, [(text, replacement), ...], what)
PF_MUTANTS = [
    ("frame_correlation", [("ac = a - a.mean()", "ac = a")], "correlation without centring"),
    ("frame_correlation", [("na = np.sqrt(np.sum(ac * ac))", "na = np.sum(ac * ac)")], "norm without the root"),
    ("frame_correlation", [("        return 0.0\n", "        return 1.0\n")], "flat frame correlates fully"),
    ("neighbour_correlations", [("frames[t + 1]", "frames[min(t + 2, T - 1)]")], "next-but-one neighbour"),
    ("kept_frames", [("if best >= corr_min:", "if best > corr_min:")], "strict correlation limit"),
    ("kept_frames", [("best = -np.inf", "best = np.inf"), ("best = max(best, c[t - 1])", "best = min(best, c[t - 1])"),
                     ("best = max(best, c[t])", "best = min(best, c[t])")], "every neighbour must correlate"),
    ("kept_frames", [("return np.array([0], dtype=np.int64)", "return np.array([], dtype=np.int64)")],
     "a one-frame window dropped"),
    ("moving_average", [("sum(axis=0) / window", "sum(axis=0) / (window + 1)")], "mean over window + 1"),
    ("moving_average", [("sel[j:j + window]", "sel[j:j + window - 1]")], "window one frame short"),
    ("moving_average", [("sel = frames[kept]", "sel = frames[:]")], "excluded frames averaged"),
    ("moving_average", [("n = K - window + 1", "n = K - window")], "last window dropped"),
    ("highpass", [("h = (window - 1) // 2", "h = window // 2")], "centre frame one late"),
    ("highpass", [("frames[kept[j + h]].astype(np.float64) - avg[j]", "avg[j] - frames[kept[j + h]].astype(np.float64)")],
     "high-pass sign"),
    ("highpass", [("frames[kept[j + h]]", "frames[j + h]")], "centre frame by raw index"),
    ("prefilter", [("filt = highpass if high_pass else moving_average", "filt = moving_average if high_pass else highpass")],
     "filters swapped"),
]


def _mutant(mod, name, edits):
    src = textwrap.dedent(inspect.getsource(getattr(mod, name)))
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    code = compile(src, f"<mutant of {name}>", "exec", flags=__future__.annotations.compiler_flag, dont_inherit=True)
    g = dict(mod.__dict__)
    exec(code, g)
    return g[name]


def _pins(module):
    out = []
    for n in dir(module):
        f = getattr(module, n)
        if n.startswith("test_") and inspect.isfunction(f) and not inspect.signature(f).parameters:
            out.append(f)
    return sorted(out, key=lambda f: f.__code__.co_firstlineno)


def _first_failing_pin(module):
    with np.errstate(all="ignore"):
        for pin in _pins(module):
            try:
                pin()
            except Exception:  # a failed assertion, or a crash on the mutant's output
                return pin.__name__
    return None


def test_pins_pass_on_the_oracles_as_written():
    assert _first_failing_pin(pins) is None
    assert _first_failing_pin(pf_pins) is None


@pytest.mark.parametrize("name,old,new,what", MUTANTS, ids=[m[3] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, what, monkeypatch):
    monkeypatch.setattr(O, name, _mutant(O, name, [(old, new)]))
    assert _first_failing_pin(pins) is not None, f"no pin notices: {what} ({name}: {old!r} -> {new!r})"


@pytest.mark.parametrize("name,edits,what", PF_MUTANTS, ids=[m[2] for m in PF_MUTANTS])
def test_planted_prefilter_mistake_fails_a_pin(name, edits, what, monkeypatch):
    monkeypatch.setattr(PF, name, _mutant(PF, name, edits))
    assert _first_failing_pin(pf_pins) is not None, f"no pin notices: {what} ({name}: {edits!r})"
