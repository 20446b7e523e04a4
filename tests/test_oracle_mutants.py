"""Planted mistakes in the oracle, on the CPU: every one must fail a pin.

The pins of tests/test_oracle.py check the oracle against closed forms, hand
derivations, certificates and brute force.  Here each test plants one
plausible mistake in one oracle function (a dropped term, a wrong sign, a
wrong threshold, a transposed operand, a misplaced step), swaps the mutated
function into the oracle module for the duration of the test, runs the pins
and requires at least one of them to fail.  A mistake that no pin notices
would mean the pins leave that part of Sec. II-A unchecked.
"""
import __future__
import inspect
import textwrap

import numpy as np
import pytest

import test_oracle as pins
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


def _mutant(name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(O, name)))
    assert src.count(old) == 1, (name, old)
    code = compile(src.replace(old, new), f"<mutant of {name}>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    g = dict(O.__dict__)
    exec(code, g)
    return g[name]


def _pins():
    out = []
    for n in dir(pins):
        f = getattr(pins, n)
        if n.startswith("test_") and inspect.isfunction(f) and not inspect.signature(f).parameters:
            out.append(f)
    return sorted(out, key=lambda f: f.__code__.co_firstlineno)


def test_pins_pass_on_the_oracle_as_written():
    for pin in _pins():
        pin()


@pytest.mark.parametrize("name,old,new,what", MUTANTS, ids=[m[3] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, what, monkeypatch):
    monkeypatch.setattr(O, name, _mutant(name, old, new))
    caught = None
    with np.errstate(all="ignore"):
        for pin in _pins():
            try:
                pin()
            except Exception:  # a failed assertion, or a crash on the mutant's output
                caught = pin.__name__
                break
    assert caught is not None, f"no pin notices: {what} ({name}: {old!r} -> {new!r})"
