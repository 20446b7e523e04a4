"""Host-side parameter validation of the C ABI, without a GPU: every rejected
combination returns the status the header documents (RPCA_ERR_ARG for values
outside their domain, RPCA_ERR_UNSUPPORTED for combinations not built), from
rpca_workspace_size and rpca_plan_create alike, before any CUDA call."""
import ctypes
import math

import pytest

from paper_2506_10257_gb300 import rpca

ARG, UNSUP = rpca.ERR_ARG, rpca.ERR_UNSUPPORTED
R32, C64 = 0, 1
FP32, TF32X3, BF16X3, TF32 = 0, 1, 2, 3
IALM, FIXED_L1 = 0, 1

# (overrides of the defaults for m = 4096, T = 20, expected status)
REJECTED = [
    (dict(m=0), ARG), (dict(T=0), ARG), (dict(T=rpca.MAX_T + 1), UNSUP),
    (dict(tol=0.0), ARG), (dict(tol=float("nan")), ARG), (dict(max_iter=0), ARG),
    (dict(mu_schedule=2), ARG), (dict(rho=0.9), ARG), (dict(mu0_scale=0.0), ARG), (dict(mu_max_factor=0.5), ARG),
    (dict(drive=3), ARG), (dict(dtype=2), ARG), (dict(precision=4), ARG), (dict(precision=-1), ARG),
    (dict(dtype=C64, T=rpca.MAX_T // 2 + 1), UNSUP), (dict(dtype=C64, precision=TF32), UNSUP),
    (dict(precision=TF32X3, drive=rpca.DRIVE_HOST), UNSUP), (dict(precision=BF16X3, T=129), UNSUP),
    (dict(precision=TF32X3, T=65, dtype=C64), UNSUP),             # complex: 2T > 128 has no tensor-core pass
    (dict(m=2 ** 36), ARG),                                   # m * T above 2^40 elements
    (dict(warm_start=2), ARG), (dict(sharded=2), ARG),
    (dict(sharded=1, dtype=C64), UNSUP), (dict(sharded=1, T=rpca.MAX_T_NARROW + 1), UNSUP),
    (dict(sharded=1, precision=TF32), UNSUP), (dict(sharded=1, mu_schedule=FIXED_L1), UNSUP),
    (dict(sharded=1, warm_start=1), UNSUP), (dict(precision=TF32), UNSUP),
    (dict(drive=rpca.DRIVE_STREAM, precision=TF32), UNSUP),
    (dict(mu_init=-1.0), ARG), (dict(mu_init=math.inf), ARG), (dict(mu_prev_scale=float("nan")), ARG),
]

# accepted by validation (on a machine without a GPU the size query then fails with RPCA_ERR_CUDA)
ACCEPTED = [
    dict(), dict(T=1), dict(T=rpca.MAX_T), dict(dtype=C64, T=rpca.MAX_T // 2), dict(precision=BF16X3, T=32),
    dict(precision=BF16X3, T=128), dict(precision=TF32X3, T=33), dict(precision=TF32X3, T=64, dtype=C64),
    dict(mu_schedule=FIXED_L1, rho=0.5),                      # rho, mu0_scale, cap only bind the IALM schedule
    dict(sharded=1), dict(warm_start=1, mu_prev_scale=0.1), dict(drive=rpca.DRIVE_STREAM, precision=TF32X3),
]


@pytest.fixture(scope="module")
def lib():
    return rpca.load()


def _params(kw):
    d = {**dict(m=4096, T=20), **kw}
    m, T = d.pop("m"), d.pop("T")
    return rpca.default_params(m, T, **d)


def _size(lib, p):
    n = ctypes.c_size_t(0)
    return lib.rpca_workspace_size(ctypes.byref(p), ctypes.byref(n))


@pytest.mark.parametrize("kw,want", REJECTED, ids=[",".join(f"{k}={v}" for k, v in kw.items()) for kw, _ in REJECTED])
def test_rejected_parameters(lib, kw, want):
    p = _params(kw)
    assert _size(lib, p) == want
    h = ctypes.c_void_p(123)
    assert lib.rpca_plan_create(ctypes.byref(p), None, 0, ctypes.byref(h)) == want


@pytest.mark.parametrize("kw", ACCEPTED, ids=[",".join(f"{k}={v}" for k, v in kw.items()) or "defaults"
                                              for kw in ACCEPTED])
def test_accepted_parameters_pass_validation(lib, kw):
    p = _params(kw)
    st = _size(lib, p)
    assert st in (rpca.OK, rpca.ERR_CUDA)                     # ERR_CUDA only where no device is visible
    assert st not in (ARG, UNSUP)


def test_null_arguments(lib):
    assert lib.rpca_workspace_size(None, None) == ARG
    p = rpca.default_params(4096, 20)
    assert lib.rpca_workspace_size(ctypes.byref(p), None) == ARG
    assert lib.rpca_plan_create(ctypes.byref(p), None, 0, None) == ARG


@pytest.mark.parametrize("fn", ["rpca_prefilter", "rpca_prefilter_highpass"])
def test_prefilter_argument_checks(lib, fn):
    # rejected before any launch, so the (never dereferenced) buffers are plain aligned addresses
    f = getattr(lib, fn)
    buf = 1 << 20
    ok = dict(X=buf, m=4096, T=30, corr_min=0.8, window=20, Y=buf, kept=buf, count=buf, corr=0, scratch=buf)

    def call(**kw):
        a = {**ok, **kw}
        return f(ctypes.c_void_p(a["X"]), a["m"], a["T"], ctypes.c_double(a["corr_min"]), a["window"],
                 ctypes.c_void_p(a["Y"]), ctypes.c_void_p(a["kept"]), ctypes.c_void_p(a["count"]),
                 ctypes.c_void_p(a["corr"]), ctypes.c_void_p(a["scratch"]), None)

    for kw in (dict(X=0), dict(Y=0), dict(kept=0), dict(count=0), dict(scratch=0), dict(m=0), dict(T=0),
               dict(window=0), dict(corr_min=float("nan")), dict(X=buf + 2), dict(Y=buf + 1)):
        assert call(**kw) == ARG, kw
    assert call(T=65536) == UNSUP
    assert lib.rpca_prefilter_scratch_bytes(0, 5) == 0 and lib.rpca_prefilter_scratch_bytes(10, 0) == 0
    assert lib.rpca_prefilter_scratch_bytes(87880, 132) >= 3 * 8 * 132   # FP64 partial sums, 3 per frame and chunk
