"""Host-side checks of the C-ABI library that need no GPU.

The library must load, export every entry point ``include/*.h`` declares,
and refuse bad arguments before touching the device.
"""
import ctypes as C
import glob
import os
import re

import pytest

from paper_0811_2111_gb300 import _lib as X
from paper_0811_2111_gb300 import build as build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(xy_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return X.lib()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("xy_create", "xy_sweep", "xy_measure", "xy_destroy", "xy_get_state",
              "xy_set_state", "xy_last_error", "xy_philox_words"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_version(lib):
    assert X.xy_version() >= 100


def _params(**kw):
    p = X.xy_params()
    p.L, p.start, p.beta, p.J, p.delta, p.seed = 8, 0, 1.0, 1.0, 3.14159, 1
    p.sincos_mode, p.reduce_mode, p.lattice_id, p.algorithm = 0, 0, 0, 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,fragment", [
    (dict(L=3), "even"), (dict(L=0), "even"), (dict(L=65536), "even"),
    (dict(beta=-1.0), "beta"), (dict(beta=float("nan")), "beta"),
    (dict(delta=0.0), "delta"), (dict(delta=4.0), "delta"),
    (dict(start=7), "start"), (dict(sincos_mode=5), "sincos"), (dict(reduce_mode=2), "reduce"),
    (dict(algorithm=9), "algorithm"), (dict(algorithm=1, L=96), "multiple of 128"),
    (dict(algorithm=3, L=96), "multiple of 128"),
    (dict(J=float("inf")), "J"),
])
def test_create_rejects_bad_parameters(lib, kw, fragment):
    ctx = C.c_void_p()
    st = lib.xy_create(C.byref(_params(**kw)), None, None, C.byref(ctx))
    assert st == X.XY_EINVAL
    assert ctx.value is None
    assert fragment in X.xy_last_error(None)


def test_null_arguments(lib):
    ctx = C.c_void_p()
    assert lib.xy_create(None, None, None, C.byref(ctx)) == X.XY_EINVAL
    assert lib.xy_create(C.byref(_params()), None, None, None) == X.XY_EINVAL
    assert lib.xy_create(C.byref(_params()), None, C.c_void_p(8), C.byref(ctx)) == X.XY_EINVAL
    assert lib.xy_sweep(None, 1) == X.XY_EINVAL
    assert lib.xy_destroy(None) == X.XY_OK
    algo = C.c_int32(-1)
    assert lib.xy_algorithm(None, C.byref(algo)) == X.XY_EINVAL and algo.value == -1
    # polls out of range: rejected before any CUDA call
    assert lib.xy_selftest_persistent_wait(None, 0) == X.XY_EINVAL
    assert lib.xy_selftest_persistent_wait(None, (1 << 24) + 1) == X.XY_EINVAL
    bogus = C.c_void_p(0x1000)
    assert lib.xy_sweep(bogus, 1) == X.XY_ESTATE        # never created: refused, not read
    assert lib.xy_destroy(bogus) == X.XY_ESTATE
    assert lib.xy_philox_words(1, 0, 0, 1, 0, 5, None, None) == X.XY_EINVAL


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    st = lib.xy_create(C.byref(_params()), None, None, C.byref(ctx))
    assert st in (X.XY_ECUDA, X.XY_ENOMEM)
    assert ctx.value is None
    assert "xy_create" in X.xy_last_error(None)


def _hmc_params(**kw):
    p = X.xy_hmc_params()
    p.L, p.start, p.beta, p.J, p.eps, p.n_md = 8, 0, 1.0, 1.0, 0.1, 10
    p.sincos_mode, p.seed, p.lattice_id, p.kernel = 0, 1, 0, 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_hmc_record_layout():
    assert C.sizeof(X.xy_hmc_record) == 96
    assert C.sizeof(X.xy_hmc_params) == 56


@pytest.mark.parametrize("kw,fragment", [
    (dict(L=1), "L must"), (dict(L=65536), "L must"),
    (dict(beta=-1.0), "beta"), (dict(beta=float("inf")), "beta"), (dict(J=float("nan")), "J"),
    (dict(eps=0.0), "eps"), (dict(eps=float("nan")), "eps"), (dict(n_md=0), "n_md"),
    (dict(start=3), "start"), (dict(sincos_mode=3), "sincos"), (dict(kernel=7), "kernel"), (dict(kernel=5, L=512), "cluster"),
    (dict(kernel=5, L=48), "cluster"),
    (dict(kernel=1, L=96), "multiple of 128"), (dict(kernel=3, L=96), "multiple of 128"),
    (dict(kernel=6, L=96), "multiple of 128"),
])
def test_hmc_create_rejects_bad_parameters(lib, kw, fragment):
    h = C.c_void_p()
    st = lib.xy_hmc_create(C.byref(_hmc_params(**kw)), None, None, C.byref(h))
    assert st == X.XY_EINVAL
    assert h.value is None
    assert fragment in X.xy_hmc_last_error(None)


def test_hmc_null_and_foreign_handles(lib):
    h = C.c_void_p()
    assert lib.xy_hmc_create(None, None, None, C.byref(h)) == X.XY_EINVAL
    assert lib.xy_hmc_create(C.byref(_hmc_params()), None, None, None) == X.XY_EINVAL
    assert lib.xy_hmc_create(C.byref(_hmc_params()), None, C.c_void_p(8), C.byref(h)) == X.XY_EINVAL
    assert lib.xy_hmc_run(None, 1) == X.XY_EINVAL
    assert lib.xy_hmc_destroy(None) == X.XY_OK
    bogus = C.c_void_p(0x2000)
    assert lib.xy_hmc_run(bogus, 1) == X.XY_ESTATE
    assert lib.xy_hmc_integrate(bogus, 1) == X.XY_ESTATE
    assert lib.xy_hmc_destroy(bogus) == X.XY_ESTATE


def test_hmc_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.xy_hmc_create(C.byref(_hmc_params()), None, None, C.byref(h))
    assert st in (X.XY_ECUDA, X.XY_ENOMEM)
    assert h.value is None
    assert "xy_hmc_create" in X.xy_hmc_last_error(None)


def test_quad_create_rejects_bad_parameters(lib):
    q = C.c_void_p()
    good = (C.c_double * 4)(1.0, 1.0, 1.0, 1.0)
    for kw in (dict(L=3), dict(L=0), dict(delta=0.0), dict(start=5), dict(sincos_mode=7),
               dict(reduce_mode=3), dict(J=float("nan")), dict(algorithm=9),
               dict(L=34, algorithm=X.XY_ALGO_PERSISTENT), dict(L=34, algorithm=X.XY_ALGO_FUSED)):
        assert lib.xy_quad_create(C.byref(_params(**kw)), good, None, C.byref(q)) == X.XY_EINVAL
        assert q.value is None
    assert "L % 32" in X.xy_quad_last_error(None)   # the last case: fused needs L % 32 == 0
    bad = (C.c_double * 4)(1.0, float("nan"), 1.0, 1.0)
    assert lib.xy_quad_create(C.byref(_params()), bad, None, C.byref(q)) == X.XY_EINVAL
    assert "beta[1]" in X.xy_quad_last_error(None)
    assert lib.xy_quad_create(C.byref(_params()), None, None, C.byref(q)) == X.XY_EINVAL
    assert lib.xy_quad_sweep(None, 1) == X.XY_EINVAL
    assert lib.xy_quad_destroy(None) == X.XY_OK
    assert lib.xy_quad_sweep(C.c_void_p(0x3000), 1) == X.XY_ESTATE
    a = C.c_int32(0)
    assert lib.xy_quad_algorithm(None, C.byref(a)) == X.XY_EINVAL


def test_sincos_polynomial_constants_are_the_fit():
    """The kernel's polynomial coefficients are the Remez fit of
    csrc/fit_sincos.py rounded to FP32, and the polynomial evaluated with the
    kernel's FP32 operations (single-rounded FMAs) stays within 7e-8 of sin and
    cos over [0, 2 pi]."""
    import importlib.util
    import numpy as np
    path = os.path.join(ROOT, "paper_0811_2111_gb300", "csrc", "fit_sincos.py")
    spec = importlib.util.spec_from_file_location("fit_sincos", path)
    fs = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fs)
    cs, es, cc, ec = fs.fit()
    assert es < 2e-9 and ec < 1e-10
    src = open(os.path.join(ROOT, "paper_0811_2111_gb300", "csrc", "xy_device.cuh")).read()
    body = src[src.index("sincos_poly"):src.index("// quadrant")]
    consts = [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    for v in list(cs) + list(cc):
        assert any(np.float32(v) == np.float32(k) for k in consts), v

    f32 = np.float32

    def fma(a, b, c):
        return f32(np.float64(a) * np.float64(b) + np.float64(c))
    S = [f32(v) for v in cs]
    Cc = [f32(v) for v in cc]
    hi, lo, magic = f32(1.57079601287841796875), f32(3.13916473532088954e-07), f32(12582912.0)
    worst = 0.0
    for t in np.linspace(0, 2 * np.pi, 20001).astype(np.float32):
        qt = fma(t, f32(0.636619772367581343), magic)
        q = int(np.frombuffer(qt.tobytes(), np.int32)[0])
        qf = f32(qt - magic)
        r = fma(-qf, lo, fma(-qf, hi, t))
        r2 = f32(r * r)
        sr = fma(f32(r * r2), fma(r2, fma(r2, S[2], S[1]), S[0]), r)
        cr = fma(r2, fma(r2, fma(r2, fma(r2, Cc[3], Cc[2]), Cc[1]), Cc[0]), f32(1.0))
        s0, c0 = (cr, sr) if q & 1 else (sr, cr)
        s = -s0 if (q & 3) in (2, 3) else s0
        c = -c0 if (q & 3) in (1, 2) else c0
        worst = max(worst, abs(float(s) - np.sin(float(t))), abs(float(c) - np.cos(float(t))))
    assert worst < 7e-8, worst


def test_fma_pipe_quadrant_step_gives_the_bits_of_the_swap_and_sign_step():
    """The accurate unit vector's quadrant step runs on the FMA pipes as
    -(a sr + b cr, a cr - b sr) with p = q - 2, a = 1 - |p|, b = p (2 - |p|):
    FP32 products with a, b in {-1, 0, 1}, never both nonzero, are exact, so
    the result is bit for bit the swap of (sr, cr) on odd q and the sign flips
    by bits 1 of q and q + 1, including signed zeros; checked for every q the
    angles in [-pi/4, 2 pi + pi/4] give, over the values the polynomials
    return on |r| <= pi/4: cr = cos r in [0.70, 1] and sr = sin r in
    [-0.71, 0.71], +0 included (sr is never -0: r = -0 gives r^3 ps = +0 as
    ps < 0, and -0 + +0 = +0).  With a cr or sr of -0 the two forms would
    differ in the sign of a zero."""
    import numpy as np
    f32 = np.float32
    rng = np.random.default_rng(5)
    srs = np.concatenate([rng.uniform(-0.71, 0.71, 20000), [0.0, np.float32(1e-30),
                                                           -np.float32(1e-30), 0.7071068]])
    crs = np.concatenate([rng.uniform(0.70, 1.0, 20000), [1.0, 0.7071068, 0.9999999, 0.75]])
    srs, crs = srs.astype(np.float32), crs.astype(np.float32)

    def fma(x, y, z):      # one FP32 rounding of the exact x * y + z
        return f32(np.float64(x) * np.float64(y) + np.float64(z))

    for q in range(0, 5):
        pq = f32(f32(q) - f32(2.0))
        a = f32(f32(1.0) - abs(pq))
        b = f32(pq * f32(f32(2.0) - abs(pq)))
        for sr, cr in zip(srs, crs):
            s_fma = fma(-a, sr, f32(-b * cr))
            c_fma = fma(b, sr, f32(-a * cr))
            s0, c0 = (cr, sr) if q & 1 else (sr, cr)
            s_bit = -s0 if (q & 2) else s0
            c_bit = -c0 if ((q + 1) & 2) else c0
            assert np.float32(s_fma).tobytes() == np.float32(s_bit).tobytes(), (q, sr, cr)
            assert np.float32(c_fma).tobytes() == np.float32(c_bit).tobytes(), (q, sr, cr)


def test_peak_measure_refuses_bad_arguments_before_the_device(lib):
    rate = C.c_double()
    for kind, iters, reps in ((-1, 16, 1), (len(X.PEAK_KINDS), 16, 1), (0, 0, 1),
                              (0, (1 << 20) + 1, 1), (0, 16, 0), (0, 16, 101)):
        st = lib.xy_peak_measure(kind, iters, reps, None, C.byref(rate), None, None)
        assert st == X.XY_EINVAL, (kind, iters, reps)
    assert lib.xy_peak_measure(0, 16, 1, None, None, None, None) == X.XY_EINVAL
    assert b"bad kind" in lib.xy_peak_last_error()
    # one microbenchmark per kind and one iteration table entry per kind
    import bench
    assert tuple(bench.PEAK_ITERS) == X.PEAK_KINDS


def test_create_refuses_a_bad_work_plan(lib):
    """ctas_per_sm must be 0 (default), 2, 3 or 4; refused before the device is touched."""
    for bad in (1, 5, -1):
        ctx = C.c_void_p()
        st = lib.xy_create(C.byref(_params(L=128, ctas_per_sm=bad)), None, None, C.byref(ctx))
        assert st == X.XY_EINVAL, bad
        assert b"ctas_per_sm" in lib.xy_last_error(None)



def test_batch_create_refuses_a_bad_work_plan(lib):
    """group_ctas in [0, 4096] and ctas_per_sm in {0, 2, 3, 4}, checked before the device."""
    Ls = (C.c_int32 * 2)(16, 16)
    betas = (C.c_double * 2)(1.0, 1.1)
    for field, bad in (("group_ctas", -1), ("group_ctas", 4097), ("ctas_per_sm", 1),
                       ("ctas_per_sm", 5)):
        p = X.xy_batch_params()
        p.n, p.L, p.beta, p.J, p.delta, p.seed = 2, Ls, betas, 1.0, 3.14159, 1
        p.sweeps_per_round = 1
        setattr(p, field, bad)
        b = C.c_void_p()
        assert lib.xy_batch_create(C.byref(p), None, C.byref(b)) == X.XY_EINVAL, (field, bad)


def test_batch_create_refuses_ladders_past_the_exchange_counter(lib):
    """The exchange's Philox counter is ladder * 65536 + pair position: a ladder
    of 65538 lattices (65537 pairs), or 65537 ladders, would reuse another
    pair's words, so either is refused before the device."""
    n = 65538
    Ls = (C.c_int32 * n)(*([2] * n))
    betas = (C.c_double * n)(*[1.0 + 1e-6 * i for i in range(n)])
    for ids, what in (([0] * n, b"65537 lattices"), (list(range(n)), b"65536 ladders")):
        ladder = (C.c_int32 * n)(*ids)
        p = X.xy_batch_params()
        p.n, p.L, p.beta, p.ladder, p.J, p.delta, p.seed = n, Ls, betas, ladder, 1.0, 3.14159, 1
        p.sweeps_per_round = 1
        b = C.c_void_p()
        assert lib.xy_batch_create(C.byref(p), None, C.byref(b)) == X.XY_EINVAL, what
        assert what in lib.xy_batch_last_error(None), what


def test_release_build_has_no_device_checks(lib):
    """The release library reports itself as such and its debug word is always 0
    (no device access: the checks are compiled out)."""
    assert lib.xy_debug_build() == 0
    w = C.c_uint32(123)
    assert lib.xy_debug_checks(C.byref(w)) == X.XY_OK and w.value == 0
    assert lib.xy_debug_checks(None) == X.XY_EINVAL
