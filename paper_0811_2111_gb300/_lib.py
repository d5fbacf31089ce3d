"""ctypes binding of the C ABI in ``include/xy.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of its own: all of the simulation runs in ``libxy.so``'s CUDA
kernels.  If the library has not been built this module raises at load time;
there is no fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# The library this process uses: libxy.so, or the debug build (libxy_debug.so)
# when XY_GB300_LIB names it (the debug-build test runs in a child process).
LIB_PATH = os.environ.get("XY_GB300_LIB") or os.path.join(HERE, "libxy.so")

XY_OK, XY_EINVAL, XY_ENOMEM, XY_ECUDA, XY_ETIMEOUT, XY_ESTATE, XY_ENUMERIC = range(7)
STATUS_NAMES = {0: "XY_OK", 1: "XY_EINVAL", 2: "XY_ENOMEM", 3: "XY_ECUDA", 4: "XY_ETIMEOUT",
                5: "XY_ESTATE", 6: "XY_ENUMERIC"}
XY_START_HOT, XY_START_COLD = 0, 1
XY_SINCOS_ACCURATE, XY_SINCOS_FAST, XY_SINCOS_LIBM = 0, 1, 2
XY_ALGO_AUTO, XY_ALGO_FUSED, XY_ALGO_TWO_PASS, XY_ALGO_PERSISTENT, XY_ALGO_FUSED2 = 0, 1, 2, 3, 4
XY_REDUCE_EXACT, XY_REDUCE_COMPENSATED = 0, 1
XY_FX_SHIFT = 30
XY_MAX_L = 32768


class XYError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class xy_params(C.Structure):
    _fields_ = [("L", C.c_int32), ("start", C.c_int32), ("beta", C.c_double), ("J", C.c_double),
                ("delta", C.c_double), ("seed", C.c_uint64), ("sincos_mode", C.c_int32),
                ("reduce_mode", C.c_int32), ("lattice_id", C.c_uint32), ("algorithm", C.c_int32),
                ("ctas_per_sm", C.c_int32)]


class xy_record(C.Structure):
    _fields_ = [("sum", C.c_int64 * 5), ("accepted", C.c_uint64), ("beta", C.c_double),
                ("flags", C.c_uint64)]


class xy_obs(C.Structure):
    _fields_ = [("e", C.c_double), ("abs_m", C.c_double), ("upsilon", C.c_double),
                ("C", C.c_double), ("Ix", C.c_double), ("Iy", C.c_double), ("Mx", C.c_double),
                ("My", C.c_double), ("accepted", C.c_uint64), ("beta", C.c_double)]


class xy_batch_params(C.Structure):
    _fields_ = [("n", C.c_int32), ("L", C.POINTER(C.c_int32)), ("beta", C.POINTER(C.c_double)),
                ("ladder", C.POINTER(C.c_int32)), ("J", C.c_double), ("delta", C.c_double),
                ("seed", C.c_uint64), ("start", C.c_int32), ("sincos_mode", C.c_int32),
                ("reduce_mode", C.c_int32), ("lattice_id0", C.c_uint32),
                ("sweeps_per_round", C.c_int32), ("target_band_sites", C.c_int32),
                ("algorithm", C.c_int32), ("group_ctas", C.c_int32), ("ctas_per_sm", C.c_int32)]


XY_BATCH_MAX_L = 256
XY_STATS_FIELDS = 8
XY_HMC_K_SHIFT = 24
XY_HMC_KERNEL_AUTO, XY_HMC_KERNEL_TILED, XY_HMC_KERNEL_SITE, XY_HMC_KERNEL_TILED2 = 0, 1, 2, 3
XY_HMC_KERNEL_TILED_TMA = 4
XY_HMC_KERNEL_CLUSTER = 5
XY_HMC_KERNEL_PERSISTENT = 6


class xy_hmc_params(C.Structure):
    _fields_ = [("L", C.c_int32), ("start", C.c_int32), ("beta", C.c_double), ("J", C.c_double),
                ("eps", C.c_double), ("n_md", C.c_int32), ("sincos_mode", C.c_int32),
                ("seed", C.c_uint64), ("lattice_id", C.c_uint32), ("kernel", C.c_int32)]


class xy_hmc_record(C.Structure):
    _fields_ = [("sum", C.c_int64 * 5), ("kinetic", C.c_int64 * 2), ("bonds", C.c_int64 * 2),
                ("dH", C.c_double), ("beta", C.c_double), ("accepted", C.c_uint64)]

_lib = None


def lib():
    """Load ``libxy.so``; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                          f"g.build()'` (the CUDA library is required, there is no fallback)")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    P = C.c_void_p
    sig = {
        "xy_create": (st, [C.POINTER(xy_params), P, P, C.POINTER(P)]),
        "xy_reserve": (st, [P, C.c_int64]),
        "xy_reset": (st, [P, C.c_uint64]),
        "xy_timing": (st, [P, C.c_int]),
        "xy_kernel_time": (st, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "xy_sweep": (st, [P, C.c_int64]),
        "xy_measure": (st, [P, C.c_int64, C.c_int64, C.POINTER(xy_obs)]),
        "xy_records_device": (st, [P, C.POINTER(P), C.POINTER(C.c_int64)]),
        "xy_info": (st, [P, C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]),
        "xy_algorithm": (st, [P, C.POINTER(C.c_int32)]),
        "xy_selftest_persistent_wait": (st, [P, C.c_int64]),
        "xy_get_state": (st, [P, P, C.POINTER(C.c_uint64)]),
        "xy_set_state": (st, [P, P, C.c_uint64]),
        "xy_set_beta": (st, [P, C.c_double]),
        "xy_synchronize": (st, [P]),
        "xy_destroy": (st, [P]),
        "xy_last_error": (C.c_char_p, [P]),
        "xy_philox_words": (st, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.c_int64, P, P]),
        "xy_version": (C.c_int32, []),
        "xy_eval_unit_vector": (st, [C.c_int32, P, P, P, C.c_int64, P]),
        "xy_sweep_noalloc": (st, [C.POINTER(xy_params), P, C.c_uint32, C.c_int64, P, P]),
        "xy_batch_create": (st, [C.POINTER(xy_batch_params), P, C.POINTER(P)]),
        "xy_batch_reserve": (st, [P, C.c_int64]),
        "xy_batch_run": (st, [P, C.c_int64]),
        "xy_batch_info": (st, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                               C.POINTER(C.c_uint64), C.POINTER(C.c_int32)]),
        "xy_batch_measure": (st, [P, C.c_int32, C.c_int64, C.c_int64, C.POINTER(xy_obs)]),
        "xy_batch_records_device": (st, [P, C.POINTER(P), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]),
        "xy_batch_betas": (st, [P, P]),
        "xy_batch_exchange_stats": (st, [P, C.POINTER(C.c_int32), P, P, P]),
        "xy_batch_get_state": (st, [P, C.c_int32, P]),
        "xy_batch_synchronize": (st, [P]),
        "xy_batch_launches_per_round": (st, [P, C.POINTER(C.c_int32)]),
        "xy_batch_series_stats": (st, [P, C.c_int64, C.c_int64, P]),
        "xy_batch_destroy": (st, [P]),
        "xy_batch_last_error": (C.c_char_p, [P]),
        "xy_noalloc_last_error": (C.c_char_p, []),
        "xy_hmc_create": (st, [C.POINTER(xy_hmc_params), P, P, C.POINTER(P)]),
        "xy_hmc_run": (st, [P, C.c_int64]),
        "xy_hmc_integrate": (st, [P, C.c_int32]),
        "xy_hmc_refresh": (st, [P]),
        "xy_hmc_last_sums": (st, [P, P]),
        "xy_hmc_measure": (st, [P, C.c_int64, C.c_int64, C.POINTER(xy_obs), P]),
        "xy_hmc_records_device": (st, [P, C.POINTER(P), C.POINTER(C.c_int64)]),
        "xy_hmc_info": (st, [P, C.POINTER(C.c_int64), C.POINTER(C.c_uint64),
                             C.POINTER(C.c_uint64)]),
        "xy_hmc_get_state": (st, [P, P, P, C.POINTER(C.c_uint64)]),
        "xy_hmc_set_state": (st, [P, P, P, C.c_uint64]),
        "xy_hmc_set_step": (st, [P, C.c_double, C.c_int32]),
        "xy_hmc_set_beta": (st, [P, C.c_double]),
        "xy_hmc_synchronize": (st, [P]),
        "xy_hmc_destroy": (st, [P]),
        "xy_hmc_last_error": (C.c_char_p, [P]),
        "xy_selftest_bounded_wait": (st, [P, C.c_int64]),
        "xy_quad_create": (st, [C.POINTER(xy_params), P, P, C.POINTER(P)]),
        "xy_quad_sweep": (st, [P, C.c_int64]),
        "xy_quad_measure": (st, [P, C.c_int32, C.c_int64, C.c_int64, C.POINTER(xy_obs)]),
        "xy_quad_get_state": (st, [P, C.c_int32, P, C.POINTER(C.c_uint64)]),
        "xy_quad_info": (st, [P, C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]),
        "xy_quad_algorithm": (st, [P, C.POINTER(C.c_int32)]),
        "xy_quad_synchronize": (st, [P]),
        "xy_quad_destroy": (st, [P]),
        "xy_quad_last_error": (C.c_char_p, [P]),
        "xy_peak_measure": (st, [C.c_int32, C.c_int32, C.c_int32, P, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "xy_peak_last_error": (C.c_char_p, []),
        "xy_debug_fail_alloc": (st, [C.c_int32]),
        "xy_debug_build": (C.c_int32, []),
        "xy_debug_checks": (st, [C.POINTER(C.c_uint32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status, ctx=None):
    if status != XY_OK:
        msg = lib().xy_last_error(ctx)
        raise XYError(status, msg.decode() if msg else "")
    return status


# -- same-named thin wrappers -------------------------------------------------

def xy_create(params, stream_ptr=None, d_angles_ptr=None):
    ctx = C.c_void_p()
    check(lib().xy_create(C.byref(params), stream_ptr, d_angles_ptr, C.byref(ctx)))
    return ctx


def xy_reserve(ctx, n_more):
    check(lib().xy_reserve(ctx, n_more), ctx)


def xy_reset(ctx, seed):
    check(lib().xy_reset(ctx, seed), ctx)


def xy_timing(ctx, every):
    check(lib().xy_timing(ctx, int(every)), ctx)


def xy_kernel_time(ctx, kernel):
    ms = C.c_double()
    n = C.c_int64()
    check(lib().xy_kernel_time(ctx, kernel, C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def xy_sweep(ctx, n):
    check(lib().xy_sweep(ctx, n), ctx)


def xy_measure(ctx, first, count):
    out = (xy_obs * max(count, 1))()
    check(lib().xy_measure(ctx, first, count, out), ctx)
    return out if count > 0 else (xy_obs * 0)()


def xy_records_device(ctx):
    p = C.c_void_p()
    n = C.c_int64()
    check(lib().xy_records_device(ctx, C.byref(p), C.byref(n)), ctx)
    return p.value, n.value


def xy_info(ctx):
    n = C.c_int64()
    s = C.c_uint64()
    check(lib().xy_info(ctx, C.byref(n), C.byref(s)), ctx)
    return n.value, s.value


def xy_algorithm(ctx):
    a = C.c_int32(0)
    check(lib().xy_algorithm(ctx, C.byref(a)), ctx)
    return a.value


def xy_get_state(ctx, host_ptr):
    s = C.c_uint64()
    check(lib().xy_get_state(ctx, host_ptr, C.byref(s)), ctx)
    return s.value


def xy_set_state(ctx, host_ptr, next_sweep):
    check(lib().xy_set_state(ctx, host_ptr, next_sweep), ctx)


def xy_set_beta(ctx, beta):
    check(lib().xy_set_beta(ctx, beta), ctx)


def xy_synchronize(ctx):
    check(lib().xy_synchronize(ctx), ctx)


def xy_destroy(ctx):
    check(lib().xy_destroy(ctx))


def xy_last_error(ctx=None):
    m = lib().xy_last_error(ctx)
    return m.decode() if m else ""


def xy_philox_words(seed, sweep, lattice_id, domain, first, n, d_out_ptr, stream_ptr=None):
    check(lib().xy_philox_words(seed, sweep, lattice_id, domain, first, n, d_out_ptr, stream_ptr))


def xy_eval_unit_vector(mode, d_theta_ptr, d_cos_ptr, d_sin_ptr, n, stream_ptr=None):
    check(lib().xy_eval_unit_vector(mode, d_theta_ptr, d_cos_ptr, d_sin_ptr, n, stream_ptr))


def xy_sweep_noalloc(params, d_angles_ptr, first_sweep, n_sweeps, d_records_ptr,
                     stream_ptr=None):
    st = lib().xy_sweep_noalloc(C.byref(params), d_angles_ptr, first_sweep, n_sweeps,
                                d_records_ptr, stream_ptr)
    if st != XY_OK:
        raise XYError(st, lib().xy_noalloc_last_error().decode())


def xy_version():
    return int(lib().xy_version())


# -- instruction-rate microbenchmarks (include/xy_peaks.h) --------------------

PEAK_KINDS = ("ffma", "imad", "imad_wide", "imad_hi", "lop3", "iadd", "mufu_sin", "mufu_ex2",
              "f2i", "dfma", "issue", "philox", "unit_vector", "unit_vector_sfu", "expf")


def xy_peak_measure(kind, iters, reps=5, stream_ptr=None):
    """(ops/s over the GPU, best launch ms, ops per launch) of one xy_peak_kind."""
    k = PEAK_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    rate, ms, ops = C.c_double(), C.c_double(), C.c_double()
    st = lib().xy_peak_measure(k, int(iters), int(reps), stream_ptr, C.byref(rate), C.byref(ms),
                               C.byref(ops))
    if st != XY_OK:
        raise XYError(st, lib().xy_peak_last_error().decode())
    return rate.value, ms.value, ops.value


# -- batches ------------------------------------------------------------------

def batch_check(status, b=None):
    if status != XY_OK:
        msg = lib().xy_batch_last_error(b)
        raise XYError(status, msg.decode() if msg else "")
    return status


def xy_batch_create(params, stream_ptr=None):
    b = C.c_void_p()
    batch_check(lib().xy_batch_create(C.byref(params), stream_ptr, C.byref(b)))
    return b


def xy_batch_reserve(b, n_rounds):
    batch_check(lib().xy_batch_reserve(b, n_rounds), b)


def xy_batch_run(b, rounds):
    batch_check(lib().xy_batch_run(b, rounds), b)


def xy_batch_info(b):
    n = C.c_int32()
    r = C.c_int64()
    s = C.c_uint64()
    c = C.c_int32()
    batch_check(lib().xy_batch_info(b, C.byref(n), C.byref(r), C.byref(s), C.byref(c)), b)
    return n.value, r.value, s.value, c.value


def xy_batch_measure(b, lattice, first, count):
    out = (xy_obs * max(count, 1))()
    batch_check(lib().xy_batch_measure(b, lattice, first, count, out), b)
    return out if count > 0 else (xy_obs * 0)()


def xy_batch_records_device(b):
    p = C.c_void_p()
    stride = C.c_int64()
    n = C.c_int64()
    batch_check(lib().xy_batch_records_device(b, C.byref(p), C.byref(stride), C.byref(n)), b)
    return p.value, stride.value, n.value


def xy_batch_betas(b, host_ptr):
    batch_check(lib().xy_batch_betas(b, host_ptr), b)


def xy_batch_exchange_stats(b, slot_ptr, acc_ptr, att_ptr):
    n = C.c_int32()
    batch_check(lib().xy_batch_exchange_stats(b, C.byref(n), slot_ptr, acc_ptr, att_ptr), b)
    return n.value


def xy_batch_get_state(b, lattice, host_ptr):
    batch_check(lib().xy_batch_get_state(b, lattice, host_ptr), b)


def xy_batch_launches_per_round(b):
    n = C.c_int32()
    batch_check(lib().xy_batch_launches_per_round(b, C.byref(n)), b)
    return n.value


def xy_batch_synchronize(b):
    batch_check(lib().xy_batch_synchronize(b), b)


def xy_batch_destroy(b):
    batch_check(lib().xy_batch_destroy(b))


def xy_batch_series_stats(b, first, count, d_out_ptr):
    batch_check(lib().xy_batch_series_stats(b, first, count, d_out_ptr), b)


# -- Hybrid Monte Carlo (include/xy_hmc.h) -------------------------------------

def hmc_check(status, h=None):
    if status != XY_OK:
        msg = lib().xy_hmc_last_error(h)
        raise XYError(status, msg.decode() if msg else "")
    return status


def xy_hmc_create(params, stream_ptr=None, d_angles_ptr=None):
    h = C.c_void_p()
    hmc_check(lib().xy_hmc_create(C.byref(params), stream_ptr, d_angles_ptr, C.byref(h)))
    return h


def xy_hmc_run(h, n_traj):
    hmc_check(lib().xy_hmc_run(h, n_traj), h)


def xy_hmc_integrate(h, n_steps):
    hmc_check(lib().xy_hmc_integrate(h, n_steps), h)


def xy_hmc_refresh(h):
    hmc_check(lib().xy_hmc_refresh(h), h)


def xy_hmc_last_sums(h):
    out = (C.c_double * 12)()
    hmc_check(lib().xy_hmc_last_sums(h, out), h)
    return list(out)


def xy_hmc_measure(h, first, count, dH_ptr=None):
    out = (xy_obs * max(count, 1))()
    hmc_check(lib().xy_hmc_measure(h, first, count, out, dH_ptr), h)
    return out if count > 0 else (xy_obs * 0)()


def xy_hmc_records_device(h):
    p = C.c_void_p()
    n = C.c_int64()
    hmc_check(lib().xy_hmc_records_device(h, C.byref(p), C.byref(n)), h)
    return p.value, n.value


def xy_hmc_info(h):
    r = C.c_int64()
    t = C.c_uint64()
    a = C.c_uint64()
    hmc_check(lib().xy_hmc_info(h, C.byref(r), C.byref(t), C.byref(a)), h)
    return r.value, t.value, a.value


def xy_hmc_get_state(h, angles_ptr, momenta_ptr=None):
    t = C.c_uint64()
    hmc_check(lib().xy_hmc_get_state(h, angles_ptr, momenta_ptr, C.byref(t)), h)
    return t.value


def xy_hmc_set_state(h, angles_ptr, momenta_ptr, next_traj):
    hmc_check(lib().xy_hmc_set_state(h, angles_ptr, momenta_ptr, next_traj), h)


def xy_hmc_set_step(h, eps, n_md):
    hmc_check(lib().xy_hmc_set_step(h, eps, n_md), h)


def xy_hmc_set_beta(h, beta):
    hmc_check(lib().xy_hmc_set_beta(h, beta), h)


def xy_hmc_synchronize(h):
    hmc_check(lib().xy_hmc_synchronize(h), h)


def xy_hmc_destroy(h):
    hmc_check(lib().xy_hmc_destroy(h))


def xy_hmc_last_error(h=None):
    m = lib().xy_hmc_last_error(h)
    return m.decode() if m else ""


# -- four replicas per site (include/xy_quad.h) ---------------------------------

XY_QUAD_REPLICAS = 4


def quad_check(status, q=None):
    if status != XY_OK:
        msg = lib().xy_quad_last_error(q)
        raise XYError(status, msg.decode() if msg else "")
    return status


def xy_quad_create(params, betas, stream_ptr=None):
    q = C.c_void_p()
    b = (C.c_double * 4)(*[float(v) for v in betas])
    quad_check(lib().xy_quad_create(C.byref(params), b, stream_ptr, C.byref(q)))
    return q


def xy_quad_sweep(q, n):
    quad_check(lib().xy_quad_sweep(q, n), q)


def xy_quad_measure(q, replica, first, count):
    out = (xy_obs * max(count, 1))()
    quad_check(lib().xy_quad_measure(q, replica, first, count, out), q)
    return out if count > 0 else (xy_obs * 0)()


def xy_quad_get_state(q, replica, host_ptr):
    t = C.c_uint64()
    quad_check(lib().xy_quad_get_state(q, replica, host_ptr, C.byref(t)), q)
    return t.value


def xy_quad_info(q):
    r = C.c_int64()
    t = C.c_uint64()
    quad_check(lib().xy_quad_info(q, C.byref(r), C.byref(t)), q)
    return r.value, t.value


def xy_quad_algorithm(q):
    a = C.c_int32(0)
    quad_check(lib().xy_quad_algorithm(q, C.byref(a)), q)
    return a.value


def xy_quad_synchronize(q):
    quad_check(lib().xy_quad_synchronize(q), q)


def xy_quad_destroy(q):
    quad_check(lib().xy_quad_destroy(q))


def xy_quad_last_error(q=None):
    m = lib().xy_quad_last_error(q)
    return m.decode() if m else ""
