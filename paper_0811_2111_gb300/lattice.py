"""Python front end of one simulated lattice (torch for memory and streams).

``Lattice`` owns a torch device buffer for the angles, passes its pointer and
the torch stream to ``xy_create``, and exposes the ABI calls with numpy
results.  All arithmetic happens in the CUDA library.
"""
import ctypes as C
import math

import numpy as np

from . import _lib as X


def _torch():
    import torch
    return torch


class Lattice:
    def __init__(self, L, beta, seed, J=1.0, delta=math.pi, start="hot", sincos="accurate",
                 reduce="exact", lattice_id=0, algorithm="auto", device=None, stream=None,
                 ctas_per_sm=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.L = int(L)
        p = X.xy_params()
        p.L = self.L
        p.start = {"hot": X.XY_START_HOT, "cold": X.XY_START_COLD}[start]
        p.beta = float(beta)
        p.J = float(J)
        p.delta = float(delta)
        p.seed = int(seed)
        p.sincos_mode = {"accurate": X.XY_SINCOS_ACCURATE, "fast": X.XY_SINCOS_FAST,
                         "libm": X.XY_SINCOS_LIBM}[sincos]
        p.reduce_mode = {"exact": X.XY_REDUCE_EXACT, "compensated": X.XY_REDUCE_COMPENSATED}[reduce]
        p.lattice_id = int(lattice_id)
        p.algorithm = {"auto": X.XY_ALGO_AUTO, "fused": X.XY_ALGO_FUSED,
                       "two_pass": X.XY_ALGO_TWO_PASS, "persistent": X.XY_ALGO_PERSISTENT,
                       "fused2": X.XY_ALGO_FUSED2}[algorithm]
        p.ctas_per_sm = int(ctas_per_sm)
        self.params = p
        self.J = float(J)
        with torch.cuda.device(self.device):
            self.angles = torch.empty(self.L * self.L, dtype=torch.float32, device=self.device)
            self.ctx = X.xy_create(p, C.c_void_p(self.stream.cuda_stream),
                                   C.c_void_p(self.angles.data_ptr()))

    # -- ABI calls ---------------------------------------------------------
    def reserve(self, n):
        X.xy_reserve(self.ctx, n)

    def reset(self, seed):
        X.xy_reset(self.ctx, int(seed))

    def timing(self, every=1):
        X.xy_timing(self.ctx, every)

    def kernel_time(self, kernel):
        return X.xy_kernel_time(self.ctx, kernel)

    def sweep(self, n=1):
        X.xy_sweep(self.ctx, n)

    def info(self):
        return X.xy_info(self.ctx)

    @property
    def algorithm(self):
        """The sweep algorithm in use: "fused", "two_pass", "persistent" or "fused2"."""
        return {X.XY_ALGO_FUSED: "fused", X.XY_ALGO_TWO_PASS: "two_pass",
                X.XY_ALGO_PERSISTENT: "persistent",
                X.XY_ALGO_FUSED2: "fused2"}[X.xy_algorithm(self.ctx)]

    def observables(self, first=0, count=None):
        n, _ = X.xy_info(self.ctx)
        count = n - first if count is None else count
        obs = X.xy_measure(self.ctx, first, count)
        names = ["e", "abs_m", "upsilon", "C", "Ix", "Iy", "Mx", "My", "beta"]
        out = {k: np.array([getattr(o, k) for o in obs], np.float64) for k in names}
        out["accepted"] = np.array([o.accepted for o in obs], np.uint64)
        return out

    def state(self):
        buf = np.empty(self.L * self.L, np.float32)
        nxt = X.xy_get_state(self.ctx, buf.ctypes.data_as(C.c_void_p))
        return buf.reshape(self.L, self.L), nxt

    def set_state(self, angles, next_sweep):
        a = np.ascontiguousarray(angles, np.float32).reshape(-1)
        if a.size != self.L * self.L:
            raise ValueError("wrong number of angles")
        X.xy_set_state(self.ctx, a.ctypes.data_as(C.c_void_p), int(next_sweep))

    def set_beta(self, beta):
        X.xy_set_beta(self.ctx, float(beta))

    def synchronize(self):
        X.xy_synchronize(self.ctx)

    def records_device(self):
        return X.xy_records_device(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            X.xy_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def unit_vectors(theta, mode="accurate", device=None):
    """(cos, sin) of float32 angles with the kernels' sincos (numpy in, numpy out)."""
    torch = _torch()
    dev = torch.device(device if device is not None else "cuda")
    t = torch.as_tensor(np.ascontiguousarray(theta, np.float32)).to(dev)
    c = torch.empty_like(t)
    s = torch.empty_like(t)
    stream = torch.cuda.current_stream(dev)
    m = {"accurate": X.XY_SINCOS_ACCURATE, "fast": X.XY_SINCOS_FAST, "libm": X.XY_SINCOS_LIBM}[mode]
    X.xy_eval_unit_vector(m, C.c_void_p(t.data_ptr()), C.c_void_p(c.data_ptr()),
                          C.c_void_p(s.data_ptr()), t.numel(), C.c_void_p(stream.cuda_stream))
    stream.synchronize()
    return c.cpu().numpy(), s.cpu().numpy()


def philox_words(seed, sweep, lattice_id, domain, first, n, device=None):
    """Device Philox words (n, 4) uint32 as a numpy array, via xy_philox_words."""
    torch = _torch()
    dev = torch.device(device if device is not None else "cuda")
    out = torch.empty((n, 4), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    X.xy_philox_words(seed, sweep, lattice_id, domain, first, n, C.c_void_p(out.data_ptr()),
                      C.c_void_p(stream.cuda_stream))
    stream.synchronize()
    return out.cpu().numpy().view(np.uint32)


class Batch:
    """Many lattices swept together (``xy_batch_*``), optional replica exchange.

    Ls, betas: per-lattice sides and initial inverse temperatures; ladders:
    per-lattice ladder ids (-1 or None for no exchange)."""

    def __init__(self, Ls, betas, seed, ladders=None, J=1.0, delta=math.pi, start="hot",
                 sincos="accurate", reduce="exact", lattice_id0=0, sweeps_per_round=10,
                 target_band_sites=0, algorithm="auto", device=None, stream=None,
                 group_ctas=0, ctas_per_sm=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = len(Ls)
        self.Ls = np.ascontiguousarray(Ls, np.int32)
        self._betas = np.ascontiguousarray(betas, np.float64)
        self._ladders = None if ladders is None else np.ascontiguousarray(ladders, np.int32)
        p = X.xy_batch_params()
        p.n = n
        p.L = self.Ls.ctypes.data_as(C.POINTER(C.c_int32))
        p.beta = self._betas.ctypes.data_as(C.POINTER(C.c_double))
        p.ladder = (None if self._ladders is None
                    else self._ladders.ctypes.data_as(C.POINTER(C.c_int32)))
        p.J = float(J)
        p.delta = float(delta)
        p.seed = int(seed)
        p.start = {"hot": X.XY_START_HOT, "cold": X.XY_START_COLD}[start]
        p.sincos_mode = {"accurate": X.XY_SINCOS_ACCURATE, "fast": X.XY_SINCOS_FAST,
                         "libm": X.XY_SINCOS_LIBM}[sincos]
        p.reduce_mode = {"exact": X.XY_REDUCE_EXACT, "compensated": X.XY_REDUCE_COMPENSATED}[reduce]
        p.lattice_id0 = int(lattice_id0)
        p.sweeps_per_round = int(sweeps_per_round)
        p.target_band_sites = int(target_band_sites)
        p.algorithm = {"auto": X.XY_ALGO_AUTO, "fused": X.XY_ALGO_FUSED,
                       "two_pass": X.XY_ALGO_TWO_PASS}[algorithm]
        p.group_ctas = int(group_ctas)
        p.ctas_per_sm = int(ctas_per_sm)
        self.params = p
        self.J = float(J)
        self.sweeps_per_round = int(sweeps_per_round)
        with torch.cuda.device(self.device):
            self.b = X.xy_batch_create(p, C.c_void_p(self.stream.cuda_stream))

    @property
    def n(self):
        return len(self.Ls)

    def reserve(self, rounds):
        X.xy_batch_reserve(self.b, rounds)

    def run(self, rounds=1):
        X.xy_batch_run(self.b, rounds)

    def info(self):
        return X.xy_batch_info(self.b)

    def launches_per_round(self):
        return X.xy_batch_launches_per_round(self.b)

    def observables(self, lattice, first=0, count=None):
        _, nrec, _, _ = X.xy_batch_info(self.b)
        count = nrec - first if count is None else count
        obs = X.xy_batch_measure(self.b, lattice, first, count)
        names = ["e", "abs_m", "upsilon", "C", "Ix", "Iy", "Mx", "My", "beta"]
        out = {k: np.array([getattr(o, k) for o in obs], np.float64) for k in names}
        out["accepted"] = np.array([o.accepted for o in obs], np.uint64)
        return out

    def betas(self):
        out = np.empty(self.n, np.float64)
        X.xy_batch_betas(self.b, out.ctypes.data_as(C.c_void_p))
        return out

    def exchange_stats(self):
        n = X.xy_batch_exchange_stats(self.b, None, None, None)
        slots = np.zeros(max(n, 1), np.int32)
        acc = np.zeros(max(n, 1), np.uint64)
        att = np.zeros(max(n, 1), np.uint64)
        X.xy_batch_exchange_stats(self.b, slots.ctypes.data_as(C.c_void_p),
                                  acc.ctypes.data_as(C.c_void_p), att.ctypes.data_as(C.c_void_p))
        return slots[:n], acc[:n], att[:n]

    def state(self, lattice):
        L = int(self.Ls[lattice])
        buf = np.empty(L * L, np.float32)
        X.xy_batch_get_state(self.b, lattice, buf.ctypes.data_as(C.c_void_p))
        return buf.reshape(L, L)

    def records_device(self):
        return X.xy_batch_records_device(self.b)

    def series_stats(self, first, count):
        """Device tensor (n, 8) float64 of xy_batch_series_stats (see include/xy.h)."""
        torch = _torch()
        out = torch.empty((self.n, X.XY_STATS_FIELDS), dtype=torch.float64, device=self.device)
        X.xy_batch_series_stats(self.b, int(first), int(count), C.c_void_p(out.data_ptr()))
        return out

    def synchronize(self):
        X.xy_batch_synchronize(self.b)

    def close(self):
        if getattr(self, "b", None) is not None:
            X.xy_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Quad:
    """Four replicas of one L x L lattice packed per site (``xy_quad_*``, the RGBA
    packing of Sec. 3.2): replica r has lattice id lattice_id + r and beta betas[r]."""

    def __init__(self, L, betas, seed, J=1.0, delta=math.pi, start="hot", sincos="accurate",
                 reduce="exact", lattice_id=0, algorithm="auto", device=None, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        if len(betas) != X.XY_QUAD_REPLICAS:
            raise ValueError("need four betas")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.L = int(L)
        p = X.xy_params()
        p.L = self.L
        p.start = {"hot": X.XY_START_HOT, "cold": X.XY_START_COLD}[start]
        p.beta = 0.0
        p.J = float(J)
        p.delta = float(delta)
        p.seed = int(seed)
        p.sincos_mode = {"accurate": X.XY_SINCOS_ACCURATE, "fast": X.XY_SINCOS_FAST,
                         "libm": X.XY_SINCOS_LIBM}[sincos]
        p.reduce_mode = {"exact": X.XY_REDUCE_EXACT, "compensated": X.XY_REDUCE_COMPENSATED}[reduce]
        p.lattice_id = int(lattice_id)
        p.algorithm = {"auto": X.XY_ALGO_AUTO, "fused": X.XY_ALGO_FUSED,
                       "two_pass": X.XY_ALGO_TWO_PASS, "persistent": X.XY_ALGO_PERSISTENT,
                       "fused2": X.XY_ALGO_FUSED2}[algorithm]
        self.params = p
        with torch.cuda.device(self.device):
            self.q = X.xy_quad_create(p, betas, C.c_void_p(self.stream.cuda_stream))

    @property
    def algorithm(self):
        """"persistent" (one launch per call), "fused" (one per sweep) or "two_pass"."""
        return {X.XY_ALGO_FUSED: "fused", X.XY_ALGO_TWO_PASS: "two_pass",
                X.XY_ALGO_PERSISTENT: "persistent"}[X.xy_quad_algorithm(self.q)]

    def sweep(self, n=1):
        X.xy_quad_sweep(self.q, n)

    def info(self):
        return X.xy_quad_info(self.q)

    def observables(self, replica, first=0, count=None):
        n, _ = X.xy_quad_info(self.q)
        count = n - first if count is None else count
        obs = X.xy_quad_measure(self.q, replica, first, count)
        names = ["e", "abs_m", "upsilon", "C", "Ix", "Iy", "Mx", "My", "beta"]
        out = {k: np.array([getattr(o, k) for o in obs], np.float64) for k in names}
        out["accepted"] = np.array([o.accepted for o in obs], np.uint64)
        return out

    def state(self, replica):
        buf = np.empty(self.L * self.L, np.float32)
        nxt = X.xy_quad_get_state(self.q, replica, buf.ctypes.data_as(C.c_void_p))
        return buf.reshape(self.L, self.L), nxt

    def synchronize(self):
        X.xy_quad_synchronize(self.q)

    def close(self):
        if getattr(self, "q", None) is not None:
            X.xy_quad_destroy(self.q)
            self.q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
