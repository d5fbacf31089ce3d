"""Hybrid Monte Carlo chains (``xy_hmc_*`` of ``include/xy_hmc.h``).

Argument marshalling only: momenta, leap-frog integration, the test and the
sums all run in ``libxy.so``'s CUDA kernels.  Angles and momenta cross the
boundary as float32 arrays in natural order [y][x].
"""
import ctypes as C

import numpy as np

from . import _lib as X

_MODES = {"accurate": X.XY_SINCOS_ACCURATE, "fast": X.XY_SINCOS_FAST, "libm": X.XY_SINCOS_LIBM}


def _torch():
    import torch
    return torch


class HMC:
    """One HMC chain on an L x L torus: H_hmc = sum p^2/2 + beta H(theta),
    trajectories of n_md leap-frog steps of size eps."""

    def __init__(self, L, beta, seed, eps, n_md, J=1.0, start="hot", sincos="accurate",
                 lattice_id=0, kernel="auto", device=None, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.L = int(L)
        p = X.xy_hmc_params()
        p.L = self.L
        p.start = {"hot": X.XY_START_HOT, "cold": X.XY_START_COLD}[start]
        p.beta = float(beta)
        p.J = float(J)
        p.eps = float(eps)
        p.n_md = int(n_md)
        p.sincos_mode = _MODES[sincos]
        p.seed = int(seed)
        p.lattice_id = int(lattice_id)
        p.kernel = {"auto": X.XY_HMC_KERNEL_AUTO, "tiled": X.XY_HMC_KERNEL_TILED,
                    "site": X.XY_HMC_KERNEL_SITE, "tiled2": X.XY_HMC_KERNEL_TILED2,
                    "tiled_tma": X.XY_HMC_KERNEL_TILED_TMA,
                    "cluster": X.XY_HMC_KERNEL_CLUSTER,
                    "persistent": X.XY_HMC_KERNEL_PERSISTENT}[kernel]
        self.params = p
        self.J = float(J)
        with torch.cuda.device(self.device):
            self.h = X.xy_hmc_create(p, C.c_void_p(self.stream.cuda_stream), None)

    # -- ABI calls ---------------------------------------------------------
    def run(self, n_traj=1):
        X.xy_hmc_run(self.h, n_traj)

    def integrate(self, n_steps):
        X.xy_hmc_integrate(self.h, n_steps)

    def refresh(self):
        X.xy_hmc_refresh(self.h)

    def last_sums(self):
        """dict of the last trajectory's/integration's sums at its start and end."""
        v = X.xy_hmc_last_sums(self.h)
        names = ["K", "C", "Ix", "Iy", "Mx", "My"]
        return {"start": dict(zip(names, v[:6])), "end": dict(zip(names, v[6:]))}

    def info(self):
        """(records, next trajectory, accepted so far)."""
        return X.xy_hmc_info(self.h)

    def observables(self, first=0, count=None):
        n, _, _ = X.xy_hmc_info(self.h)
        count = n - first if count is None else count
        dH = np.zeros(max(count, 1), np.float64)
        obs = X.xy_hmc_measure(self.h, first, count, dH.ctypes.data_as(C.c_void_p))
        names = ["e", "abs_m", "upsilon", "C", "Ix", "Iy", "Mx", "My", "beta"]
        out = {k: np.array([getattr(o, k) for o in obs], np.float64) for k in names}
        out["accepted"] = np.array([o.accepted for o in obs], np.uint64)
        out["dH"] = dH[:count]
        return out

    def records_device(self):
        return X.xy_hmc_records_device(self.h)

    def state(self):
        """(angles [L, L] float32, momenta [L, L] float32, next trajectory)."""
        th = np.empty(self.L * self.L, np.float32)
        p = np.empty(self.L * self.L, np.float32)
        t = X.xy_hmc_get_state(self.h, th.ctypes.data_as(C.c_void_p), p.ctypes.data_as(C.c_void_p))
        return th.reshape(self.L, self.L), p.reshape(self.L, self.L), t

    def set_state(self, angles, momenta=None, next_traj=0):
        a = np.ascontiguousarray(angles, np.float32).reshape(-1)
        if a.size != self.L * self.L:
            raise ValueError("wrong number of angles")
        pp = None
        if momenta is not None:
            m = np.ascontiguousarray(momenta, np.float32).reshape(-1)
            if m.size != a.size:
                raise ValueError("wrong number of momenta")
            pp = m.ctypes.data_as(C.c_void_p)
        X.xy_hmc_set_state(self.h, a.ctypes.data_as(C.c_void_p), pp, int(next_traj))

    def set_step(self, eps, n_md):
        X.xy_hmc_set_step(self.h, float(eps), int(n_md))

    def set_beta(self, beta):
        X.xy_hmc_set_beta(self.h, float(beta))

    def synchronize(self):
        X.xy_hmc_synchronize(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            X.xy_hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
