"""The allocation-free sweep entry point against the regular one (GPU).

xy_sweep_noalloc exists for callers that cannot allocate device memory while
they run; it uses a fixed buffer inside the library instead.  This file is
collected last so that a run stopping at its first failure has already run
every other test.  It calls both entry points through the C ABI on the same
parameters and checks, on two calls in a row, that the angles and per-sweep
records agree within the tolerances the other GPU tests use.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300.lattice import Lattice  # noqa: E402
from gpu_util import ANGLE_TOL, circ, record_tolerance  # noqa: E402


def _obs_from_records(raw, L, beta, J=1.0):
    """(C, Ix, Iy, Mx, My, accepted) from raw device records (n, 8) int64."""
    sums = raw[:, :5].astype(np.float64) * 2.0 ** -X.XY_FX_SHIFT
    return sums, raw[:, 5].astype(np.uint64)


@pytest.mark.parametrize("L,sincos", [(256, "accurate"), (1024, "fast")])
def test_noalloc_matches_regular_sweeps(L, sincos):
    beta, seed, n = 1.1, 77, 7
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    with Lattice(L, beta, seed, sincos=sincos, algorithm="fused") as ref:
        start, _ = ref.state()
        # the regular path's split-layout start state, copied to a caller buffer
        angles = ref.angles.clone()
        ref.sweep(n)
        s1, _ = ref.state()
        o1 = ref.observables()
        ref.sweep(n)
        s2, _ = ref.state()
        o2 = ref.observables(n, n)
        params = ref.params
    recs = torch.zeros((n, 8), dtype=torch.int64, device=dev)
    got = []
    for call in range(2):                                # two calls in a row
        X.xy_sweep_noalloc(params, C.c_void_p(angles.data_ptr()), call * n, n,
                           C.c_void_p(recs.data_ptr()), C.c_void_p(stream.cuda_stream))
        stream.synchronize()
        # back to natural order through the regular ABI for the comparison
        with Lattice(L, beta, seed, sincos=sincos, algorithm="fused") as view:
            view.angles.copy_(angles)
            torch.cuda.synchronize()
            state, _ = view.state()
        got.append((state, _obs_from_records(recs.cpu().numpy(), L, beta)))
    tol = record_tolerance(L * L, fast=(sincos == "fast"))
    for (state, (sums, acc)), s_ref, o_ref in ((got[0], s1, o1), (got[1], s2, o2)):
        assert circ(state.reshape(-1), s_ref.reshape(-1)).max() <= ANGLE_TOL
        ref_sums = np.stack([o_ref[k] for k in ("C", "Ix", "Iy", "Mx", "My")], axis=1)
        assert np.max(np.abs(sums - ref_sums)) <= tol
        assert np.array_equal(acc, o_ref["accepted"])


def test_noalloc_rejects_sizes_beyond_its_buffer():
    p = X.xy_params()
    p.L, p.beta, p.J, p.delta, p.seed = 2048, 1.0, 1.0, 3.14159, 1
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(X.XYError) as ei:
        X.xy_sweep_noalloc(p, C.c_void_p(buf.data_ptr()), 0, 1, C.c_void_p(buf.data_ptr()))
    assert ei.value.status == X.XY_EINVAL
    assert "1024" in str(ei.value)
