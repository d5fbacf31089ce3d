"""The allocation-free sweep entry point against the regular one (GPU).

xy_sweep_noalloc exists for callers that cannot allocate device memory while
they run; it uses a fixed buffer inside the library instead.  This file is
collected last so that a run stopping at its first failure has already run
every other test.  It calls both entry points through the C ABI on the same
parameters and checks, on two calls in a row, that the angles and the raw
per-sweep record words are identical: both run the same fused kernel on the
same Philox words, and the record sums are fixed-point integers added by
atomics, whose order does not matter, so nothing may differ by even one bit.
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


def _device_records(ptr, n):
    """Copy of n xy_record structs (8 words of 64 bits each) at a device address."""
    class _View:
        __cuda_array_interface__ = {"shape": (n, 8), "typestr": "<i8", "data": (ptr, False),
                                    "version": 3}
    return torch.as_tensor(_View(), device="cuda").clone()


@pytest.mark.parametrize("L,sincos", [(256, "accurate"), (1024, "fast")])
def test_noalloc_matches_regular_sweeps(L, sincos):
    beta, seed, n = 1.1, 77, 7
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    with Lattice(L, beta, seed, sincos=sincos, algorithm="fused") as ref:
        # the regular path's split-layout start state, copied to a caller buffer
        angles = ref.angles.clone()
        ref.sweep(n)
        torch.cuda.synchronize()
        a1 = ref.angles.clone()
        ref.sweep(n)
        torch.cuda.synchronize()
        a2 = ref.angles.clone()
        ptr, count = ref.records_device()
        assert count == 2 * n
        rec_ref = _device_records(ptr, count)
        params = ref.params
    recs = torch.zeros((n, 8), dtype=torch.int64, device=dev)
    for call, a_ref in enumerate((a1, a2)):                # two calls in a row
        X.xy_sweep_noalloc(params, C.c_void_p(angles.data_ptr()), call * n, n,
                           C.c_void_p(recs.data_ptr()), C.c_void_p(stream.cuda_stream))
        stream.synchronize()
        assert torch.equal(angles, a_ref), f"call {call}: angles differ"
        assert torch.equal(recs, rec_ref[call * n:(call + 1) * n]), f"call {call}: records differ"


def test_noalloc_rejects_sizes_beyond_its_buffer():
    p = X.xy_params()
    p.L, p.beta, p.J, p.delta, p.seed = 2048, 1.0, 1.0, 3.14159, 1
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(X.XYError) as ei:
        X.xy_sweep_noalloc(p, C.c_void_p(buf.data_ptr()), 0, 1, C.c_void_p(buf.data_ptr()))
    assert ei.value.status == X.XY_EINVAL
    assert "1024" in str(ei.value)
