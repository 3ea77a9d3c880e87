"""The allocation-free time-step entry point (sidp_compute_dt_static) agrees with sidp_compute_dt.

sidp_compute_dt_static exists for callers that cannot allocate device memory where they need a
time step (their pool allocator owns the device, or cudaMalloc's synchronisation is not
acceptable in their loop).  It keeps its scratch in a fixed device array shared by all calls, so
this test makes two calls in a row on different states and checks each against the context-based
entry point.  It sits in its own file, collected last.
"""
import numpy as np
import pytest

from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_dt_matches_context_dt_twice(precision):
    import torch
    torch.cuda.init()
    cfgs = [dict(law="euler", p=4, nx=16, ny=16, bc=("outflow",) * 4),
            dict(law="burgers", p=3, nx=8, ny=8, bc=("periodic",) * 4, cfl=0.2)]
    for seed, kw in enumerate(cfgs):
        sv = sidp.Solver(precision=precision, **kw)
        x, y = sv.node_coords()
        U = inputs.four_quadrant(x, y, seed) if kw["law"] == "euler" else inputs.burgers_pulse(x, y)
        sv.set_state(U)
        ref = sv.compute_dt()
        dptr, _, _ = sidp.sidp_device_state(sv.ctx)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        sidp.sidp_compute_dt_static(sv.cfg, dptr, out.data_ptr(), None)
        torch.cuda.synchronize()
        got = float(out.item())
        # the same per-node arithmetic as the context's kernel; float32 allows a few ulp where the
        # compiler contracts the face sum into fused multiply-adds differently
        tol = 1e-13 if precision == "fp64" else 4e-7
        assert ref > 0 and abs(got - ref) <= tol * ref, (got, ref)
        sv.close()


def test_static_dt_rejects_oversized_and_unsupported():
    """Each rejection happens on the host, before the (dummy) device pointers are touched."""
    lib = sidp.load()
    big = sidp.make_config(law="euler", p=7, nx=600, ny=600)  # 23M nodes > 16.7M
    assert lib.sidp_compute_dt_static(big, 1, 1, None) == 1
    ex = sidp.make_config(law="euler", p=3, nx=4, ny=4, bc=("exact",) * 4)
    assert lib.sidp_compute_dt_static(ex, 1, 1, None) == 1
    # the unsparsified operator has a smaller time step than the one computed here
    dense = sidp.make_config(law="euler", p=3, nx=4, ny=4, sparsify=False)
    assert lib.sidp_compute_dt_static(dense, 1, 1, None) == 1
    bad_gamma = sidp.make_config(law="euler", p=3, nx=4, ny=4)
    bad_gamma.gamma = 1.0
    assert lib.sidp_compute_dt_static(bad_gamma, 1, 1, None) == 1
    unpaired = sidp.make_config(law="burgers", p=3, nx=4, ny=4, bc=("periodic", "outflow", "periodic", "periodic"))
    assert lib.sidp_compute_dt_static(unpaired, 1, 1, None) == 1
