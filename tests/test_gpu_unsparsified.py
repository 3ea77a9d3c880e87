"""Unsparsified comparison mode (Sec. 3.4) on the GPU path against the oracle (sparsify=False):
time step, per-stage updates for every limiter, and the sine-wave comparison."""
import numpy as np
import pytest

from fe_compare import elementwise_fe_check, euler_fe_check
from oracle import laws, scheme
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def rel(a, b):
    a = a.reshape(b.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)


def make(lawname, p, limiter, bc=("outflow",) * 4, nx=5, ny=3):
    dom = (0.0, 1.0, 0.0, ny / nx)
    law = laws.Burgers() if lawname == "burgers" else laws.Euler(G)
    pb = scheme.Problem(law, p, nx, ny, domain=dom, bc=bc, limiter=limiter, sparsify=False)
    sv = sidp.Solver(law=lawname, p=p, nx=nx, ny=ny, domain=dom, bc=bc, limiter=limiter, gamma=G, sparsify=False)
    X, Y = pb.node_coords()
    if lawname == "burgers":
        U = inputs.burgers_pulse(X, Y)
    else:
        U = inputs.four_quadrant(X, Y, p)
        U = scheme.Problem(law, p, nx, ny, domain=dom, bc=bc, sparsify=False).ssp_rk3_step(U)[0]
    return pb, sv, U


@pytest.mark.parametrize("lawname,p", [("burgers", 2), ("burgers", 5), ("euler", 3), ("euler", 7)])
def test_dt(lawname, p):
    pb, sv, U = make(lawname, p, "subcell")
    sv.set_state(U.reshape(U.shape[0], -1))
    dt = pb.compute_dt(U)
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt


@pytest.mark.parametrize("limiter", ["none", "lo", "subcell", "elementwise"])
@pytest.mark.parametrize("lawname,p", [("burgers", 1), ("burgers", 3), ("burgers", 6), ("euler", 2), ("euler", 4)])
def test_stage_parity(lawname, p, limiter):
    pb, sv, U0 = make(lawname, p, limiter, bc=("periodic", "periodic", "outflow", "outflow"))
    nc = U0.shape[0]
    dt = pb.compute_dt(U0)
    cur = U0
    sv.set_debug(True)
    for k in (1, 2, 3):
        sv.set_state(cur.reshape(nc, -1))
        sv.stage(1, dt)
        got = sv.get_state(1)
        if limiter == "elementwise":
            elementwise_fe_check(pb, cur, dt, got, sv.bounds()["alpha"])
        elif limiter == "subcell" and lawname == "euler":
            euler_fe_check(pb, cur, dt, got, sv.bounds()["alpha"])
        else:
            exp, info = pb.fe_stage(cur, dt, full=True)
            assert np.all(rel(got, exp) <= 1e-12), rel(got, exp)
            if limiter == "subcell":
                bd = sv.bounds()
                np.testing.assert_allclose(bd["lo"], info["lo"].ravel(), rtol=1e-13, atol=1e-13)
                np.testing.assert_allclose(bd["hi"], info["hi"].ravel(), rtol=1e-13, atol=1e-13)
        cur = pb.stage(cur, U0, dt, k)


def test_sine_wave_comparison_on_gpu():
    """Sec. 3.4: 1D sine wave, 64 degrees of freedom, low-order operators, t = 2."""
    out = {}
    for p in (1, 3, 7):
        ne = 64 // (p + 1)
        h = 2.0 / ne
        for sp in (True, False):
            sv = sidp.Solver(law="advection", p=p, nx=ne, ny=1, domain=(-1.0, 1.0, 0.0, h), beta=(1.0, 0.0),
                             limiter="lo", sparsify=sp)
            x, y = sv.node_coords()
            sv.set_state(np.sin(np.pi * x)[None])
            nsteps = int(np.ceil(2.0 / sv.compute_dt()))
            for _ in range(nsteps):
                for k in (1, 2, 3):
                    sv.stage(k, 2.0 / nsteps)
            out[(p, sp)] = float(sv.get_state(0).max())
    assert out[(1, True)] == pytest.approx(out[(1, False)], rel=1e-12)
    assert out[(7, False)] < 0.3 * out[(7, True)]
    assert out[(7, True)] > 0.8 * out[(3, True)]


def test_batch_rejects_unsparsified():
    with pytest.raises(Exception):
        sidp.sidp_batch_create([sidp.make_config(law="burgers", p=2, nx=2, ny=2, sparsify=False)])
