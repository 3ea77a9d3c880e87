"""Slip-wall boundary (Sec. 5.7) on the GPU path: per-stage parity with the FP64 oracle (strict for
the unlimited and low-order operators, conditioning-aware for the entropy-limited stage), and the
mirror symmetry checked on the GPU alone over whole steps."""
import numpy as np
import pytest

import test_oracle_wall as tw
from fe_compare import euler_fe_check
from oracle import laws, scheme
from paper_2004_08503_gb300 import build, sidp

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


@pytest.mark.parametrize("limiter", ["none", "lo", "subcell"])
@pytest.mark.parametrize("p,bc", [(2, ("wall", "outflow", "wall", "outflow")), (3, ("outflow", "wall", "outflow", "wall")),
                                  (5, ("wall",) * 4), (7, ("wall", "wall", "periodic", "periodic"))])
def test_wall_stage_parity(p, bc, limiter):
    nx, ny = 5, 3
    dom = (0.0, 1.0, 0.0, 0.6)
    pb = scheme.Problem(laws.Euler(G), p, nx, ny, domain=dom, bc=bc, limiter=limiter)
    sv = sidp.Solver(law="euler", p=p, nx=nx, ny=ny, domain=dom, bc=bc, limiter=limiter, gamma=G)
    X, Y = pb.node_coords()
    U0 = pb.law.prim_to_cons(*tw._data(X, Y))
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(4, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    sv.set_debug(True)
    cur = U0
    for k in (1, 2, 3):
        sv.set_state(cur.reshape(4, -1))
        sv.stage(1, dt)
        got = sv.get_state(1)
        if limiter == "subcell":
            euler_fe_check(pb, cur, dt, got, sv.bounds()["alpha"])
        else:
            assert np.all(rel(got, pb.fe_stage(cur, dt)) <= 1e-12)
        cur = pb.stage(cur, U0, dt, k)


@pytest.mark.parametrize("side", ["W", "S"])
def test_wall_mirror_symmetry_on_gpu(side):
    """GPU alone: wall problem == mirrored doubled problem restricted (low-order operator, whole
    steps with the device time step, to 1e-12)."""
    p = 3
    law, wall, full = tw._problems(p, side, "lo")
    n = tw.N_EL
    bcw = ["outflow"] * 4
    bcw[{"W": 0, "S": 2}[side]] = "wall"
    sw = sidp.Solver(law="euler", p=p, nx=n, ny=n, bc=tuple(bcw), limiter="lo", gamma=G)
    if side == "W":
        sf = sidp.Solver(law="euler", p=p, nx=2 * n, ny=n, domain=(-1, 1, 0, 1), bc=("outflow",) * 4, limiter="lo", gamma=G)
    else:
        sf = sidp.Solver(law="euler", p=p, nx=n, ny=2 * n, domain=(0, 1, -1, 1), bc=("outflow",) * 4, limiter="lo", gamma=G)
    Uw = tw._initial(wall)
    sw.set_state(Uw.reshape(4, -1))
    sf.set_state(tw._mirror(Uw, p, side).reshape(4, -1))
    for _ in range(5):
        sw.step()
        sf.step()
        a = sw.get_state(0).reshape(Uw.shape)
        b = tw._restrict(sf.get_state(0).reshape(4, -1, (p + 1) ** 2), p, side)
        assert np.all(rel(b, a) <= 1e-12)


def test_wall_rejected_for_scalar_law():
    with pytest.raises(Exception):
        sidp.Solver(law="burgers", p=2, nx=2, ny=2, bc=("wall", "outflow", "outflow", "outflow"))
