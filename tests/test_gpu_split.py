"""Split boundaries (the moving two-state ghost of the double Mach reflection, Sec. 5.7) on the GPU
path against the FP64 oracle: stage times, whole steps with the device clock, the limited stage,
and a mixed-precision double Mach reflection run against the exact incident-shock path."""
import numpy as np
import pytest

from fe_compare import euler_fe_check
from oracle import laws, scheme
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu
G = 1.4
DMR_BC = ("split", "outflow", "split", "split")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def rel(a, b):
    a = a.reshape(b.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)


def make(p, nx, ny, limiter, precision="fp64", split=None):
    split = inputs.double_mach_boundaries() if split is None else split
    dom = (0.0, nx / ny, 0.0, 1.0)   # square elements, unit height
    pb = scheme.Problem(laws.Euler(G), p, nx, ny, domain=dom, bc=DMR_BC, limiter=limiter, split=split)
    sv = sidp.Solver(law="euler", p=p, nx=nx, ny=ny, domain=dom, bc=DMR_BC, limiter=limiter, gamma=G,
                     precision=precision)
    for side, sp in split.items():
        sv.set_split(side, sp["s0"], sp["speed"], sp["a"], sp["b"])
    return pb, sv


@pytest.mark.parametrize("limiter", ["lo"])
@pytest.mark.parametrize("p", [2, 3, 5])
def test_stage_times_parity(p, limiter):
    """Three explicit stages at t^n = 0.013: ghosts at t^n, t^n + dt, t^n + dt/2 (the moving top
    split crosses face nodes within the step).  The low-order operator (the unlimited high-order
    one loses positivity on this Mach 10 shock within a stage, as the paper's limiting expects)."""
    pb, sv = make(p, 12, 3, limiter)
    X, Y = pb.node_coords()
    U0 = inputs.double_mach(X, Y)
    pb.time = 0.013
    sv.set_time(0.013)
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(4, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    cur = U0
    for k in (1, 2, 3):
        expect = pb.stage(cur, U0, dt, k)
        sv.stage(k, dt)
        got = sv.get_state({1: 1, 2: 2, 3: 0}[k])
        assert np.all(rel(got, expect) <= 1e-12), (k, rel(got, expect))
        cur = expect


@pytest.mark.parametrize("t0", [0.0, 0.021])
def test_limited_stage_parity(t0):
    pb, sv = make(3, 12, 3, "subcell")
    X, Y = pb.node_coords()
    U0 = inputs.double_mach(X, Y)
    pb.time = t0
    sv.set_time(t0)
    dt = pb.compute_dt(U0)
    cur = U0
    for k in (1, 2, 3):
        ts = t0 + (0.0, 1.0, 0.5)[k - 1] * dt   # the stage time, as a stage-1 call of its own
        pb.time = pb.t_eval = ts                # (the oracle's forward-Euler operator reads t_eval)
        sv.set_time(ts)
        sv.set_state(cur.reshape(4, -1))
        sv.set_debug(True)
        sv.stage(1, dt)
        euler_fe_check(pb, cur, dt, sv.get_state(1), sv.bounds()["alpha"])
        pb.time = t0
        cur = pb.stage(cur, U0, dt, k)


def test_whole_steps_with_the_device_clock():
    """sidp_step: dt on the device at t^n, the clock advanced, the stage times from t^n."""
    pb, sv = make(2, 12, 3, "lo")
    X, Y = pb.node_coords()
    U = inputs.double_mach(X, Y)
    sv.set_state(U.reshape(4, -1))
    for _ in range(6):
        U, dt = pb.ssp_rk3_step(U)
        sv.step()
        d = sv.diag()
        assert abs(d["last_dt"] - dt) <= 1e-13 * dt
    assert abs(sv.diag()["t"] - pb.time) <= 1e-13 * pb.time
    assert np.all(rel(sv.get_state(0), U) <= 1e-11)


def test_double_mach_mixed_precision_shock_path():
    """96x24 elements, p = 3, mixed precision, to t = 0.05 with the device time step: positive
    density and pressure, and the incident shock on its exact path at the top (within an element)."""
    pb, sv = make(3, 96, 24, "subcell", precision="mixed")
    x, y = sv.node_coords()
    sv.set_state(inputs.double_mach(x, y))
    while sv.diag()["t"] < 0.05:
        sv.step(10)
    d = sv.diag()
    assert d["rho_min"] > 0 and d["p_min"] > 0 and d["nonfinite"] == 0
    u = sv.get_state(0)
    top = np.abs(y - 1.0) < 1e-12
    order = np.argsort(x[top])
    xs, rs = x[top][order], u[0][top][order]
    mid = 0.5 * (inputs.DMR_PRE[0] + inputs.DMR_POST[0])
    cross = xs[np.argmax(rs < mid)]
    assert abs(cross - inputs.dmr_shock_x(1.0, d["t"])) < 4.0 / 96


def test_split_errors():
    sv = sidp.Solver(law="euler", p=2, nx=2, ny=2, bc=("outflow",) * 4)
    with pytest.raises(sidp.SidpError):
        sv.set_split("W", 0.0, 0.0, inputs.dmr_cons(inputs.DMR_PRE))   # not a split side
    sb = sidp.Solver(law="burgers", p=2, nx=2, ny=2, bc=("split", "outflow", "outflow", "outflow"))
    with pytest.raises(sidp.SidpError):
        sb.set_split("W", 0.0, 0.0, np.array([1.0]))                    # wall part for a scalar law
    sb.set_split("W", 0.5, 1.0, np.array([1.0]), np.array([0.0]))
    with pytest.raises(Exception):
        sidp.sidp_batch_create([sidp.make_config(law="euler", p=2, nx=2, ny=2, bc=("split",) + ("outflow",) * 3)])
