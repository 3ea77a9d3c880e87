"""Pins of the oracle's split boundary (the moving two-state ghost of the double Mach reflection,
Sec. 5.7) against the exact-state and slip-wall boundaries, against hand-built ghost states at the
SSP-RK3 stage times, and against the exact incident-shock path."""
import numpy as np
import pytest

from oracle import laws, scheme
from paper_2004_08503_gb300 import inputs

G = 1.4


def test_double_mach_data_satisfy_rankine_hugoniot():
    """Sec. 5.7 data: a Mach 10 shock (speed 10 along its normal into gas at rest with sound speed
    1) with the printed post-shock state conserves mass, normal momentum and energy across it."""
    law = laws.Euler(G)
    pre, post = inputs.dmr_cons(inputs.DMR_PRE), inputs.dmr_cons(inputs.DMR_POST)
    nrm = np.array([np.cos(np.pi / 6), -np.sin(np.pi / 6)])   # shock normal, pointing downstream
    S = 10.0
    assert np.sqrt(G * inputs.DMR_PRE[3] / inputs.DMR_PRE[0]) == pytest.approx(1.0)
    Fx0, Fy0 = law.flux(pre[:, None])
    Fx1, Fy1 = law.flux(post[:, None])
    Fn0 = Fx0[:, 0] * nrm[0] + Fy0[:, 0] * nrm[1]
    Fn1 = Fx1[:, 0] * nrm[0] + Fy1[:, 0] * nrm[1]
    np.testing.assert_allclose(Fn1 - Fn0, S * (post - pre), rtol=2e-3, atol=1e-9)
    # the tangential velocity of the post-shock state is zero (the normal shock moves at S)
    v = np.array(inputs.DMR_POST[1:3])
    assert abs(v @ np.array([np.sin(np.pi / 6), np.cos(np.pi / 6)])) < 1e-12


def _euler_data(pb, seed=2):
    X, Y = pb.node_coords()
    return inputs.four_quadrant(X, Y, seed)


@pytest.mark.parametrize("side", ["W", "S", "N"])
def test_constant_split_equals_exact_state(side):
    law = laws.Euler(G)
    c = inputs.dmr_cons((0.9, 0.3, -0.2, 0.7))
    bc = ["outflow"] * 4
    bc[scheme.SIDES.index(side)] = "split"
    ps = scheme.Problem(law, 3, 4, 3, domain=(0, 1, 0, 0.75), bc=tuple(bc),
                        split={side: dict(s0=0.4, speed=2.0, a=c, b=c)})
    bc[scheme.SIDES.index(side)] = "exact"
    nside = 3 if side in ("W", "E") else 4
    ghost = {side: np.broadcast_to(c[:, None, None], (4, nside, 4)).copy()}
    pe = scheme.Problem(law, 3, 4, 3, domain=(0, 1, 0, 0.75), bc=tuple(bc), ghost=ghost)
    U = _euler_data(ps)
    U1, dt1 = ps.ssp_rk3_step(U)
    U2, dt2 = pe.ssp_rk3_step(U)
    assert dt1 == dt2
    np.testing.assert_array_equal(U1, U2)


def test_split_with_wall_part_equals_wall():
    law = laws.Euler(G)
    c = inputs.dmr_cons((0.9, 0.3, -0.2, 0.7))
    ps = scheme.Problem(law, 2, 4, 3, domain=(0, 1, 0, 0.75), bc=("outflow", "outflow", "split", "outflow"),
                        split={"S": dict(s0=-1e30, speed=0.0, a=c, b=None)})
    pw = scheme.Problem(law, 2, 4, 3, domain=(0, 1, 0, 0.75), bc=("outflow", "outflow", "wall", "outflow"))
    U = _euler_data(ps)
    np.testing.assert_array_equal(ps.ssp_rk3_step(U)[0], pw.ssp_rk3_step(U)[0])


@pytest.mark.parametrize("side", ["N", "W"])
def test_moving_split_uses_the_stage_times(side):
    """The ghost of stage k is the split state at t^n + (0, 1, 1/2)[k-1] dt: three forward-Euler
    stages with hand-built exact-state ghosts at those times reproduce the step (the coordinate
    along the side is x on S/N sides and y on W/E sides)."""
    law = laws.Euler(G)
    a, b = inputs.dmr_cons((1.2, 0.1, 0.0, 1.5)), inputs.dmr_cons((0.6, -0.2, 0.1, 0.4))
    p, nx, ny = 3, 5, 3
    dom = (0, 1, 0.1, 0.7)
    sp = dict(s0=0.2, speed=15.0, a=a, b=b)
    bc = ["outflow"] * 4
    bc[scheme.SIDES.index(side)] = "split"
    ps = scheme.Problem(law, p, nx, ny, domain=dom, bc=tuple(bc), split={side: sp})
    U0 = _euler_data(ps)
    ps.time = 0.01
    dt = ps.compute_dt(U0)
    ne, lo = (nx, ps.x0) if side == "N" else (ny, ps.y0)
    C = lo + ps.h * (np.arange(ne)[:, None] + ps.xi[None, :])   # along-side coordinate of the face nodes
    # put the split half a step's travel before a face node: it crosses the node between stages
    sp["s0"] = C[1, 1] - sp["speed"] * (0.01 + 0.5 * dt)
    U1, _ = ps.ssp_rk3_step(U0, dt)
    assert ps.time == pytest.approx(0.01 + dt)

    def ghost_at(t):
        below = C < sp["s0"] + sp["speed"] * t
        return {side: np.where(below[None], a[:, None, None], b[:, None, None])}

    bc[scheme.SIDES.index(side)] = "exact"
    cur = U0
    for k, c in ((1, 0.0), (2, 1.0), (3, 0.5)):
        pe = scheme.Problem(law, p, nx, ny, domain=dom, bc=tuple(bc), ghost=ghost_at(0.01 + c * dt))
        cur = pe.stage(cur, U0, dt, k)
    np.testing.assert_array_equal(U1, cur)
    # the split point crosses a face node during the step (the test exercises the time)
    assert np.any(ghost_at(0.01)[side] != ghost_at(0.01 + dt)[side])


def test_double_mach_incident_shock_moves_at_its_exact_speed():
    """Coarse double Mach reflection (Sec. 5.7 boundaries and data), p = 2, to t = 0.02: the
    incident shock along the top of the domain stays at x = 1/6 + (1 + 20 t)/sqrt(3) (to within an
    element), and density and pressure stay positive."""
    law = laws.Euler(G)
    pb = scheme.Problem(law, 2, 24, 6, domain=(0, 4, 0, 1), bc=("split", "outflow", "split", "split"),
                        split=inputs.double_mach_boundaries())
    X, Y = pb.node_coords()
    U = inputs.double_mach(X, Y)
    while pb.time < 0.02 - 1e-12:
        U, _ = pb.ssp_rk3_step(U, min(pb.compute_dt(U), 0.02 - pb.time))
    assert U[0].min() > 0 and law.pressure(U).min() > 0
    top = np.abs(Y - 1.0) < 1e-12
    xs, rs = X[top], U[0][top]
    order = np.argsort(xs)
    xs, rs = xs[order], rs[order]
    mid = 0.5 * (inputs.DMR_PRE[0] + inputs.DMR_POST[0])
    cross = xs[np.argmax(rs < mid)]   # first node below the mid density, from the left
    assert abs(cross - inputs.dmr_shock_x(1.0, pb.time)) < pb.h
