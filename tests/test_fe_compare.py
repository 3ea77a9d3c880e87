"""The conditioning-aware comparators of tests/fe_compare.py must reject an over-limiting candidate.

Sec. 4.1.3 and Sec. 4.2 define alpha-tilde as the largest admissible coefficient.  The comparators
relax the strict 1e-12 match at ill-conditioned nodes; these tests plant, on the CPU, a candidate
that sets alpha = 0 (or scales alpha down) exactly where the strict match is relaxed, builds its
update with the oracle's own arithmetic, and check that the comparator rejects it while it accepts
the unmodified oracle.  The planted candidates are consistent (their state is the update of their
coefficients), admissible and inside the bounds, so only the maximality test can catch them at
the relaxed nodes.
"""
import numpy as np
import pytest

import fe_compare
from oracle import laws, scheme
from paper_2004_08503_gb300 import inputs

G = 1.4


def _euler_case(p):
    law = laws.Euler(G)
    pb = scheme.Problem(law, p, 5, 3, domain=(0.0, 1.0, 0.0, 0.6), bc=("outflow",) * 4)
    X, Y = pb.node_coords()
    rho = 1.0 + 0.5 * np.exp(-((X - 0.3) ** 2 + (Y - 0.55) ** 2) / 0.02) + 0.4 * (X + 0.3 * Y > 0.5)
    vx = 0.8 * np.sin(3.0 * Y + 1.0) - 0.6
    vy = 0.3 * np.cos(2.0 * X)
    pr = 1.0 + 0.7 * (X > 0.6)
    U = law.prim_to_cons(rho, vx, vy, pr)
    return pb, U


def _ill_conditioned_euler(pb, info, dt):
    """The ill-conditioned nodes themselves (the comparator also relaxes their face neighbours,
    so changing alpha here changes no strictly checked node)."""
    uL, K = info["uL"], info["K"]
    rhoe = pb.law.pressure(uL) / (pb.law.gamma - 1.0)
    ic = pb.law.psi(uL, K) < 1e-6 * rhoe
    return ic | fe_compare.zalesak_ill_conditioned(pb, info, dt)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_euler_comparator_rejects_zero_alpha_at_relaxed_nodes(p):
    pb, U = _euler_case(p)
    dt = pb.compute_dt(U)
    exp, info = pb.fe_stage(U, dt, full=True)
    fe_compare.euler_fe_check(pb, U, dt, exp, info["alpha_tilde"])  # the oracle itself passes
    bad = _ill_conditioned_euler(pb, info, dt)
    at = info["alpha_tilde"]
    assert np.any(bad & (at > 0.1)), "no relaxed node with room for antidiffusion in this data"
    planted = np.where(bad, 0.0, at)
    got = fe_compare.apply_alpha(pb, info, dt, planted)
    with pytest.raises(AssertionError, match="not maximal"):
        fe_compare.euler_fe_check(pb, U, dt, got, planted)


@pytest.mark.parametrize("p", [2, 4])
def test_euler_comparator_rejects_uniformly_scaled_alpha(p):
    """alpha scaled by 0.99 everywhere: admissible, consistent, 1% short of maximal."""
    pb, U = _euler_case(p)
    dt = pb.compute_dt(U)
    exp, info = pb.fe_stage(U, dt, full=True)
    planted = 0.99 * info["alpha_tilde"]
    got = fe_compare.apply_alpha(pb, info, dt, planted)
    with pytest.raises(AssertionError):
        fe_compare.euler_fe_check(pb, U, dt, got, planted)


def test_euler_comparator_rejects_inconsistent_state():
    """A state that is not the update of the coefficients it reports."""
    pb, U = _euler_case(3)
    dt = pb.compute_dt(U)
    exp, info = pb.fe_stage(U, dt, full=True)
    bad = fe_compare.spread_faces(_ill_conditioned_euler(pb, info, dt), pb.n)
    got = exp.copy()
    i = np.argwhere(bad)[0]
    got[1, i[0], i[1]] += 1e-9 * np.max(np.abs(exp[1]))  # inside the old validity slack
    with pytest.raises(AssertionError):
        fe_compare.euler_fe_check(pb, U, dt, got, info["alpha_tilde"])


@pytest.mark.parametrize("p", [3, 5])
def test_scalar_comparator_zero_over_zero_and_over_limiting(p):
    """The solid body data with the Sec. 4.4 relaxed bounds.  Every relaxed node of this scalar
    data sits on its bound with antidiffusive fluxes of that sign at rounding level: Zalesak's
    ratio is a 0/0 there and any alpha in [0, 1] is a correct result (the oracle under one-ulp
    input noise produces both 0 and 1), so alpha = 0 there is accepted.  A candidate that
    over-limits where the bounds leave room (alpha scaled by 0.9) is rejected."""
    si = dict(gmin=0.0, gmax=1.0)
    pb = scheme.Problem(laws.AdvectionVar(*inputs.SOLID_BODY_VELOCITY), p, 7, 6, domain=(0, 1, 0, 6 / 7),
                        bc=("outflow",) * 4, smoothness=si)
    X, Y = pb.node_coords()
    U = inputs.solid_body(X, Y)
    dt = pb.compute_dt(U)
    exp, info = pb.fe_stage(U, dt, full=True)
    fe_compare.scalar_fe_check(pb, U, dt, exp, info["alpha_tilde"])
    bad = fe_compare.zalesak_ill_conditioned(pb, info, dt)
    at = info["alpha_tilde"]
    uL = info["uL"][0]
    on_bound = np.minimum(info["hi"] - uL, uL - info["lo"]) <= 1e-9 * np.max(np.abs(uL))
    assert np.all(on_bound[bad])
    planted = np.where(bad, 0.0, at)
    fe_compare.scalar_fe_check(pb, U, dt, fe_compare.apply_alpha(pb, info, dt, planted), planted)
    room = ~on_bound & (at > 0.1)
    assert np.any(room)
    planted = np.where(room, 0.9 * at, at)
    with pytest.raises(AssertionError):
        fe_compare.scalar_fe_check(pb, U, dt, fe_compare.apply_alpha(pb, info, dt, planted), planted)


@pytest.mark.parametrize("lawname,p", [("burgers", 3), ("euler", 3)])
def test_elementwise_comparator_rejects_zero_alpha(lawname, p):
    law = laws.Burgers() if lawname == "burgers" else laws.Euler(G)
    pb = scheme.Problem(law, p, 4, 3, domain=(0, 1, 0, 0.75), limiter="elementwise", bc=("outflow",) * 4)
    X, Y = pb.node_coords()
    U = (1.0 + inputs.sine_advection(X, Y)) if lawname == "burgers" else inputs.four_quadrant(X, Y, p)
    if lawname == "euler":
        U, _ = scheme.Problem(law, p, 4, 3, domain=(0, 1, 0, 0.75), bc=("outflow",) * 4).ssp_rk3_step(U)
    dt = pb.compute_dt(U)
    exp, info = pb.fe_stage(U, dt, full=True)
    fe_compare.elementwise_fe_check(pb, U, dt, exp, info["alpha_tilde"])
    at = info["alpha_tilde"]
    e = int(np.argmax(info["alpha_K"]))  # the element with the most room
    assert info["alpha_K"][e] > 0.01
    planted = at.copy()
    planted[e] = 0.0
    m = pb._mass(None)
    got = info["uL"] + dt / m[None] * np.min(planted, axis=1)[None, :, None] * info["rn"]
    with pytest.raises(AssertionError):
        fe_compare.elementwise_fe_check(pb, U, dt, got, planted)
