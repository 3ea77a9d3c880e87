"""Pins of the whole limited scheme to numbers the paper prints, and design-order checks."""
import os

import numpy as np
import pytest

from oracle import laws, scheme
from paper_2004_08503_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "advection_convergence_si_disabled.txt")


def _table():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            p, nel, err = line.split()
            rows.append((int(p), int(nel), float(err)))
    return rows


def advection_l1(p, nel):
    """y-invariant 2D run of u_t + u_x = 0 on nel x 1 square elements, periodic, to t = 1."""
    h = 1.0 / nel
    pb = scheme.Problem(laws.Advection((1.0, 0.0)), p, nel, 1, domain=(0, 1, 0, h))
    X, Y = pb.node_coords()
    U = inputs.sine_advection(X, Y)
    nst = int(np.ceil(1.0 / pb.compute_dt(U)))
    for _ in range(nst):
        U, _ = pb.ssp_rk3_step(U, 1.0 / nst)
    return np.sum(np.abs(U[0] - np.sin(2 * np.pi * X)) * pb.mass) / h


@pytest.mark.parametrize("p,nel,err", _table())
def test_advection_table_si_disabled(p, nel, err):
    """Table tab:convergence, S.I. disabled.  The paper integrates with an 8th-order RK and an
    unstated dt; with SSP-RK3 at CFL 1/2 (Sec. 5) the oracle lands within 5% of every entry."""
    got = advection_l1(p, nel)
    assert abs(got - err) <= 0.05 * err, (p, nel, got, err)


GOLD_SI = os.path.join(os.path.dirname(__file__), "golden", "advection_convergence_si_enabled.txt")


def _table_si():
    rows = []
    for line in open(GOLD_SI):
        if line.strip() and not line.startswith("#"):
            p, nel, err, tol = line.split()
            rows.append((int(p), int(nel), float(err), float(tol)))
    return rows


@pytest.mark.parametrize("p,nel,err,tol", _table_si())
def test_advection_table_si_enabled(p, nel, err, tol):
    """Table tab:convergence, S.I. enabled (Sec. 4.4 indicator, global bounds [-1, 1] from the
    initial data).  dt = 1/4 of the CFL step removes the SSP-RK3 temporal error the paper's 8th-order
    RK avoids.  p=4 on 8 elements lands within 0.1% of the printed value."""
    h = 1.0 / nel
    pb = scheme.Problem(laws.Advection((1.0, 0.0)), p, nel, 1, domain=(0, 1, 0, h),
                        smoothness=dict(gmin=-1.0, gmax=1.0))
    X, Y = pb.node_coords()
    U = inputs.sine_advection(X, Y)
    nst = int(np.ceil(1.0 / (0.25 * pb.compute_dt(U))))
    for _ in range(nst):
        U, _ = pb.ssp_rk3_step(U, 1.0 / nst)
    got = np.sum(np.abs(U[0] - np.sin(2 * np.pi * X)) * pb.mass) / h
    assert abs(got - err) <= tol * err, (p, nel, got, err)


def test_smoothness_indicator_detects_discontinuity_and_smoothness():
    """Sec. 4.4: a smooth element gets eps = 0 (global bounds), an element with a jump eps = 1."""
    pb = scheme.Problem(laws.Advection((1.0, 0.0)), 3, 4, 4, smoothness=dict(gmin=0.0, gmax=1.0))
    X, Y = pb.node_coords()
    U = np.where(X < 0.3, 1.0, 0.0)[None] + 0.0
    eps, sK = pb.smoothness_factor(U, np.arange(pb.Ne))
    jump = np.array([(X[e].min() < 0.3) and (X[e].max() >= 0.3) for e in range(pb.Ne)])
    assert np.all(eps[jump] == 1.0) and np.all(eps[~jump] == 0.0)
    smooth = np.sin(np.pi * X)[None] * 0.5 + 0.5
    eps2, _ = pb.smoothness_factor(smooth, np.arange(pb.Ne))
    assert np.all(eps2 == 0.0)


def vortex_ho_error(p, nel):
    g = 1.4
    pb0 = scheme.Problem(laws.Euler(g), p, nel, nel)
    xi, h = pb0.xi, pb0.h
    ghost = {}
    pos = (np.arange(nel)[:, None] + xi[None, :]) * h
    ghost["W"] = inputs.vortex(0 * pos, pos, g)
    ghost["E"] = inputs.vortex(0 * pos + 1.0, pos, g)
    ghost["S"] = inputs.vortex(pos, 0 * pos, g)
    ghost["N"] = inputs.vortex(pos, 0 * pos + 1.0, g)
    pb = scheme.Problem(laws.Euler(g), p, nel, nel, bc=("exact",) * 4, ghost=ghost, limiter="none")
    X, Y = pb.node_coords()
    U0 = inputs.vortex(X, Y, g)
    U = U0.copy()
    T = 0.02
    dt0 = 0.25 * pb.compute_dt(U) * (nel / 8.0) ** (-max(0.0, (p + 1) / 3.0 - 1.0))
    nst = int(np.ceil(T / dt0))
    for _ in range(nst):
        U, _ = pb.ssp_rk3_step(U, T / nst)
    return np.sum(np.abs(U[0] - U0[0]) * pb.mass[None])


@pytest.mark.parametrize("p,n1,min_rate", [(3, 8, 3.3), pytest.param(2, 16, 2.6, marks=pytest.mark.slow)])
def test_vortex_ho_design_order(p, n1, min_rate):
    """The unlimited target scheme (Eq. dg-strong) converges at order ~p+1 on a smooth steady
    isentropic vortex with exact-state boundary data (Sec. 2; order gate on the HO scheme).
    Measured: p=3 rates 3.43 (8->16) and 3.88 (16->32); p=2: 2.14, 2.69."""
    e1, e2 = vortex_ho_error(p, n1), vortex_ho_error(p, 2 * n1)
    rate = np.log2(e1 / e2)
    assert rate > min_rate, (e1, e2, rate)
