"""Pins of the oracle's variable-velocity advection (Sec. 3.3, solid body rotation of Sec. 5.4).

The velocity class is beta = (bx0 + bxy y, by0 + byx x): divergence-free, and beta.n continuous
across every face of a Cartesian mesh.  None of these tests re-types the oracle's formulas: they
check it against the constant-velocity path (an independent code path), against exact
differentiation of polynomials, against invariants (free stream, conservation, convex
combination of bar states, discrete maximum principle) and against the exact rotated solution.
"""
import os

import numpy as np
import pytest

from oracle import laws, scheme
from paper_2004_08503_gb300 import inputs

ROT = inputs.SOLID_BODY_VELOCITY


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("limiter", ["none", "lo", "subcell"])
def test_constant_velocity_matches_constant_advection(p, limiter):
    """bxy = byx = 0 must reduce every residual, bar state, dt and limited update to the
    constant-beta law (Sec. 3.3 coefficients reduce to Eq. dij)."""
    beta = (0.7, -0.4)
    kw = dict(domain=(0, 1, 0, 0.75), limiter=limiter)
    pa = scheme.Problem(laws.Advection(beta), p, 4, 3, **kw)
    pv = scheme.Problem(laws.AdvectionVar(beta[0], 0.0, beta[1], 0.0), p, 4, 3, **kw)
    X, Y = pa.node_coords()
    U = (np.sin(2 * np.pi * X) + (X > 0.5) + 0.3 * np.cos(4 * np.pi * Y))[None]
    assert pa.compute_dt(U) == pytest.approx(pv.compute_dt(U), rel=1e-14)
    np.testing.assert_allclose(pv.ho_residual(U), pa.ho_residual(U), atol=1e-13)
    ra, ba, da, fa = pa.lo_residual(U, want_bars=True)
    rv, bv, dv, fv = pv.lo_residual(U, want_bars=True)
    np.testing.assert_allclose(rv, ra, atol=1e-13)
    np.testing.assert_allclose(dv, da, atol=1e-14)
    np.testing.assert_allclose(bv["pairs"], ba["pairs"], atol=1e-13)
    dt = pa.compute_dt(U)
    np.testing.assert_allclose(pv.fe_stage(U, dt), pa.fe_stage(U, dt), atol=1e-13)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_free_stream_rotation(p):
    """A constant state is steady: the discrete divergence sum_j c-hat_ij . beta_j vanishes
    because x-pairs share y (and beta_x) and y-pairs share x (and beta_y)."""
    pb = scheme.Problem(laws.AdvectionVar(*ROT), p, 3, 4, domain=(0, 0.75, 0, 1), bc=("outflow",) * 4)
    U = np.full((1, pb.Ne, pb.n ** 2), 0.6)
    assert np.abs(pb.ho_residual(U)).max() < 1e-12
    assert np.abs(pb.lo_residual(U)).max() < 1e-12


@pytest.mark.parametrize("p", [1, 3, 6])
def test_conservation_periodic(p):
    """Prop. (conservation) for Eq. dg-strong and Eq. dg-idp with variable velocity: beta_x
    depends on y only and beta_y on x only, so the periodic faces carry equal normal fluxes."""
    rng = np.random.default_rng(p)
    pb = scheme.Problem(laws.AdvectionVar(0.3, 1.7, -0.2, -1.1), p, 3, 4, domain=(0, 0.75, 0, 1))
    U = rng.uniform(-1, 2, (1, pb.Ne, pb.n ** 2))
    for r in (pb.ho_residual(U), pb.lo_residual(U)):
        tot = r.sum(axis=(0, 2, 3))
        assert np.all(np.abs(tot) <= 1e-14 * np.abs(r).sum(axis=(0, 2, 3)))


@pytest.mark.parametrize("p", [2, 3, 5])
def test_ho_exact_on_polynomials(p):
    """Strong form Eq. dg-strong: for u of degree p-1 and affine beta, beta u has degree p and
    r^H_i = -m_i beta(x_i) . grad u(x_i) exactly (div beta = 0); with outflow ghosts equal to
    the trace and continuous u, no face term remains."""
    bx0, bxy, by0, byx = 0.4, -1.3, 0.9, 2.1
    pb = scheme.Problem(laws.AdvectionVar(bx0, bxy, by0, byx), p, 3, 2, domain=(-0.3, 1.2, 0.1, 1.1),
                        bc=("outflow",) * 4)
    X, Y = pb.node_coords()
    q = p - 1
    rng = np.random.default_rng(11 + p)
    C = rng.uniform(-1, 1, (q + 1, q + 1))
    C[np.add.outer(np.arange(q + 1), np.arange(q + 1)) > q] = 0.0   # total degree <= p-1
    u = np.polynomial.polynomial.polyval2d(X, Y, C)
    ux = np.polynomial.polynomial.polyval2d(X, Y, np.polynomial.polynomial.polyder(C, axis=0))
    uy = np.polynomial.polynomial.polyval2d(X, Y, np.polynomial.polynomial.polyder(C, axis=1))
    expect = -pb.mass[None] * ((bx0 + bxy * Y) * ux + (by0 + byx * X) * uy)
    r = pb.ho_residual(u[None])
    np.testing.assert_allclose((r[0] + r[1])[0], expect, atol=1e-12 * np.abs(expect).max())


def test_lo_convex_combination_and_bar_state_bounds():
    """Eq. convex-combination with the Sec. 3.3 coefficients: u^L is a convex combination of
    u_i and bar states, and each bar state of linear advection lies between u_i and u_j."""
    rng = np.random.default_rng(5)
    pb = scheme.Problem(laws.AdvectionVar(*ROT), 3, 3, 3, bc=("outflow",) * 4)
    U = rng.uniform(-1, 2, (1, pb.Ne, 16))
    dt = pb.compute_dt(U)
    rL, bars, dij, dface = pb.lo_residual(U, want_bars=True)
    uL = U + dt / pb.mass * (rL[0] + rL[1])
    ui, uj = U[:, :, pb.pI], U[:, :, pb.pJ]
    tol = 1e-13
    assert np.all(bars["pairs"] >= np.minimum(ui, uj) - tol)
    assert np.all(bars["pairs"] <= np.maximum(ui, uj) + tol)
    acc = np.zeros_like(U)
    wsum = np.zeros(U.shape[1:])
    wgt = 2 * dt * dij / pb.mass[pb.pI]
    np.add.at(acc, (slice(None), slice(None), pb.pI), wgt[None] * bars["pairs"])
    np.add.at(wsum, (slice(None), pb.pI), wgt)
    for s in scheme.SIDES:
        idx = pb.fnodes[s]
        wf = 2 * dt * dface[s] / pb.mass[idx]
        acc[:, :, idx] += wf[None] * bars["faces"][s]
        wsum[:, idx] += wf
    assert wsum.max() <= pb.cfl * (1 + 1e-12)
    np.testing.assert_allclose(uL, (1 - wsum)[None] * U + acc, atol=1e-13, rtol=1e-12)


def _rotate_back(X, Y, t):
    """Foot of the characteristic of the solid body rotation (angular speed 2 pi about (1/2,1/2))."""
    c, s = np.cos(2 * np.pi * t), np.sin(2 * np.pi * t)
    dx, dy = X - 0.5, Y - 0.5
    return 0.5 + c * dx + s * dy, 0.5 - s * dx + c * dy


def _rotation_error(ne, p, T, limiter):
    pb = scheme.Problem(laws.AdvectionVar(*ROT), p, ne, ne, bc=("outflow",) * 4, limiter=limiter)
    X, Y = pb.node_coords()
    U = inputs.smooth_bump(X, Y)
    dt0 = pb.compute_dt(U)
    nsteps = int(np.ceil(T / dt0))
    for _ in range(nsteps):
        U, _ = pb.ssp_rk3_step(U, T / nsteps)
    Xb, Yb = _rotate_back(X, Y, T)
    ex = inputs.smooth_bump(Xb, Yb)
    return float(np.sum(pb.mass[None] * np.abs(U - ex))), U


def test_rotation_ho_converges_to_exact_rotation():
    """The unlimited DG-SEM solution of the rotated C^5 bump converges to the exactly rotated
    bump at high order (p = 3: order about 3.5 between 8x8 and 16x16 elements, still
    pre-asymptotic toward p + 1; a dropped face or volume term stalls it at O(1) or O(h))."""
    T = 0.05
    e8, _ = _rotation_error(8, 3, T, "none")
    e16, _ = _rotation_error(16, 3, T, "none")
    assert e16 < 2.5e-4
    assert np.log2(e8 / e16) > 3.2


def test_rotation_limited_maximum_principle_and_accuracy():
    """Subcell limiting (Sec. 4.1) keeps the rotated bump inside [0, 1] (global DMP) and stays
    close to the HO accuracy on a smooth profile."""
    T = 0.05
    eH, _ = _rotation_error(8, 3, T, "none")
    eS, U = _rotation_error(8, 3, T, "subcell")
    assert U.min() >= -1e-14 and U.max() <= 1 + 1e-14
    assert eS < 3 * eH


def _golden_rows(ne):
    path = os.path.join(os.path.dirname(__file__), "golden", "solid_body_rotation.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            if int(f[0]) == ne:
                rows.append((f[1], int(f[2]), float(f[3]), float(f[4]), float(f[5]), float(f[6]), float(f[7])))
    return rows


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("SIDP_LONG_ORACLE"), reason="about 4 minutes per case: set SIDP_LONG_ORACLE=1")
@pytest.mark.parametrize("limiter,si,lo,hi,l1,tol,rtol", _golden_rows(25))
def test_solid_body_25_p3_matches_paper(limiter, si, lo, hi, l1, tol, rtol):
    """Sec. 5.4 / Sec. 4.4 on 25x25 elements, p = 3, one revolution at half of the CFL bound:
    the oracle's extrema and L1 error against the paper's printed values."""
    smooth = dict(gmin=0.0, gmax=1.0) if si else None
    pb = scheme.Problem(laws.AdvectionVar(*ROT), 3, 25, 25, bc=("outflow",) * 4, limiter=limiter,
                        smoothness=smooth)
    X, Y = pb.node_coords()
    U0 = inputs.solid_body(X, Y)
    nsteps = int(np.ceil(1.0 / pb.compute_dt(U0)))
    U = U0
    for _ in range(nsteps):
        U, _ = pb.ssp_rk3_step(U, 1.0 / nsteps)
    err = float(np.sum(pb.mass[None] * np.abs(U - U0)))
    assert abs(U.min() - lo) <= tol and abs(U.max() - hi) <= tol, (U.min(), U.max())
    assert U.min() >= -1e-12 and U.max() <= 1 + 1e-12
    assert abs(err / l1 - 1) <= rtol, err


@pytest.mark.parametrize("p", [3, 5])
def test_zalesak_zero_over_zero_comparator_on_oracle_noise(p):
    """The limited stage with the Sec. 4.4 relaxed bounds is ill-conditioned where Zalesak's
    R = min(1, Q/P) is a rounding-level 0/0 (a state on its bound, noise-level antidiffusion of
    that sign): the oracle against itself under one-ulp input noise differs there by far more
    than rounding.  The GPU parity comparator must accept every such noisy oracle result.  (On
    this plateau-heavy data about a quarter of the nodes touch an ill-conditioned node; those are
    still held to the bounds and to the size of their antidiffusive correction.)"""
    import fe_compare
    si = dict(gmin=0.0, gmax=1.0)
    pb = scheme.Problem(laws.AdvectionVar(*ROT), p, 7, 6, domain=(0, 1, 0, 6 / 7), bc=("outflow",) * 4,
                        smoothness=si)
    X, Y = pb.node_coords()
    U0 = inputs.solid_body(X, Y)
    dt = pb.compute_dt(U0)
    cur = U0
    worst, frac = 0.0, 0.0
    for k in (1, 2, 3):
        base = pb.fe_stage(cur, dt)
        for seed in range(8):
            rng = np.random.default_rng(100 * k + seed)
            noisy = cur * (1 + 2.2e-16 * rng.standard_normal(cur.shape))
            got, info = pb.fe_stage(noisy, dt, full=True)
            worst = max(worst, float(np.abs(got - base).max()))
            frac = max(frac, fe_compare.scalar_fe_check(pb, cur, dt, got, info["alpha_tilde"], tol=1e-12))
        cur = pb.stage(cur, U0, dt, k)
    assert worst > 1e-8          # the sensitivity is real (strict parity cannot hold here)
    assert frac < 0.35
