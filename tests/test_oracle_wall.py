"""Pin of the slip-wall boundary (Sec. 5.7) by symmetry: a wall at x = 0 (or y = 0) on [0,1]^2 must
give, to rounding, the solution on [-1,1] x [0,1] (or [0,1] x [-1,1]) of the mirrored data
restricted to [0,1]^2 - the face between the mirrored halves is a plane of symmetry.

Unlimited and low-order runs agree to 1e-12 over whole steps.  With subcell limiting the entropy
roots of nodes near the entropy bound amplify rounding (the two problems sum in different orders),
so the limited stage is compared per stage from mirrored identical inputs with the
conditioning-aware check used for the GPU path.
"""
import numpy as np
import pytest

from fe_compare import euler_fe_check
from oracle import laws, scheme

G = 1.4
N_EL = 4


def _data(X, Y):
    rho = 1.0 + 0.5 * np.exp(-((X - 0.3) ** 2 + (Y - 0.55) ** 2) / 0.02) + 0.4 * (X + 0.3 * Y > 0.5)
    vx = 0.8 * np.sin(3.0 * Y + 1.0) - 0.6
    vy = 0.3 * np.cos(2.0 * X)
    p = 1.0 + 0.7 * (X > 0.6)
    return rho, vx, vy, p


def _problems(p, side, limiter):
    law = laws.Euler(G)
    n = N_EL
    bc = ["outflow"] * 4
    bc[{"W": 0, "S": 2}[side]] = "wall"
    wall = scheme.Problem(law, p, n, n, bc=tuple(bc), limiter=limiter)
    if side == "W":
        full = scheme.Problem(law, p, 2 * n, n, domain=(-1, 1, 0, 1), bc=("outflow",) * 4, limiter=limiter)
    else:
        full = scheme.Problem(law, p, n, 2 * n, domain=(0, 1, -1, 1), bc=("outflow",) * 4, limiter=limiter)
    return law, wall, full


def _mirror(Uw, p, side):
    """The state on the doubled mesh: Uw on [0,1]^2 and its mirror image (normal momentum negated)."""
    n, q = N_EL, p + 1
    nc = Uw.shape[0]
    W = Uw.reshape(nc, n, n, q, q)          # [f, ey, ex, a, b]
    M = W.copy()
    if side == "W":
        M = M[:, :, ::-1, :, ::-1].copy()
        M[1] *= -1.0
        F = np.concatenate([M, W], axis=2)  # ex: mirrored half first
    else:
        M = M[:, ::-1, :, ::-1, :].copy()
        M[2] *= -1.0
        F = np.concatenate([M, W], axis=1)
    return F.reshape(nc, -1, q * q)


def _restrict(Uf, p, side):
    n, q = N_EL, p + 1
    nc = Uf.shape[0]
    if side == "W":
        return Uf.reshape(nc, n, 2 * n, q * q)[:, :, n:].reshape(nc, -1, q * q)
    return Uf.reshape(nc, 2 * n, n, q * q)[:, n:].reshape(nc, -1, q * q)


def _initial(wall):
    X, Y = wall.node_coords()
    return wall.law.prim_to_cons(*_data(X, Y))


@pytest.mark.parametrize("limiter", ["none", "lo"])
@pytest.mark.parametrize("p,side", [(2, "W"), (3, "S"), (5, "W")])
def test_wall_equals_mirrored_problem(p, side, limiter):
    law, wall, full = _problems(p, side, limiter)
    Uw = _initial(wall)
    Uf = _mirror(Uw, p, side)
    # the mirror of the data is the data of the mirrored problem (independent construction)
    Xf, Yf = full.node_coords()
    if side == "W":
        sgn = np.sign(Xf.mean(axis=1, keepdims=True))
        rho, vx, vy, pr = _data(np.abs(Xf), Yf)
        vx = sgn * vx
    else:
        sgn = np.sign(Yf.mean(axis=1, keepdims=True))
        rho, vx, vy, pr = _data(Xf, np.abs(Yf))
        vy = sgn * vy
    np.testing.assert_allclose(Uf, law.prim_to_cons(rho, vx, vy, pr), atol=1e-14)
    for _ in range(4):
        dt = full.compute_dt(Uf)
        assert wall.compute_dt(Uw) == pytest.approx(dt, rel=1e-13)
        Uf, _ = full.ssp_rk3_step(Uf, dt)
        Uw, _ = wall.ssp_rk3_step(Uw, dt)
        scale = np.max(np.abs(Uw), axis=(1, 2))
        err = np.max(np.abs(_restrict(Uf, p, side) - Uw), axis=(1, 2)) / scale
        assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("p,side", [(2, "W"), (3, "S"), (4, "W")])
def test_wall_limited_stage_equals_mirrored_problem(p, side):
    law, wall, full = _problems(p, side, "subcell")
    Uw = _initial(wall)
    dt = full.compute_dt(_mirror(Uw, p, side))
    U0 = Uw
    for k in (1, 2, 3):
        fe_full, info = full.fe_stage(_mirror(Uw, p, side), dt, full=True)
        alpha = _restrict(info["alpha_tilde"][None], p, side)[0]
        euler_fe_check(wall, Uw, dt, _restrict(fe_full, p, side), alpha)
        Uw = wall.stage(Uw, U0, dt, k)


def test_wall_rejects_scalar_laws():
    with pytest.raises(ValueError):
        scheme.Problem(laws.Burgers(), 2, 2, 2, bc=("wall", "outflow", "outflow", "outflow"))


@pytest.mark.parametrize("p,bc", [(2, ("wall", "outflow", "wall", "outflow")), (5, ("wall",) * 4),
                                  (3, ("outflow",) * 4)])
def test_euler_comparator_accepts_oracle_under_input_noise(p, bc):
    """The conditioning-aware Euler check must accept the oracle against itself under one-ulp
    input noise: entropy roots near the entropy bound, and Zalesak's density ratio on the density
    plateau of this data (lo = u^L exactly, noise-level density fluxes, genuine momentum fluxes),
    move under rounding by far more than 1e-12."""
    law = laws.Euler(G)
    pb = scheme.Problem(law, p, 5, 3, domain=(0.0, 1.0, 0.0, 0.6), bc=bc)
    X, Y = pb.node_coords()
    U = law.prim_to_cons(*_data(X, Y))
    dt = pb.compute_dt(U)
    base = pb.fe_stage(U, dt)
    worst = 0.0
    for seed in range(6):
        rng = np.random.default_rng(seed)
        noisy = U * (1 + 2.2e-16 * rng.standard_normal(U.shape))
        got, info = pb.fe_stage(noisy, dt, full=True)
        worst = max(worst, float(np.max(np.abs(got - base) / np.max(np.abs(base), axis=(1, 2))[:, None, None])))
        euler_fe_check(pb, U, dt, got, info["alpha_tilde"])
    assert worst > 1e-12   # the sensitivity is real
