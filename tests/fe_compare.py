"""Comparison of a forward-Euler limited stage with the oracle's where Zalesak's ratio is 0/0.

Sec. 4.1.3 limits node i by alpha_i = min(R+, R-), R+- = min(1, Q+-/P+-).  Where the low-order
state sits on its bound (Q = 0 up to rounding) and the antidiffusive fluxes of that sign are
rounding noise (P = 0 up to rounding), R is a 0/0 that rounding decides anywhere in [0, 1]: one
ulp of input moves it.  alpha_i also limits the node's fluxes of the other sign and, through the
face minimum, its neighbours' - genuine fluxes - so two correct evaluations of the method may
differ there by much more than rounding (the oracle against itself under one-ulp input noise
shows it).  Both results are valid: every candidate stays inside the bounds.

The check: nodes where that rounding moves the update by more than `tol` (a binding ratio whose
P is small beside the node's other fluxes, or a rounding-level 0/0), together with their
subcell-face neighbours, must lie inside the (relaxed) bounds and differ from the oracle by
no more than the node's full antidiffusive correction dt/m sum |r-bar|; every other node must
match to `tol` (normwise).
"""
import numpy as np


def zalesak_ill_conditioned(pb, info, dt, tol=1e-12, kappa=64.0, tau=1e-10, elems=None):
    """Nodes (Ne, n*n) whose limited update the rounding of the Zalesak ratio moves by more
    than `tol` in some field (relative to that field's max |u|).

    The ratio limits the limited field (the scalar, or rho).  Rounding perturbs Q = m/dt (bound -
    u^L) by about kappa ulp m/dt max|u|, so a ratio R = Q/P that binds (R < 1) moves by about that
    over P; a rounding-level 0/0 (Q and P of one sign below the noise floor tau m/dt max|u|) may
    take any value in [0, 1].  Through alpha_i the change reaches every flux the node governs, in
    every field: at most dt/m sum_faces |r-bar_q| per unit of alpha."""
    ulp = np.finfo(float).eps
    xp, xm, yp, ym = pb._node_face_fluxes(info["rbar"])
    c = np.stack([xp[0], -xm[0], yp[0], -ym[0]])
    Pp = np.sum(np.maximum(c, 0.0), axis=0)
    Pm = -np.sum(np.minimum(c, 0.0), axis=0)
    uL = info["uL"]
    s0 = max(np.max(np.abs(uL[0])), 1e-300)
    m = pb._mass(elems)
    eta = tau * m / dt * s0
    Qp = m / dt * np.maximum(info["hi"] - uL[0], 0.0)
    Qm = m / dt * np.maximum(uL[0] - info["lo"], 0.0)
    fsc = np.maximum(np.max(np.abs(uL), axis=(1, 2)), 1e-300)[:, None, None]
    impact = np.max(dt / m[None] * (np.abs(xp) + np.abs(xm) + np.abs(yp) + np.abs(ym)) / fsc, axis=0)
    flag = np.zeros(Pp.shape, bool)
    for P, Q in ((Pp, Qp), (Pm, Qm)):
        zero_zero = (P <= eta) & (Q <= eta)
        binding = (P > eta) & (Q < P * (1 + 1e-8))
        dR = kappa * ulp * (m / dt) * s0 / np.where(P > 0, P, np.inf)
        flag |= zero_zero & (impact > tol)
        flag |= binding & (dR * impact > tol)
    return flag


def spread_faces(flag, n):
    A = flag.reshape(-1, n, n)
    out = A.copy()
    out[:, :, 1:] |= A[:, :, :-1]
    out[:, :, :-1] |= A[:, :, 1:]
    out[:, 1:, :] |= A[:, :-1, :]
    out[:, :-1, :] |= A[:, 1:, :]
    return out.reshape(flag.shape)


def scalar_fe_check(pb, U, dt, got, tol=1e-12, tau=1e-10):
    """Compare a scalar forward-Euler limited stage `got` (any shape of nc*N values) with the
    oracle's from the same input U.  Returns the fraction of nodes checked by validity."""
    exp, info = pb.fe_stage(U, dt, full=True)
    got = np.asarray(got).reshape(exp.shape)
    scale = max(np.max(np.abs(exp)), 1e-300)
    bad = spread_faces(zalesak_ill_conditioned(pb, info, dt, tol=tol, tau=tau), pb.n)
    err = np.abs(got - exp)[0] / scale
    assert np.all(err[~bad] <= tol), np.max(err[~bad])
    xp, xm, yp, ym = pb._node_face_fluxes(info["rbar"])
    corr = dt / pb._mass(None) * (np.abs(xp) + np.abs(xm) + np.abs(yp) + np.abs(ym))[0] / scale
    assert np.all(err[bad] <= corr[bad] + tol)
    g = got[0]
    slack = tol * scale
    assert np.all(g[bad] >= info["lo"][bad] - slack) and np.all(g[bad] <= info["hi"][bad] + slack)
    return float(bad.mean())


def elementwise_fe_check(pb, U, dt, got, tol=1e-12, ulp=None, kappa=64.0, tau=1e-6, eta_rel=1e-10):
    """Elementwise limiting (Sec. 4.1.2, 4.2.1): compare `got` with the oracle's stage from U.

    alpha_K = min over the element of alpha-tilde_i.  Rounding moves alpha-tilde_i of a binding
    Zalesak ratio Q/|r_i| by about kappa ulp (m/dt) max|u| / |r_i|; a rounding-level 0/0 (node on
    its bound, noise-level r_i) may take any value in [0, 1]; for Euler a node whose psi_K(u^L) is
    below tau rho e has an entropy root that rounding can move anywhere below its density value.
    The interval of alpha_K follows; each node may then differ by (its width) |dt/m r_i| plus
    tol max|u|, and must stay inside the bounds (and sigma >= K for Euler)."""
    ulp = np.finfo(float).eps if ulp is None else ulp
    exp, info = pb.fe_stage(U, dt, full=True)
    got = np.asarray(got).reshape(exp.shape)
    at, aK, rn, uL = info["alpha_tilde"], info["alpha_K"], info["rn"], info["uL"]
    m = pb._mass(None)
    scale = max(np.max(np.abs(exp)), 1e-300)
    s0 = max(np.max(np.abs(uL[0])), 1e-300)
    r0 = np.abs(rn[0])
    delta = kappa * ulp * (m / dt) * s0 / np.where(r0 > 0, r0, np.inf)
    eta = eta_rel * (m / dt) * s0
    Qp = m / dt * np.maximum(info["hi"] - uL[0], 0.0)
    Qm = m / dt * np.maximum(uL[0] - info["lo"], 0.0)
    zero_zero = (r0 <= eta) & (np.minimum(Qp, Qm) <= eta)
    lo_i = np.where(zero_zero, 0.0, at - delta)
    hi_i = np.where(zero_zero, 1.0, at + delta)
    if pb.law.name == "euler":
        rhoe = pb.law.pressure(uL) / (pb.law.gamma - 1.0)
        ill = pb.law.psi(uL, info["K"]) < tau * rhoe
        lo_i = np.where(ill, 0.0, lo_i)
        hi_i = np.where(ill, 1.0, hi_i)
    width = np.clip(np.min(hi_i, axis=1), 0, 1) - np.clip(np.min(lo_i, axis=1), 0, 1)
    w = dt / m[None] * np.abs(rn)
    allowed = width[None, :, None] * w + tol * scale
    err = np.abs(got - exp)
    assert np.all(err <= allowed), np.max(err - allowed)
    slack = 10 * tol * scale
    assert np.all(got[0] >= info["lo"] - slack) and np.all(got[0] <= info["hi"] + slack)
    if pb.law.name == "euler":
        assert np.all(pb.law.sigma(got) >= info["K"] * (1 - 10 * tol))
    return float(np.mean(width > 0))


def euler_fe_check(pb, U, dt, got, tol=1e-12, tau=1e-6, elems=None):
    """Compare a GPU forward-Euler stage with the oracle's on the entropy-limited Euler path.

    The entropy coefficient of node i is the root t* of psi_K(u^L + t w) = min(0, psi_K(u^L)),
    psi_K concave.  Concavity gives |psi'(t*)| >= psi_0 / t* with psi_0 = psi_K(u^L), so a
    rounding-level change delta of psi moves the root by at most t* delta / psi_0: nodes with
    psi_0 >= tau rho e have roots fixed to relative precision ~eps/tau.  Nodes closer than tau to
    the bound (constant regions, isentropic flow) have roots that rounding-level differences of
    the inputs can move far (the oracle itself moves there under 1e-16 input noise).  Those nodes
    and their face neighbours (alpha on a subcell face is the min of the two nodes) are checked
    for validity instead: density inside its bounds, sigma >= K_i, and a difference no larger than
    the sum of the node's absolute subcell corrections dt/m sum |r-bar|.  All other nodes must
    match to `tol` (normwise per field).  `elems`: check only these elements (`got` holds their
    values).  Returns the fraction of nodes checked by validity."""
    exp, info = pb.fe_stage(U, dt, elems=elems, full=True)
    n = pb.n
    got = got.reshape(exp.shape)
    scale = np.max(np.abs(exp), axis=(1, 2))
    uL, K = info["uL"], info["K"]
    rhoe = pb.law.pressure(uL) / (pb.law.gamma - 1.0)
    ic = pb.law.psi(uL, K) < tau * rhoe
    # plus nodes where Zalesak's density ratio is ill-conditioned (a density plateau on its bound)
    bad = spread_faces(ic | zalesak_ill_conditioned(pb, info, dt, tol=tol, elems=elems), n)
    err = np.abs(got - exp) / scale[:, None, None]
    assert np.all(err[:, ~bad] <= tol), np.max(err[:, ~bad], axis=1)
    xp, xm, yp, ym = pb._node_face_fluxes(info["rbar"])
    corr = dt / pb._mass(elems) * (np.abs(xp) + np.abs(xm) + np.abs(yp) + np.abs(ym)) / scale[:, None, None]
    assert np.all(err[:, bad] <= corr[:, bad] + tol)
    assert np.all(got[0][bad] >= info["lo"][bad] * (1 - 1e-12)) and np.all(got[0][bad] <= info["hi"][bad] * (1 + 1e-12))
    assert np.all(pb.law.sigma(got)[bad] >= K[bad] * (1 - 1e-12))
    return float(bad.mean())
