"""Comparison of a forward-Euler limited stage with the oracle's where the limiter is ill-conditioned.

Sec. 4.1.3 limits node i by alpha_i = min(R+, R-), R+- = min(1, Q+-/P+-).  Where the low-order
state sits on its bound (Q = 0 up to rounding) and the antidiffusive fluxes of that sign are
rounding noise (P = 0 up to rounding), R is a 0/0 that rounding decides anywhere in [0, 1]: one
ulp of input moves it.  Sec. 4.3 limits the Euler density's nodes further by the entropy line
search, whose root is ill-conditioned where u^L is within rounding of the entropy bound.
alpha_i also limits the node's other fluxes and, through the face minimum, its neighbours', so
two correct evaluations of the method may differ there by much more than rounding (the oracle
against itself under one-ulp input noise shows it).

The check, given the candidate's output state `got` and its nodal coefficients `alpha`
(alpha-tilde_i, from the GPU's debug capture or the candidate oracle's own):
  * nodes that are well conditioned must match the oracle to `tol` (normwise per field);
  * at every node alpha_i must be admissible and maximal under the oracle's own float64
    constraints (Sec. 4.1.3 and 4.2 define alpha-tilde as the LARGEST admissible coefficient):
    every constraint holds at alpha_i up to its rounding scale, and either alpha_i = 1 or some
    constraint is violated (again up to its rounding scale) at alpha_i (1 + 1e-6) + 1e-12;
  * the oracle's update rebuilt with those coefficients (alpha_{m,k} = min of the two nodes)
    must equal `got` to `tol`, so `got` is the limited update of an admissible, maximal alpha;
  * the ill-conditioned nodes (and their subcell-face neighbours) stay inside the bounds (and,
    for Euler, sigma >= K);
  * their share of the mesh is printed and must stay below `max_relaxed` (default 0.45 of the
    nodes, 0.75 of the elements for elementwise limiting, where one binding node sets the whole
    element's coefficient: the plateau-heavy test data of the
    solid body rotation and of the slip-wall mirror test reach 0.40; callers state tighter
    bounds where their data allow).
An over-limiting candidate (alpha = 0 where the constraints leave room) fails the maximality
test even at ill-conditioned nodes.
"""
import numpy as np

KAPPA = 64.0  # rounding allowance, in units of the last place of each constraint's operands
BUMP_REL, BUMP_ABS = 1e-6, 1e-12


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


def operand_scale(pb, U, uL, elems):
    """Per node and field, the magnitude of the operands its low-order state is computed from:
    the largest |u| over the node's element and the four face-adjacent elements (their traces
    enter its face fluxes, and dt/m times a flux is of the order of the states), and the node's
    own |u^L|.  Shape (nc, Ne, n*n).  With a subset of elements the subset's maximum is used."""
    nc = U.shape[0]
    if elems is not None:
        s = np.max(np.abs(U[:, elems]), axis=(1, 2))[:, None, None]
        return np.maximum(s, np.abs(uL))
    se = np.max(np.abs(U), axis=2).reshape(nc, pb.ny, pb.nx)
    out = se.copy()
    for ax in (1, 2):
        for sh in (1, -1):
            out = np.maximum(out, np.roll(se, sh, axis=ax))
    return np.maximum(out.reshape(nc, -1)[:, :, None], np.abs(uL))


def _psi_scale(law, u, K, S):
    """Rounding scale of psi_K at the state u whose operands are known to the scales S (per field):
    the magnitudes of rho E, |m|^2/(2 rho) and K rho^gamma, plus |grad psi| . S."""
    rho = u[0]
    v = np.sqrt(u[1] ** 2 + u[2] ** 2) / np.where(rho > 0, rho, np.inf)
    rg = K * np.abs(rho) ** law.gamma
    d_rho = 0.5 * v * v + law.gamma * K * np.abs(rho) ** (law.gamma - 1.0)
    return np.abs(u[3]) + 0.5 * rho * v * v + rg + d_rho * S[0] + v * (S[1] + S[2]) + S[3]


def _constraints(pb, info, dt, alpha, dirs, zal, S, elems, ulp, kappa):
    """Slack g >= 0 (admissible) and rounding scale eta of every constraint at coefficient alpha
    (Ne, n*n): Zalesak's two (in state units: bound - u^L - alpha dt/m P) and, for Euler, rho > 0
    and psi_K >= min(0, psi_K(u^L)) along each direction w of `dirs` (u^L + alpha w).
    Returns lists of (g, eta) arrays."""
    uL = info["uL"]
    m = pb._mass(elems)
    Pp, Pm = zal
    out = []
    s0 = S[0]
    up = info["hi"] - uL[0]
    dn = uL[0] - info["lo"]
    out.append((np.maximum(up, 0.0) - alpha * dt / m * Pp, kappa * ulp * (s0 + dt / m * Pp)))
    out.append((np.maximum(dn, 0.0) - alpha * dt / m * Pm, kappa * ulp * (s0 + dt / m * Pm)))
    if pb.law.name == "euler":
        law, K = pb.law, info["K"]
        target = np.minimum(0.0, law.psi(uL, K))
        for w in dirs:
            u = uL + alpha[None] * w
            out.append((u[0], kappa * ulp * S[0]))
            with np.errstate(invalid="ignore", divide="ignore"):
                g = np.where(u[0] > 0, law.psi(u, K) - target, -np.inf)
            out.append((g, kappa * ulp * _psi_scale(law, u, K, S)))
    return out


def _check_alpha(pb, U, info, dt, alpha, dirs, zal, elems, ulp, kappa, where=None):
    """alpha (Ne, n*n) admissible and maximal under the oracle's float64 constraints."""
    S = operand_scale(pb, U, info["uL"], elems)
    at = np.clip(alpha, 0.0, 1.0)
    assert np.all(alpha >= 0.0) and np.all(alpha <= 1.0 + 1e-15), "alpha outside [0, 1]"
    sel = np.ones(at.shape, bool) if where is None else where
    for g, eta in _constraints(pb, info, dt, at, dirs, zal, S, elems, ulp, kappa):
        bad = sel & (g < -eta)
        assert not np.any(bad), f"alpha not admissible at {int(bad.sum())} nodes (worst slack {np.min((g + eta)[bad]):.3e})"
    bumped = np.minimum(at * (1.0 + BUMP_REL) + BUMP_ABS, 1.0)
    tight = at >= 1.0 - 1e-12
    for g, eta in _constraints(pb, info, dt, bumped, dirs, zal, S, elems, ulp, kappa):
        tight |= g <= eta
    loose = sel & ~tight
    assert not np.any(loose), (f"alpha not maximal at {int(loose.sum())} of {int(sel.sum())} nodes "
                               f"(alpha there {at[loose][:5]}, oracle {info['alpha_tilde'][loose][:5]})")


def apply_alpha(pb, info, dt, at, elems=None):
    """The subcell update of Eq. subcell-fct / convex-fct with nodal coefficients `at` (Ne, n*n):
    alpha_{m,k} = min of the two nodes of each interior subcell face, applied to the oracle's r-bar."""
    n = pb.n
    ne = at.shape[0]
    A = at.reshape(ne, n, n)
    ax = np.zeros((ne, n, n + 1))
    ay = np.zeros((ne, n, n + 1))
    ax[:, :, 1:n] = np.minimum(A[:, :, :-1], A[:, :, 1:])
    At = A.swapaxes(1, 2)
    ay[:, :, 1:n] = np.minimum(At[:, :, :-1], At[:, :, 1:])
    lim = np.stack([ax, ay])[:, None] * info["rbar"]
    xp, xm, yp, ym = pb._node_face_fluxes(lim)
    return info["uL"] + dt / pb._mass(elems)[None] * (xp - xm + yp - ym)


def _subcell_parts(pb, info, dt, elems):
    xp, xm, yp, ym = pb._node_face_fluxes(info["rbar"])
    c = np.stack([xp[0], -xm[0], yp[0], -ym[0]])
    zal = (np.sum(np.maximum(c, 0.0), axis=0), -np.sum(np.minimum(c, 0.0), axis=0))
    sc = 4.0 * dt / pb._mass(elems)[None]
    dirs = [sc * v for v in (xp, -xm, yp, -ym)]
    return zal, dirs


def _report(name, frac, max_relaxed):
    print(f"{name}: relaxed share {frac:.4f} (bound {max_relaxed})")
    assert frac <= max_relaxed, f"{name}: {frac:.4f} of the nodes checked by validity > {max_relaxed}"


def _reshape_alpha(alpha, shape):
    a = np.asarray(alpha, dtype=float).reshape(shape)
    return a


def scalar_fe_check(pb, U, dt, got, alpha, tol=1e-12, tau=1e-10, max_relaxed=0.45, ulp=None, kappa=KAPPA):
    """Compare a scalar forward-Euler limited stage `got` (nc*N values) and its nodal coefficients
    `alpha` (N values) with the oracle's from the same input U.  Returns the share of nodes
    checked by validity."""
    ulp = np.finfo(float).eps if ulp is None else ulp
    exp, info = pb.fe_stage(U, dt, full=True)
    got = np.asarray(got).reshape(exp.shape)
    alpha = _reshape_alpha(alpha, info["alpha_tilde"].shape)
    scale = max(np.max(np.abs(exp)), 1e-300)
    bad = spread_faces(zalesak_ill_conditioned(pb, info, dt, tol=tol, tau=tau), pb.n)
    err = np.abs(got - exp)[0] / scale
    assert np.all(err[~bad] <= tol), np.max(err[~bad])
    zal, dirs = _subcell_parts(pb, info, dt, None)
    _check_alpha(pb, U, info, dt, alpha, dirs, zal, None, ulp, kappa)
    rebuilt = apply_alpha(pb, info, dt, alpha)
    assert np.max(np.abs(rebuilt - got)) / scale <= tol, np.max(np.abs(rebuilt - got)) / scale
    g = got[0]
    slack = tol * scale
    assert np.all(g[bad] >= info["lo"][bad] - slack) and np.all(g[bad] <= info["hi"][bad] + slack)
    frac = float(bad.mean())
    _report("scalar subcell", frac, max_relaxed)
    return frac


def elementwise_fe_check(pb, U, dt, got, alpha, tol=1e-12, ulp=None, kappa=KAPPA, tau=1e-6, eta_rel=1e-10,
                         max_relaxed=0.75):
    """Elementwise limiting (Sec. 4.1.2, 4.2.1): compare `got` and the nodal coefficients `alpha`
    (alpha-tilde_i before the element minimum) with the oracle's stage from U.

    alpha_K = min over the element of alpha-tilde_i.  Rounding moves alpha-tilde_i of a binding
    Zalesak ratio Q/|r_i| by about kappa ulp (m/dt) max|u| / |r_i|; a rounding-level 0/0 (node on
    its bound, noise-level r_i) may take any value in [0, 1]; for Euler a node whose psi_K(u^L) is
    below tau rho e has an entropy root that rounding can move anywhere below its density value.
    The interval of alpha_K follows; each node may then differ by (its width) |dt/m r_i| plus
    tol max|u|, and must stay inside the bounds (and sigma >= K for Euler).  Every alpha-tilde_i
    must be admissible and maximal under the oracle's constraints, and the update rebuilt from
    min_K alpha must equal `got`."""
    ulp = np.finfo(float).eps if ulp is None else ulp
    exp, info = pb.fe_stage(U, dt, full=True)
    got = np.asarray(got).reshape(exp.shape)
    at, aK, rn, uL = info["alpha_tilde"], info["alpha_K"], info["rn"], info["uL"]
    alpha = _reshape_alpha(alpha, at.shape)
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
    # admissible and maximal alpha-tilde_i (single flux r_i, no gamma_d), then the rebuilt update
    zal = (np.maximum(rn[0], 0.0), -np.minimum(rn[0], 0.0))
    dirs = [dt / m[None] * rn]
    _check_alpha(pb, U, info, dt, alpha, dirs, zal, None, ulp, kappa)
    rebuilt = uL + dt / m[None] * np.min(alpha, axis=1)[None, :, None] * rn
    assert np.max(np.abs(rebuilt - got)) <= 10 * tol * scale, np.max(np.abs(rebuilt - got)) / scale
    slack = 10 * tol * scale
    assert np.all(got[0] >= info["lo"] - slack) and np.all(got[0] <= info["hi"] + slack)
    if pb.law.name == "euler":
        assert np.all(pb.law.sigma(got) >= info["K"] * (1 - 10 * tol))
    # share of elements whose rounding interval of alpha_K moves some node by more than tol
    frac = float(np.mean(np.max(width[None, :, None] * w, axis=(0, 2)) > tol * scale))
    _report("elementwise", frac, max_relaxed)
    return frac


def euler_fe_check(pb, U, dt, got, alpha, tol=1e-12, tau=1e-6, elems=None, max_relaxed=0.45, ulp=None,
                   kappa=KAPPA):
    """Compare a forward-Euler stage `got` and its nodal coefficients `alpha` with the oracle's on
    the entropy-limited Euler path.

    The entropy coefficient of node i is the root t* of psi_K(u^L + t w) = min(0, psi_K(u^L)),
    psi_K concave.  Concavity gives |psi'(t*)| >= psi_0 / t* with psi_0 = psi_K(u^L), so a
    rounding-level change delta of psi moves the root by at most t* delta / psi_0: nodes with
    psi_0 >= tau rho e have roots fixed to relative precision ~eps/tau.  Nodes closer than tau to
    the bound (constant regions, isentropic flow) have roots that rounding-level differences of
    the inputs can move far (the oracle itself moves there under 1e-16 input noise).  Those nodes
    whose subcell fluxes can move the update by more than tol, and their face neighbours (alpha on a subcell face is the min of the two nodes) are held to
    validity: an admissible and maximal alpha, the update rebuilt from it, density inside its
    bounds and sigma >= K_i.  All other nodes must match to `tol` (normwise per field).  `elems`:
    check only these elements (`got` and `alpha` hold their values).  Returns the share of nodes
    checked by validity."""
    ulp = np.finfo(float).eps if ulp is None else ulp
    exp, info = pb.fe_stage(U, dt, elems=elems, full=True)
    n = pb.n
    got = got.reshape(exp.shape)
    alpha = _reshape_alpha(alpha, info["alpha_tilde"].shape)
    scale = np.max(np.abs(exp), axis=(1, 2))
    uL, K = info["uL"], info["K"]
    rhoe = pb.law.pressure(uL) / (pb.law.gamma - 1.0)
    # a node whose subcell fluxes move no field by more than tol cannot be moved by its alpha
    # (nor its face neighbours through the shared face coefficient: that face's flux is its own)
    xp, xm, yp, ym = pb._node_face_fluxes(info["rbar"])
    fsc = np.maximum(np.max(np.abs(uL), axis=(1, 2)), 1e-300)[:, None, None]
    impact = np.max(dt / pb._mass(elems)[None] * (np.abs(xp) + np.abs(xm) + np.abs(yp) + np.abs(ym)) / fsc, axis=0)
    ic = (pb.law.psi(uL, K) < tau * rhoe) & (impact > tol)
    # plus nodes where Zalesak's density ratio is ill-conditioned (a density plateau on its bound)
    bad = spread_faces(ic | zalesak_ill_conditioned(pb, info, dt, tol=tol, elems=elems), n)
    err = np.abs(got - exp) / scale[:, None, None]
    assert np.all(err[:, ~bad] <= tol), np.max(err[:, ~bad], axis=1)
    zal, dirs = _subcell_parts(pb, info, dt, elems)
    _check_alpha(pb, U, info, dt, alpha, dirs, zal, elems, ulp, kappa)
    rebuilt = apply_alpha(pb, info, dt, alpha, elems)
    rerr = np.max(np.abs(rebuilt - got), axis=(1, 2)) / scale
    assert np.all(rerr <= tol), rerr
    assert np.all(got[0][bad] >= info["lo"][bad] * (1 - 1e-12)) and np.all(got[0][bad] <= info["hi"][bad] * (1 + 1e-12))
    assert np.all(pb.law.sigma(got)[bad] >= K[bad] * (1 - 1e-12))
    frac = float(bad.mean())
    _report("euler subcell", frac, max_relaxed)
    return frac
