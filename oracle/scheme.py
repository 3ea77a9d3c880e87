"""The sparse IDP DG stage update written out literally (oracle; test infrastructure only).

Mesh: nx x ny uniform Cartesian quads of side h on [x0,x1]x[y0,y1].  Element
e = ey*nx + ex; inside it node i = a*n + b (a: y index, b: x index, n = p+1) sits
at (x0 + (ex + xi_b) h, y0 + (ey + xi_a) h).  A state is an array (nc, Ne, n*n).

On such a mesh the element map has J = h I, so G = det J = h^2 and G J^{-1} = h I
(Sec. 2.3); the mass is m_i = h^2 w_a w_b (M_K = M_R G).  The conservative metric
correction C of Sec. 3.1 vanishes (the right-hand side of Eq. metric-perturbation
is zero by (P2)), so G J^-1-hat = G J^-1.

Order of operations of one forward-Euler stage (Sec. 4, Eq. subcell-fct / convex-fct):
  1. r^H  (Eq. ho-update, strong form Eq. dg-strong, Lax-Friedrichs flux Eq. lax-friedrichs)
  2. r^L  (Eq. dg-idp: pairwise c-hat_ij . F_j and graph viscosity d-hat_ij (u_j - u_i),
           d_ij from Eq. dij; face terms from Eq. lf-alternative)
  3. bar states (Eq. bar-states) and local bounds (Sec. 4.1.1; Sec. 4.3 for Euler)
  4. r_{i,k} = r^H_{i,k} - r^L_{i,k} and subcell fluxes r-bar_{m,k} (Sec. 4.1.3)
  5. nodal alpha-tilde (Zalesak on the scalar or on density; Euler: largest t with all
     gamma-scaled candidates of Eq. convex-provisional in the entropy set)
  6. alpha_{m,k} = min of the two adjacent alpha-tilde; limited update.
Time stepping: SSP-RK3 (Sec. 5) with dt = CFL min_i m_i / (2 sum_{j!=i} d-hat_ij) (Eq. cfl-low).

Readings of points the paper leaves open are marked "reading:" below.
"""
import numpy as np

from . import gll as _gll

SIDES = ("W", "E", "S", "N")
_NORMALS = {"W": (-1.0, 0.0), "E": (1.0, 0.0), "S": (0.0, -1.0), "N": (0.0, 1.0)}
_DIR = {"W": 0, "E": 0, "S": 1, "N": 1}  # coordinate direction k of the face normal


class Problem:
    """Mesh, law, reference operators and boundary data of one simulation."""

    def __init__(self, law, p, nx, ny, domain=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4,
                 ghost=None, cfl=0.5, limiter="subcell", sparsify=True, smoothness=None, split=None):
        """sparsify=False swaps D-hat for the dense D in the low-order operator: the
        unsparsified graph-viscosity method the paper compares against (Sec. 3.4).
        smoothness: None, or dict(gmin, gmax[, s0, kappa]) enabling the subcell-resolution
        smoothness indicator of Sec. 4.4 (relaxed bounds of the limited field).
        split: {side: dict(s0, speed, a, b)} for sides with bc "split": the ghost state is `a`
        where the coordinate along the side is below s0 + speed t and `b` elsewhere (b None: a
        slip wall there), t the time of the stage (the boundaries of the double Mach reflection,
        Sec. 5.7)."""
        x0, x1, y0, y1 = map(float, domain)
        h = (x1 - x0) / nx
        if abs((y1 - y0) / ny - h) > 1e-14 * max(1.0, abs(h)):
            raise ValueError("square elements required")
        self.law, self.p, self.n = law, int(p), int(p) + 1
        self.nx, self.ny, self.Ne = int(nx), int(ny), int(nx) * int(ny)
        self.x0, self.y0, self.h = x0, y0, h
        self.bc = dict(zip(SIDES, bc))
        for s in SIDES:
            if self.bc[s] not in ("periodic", "outflow", "exact", "wall", "split"):
                raise ValueError(self.bc[s])
            if self.bc[s] == "wall" and law.name != "euler":
                raise ValueError("slip walls are defined for the Euler equations")
            if self.bc[s] == "split" and (split is None or s not in split):
                raise ValueError("split side without parameters")
        self.ghost = ghost or {}
        self.split = split or {}
        # simulated time t^n, and the time at which time-dependent ghost states are evaluated
        # (t^n for dt and stage 1, t^n + dt for stage 2, t^n + dt/2 for stage 3 of SSP-RK3)
        self.time = 0.0
        self.t_eval = 0.0
        self.cfl, self.limiter = float(cfl), limiter
        self.smoothness = None
        if smoothness is not None:
            si = dict(smoothness)
            si.setdefault("s0", np.log10(float(p) ** -4))  # Sec. 4.4: s0 ~ log10(p^-4)
            si.setdefault("kappa", 1.0)
            self.smoothness = si
        n = self.n
        self.xi, self.w = _gll.gll(self.p)
        D = _gll.diff_matrix(self.p)
        Dh = _gll.sparse_diff_matrix(self.p) if sparsify else D
        M1 = np.diag(self.w)
        B0 = np.zeros((n, n)); B0[0, 0] = 1.0
        B1 = np.zeros((n, n)); B1[n - 1, n - 1] = 1.0
        # Eq. (kronecker): D_{1,R} = M (x) D acts along x (fast index b), D_{2,R} = D (x) M.
        self.DX, self.DY = np.kron(M1, D), np.kron(D, M1)
        self.DhX, self.DhY = np.kron(M1, Dh), np.kron(Dh, M1)
        # Boundary operators of Sec. 2.2.
        self.B = {"W": np.kron(M1, B0), "E": np.kron(M1, B1), "S": np.kron(B0, M1), "N": np.kron(B1, M1)}
        self.mass = h * h * np.kron(self.w, self.w)  # m_i, Sec. 2.3 (M_K = M_R G)
        # Volume coefficients c_ij of Eq. (dg-lo-cij): sum_i D-hat_i^T (G J^-1)_ii F_i = sum_j c_ij . F_j
        self.cX, self.cY = h * self.DhX.T, h * self.DhY.T
        # E(i): in-element stencil pairs (i != j with c_ij or c_ji nonzero).
        nz = (np.abs(self.cX) + np.abs(self.cY) + np.abs(self.cX.T) + np.abs(self.cY.T)) > 0
        np.fill_diagonal(nz, False)
        I, J = np.nonzero(nz)
        self.pI, self.pJ = I, J
        self.p_cij = np.stack([self.cX[I, J], self.cY[I, J]])
        self.p_cji = np.stack([self.cX[J, I], self.cY[J, I]])
        kx = np.abs(self.p_cij[0]) + np.abs(self.p_cji[0]) > 0
        ky = np.abs(self.p_cij[1]) + np.abs(self.p_cji[1]) > 0
        if np.any(kx & ky):
            raise AssertionError("a stencil pair couples both directions")
        self.p_dir = np.where(kx, 0, 1)
        # face nodes (element-local index) in order along the face, and the matching
        # node of the neighbouring element across the face
        a = np.arange(n)
        self.fnodes = {"W": a * n, "E": a * n + (n - 1), "S": a, "N": (n - 1) * n + a}
        self.fopp = {"W": self.fnodes["E"], "E": self.fnodes["W"], "S": self.fnodes["N"], "N": self.fnodes["S"]}
        self.fw = {s: self.w.copy() for s in SIDES}  # face quadrature weight at each face node
        # variable-velocity advection (Sec. 3.3): beta at every node
        self.var = law.name == "advection_var"
        if self.var:
            X, Y = self.node_coords()
            self.BX, self.BY = law.velocity(X, Y)

    # ------------------------------------------------------------------ geometry
    def _mass(self, elems):
        """m_i of the nodes of `elems`, broadcastable against (len(elems), n*n): on a Cartesian
        mesh every element has the same masses, so a single row (1, n*n)."""
        return self.mass[None, :]

    def node_coords(self):
        """Physical coordinates (Ne, n*n) of all nodes."""
        n, nx = self.n, self.nx
        e = np.arange(self.Ne)
        ex, ey = e % nx, e // nx
        bb, aa = np.meshgrid(np.arange(n), np.arange(n))
        X = self.x0 + (ex[:, None] + self.xi[bb.ravel()][None, :]) * self.h
        Y = self.y0 + (ey[:, None] + self.xi[aa.ravel()][None, :]) * self.h
        return X, Y

    def neighbor_trace(self, U, side, elems):
        """u^+ at the face nodes of `side` for elements `elems`: (nc, len(elems), n).

        periodic: trace of the neighbouring element; outflow (reading: ghost = interior
        trace, u^+ = u^-); exact: user ghost trace self.ghost[side] of shape (nc, n_side, n);
        wall (slip, Sec. 5.7): the mirror image of the interior trace, normal momentum negated, so
        that the face flux carries no mass and the face is a plane of symmetry; split: the state a
        below the moving split point s0 + speed t_eval along the side, b (or a wall) above it.
        """
        nx, ny = self.nx, self.ny
        ex, ey = elems % nx, elems // nx
        bc = self.bc[side]
        if side == "W":
            nb_ex, nb_ey, inside = ex - 1, ey, ex > 0
        elif side == "E":
            nb_ex, nb_ey, inside = ex + 1, ey, ex < nx - 1
        elif side == "S":
            nb_ex, nb_ey, inside = ex, ey - 1, ey > 0
        else:
            nb_ex, nb_ey, inside = ex, ey + 1, ey < ny - 1
        nbe = (nb_ey % ny) * nx + (nb_ex % nx)
        out = U[:, nbe][:, :, self.fopp[side]]
        if bc == "periodic":
            return out
        own = U[:, elems][:, :, self.fnodes[side]]
        if bc == "outflow":
            alt = own
        elif bc == "wall":
            alt = own.copy()
            alt[1 if side in ("W", "E") else 2] *= -1.0
        elif bc == "split":
            sp = self.split[side]
            if side in ("W", "E"):   # coordinate along the side of each face node: y
                coord = self.y0 + self.h * (ey[:, None] + self.xi[None, :])
            else:
                coord = self.x0 + self.h * (ex[:, None] + self.xi[None, :])
            below = coord < sp["s0"] + sp["speed"] * self.t_eval
            a = np.asarray(sp["a"], dtype=float)[:, None, None] * np.ones_like(own)
            if sp.get("b") is None:
                b = own.copy()
                b[1 if side in ("W", "E") else 2] *= -1.0
            else:
                b = np.asarray(sp["b"], dtype=float)[:, None, None] * np.ones_like(own)
            alt = np.where(below[None], a, b)
        else:
            pos = ey if side in ("W", "E") else ex
            alt = np.asarray(self.ghost[side])[:, pos, :]
        return np.where(inside[None, :, None], out, alt)

    # ------------------------------------------------------------------ residuals
    def lf_flux(self, um, up, nvec):
        """Eq. (lax-friedrichs): 1/2 (F(u^-) + F(u^+)).n - lambda/2 (u^+ - u^-)."""
        nx_, ny_ = nvec
        Fm, Fp = self.law.flux(um), self.law.flux(up)
        lam = self.law.lam(um, up, nx_, ny_)
        Fn = 0.5 * ((Fm[0] + Fp[0]) * nx_ + (Fm[1] + Fp[1]) * ny_)
        return Fn - 0.5 * lam * (up - um), lam

    def ho_residual(self, U, elems=None):
        """r^H per direction, Eq. (ho-update): r^H = -(sum_i D_{i,R} (G J^-1 F)_i + sum_e B_e (F-hat_e - F_e.n)).

        Returns (2, nc, len(elems), n*n); index 0 collects D_{1,R} and the x faces.
        """
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        Ue = U[:, elems]
        h = self.h
        Fx, Fy = self._flux(Ue, elems)
        r = np.zeros((2,) + Ue.shape)
        r[0] = -(h * Fx) @ self.DX.T
        r[1] = -(h * Fy) @ self.DY.T
        for s in SIDES:
            nvec = _NORMALS[s]
            idx = self.fnodes[s]
            um = Ue[:, :, idx]
            up = self.neighbor_trace(U, s, elems)
            if self.var:
                bn = self.BX[elems][:, idx] * nvec[0] + self.BY[elems][:, idx] * nvec[1]
                fhat = 0.5 * bn * (um + up) - 0.5 * np.abs(bn) * (up - um)
                G = np.zeros_like(Ue)
                G[:, :, idx] = h * (fhat - bn * um)
                r[_DIR[s]] -= G @ self.B[s].T
                continue
            fhat, _ = self.lf_flux(um, up, nvec)
            Fm = self.law.flux(um)
            G = np.zeros_like(Ue)
            G[:, :, idx] = h * (fhat - (Fm[0] * nvec[0] + Fm[1] * nvec[1]))  # scaled normal carries h
            r[_DIR[s]] -= G @ self.B[s].T
        return r

    def _flux(self, Ue, elems):
        """F at the nodes of `elems`; beta(x_i) u_i for variable-velocity advection."""
        if self.var:
            return self.BX[elems][None] * Ue, self.BY[elems][None] * Ue
        return self.law.flux(Ue)

    def _pair_viscosity_var(self, elems):
        """Sec. 3.3 modified coefficients: d-hat_ij = max(|c-hat_ij . beta_i|, |c-hat_ji . beta_j|)."""
        bxi, byi = self.BX[elems][:, self.pI], self.BY[elems][:, self.pI]
        bxj, byj = self.BX[elems][:, self.pJ], self.BY[elems][:, self.pJ]
        a = np.abs(self.p_cij[0] * bxi + self.p_cij[1] * byi)
        b = np.abs(self.p_cji[0] * bxj + self.p_cji[1] * byj)
        return np.maximum(a, b)

    def _pair_viscosity(self, Ue):
        """d_ij of Eq. (dij) on the in-element pairs (pI, pJ): (len(elems), npairs).

        reading: Eq. (dij) takes n_ij = c_ij/|c_ij| from Guermond-Popov, whose c_ij carries the
        opposite sign (their flux term sits on the left-hand side).  With the sign of Eq. (dg-idp)
        the direction of the pair's Riemann problem, from i toward j, is n_ij = -c_ij/|c_ij|.
        """
        ui, uj = Ue[:, :, self.pI], Ue[:, :, self.pJ]
        ncij = np.linalg.norm(self.p_cij, axis=0)
        ncji = np.linalg.norm(self.p_cji, axis=0)
        nij = -self.p_cij / np.where(ncij > 0, ncij, 1.0)
        nji = -self.p_cji / np.where(ncji > 0, ncji, 1.0)
        l1 = self.law.lam(ui, uj, nij[0], nij[1]) * ncij
        l2 = self.law.lam(uj, ui, nji[0], nji[1]) * ncji
        return np.maximum(l1, l2)

    def lo_residual(self, U, elems=None, want_bars=False):
        """r^L per direction from Eq. (dg-idp): m_i du_i/dt = sum_j c-hat_ij.F_j + sum_j d-hat_ij (u_j - u_i).

        c-hat_ij = c_ij + b_ij; the face coefficients come from Eq. (lf-alternative):
        b_ii = -1/2 sum_{faces of i} wn_ii, b_ij = -1/2 wn_ij, d-hat_ij = lambda |wn_ij| / 2,
        wn = h * w_face * outward normal.  Optionally returns the bar states of Eq. (bar-states).
        """
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        Ue = U[:, elems]
        h = self.h
        Fx, Fy = self._flux(Ue, elems)
        r = np.zeros((2,) + Ue.shape)
        # volume: sum_j c_ij . F_j (c_ij = h (D-hat_{1,R}^T, D-hat_{2,R}^T)_ij)
        r[0] = Fx @ self.cX.T
        r[1] = Fy @ self.cY.T
        # in-element graph viscosity, Eq. (dij) (Sec. 3.3 coefficients for variable velocity)
        dij = self._pair_viscosity_var(elems) if self.var else self._pair_viscosity(Ue)
        ui, uj = Ue[:, :, self.pI], Ue[:, :, self.pJ]
        visc = dij[None] * (uj - ui)
        for k in (0, 1):
            sel = self.p_dir == k
            acc = np.zeros_like(Ue)
            np.add.at(acc, (slice(None), slice(None), self.pI[sel]), visc[:, :, sel])
            r[k] += acc
        bars = None
        if want_bars:
            if self.var:  # Sec. 3.3 modified bar states: (c-hat_ij . beta_j) (u_j - u_i)
                cb = self.p_cij[0] * self.BX[elems][:, self.pJ] + self.p_cij[1] * self.BY[elems][:, self.pJ]
                cdF = cb[None] * (uj - ui)
            else:
                FI = (Fx[:, :, self.pI], Fy[:, :, self.pI])
                FJ = (Fx[:, :, self.pJ], Fy[:, :, self.pJ])
                cdF = self.p_cij[0] * (FJ[0] - FI[0]) + self.p_cij[1] * (FJ[1] - FI[1])
            dsafe = np.where(dij > 0, dij, 1.0)
            ubar = 0.5 * (ui + uj) + np.where(dij > 0, cdF / (2.0 * dsafe), 0.0)
            bars = {"pairs": ubar, "faces": {}}
        # element faces
        dface = {}
        for s in SIDES:
            nvec = _NORMALS[s]
            idx = self.fnodes[s]
            um = Ue[:, :, idx]
            up = self.neighbor_trace(U, s, elems)
            wn = h * self.fw[s]  # |wn_ij|
            bcoef = -0.5 * wn  # b_ii^(face) = b_ij = -1/2 wn (times the normal)
            if self.var:  # beta.n is continuous across the face (Sec. 3.3 velocity class)
                bn = self.BX[elems][:, idx] * nvec[0] + self.BY[elems][:, idx] * nvec[1]
                FnI, FnJ = bn * um, bn * up
                lam = np.abs(bn)
            else:
                Fm, Fp = self.law.flux(um), self.law.flux(up)
                lam = self.law.lam(um, up, nvec[0], nvec[1])
                FnI = Fm[0] * nvec[0] + Fm[1] * nvec[1]
                FnJ = Fp[0] * nvec[0] + Fp[1] * nvec[1]
            dhat = 0.5 * lam * wn
            contrib = bcoef * (FnI + FnJ) + dhat * (up - um)
            G = np.zeros_like(Ue)
            G[:, :, idx] = contrib
            r[_DIR[s]] += G
            dface[s] = dhat
            if want_bars:
                dsafe = np.where(dhat > 0, dhat, 1.0)
                ub = 0.5 * (um + up) + np.where(dhat > 0, bcoef * (FnJ - FnI) / (2.0 * dsafe), 0.0)
                bars["faces"][s] = ub
        if want_bars:
            return r, bars, dij, dface
        return r

    def sum_dhat(self, U, elems=None):
        """sum_{j != i} d-hat_ij per node (the quantity in Eq. cfl-low)."""
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        _, _, dij, dface = self.lo_residual(U, elems, want_bars=True)
        tot = np.zeros((len(elems), self.n * self.n))
        np.add.at(tot, (slice(None), self.pI), dij)
        for s in SIDES:
            tot[:, self.fnodes[s]] += dface[s]
        return tot

    def compute_dt(self, U):
        """Eq. (cfl-low) with the CFL constant of Sec. 5.

        reading: Eq. (cfl-low) divides by d-hat_ii = -sum d-hat_ij < 0; the convex-combination
        form Eq. (convex-combination) needs dt <= m_i / (2 sum_{j != i} d-hat_ij), used here.
        """
        self.t_eval = self.time
        tot = self.sum_dhat(U)
        # a node with sum d-hat = 0 (a stagnation point of a velocity field) puts no limit on dt
        with np.errstate(divide="ignore"):
            return self.cfl * float(np.min(self._mass(None) / (2.0 * tot)))

    # ------------------------------------------------------------------ limiting
    def bounds(self, U, bars, elems):
        """Local bounds over N(i) including i itself (reading: u-bar_ii = u_i).

        Scalar: u_i^min/max = min/max of the bar states (Sec. 4.1.1).
        Euler: rho bounds from bar-state densities; K_i = min_{j in N(i)} sigma(u_j) (Sec. 4.3),
        i.e. s_i^min = log(K_i)/(gamma-1).
        """
        Ue = U[:, elems]
        f = 0  # the limited field: the scalar, or the density
        lo = Ue[f].copy()
        hi = Ue[f].copy()
        np.minimum.at(lo, (slice(None), self.pI), bars["pairs"][f])
        np.maximum.at(hi, (slice(None), self.pI), bars["pairs"][f])
        for s in SIDES:
            idx = self.fnodes[s]
            lo[:, idx] = np.minimum(lo[:, idx], bars["faces"][s][f])
            hi[:, idx] = np.maximum(hi[:, idx], bars["faces"][s][f])
        K = None
        if self.law.name == "euler":
            sig = self.law.sigma(Ue)
            K = sig.copy()
            np.minimum.at(K, (slice(None), self.pI), sig[:, self.pJ])
            for s in SIDES:
                idx = self.fnodes[s]
                K[:, idx] = np.minimum(K[:, idx], self.law.sigma(self.neighbor_trace(U, s, elems)))
        return lo, hi, K

    def subcell_fluxes(self, r):
        """r-bar_{m,k} = sum_{i in M(m,k)} r_{i,k} (Sec. 4.1.3).

        reading: M(m,k) is the set of nodes of the line with a lower index than the face.
        Returns (2, nc, Ne, n, n+1): x faces indexed [a, q], y faces [b, q], q = 0..n; q = 0 and
        q = n are the element boundary (zero by Prop. line-zero-sum, set exactly to zero).
        """
        n = self.n
        nc, ne = r.shape[1], r.shape[2]
        rx = r[0].reshape(nc, ne, n, n)            # [a, b]
        ry = r[1].reshape(nc, ne, n, n).swapaxes(2, 3)  # [b, a]
        out = np.zeros((2, nc, ne, n, n + 1))
        for k, rl in enumerate((rx, ry)):
            for q in range(1, n):
                out[k, :, :, :, q] = np.sum(rl[:, :, :, :q], axis=3)
        return out

    def _node_face_fluxes(self, rbar):
        """For every node, r-bar at m_i^+ and m_i^- in x and y: each (nc, Ne, n*n)."""
        n = self.n
        nc, ne = rbar.shape[1], rbar.shape[2]
        xp = rbar[0][:, :, :, 1:n + 1].reshape(nc, ne, n * n)
        xm = rbar[0][:, :, :, 0:n].reshape(nc, ne, n * n)
        yp = rbar[1][:, :, :, 1:n + 1].swapaxes(2, 3).reshape(nc, ne, n * n)
        ym = rbar[1][:, :, :, 0:n].swapaxes(2, 3).reshape(nc, ne, n * n)
        return xp, xm, yp, ym

    def smoothness_factor(self, U, elems):
        """epsilon_K of Sec. 4.4 for each element, from the limited field of the stage input.

        u_K is expanded in the tensor Legendre basis on the element (solving the nodal
        interpolation V c = u exactly, V_ij = L_j(x_i) on [0,1]); u-hat_K drops every mode of
        degree p in either variable; the norms are the exact L2 norms of the polynomials
        (||L_k||^2 = 1/(2k+1) on [0,1]); s_K = log10(||u - u-hat||^2 / ||u||^2).
        reading: the printed middle branch 1/2 - 1/2 sin(pi (s_K - s0)/(2 kappa)) is 1 at the lower
        end and 0 at the upper end, contradicting the outer branches (0 below, 1 above); the
        continuous form 1/2 + 1/2 sin(...) (Persson-Peraire) is used.
        """
        from numpy.polynomial import legendre as npleg
        n, p = self.n, self.p
        Lv = np.stack([npleg.legval(2.0 * self.xi - 1.0, np.eye(n)[k]) for k in range(n)], axis=1)  # V[i,k]
        Vinv = np.linalg.inv(Lv)
        u = U[0, elems].reshape(len(elems), n, n)  # [e, a, b]
        c = np.einsum("ja,kb,eab->ejk", Vinv, Vinv, u)  # c[e, j (y degree), k (x degree)]
        norms = 1.0 / (2.0 * np.arange(n) + 1.0)
        wgt = norms[:, None] * norms[None, :]
        tot = np.sum(c * c * wgt, axis=(1, 2))
        mask = np.zeros((n, n), bool)
        mask[p, :] = True
        mask[:, p] = True
        top = np.sum(c * c * wgt * mask, axis=(1, 2))
        with np.errstate(divide="ignore", invalid="ignore"):
            sK = np.where(tot > 0, np.log10(np.maximum(top, 1e-300) / tot), -np.inf)
        s0, kap = self.smoothness["s0"], self.smoothness["kappa"]
        with np.errstate(invalid="ignore"):  # sin(-inf) on all-zero elements, discarded by the branch
            eps = np.where(sK < s0 - kap, 0.0,
                           np.where(sK > s0 + kap, 1.0, 0.5 + 0.5 * np.sin(np.pi * (sK - s0) / (2.0 * kap))))
        return eps, sK

    def zalesak(self, uL, lo, hi, rbar, dt, field=0, elems=None):
        """Nodal alpha-tilde from the sums of positive and negative parts of the adjacent
        subcell fluxes (Sec. 4.1.3), Zalesak-style.

        reading: P+ = sum of positive parts of (+r-bar_{m+,k}, -r-bar_{m-,k}), P- of negative parts;
        Q+ = max(0, m/dt (u^max - u^L)), Q- = min(0, m/dt (u^min - u^L)); R = min(1, Q/P), 1 where
        P = 0; alpha-tilde = min(R+, R-).
        """
        xp, xm, yp, ym = self._node_face_fluxes(rbar)
        c = np.stack([xp[field], -xm[field], yp[field], -ym[field]])
        Pp = np.sum(np.maximum(c, 0.0), axis=0)
        Pm = np.sum(np.minimum(c, 0.0), axis=0)
        m = self._mass(elems)
        Qp = np.maximum(0.0, m / dt * (hi - uL[field]))
        Qm = np.minimum(0.0, m / dt * (lo - uL[field]))
        Rp = np.where(Pp > 0, np.minimum(1.0, Qp / np.where(Pp > 0, Pp, 1.0)), 1.0)
        Rm = np.where(Pm < 0, np.minimum(1.0, Qm / np.where(Pm < 0, Pm, -1.0)), 1.0)
        return np.minimum(Rp, Rm)

    def entropy_limit(self, uL, K, rbar, dt, amax, iters=80, elems=None):
        """Largest t in [0, amax] with every candidate of Eq. (convex-provisional),
        u^L + gamma_d t (dt/m_i)(+-r-bar_{m_i^+-,k}), gamma_d = 2d = 4, in the entropy set (Sec. 4.3).

        The set is {rho > 0, psi_K >= min(0, psi_K(u^L))} (reading: u^L belongs to it in exact
        arithmetic; the min keeps roundoff in u^L from zeroing the coefficient).  psi_K is concave,
        so along a candidate the admissible t form an interval [0, t*]; t* is found by bisection.
        """
        xp, xm, yp, ym = self._node_face_fluxes(rbar)
        scale = 4.0 * dt / self._mass(elems)
        return self.entropy_line_search(uL, K, [scale[None] * v for v in (xp, -xm, yp, -ym)], amax, iters)

    def entropy_line_search(self, uL, K, dirs, amax, iters=80):
        """Largest t in [0, amax] with u^L + t w in the entropy set for every direction w of `dirs`
        (bisection on each line; the admissible t of a line form an interval since psi_K is concave)."""
        law = self.law
        psi0 = law.psi(uL, K)
        target = np.minimum(0.0, psi0)
        t_all = amax.copy()
        for wdir in dirs:

            def ok(t):
                u = uL + t[None] * wdir
                return (u[0] > 0) & (law.psi(u, K) >= target)

            good = ok(amax)
            lo = np.zeros_like(amax)
            hi = amax.copy()
            for _ in range(iters):
                mid = 0.5 * (lo + hi)
                f = ok(mid)
                lo = np.where(f, mid, lo)
                hi = np.where(f, hi, mid)
            t = np.where(good, amax, lo)
            t_all = np.minimum(t_all, t)
        return t_all

    def elementwise_alpha(self, uL, lo, hi, K, rn, dt, elems=None):
        """Elementwise limiting (Sec. 4.1.2 linear, Sec. 4.2.1 convex constraints).

        alpha-tilde_i is the largest value in [0,1] for which u^L_i + alpha (dt/m_i) r_i, with the
        nodal antidiffusive flux r_i = r^H_i - r^L_i (summed over dimensions), stays inside the
        bounds of the limited field (Zalesak with the single flux r_i: R+- = min(1, Q+-/P+-),
        P+ = max(0, r_i), P- = min(0, r_i), 1 where P = 0) and, for Euler, in the entropy set
        (Eq. convex-provisional-elementwise, one candidate, no gamma_d factor).  Every node of the
        element then takes alpha_K = min of alpha-tilde over the element.  Returns (Ne, 1).
        """
        m = self._mass(elems)
        r0 = rn[0]
        Pp = np.maximum(r0, 0.0)
        Pm = np.minimum(r0, 0.0)
        Qp = np.maximum(0.0, m / dt * (hi - uL[0]))
        Qm = np.minimum(0.0, m / dt * (lo - uL[0]))
        Rp = np.where(Pp > 0, np.minimum(1.0, Qp / np.where(Pp > 0, Pp, 1.0)), 1.0)
        Rm = np.where(Pm < 0, np.minimum(1.0, Qm / np.where(Pm < 0, Pm, -1.0)), 1.0)
        at = np.minimum(Rp, Rm)
        if self.law.name == "euler":
            at = self.entropy_line_search(uL, K, [(dt / m)[None] * rn], at)
        return at.min(axis=1, keepdims=True), at

    # ------------------------------------------------------------------ one stage
    def fe_stage(self, U, dt, elems=None, limiter=None, full=False):
        """Forward-Euler limited update u^{FE}(U) of Eq. (subcell-fct) / (convex-fct)."""
        limiter = self.limiter if limiter is None else limiter
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        Ue = U[:, elems]
        m = self._mass(elems)[None]
        rH = self.ho_residual(U, elems)
        rL, bars, dij, dface = self.lo_residual(U, elems, want_bars=True)
        uH = Ue + dt / m * (rH[0] + rH[1])
        uL = Ue + dt / m * (rL[0] + rL[1])
        info = {"rH": rH, "rL": rL, "uH": uH, "uL": uL, "bars": bars}
        if limiter == "none":
            out = uH
        elif limiter == "lo":
            out = uL
        elif limiter == "elementwise":
            lo, hi, K = self.bounds(U, bars, elems)
            if self.smoothness is not None:
                eps, _ = self.smoothness_factor(U, elems)
                lo = eps[:, None] * lo + (1.0 - eps[:, None]) * self.smoothness["gmin"]
                hi = eps[:, None] * hi + (1.0 - eps[:, None]) * self.smoothness["gmax"]
            rn = (rH[0] + rH[1]) - (rL[0] + rL[1])
            aK, at = self.elementwise_alpha(uL, lo, hi, K, rn, dt, elems)
            out = uL + dt / m * aK[None] * rn
            info.update({"lo": lo, "hi": hi, "K": K, "alpha_tilde": at, "alpha_K": aK[:, 0], "rn": rn})
        elif limiter == "subcell":
            r = rH - rL
            rbar = self.subcell_fluxes(r)
            lo, hi, K = self.bounds(U, bars, elems)
            if self.smoothness is not None:
                # Eq. relaxed-bounds: eps_K u^min + (1 - eps_K) g^min (and likewise the maximum)
                eps, _ = self.smoothness_factor(U, elems)
                lo = eps[:, None] * lo + (1.0 - eps[:, None]) * self.smoothness["gmin"]
                hi = eps[:, None] * hi + (1.0 - eps[:, None]) * self.smoothness["gmax"]
            at = self.zalesak(uL, lo, hi, rbar, dt, elems=elems)
            if self.law.name == "euler":
                at = self.entropy_limit(uL, K, rbar, dt, at, elems=elems)
            n = self.n
            ne = len(elems)
            A = at.reshape(ne, n, n)
            ax = np.zeros((ne, n, n + 1))
            ay = np.zeros((ne, n, n + 1))
            ax[:, :, 1:n] = np.minimum(A[:, :, :-1], A[:, :, 1:])        # x faces [a, q]
            At = A.swapaxes(1, 2)
            ay[:, :, 1:n] = np.minimum(At[:, :, :-1], At[:, :, 1:])      # y faces [b, q]
            lim = np.stack([ax, ay])[:, None] * rbar                      # alpha_{m,k} r-bar_{m,k}
            xp, xm, yp, ym = self._node_face_fluxes(lim)
            out = uL + dt / m * (xp - xm + yp - ym)
            info.update({"r": r, "rbar": rbar, "lo": lo, "hi": hi, "K": K, "alpha_tilde": at,
                         "alpha_x": ax, "alpha_y": ay})
        else:
            raise ValueError(limiter)
        if full:
            return out, info
        return out

    def ssp_rk3_step(self, U, dt=None):
        """One SSP-RK3 step (Sec. 5): u1 = FE(u), u2 = 3/4 u + 1/4 FE(u1), u+ = 1/3 u + 2/3 FE(u2).

        reading: dt is computed once per step from u^n and used in all three stages.
        """
        if dt is None:
            dt = self.compute_dt(U)
        t = self.time
        self.t_eval = t
        u1 = self.fe_stage(U, dt)
        self.t_eval = t + dt
        u2 = 0.75 * U + 0.25 * self.fe_stage(u1, dt)
        self.t_eval = t + 0.5 * dt
        out = U / 3.0 + (2.0 / 3.0) * self.fe_stage(u2, dt)
        self.time = self.t_eval = t + dt
        return out, dt

    def stage(self, U, U0, dt, k, elems=None):
        """SSP-RK3 stage k in {1,2,3} on elements `elems`: FE update plus the RK combination.
        Time-dependent ghost states are evaluated at self.time + (0, 1, 1/2)[k-1] dt (self.time
        is not advanced)."""
        self.t_eval = self.time + (0.0, 1.0, 0.5)[k - 1] * dt
        fe = self.fe_stage(U, dt, elems)
        U0e = U0[:, np.arange(self.Ne) if elems is None else np.asarray(elems)]
        if k == 1:
            return fe
        if k == 2:
            return 0.75 * U0e + 0.25 * fe
        return U0e / 3.0 + (2.0 / 3.0) * fe

    def total_mass(self, U):
        """sum_i m_i u_i per field (Sec. 2.4, conservation)."""
        return np.sum(U * self._mass(None)[None], axis=(1, 2))
