"""Curved (mapped) quadrilateral meshes in the oracle (test infrastructure only).

The mesh keeps the nx x ny element topology of the Cartesian oracle, but each element carries
its own map T_K: the caller gives the physical coordinates (X, Y) of every Gauss-Lobatto node
(shape (Ne, n*n), node order as in `scheme`).  Everything below follows Sec. 2.3 and Sec. 3.1:

  * metric terms at the nodes (Sec. 2.3): the Jacobian J of the interpolated map, with the
    reference derivatives taken by the nodal Lagrange derivative matrix; G = det J and the rows
    of G J^-1, row 1 = (y_eta, -x_eta), row 2 = (-y_xi, x_xi).  In two dimensions this
    cross-product form satisfies the metric identity Eq. (metric) exactly (the two derivative
    matrices commute), which is the free-stream preserving evaluation the paper calls for;
  * m_i = w_a w_b G_i (M_K = M_R G);
  * high-order residual: Eq. (dg-strong) with the contravariant fluxes F~_k = (G J^-1)_k . F;
  * face normals: the scaled outward normal of a face node is the row of G J^-1 normal to the
    face (W: -row 1, E: +row 1, S: -row 2, N: +row 2).
    reading: on a conforming mesh the two elements' rows agree in exact arithmetic; the oracle
    takes their mean (own row minus the neighbour's outward row, halved), so both elements use
    one normal, exactly opposite; a boundary face that is not periodic uses its own row;
  * the conservative correction (Sec. 3.1): G J^-1-hat = G J^-1 + C with C the minimum-norm
    solution of Eq. (metric-perturbation), computed with the pseudo-inverse (an SVD) of the
    reference-element matrix (D-hat_{1,R}^T  D-hat_{2,R}^T), formed once and reused for every
    element;
  * low-order residual: Eq. (dg-lo-modified) in the pairwise form of Eq. (dg-lo-cij) with
    c_ij = D-hat_{1,R}^T[i,j] (row 1-hat)_j + D-hat_{2,R}^T[i,j] (row 2-hat)_j (the metric
    at node j), d_ij of Eq. (dij) (n_ij = -c_ij/|c_ij|, c21) and the bar states of
    Eq. (bar-states) per ordered pair (on a curved element c_ij != -c_ji, so the two nodes of a
    pair have different bar states); face terms of Eq. (lf-alternative) with the face normals;
  * limiting, CFL and SSP-RK3 as on Cartesian meshes, with the per-node masses;
  * the smoothness indicator of Sec. 4.4 on the reference element.
    reading: the modal expansion and its L2 norms are those of the reference element (the map's
    Jacobian does not weight them), so s_K measures the polynomial on the reference square.

Boundaries: periodic (the mapped mesh must then be periodic: coordinates across a periodic
side differ by the period), outflow, and slip walls for the Euler equations (Sec. 5.7):
    reading: the ghost state is the mirror image of the interior trace across the face, the
    momentum reflected about the face's unit normal, m - 2 (m . n) n (n the face node's normal,
    the row of G J^-1 normal to the face); on a Cartesian face this negates the normal
    component, as on Cartesian meshes.  Density and energy are unchanged, so no mass or energy
    crosses the wall.
"""
import numpy as np

from . import gll as _gll
from .scheme import SIDES, Problem, _DIR

_ROW_SIGN = {"W": -1.0, "E": 1.0, "S": -1.0, "N": 1.0}


class CurvedProblem(Problem):
    """A Problem on the mapped mesh with node coordinates (X, Y).  correct=False keeps the
    uncorrected metric terms in the low-order operator (for the tests of Sec. 3.1)."""

    def __init__(self, law, p, nx, ny, X, Y, bc=("periodic",) * 4, cfl=0.5, limiter="subcell", correct=True,
                 smoothness=None):
        for s in bc:
            if s not in ("periodic", "outflow", "wall"):
                raise ValueError("curved meshes take periodic, outflow or slip-wall boundaries")
            if s == "wall" and law.name != "euler":
                raise ValueError("slip walls are defined for the Euler equations")
        if law.name == "advection_var":
            raise ValueError("variable-velocity advection is defined on Cartesian meshes")
        # reference operators and pair structure of a unit Cartesian mesh (h = 1)
        super().__init__(law, p, nx, ny, domain=(0.0, float(nx), 0.0, float(ny)), bc=bc, cfl=cfl, limiter=limiter,
                         smoothness=smoothness)
        n, NN, Ne = self.n, self.n * self.n, self.Ne
        self.X = np.asarray(X, dtype=float).reshape(Ne, NN).copy()
        self.Y = np.asarray(Y, dtype=float).reshape(Ne, NN).copy()
        A = _gll.lagrange_derivatives(self.xi)  # A[i, j] = phi_j'(xi_i)
        # [e, a (eta), b (xi)], relative to each element's first node: the derivative of a constant
        # vanishes (P1), so this is the same map, and the derivatives keep their relative precision
        # on fine meshes instead of losing |x|/h of it to the absolute coordinates
        Xe = (self.X - self.X[:, :1]).reshape(Ne, n, n)
        Ye = (self.Y - self.Y[:, :1]).reshape(Ne, n, n)
        x_xi = np.einsum("bc,eac->eab", A, Xe)
        y_xi = np.einsum("bc,eac->eab", A, Ye)
        x_eta = np.einsum("ac,ecb->eab", A, Xe)
        y_eta = np.einsum("ac,ecb->eab", A, Ye)
        self.G = (x_xi * y_eta - x_eta * y_xi).reshape(Ne, NN)
        if not np.all(self.G > 0):
            raise ValueError("the node coordinates give an element with det J <= 0")
        self.R1 = np.stack([y_eta, -x_eta]).reshape(2, Ne, NN)  # row 1 of G J^-1
        self.R2 = np.stack([-y_xi, x_xi]).reshape(2, Ne, NN)    # row 2 of G J^-1
        self.mK = np.kron(self.w, self.w)[None, :] * self.G    # m_i = w_a w_b G_i
        self.nface = self._face_normals()
        if correct:
            self.Q1, self.Q2, self.C = self._corrected_rows()
        else:
            self.Q1, self.Q2, self.C = self.R1, self.R2, np.zeros((2, 2, Ne, NN))
        # c_ij and c_ji of the in-element pairs, per element: (2, Ne, npairs)
        I, J = self.pI, self.pJ
        DXt, DYt = self.DhX.T, self.DhY.T
        self.e_cij = np.stack([DXt[I, J] * self.Q1[k][:, J] + DYt[I, J] * self.Q2[k][:, J] for k in (0, 1)])
        self.e_cji = np.stack([DXt[J, I] * self.Q1[k][:, I] + DYt[J, I] * self.Q2[k][:, I] for k in (0, 1)])

    # ------------------------------------------------------------------ geometry
    def _mass(self, elems):
        return self.mK if elems is None else self.mK[np.asarray(elems)]

    def node_coords(self):
        return self.X, self.Y

    def _neighbour(self, side):
        """Element across `side` of every element (wrapped), and whether it exists."""
        e = np.arange(self.Ne)
        ex, ey = e % self.nx, e // self.nx
        if side == "W":
            nb_ex, nb_ey, inside = ex - 1, ey, ex > 0
        elif side == "E":
            nb_ex, nb_ey, inside = ex + 1, ey, ex < self.nx - 1
        elif side == "S":
            nb_ex, nb_ey, inside = ex, ey - 1, ey > 0
        else:
            nb_ex, nb_ey, inside = ex, ey + 1, ey < self.ny - 1
        nbe = (nb_ey % self.ny) * self.nx + (nb_ex % self.nx)
        return nbe, inside | (self.bc[side] == "periodic")

    def _face_normals(self):
        """Scaled outward normal at the face nodes of every side: {side: (2, Ne, n)}."""
        own = {}
        for s in SIDES:
            R = self.R1 if _DIR[s] == 0 else self.R2
            own[s] = _ROW_SIGN[s] * R[:, :, self.fnodes[s]]
        opp = {"W": "E", "E": "W", "S": "N", "N": "S"}
        out = {}
        for s in SIDES:
            nbe, shared = self._neighbour(s)
            mean = 0.5 * (own[s] - own[opp[s]][:, nbe, :])
            out[s] = np.where(shared[None, :, None], mean, own[s])
        return out

    def _corrected_rows(self):
        """G J^-1-hat = G J^-1 + C, C the minimum-norm solution of Eq. (metric-perturbation)."""
        NN = self.n * self.n
        Amat = np.hstack([self.DhX.T, self.DhY.T])  # (NN, 2 NN)
        # SVD, once for the reference element.  The matrix has exactly one zero singular value
        # (its left null space is the constants); the cut-off drops it and nothing else (the
        # smallest other singular value is above 1e-2 for p <= 7).
        Apinv = np.linalg.pinv(Amat, rcond=1e-8)
        C = np.zeros((2, 2, self.Ne, NN))            # C[i, j]: correction of row i, component j
        for j in (0, 1):
            bnd = np.zeros((self.Ne, NN))            # sum_e B_e n_{e,j} 1
            for s in SIDES:
                bnd[:, self.fnodes[s]] += self.fw[s][None, :] * self.nface[s][j]
            rhs = bnd - (self.R1[j] @ self.DhX + self.R2[j] @ self.DhY)
            sol = rhs @ Apinv.T
            C[0, j], C[1, j] = sol[:, :NN], sol[:, NN:]
        return self.R1 + C[0], self.R2 + C[1], C

    def neighbor_trace(self, U, side, elems):
        """u^+ at the face nodes of `side`: as on Cartesian meshes, except that a slip wall mirrors
        the interior trace across the face's own normal (the module's reading)."""
        out = super().neighbor_trace(U, side, elems)
        if self.bc[side] != "wall":
            return out
        nbe, shared = self._neighbour(side)
        wall = ~shared[elems]
        own = U[:, elems][:, :, self.fnodes[side]]
        nv = self.nface[side][:, elems]
        nh = nv / np.sqrt(nv[0] ** 2 + nv[1] ** 2)[None]
        mn = own[1] * nh[0] + own[2] * nh[1]
        ghost = own.copy()
        ghost[1] = own[1] - 2.0 * mn * nh[0]
        ghost[2] = own[2] - 2.0 * mn * nh[1]
        return np.where(wall[None, :, None], ghost, out)

    # ------------------------------------------------------------------ residuals
    def _face_data(self, U, s, elems):
        nv = self.nface[s][:, elems]  # (2, ne, n)
        nn = np.sqrt(nv[0] ** 2 + nv[1] ** 2)
        return nv, nn, nv / nn[None]

    def ho_residual(self, U, elems=None):
        """r^H per reference direction, Eq. (dg-strong) with F~_k = (G J^-1)_k . F."""
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        Ue = U[:, elems]
        Fx, Fy = self.law.flux(Ue)
        R1, R2 = self.R1[:, elems], self.R2[:, elems]
        F1 = R1[0] * Fx + R1[1] * Fy
        F2 = R2[0] * Fx + R2[1] * Fy
        r = np.zeros((2,) + Ue.shape)
        r[0] = -F1 @ self.DX.T
        r[1] = -F2 @ self.DY.T
        for s in SIDES:
            idx = self.fnodes[s]
            nv, nn, nh = self._face_data(U, s, elems)
            um = Ue[:, :, idx]
            up = self.neighbor_trace(U, s, elems)
            Fm, Fp = self.law.flux(um), self.law.flux(up)
            lam = self.law.lam(um, up, nh[0], nh[1])
            fhat = 0.5 * ((Fm[0] + Fp[0]) * nv[0] + (Fm[1] + Fp[1]) * nv[1]) - 0.5 * lam * nn * (up - um)
            G = np.zeros_like(Ue)
            G[:, :, idx] = fhat - (Fm[0] * nv[0] + Fm[1] * nv[1])
            r[_DIR[s]] -= G @ self.B[s].T
        return r

    def lo_residual(self, U, elems=None, want_bars=False):
        """r^L per reference direction, Eq. (dg-lo-modified) in the form of Eq. (dg-lo-cij)."""
        elems = np.arange(self.Ne) if elems is None else np.asarray(elems)
        Ue = U[:, elems]
        Fx, Fy = self.law.flux(Ue)
        Q1, Q2 = self.Q1[:, elems], self.Q2[:, elems]
        r = np.zeros((2,) + Ue.shape)
        r[0] = (Q1[0] * Fx + Q1[1] * Fy) @ self.DhX  # sum_j D-hat_1^T[i,j] (row 1-hat . F)_j
        r[1] = (Q2[0] * Fx + Q2[1] * Fy) @ self.DhY
        cij, cji = self.e_cij[:, elems], self.e_cji[:, elems]
        ui, uj = Ue[:, :, self.pI], Ue[:, :, self.pJ]
        ncij = np.sqrt(cij[0] ** 2 + cij[1] ** 2)
        ncji = np.sqrt(cji[0] ** 2 + cji[1] ** 2)
        nij, nji = -cij / ncij[None], -cji / ncji[None]
        dij = np.maximum(self.law.lam(ui, uj, nij[0], nij[1]) * ncij, self.law.lam(uj, ui, nji[0], nji[1]) * ncji)
        visc = dij[None] * (uj - ui)
        for k in (0, 1):
            sel = self.p_dir == k
            acc = np.zeros_like(Ue)
            np.add.at(acc, (slice(None), slice(None), self.pI[sel]), visc[:, :, sel])
            r[k] += acc
        bars = None
        if want_bars:
            FI = (Fx[:, :, self.pI], Fy[:, :, self.pI])
            FJ = (Fx[:, :, self.pJ], Fy[:, :, self.pJ])
            cdF = cij[0] * (FJ[0] - FI[0]) + cij[1] * (FJ[1] - FI[1])
            dsafe = np.where(dij > 0, dij, 1.0)
            bars = {"pairs": 0.5 * (ui + uj) + np.where(dij > 0, cdF / (2.0 * dsafe), 0.0), "faces": {}}
        dface = {}
        for s in SIDES:
            idx = self.fnodes[s]
            nv, nn, nh = self._face_data(U, s, elems)
            um = Ue[:, :, idx]
            up = self.neighbor_trace(U, s, elems)
            wn = self.fw[s][None, :] * nv  # weighted normal wn_ij (2, ne, n)
            wnn = self.fw[s][None, :] * nn
            Fm, Fp = self.law.flux(um), self.law.flux(up)
            FnI = Fm[0] * wn[0] + Fm[1] * wn[1]
            FnJ = Fp[0] * wn[0] + Fp[1] * wn[1]
            lam = self.law.lam(um, up, nh[0], nh[1])
            dhat = 0.5 * lam * wnn
            G = np.zeros_like(Ue)
            G[:, :, idx] = -0.5 * (FnI + FnJ) + dhat * (up - um)
            r[_DIR[s]] += G
            dface[s] = dhat
            if want_bars:
                dsafe = np.where(dhat > 0, dhat, 1.0)
                bars["faces"][s] = 0.5 * (um + up) + np.where(dhat > 0, -0.5 * (FnJ - FnI) / (2.0 * dsafe), 0.0)
        if want_bars:
            return r, bars, dij, dface
        return r
