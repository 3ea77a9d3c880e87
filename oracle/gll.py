"""Reference-element tables of the oracle (test infrastructure only).

Sec. 2.1 (nodal Gauss-Lobatto basis on [0,1]) and Sec. 2.2 (collocated 1D operators):
  * ``gll(p)``          nodes xi_i and quadrature weights w_i on [0,1]  (M_1D = diag(w))
  * ``diff_matrix(p)``  weighted differentiation matrix (D_1D)_ij = w_i * phi_j'(xi_i)
  * ``sparse_diff_matrix(p)``  the sparsified first-order matrix D-hat_1D of Eq. (didp)

Everything is float64.  Nodes come from numpy's Legendre root finder (a library
primitive) polished by Newton steps; derivatives of the Lagrange basis use the
barycentric formula.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll(p):
    """Gauss-Lobatto nodes and weights on [0,1] for degree p >= 1 (Sec. 2.1).

    The interior nodes on [-1,1] are the roots of P_p'; the weights are
    2 / (p (p+1) P_p(x_i)^2).  Both are mapped to [0,1] (weights halved, sum 1).
    """
    if p < 1:
        raise ValueError("p >= 1 required")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    dcp = npleg.legder(cp)
    ddcp = npleg.legder(dcp)
    if p > 1:
        r = np.sort(npleg.legroots(dcp).real)
        for _ in range(3):  # Newton polish of P_p'(x) = 0
            r = r - npleg.legval(r, dcp) / npleg.legval(r, ddcp)
        x = np.concatenate([[-1.0], r, [1.0]])
    else:
        x = np.array([-1.0, 1.0])
    Pp = npleg.legval(x, cp)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_derivatives(xi):
    """A[i, j] = phi_j'(xi_i) for the Lagrange basis on nodes xi (barycentric form)."""
    n = len(xi)
    lam = np.array([1.0 / np.prod([xi[j] - xi[k] for k in range(n) if k != j]) for j in range(n)])
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                A[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])
        A[i, i] = -np.sum(A[i, :])
    return A


def diff_matrix(p):
    """Weighted 1D differentiation matrix (D_1D)_ij = w_i phi_j'(xi_i) (Sec. 2.2)."""
    xi, w = gll(p)
    return w[:, None] * lagrange_derivatives(xi)


def sparse_diff_matrix(p):
    """Sparsified derivative D-hat_1D of Eq. (didp), Sec. 3.

    Row 0: (-1/2, 1/2, 0, ...); interior row i: -1/2 at i-1 and +1/2 at i+1;
    last row: -1/2 at p-1 and +1/2 at p.  The paper prints only the first rows;
    the last row is the one forced by the row- and column-sum properties (P1),
    (P2) that the paper states D-hat satisfies.
    """
    n = p + 1
    Dh = np.zeros((n, n))
    Dh[0, 0], Dh[0, 1] = -0.5, 0.5
    for i in range(1, n - 1):
        Dh[i, i - 1], Dh[i, i + 1] = -0.5, 0.5
    Dh[n - 1, n - 2], Dh[n - 1, n - 1] = -0.5, 0.5
    return Dh
