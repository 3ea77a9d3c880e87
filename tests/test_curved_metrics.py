"""The library's curved-mesh metric arrays (sidp_curved_metrics, computed on the host, no GPU)
against the oracle's (Sec. 2.3 metric terms, face normals; Sec. 3.1 corrected rows)."""
import numpy as np
import pytest

from oracle import laws, scheme
from oracle.curved import CurvedProblem
from paper_2004_08503_gb300 import build, inputs, sidp


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def _oracle_tables(cw):
    N = cw.X.size
    n, NN = cw.n, cw.n * cw.n
    nxf = np.zeros((2, cw.Ne, NN))
    nyf = np.zeros((2, cw.Ne, NN))
    nxf[:, :, cw.fnodes["W"]] = -cw.nface["W"]   # +xi normal = minus the outward one on W
    nxf[:, :, cw.fnodes["E"]] = cw.nface["E"]
    nyf[:, :, cw.fnodes["S"]] = -cw.nface["S"]
    nyf[:, :, cw.fnodes["N"]] = cw.nface["N"]
    return np.concatenate([cw.R1.reshape(2, N), cw.R2.reshape(2, N), cw.Q1.reshape(2, N), cw.Q2.reshape(2, N),
                           cw.mK.reshape(1, N), nxf.reshape(2, N), nyf.reshape(2, N)])


@pytest.mark.parametrize("bc", [("periodic",) * 4, ("outflow",) * 4, ("outflow", "outflow", "periodic", "periodic")])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_metric_arrays_match_the_oracle(p, bc):
    nx, ny = 4, 3
    X, Y = scheme.Problem(laws.Burgers(), p, nx, ny, domain=(0, 1, 0, 0.75)).node_coords()
    Xw, Yw = inputs.warped_coords(X, Y, 0.08, (1.0, 0.75))
    cw = CurvedProblem(laws.Burgers(), p, nx, ny, Xw, Yw, bc=bc)
    got = sidp.sidp_curved_metrics(p, nx, ny, bc, Xw, Yw)
    ref = _oracle_tables(cw)
    assert got.shape == ref.shape == (sidp.GEO_FIELDS, Xw.size)
    # the two sides differentiate the map with differently rounded derivative matrices (rows of
    # size ~p^2): agreement to a few hundred ulp
    scale = np.abs(ref[:8]).max()
    np.testing.assert_allclose(got[:8], ref[:8], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(got[8], ref[8], rtol=1e-12)
    np.testing.assert_allclose(got[9:], ref[9:], rtol=0, atol=1e-12 * scale)


def test_metric_errors():
    X, Y = scheme.Problem(laws.Burgers(), 2, 3, 3).node_coords()
    with pytest.raises(sidp.SidpError):
        sidp.sidp_curved_metrics(2, 3, 3, ("periodic",) * 4, -X, Y)          # mirrored: det J < 0
    with pytest.raises(sidp.SidpError):
        sidp.sidp_curved_metrics(2, 3, 3, ("exact",) + ("outflow",) * 3, X, Y)
    with pytest.raises(sidp.SidpError):
        sidp.sidp_curved_metrics(8, 3, 3, ("periodic",) * 4, X, Y)


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_library_arrays_satisfy_the_identities(p):
    """The library's own arrays, checked against the mathematics rather than the oracle: the
    metric identity Eq. metric for its rows of G J^-1, Eq. idp-sbp for its corrected rows with its
    face normals, and sum_i m_i = the area of the mapped domain (periodic warp: the area of the
    undeformed one)."""
    from oracle import gll
    nx, ny = 4, 3
    X, Y = scheme.Problem(laws.Burgers(), p, nx, ny, domain=(0, 1, 0, 0.75)).node_coords()
    Xw, Yw = inputs.warped_coords(X, Y, 0.08, (1.0, 0.75))
    g = sidp.sidp_curved_metrics(p, nx, ny, ("periodic",) * 4, Xw, Yw)
    n, Ne = p + 1, nx * ny
    xi, w = gll.gll(p)
    M1 = np.diag(w)
    D, Dh = gll.diff_matrix(p), gll.sparse_diff_matrix(p)
    DX, DY = np.kron(M1, D), np.kron(D, M1)
    DhX, DhY = np.kron(M1, Dh), np.kron(Dh, M1)
    R = g[0:4].reshape(4, Ne, n * n)
    Q = g[4:8].reshape(4, Ne, n * n)
    NXf = g[9:11].reshape(2, Ne, n, n)
    NYf = g[11:13].reshape(2, Ne, n, n)
    scale = np.abs(R).max()
    for j in (0, 1):
        ident = R[j] @ DX.T + R[2 + j] @ DY.T          # sum_i D_i (G J^-1)_ij 1
        assert np.abs(ident).max() < 1e-13 * scale
        bnd = np.zeros((Ne, n, n))                      # sum_e B_e n_{e,j} 1, outward normals
        bnd[:, :, 0] -= w[None, :] * NXf[j][:, :, 0]
        bnd[:, :, p] += w[None, :] * NXf[j][:, :, p]
        bnd[:, 0, :] -= w[None, :] * NYf[j][:, 0, :]
        bnd[:, p, :] += w[None, :] * NYf[j][:, p, :]
        lhs = Q[j] @ DhX + Q[2 + j] @ DhY
        assert np.abs(lhs - bnd.reshape(Ne, -1)).max() < 1e-13 * scale
    assert np.sum(g[8]) == pytest.approx(0.75, rel=1e-12)


def test_metric_arrays_agree_on_a_fine_mesh():
    """On a 256x256 warped mesh (h = 1/256) the two sides still agree to a few ulp of each array:
    both differentiate the coordinates relative to the element's first node (the same map, since
    the derivative of a constant vanishes), so no precision is lost to the absolute coordinates as
    the elements shrink."""
    p, nel = 3, 256
    X, Y = scheme.Problem(laws.Euler(1.4), p, nel, nel).node_coords()
    Xw, Yw = inputs.warped_coords(X, Y, 0.05)
    cw = CurvedProblem(laws.Euler(1.4), p, nel, nel, Xw, Yw, bc=("periodic",) * 4)
    got = sidp.sidp_curved_metrics(p, nel, nel, ("periodic",) * 4, Xw, Yw)
    ref = _oracle_tables(cw)
    for k in range(sidp.GEO_FIELDS):
        scale = np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() <= 2e-14 * scale, k
