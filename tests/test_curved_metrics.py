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
