"""Pins of the oracle's reference-element tables (Sec. 2.1, 2.2, Eq. didp) to closed forms."""
import numpy as np
import pytest

from oracle import gll

# Textbook Gauss-Lobatto nodes/weights on [-1,1], mapped to [0,1].
CLOSED = {
    1: ([-1, 1], [1, 1]),
    2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_closed_forms(p):
    x, w = gll.gll(p)
    xs, ws = CLOSED[p]
    np.testing.assert_allclose(x, 0.5 * (np.array(xs) + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * np.array(ws), atol=1e-15)


@pytest.mark.parametrize("p", range(1, 8))
def test_gll_quadrature_exact_to_degree_2p_minus_1(p):
    x, w = gll.gll(p)
    for k in range(2 * p):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    # and not exact at degree 2p (Lobatto rules are exact to 2p-1 only)
    assert abs(np.sum(w * x ** (2 * p)) - 1.0 / (2 * p + 1)) > 1e-12


@pytest.mark.parametrize("p", range(1, 8))
def test_diff_matrix_differentiates_polynomials(p):
    x, w = gll.gll(p)
    D = gll.diff_matrix(p)
    for k in range(p + 1):
        f = x ** k
        df = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(D @ f, w * df, atol=1e-12)


@pytest.mark.parametrize("p", range(1, 8))
def test_P1_P2(p):
    D = gll.diff_matrix(p)
    Dh = gll.sparse_diff_matrix(p)
    e = np.zeros(p + 1)
    e[0], e[-1] = -1.0, 1.0
    for M in (D, Dh):
        np.testing.assert_allclose(M.sum(axis=1), 0.0, atol=1e-14)   # (P1)
        np.testing.assert_allclose(M.sum(axis=0), e, atol=1e-14)     # (P2)


def test_sparse_diff_matrix_entries_and_p1_identity():
    Dh = gll.sparse_diff_matrix(4)
    expect = np.array([[-.5, .5, 0, 0, 0], [-.5, 0, .5, 0, 0], [0, -.5, 0, .5, 0],
                       [0, 0, -.5, 0, .5], [0, 0, 0, -.5, .5]])
    np.testing.assert_array_equal(Dh, expect)
    np.testing.assert_allclose(gll.diff_matrix(1), gll.sparse_diff_matrix(1), atol=1e-15)
