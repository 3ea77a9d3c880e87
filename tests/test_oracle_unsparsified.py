"""Pin of the unsparsified comparison mode (Sec. 3.4): graph viscosity on the dense DG-SEM operator.

At p = 1 the dense and sparsified operators coincide (D-hat = D).  At fixed degrees of freedom the
dense operator couples each node with O(p) others, and every such pair adds viscosity: its
low-order solution of an advected sine wave degrades quickly as p grows, while the sparsified one
does not (the paper's sine-wave comparison, here with 64 instead of 128 degrees of freedom).
"""
import numpy as np

from oracle import laws, scheme


def _sine_lo(p, sparsify, dofs=64, T=1.0):
    ne = dofs // (p + 1)
    h = 2.0 / ne
    pb = scheme.Problem(laws.Advection((1.0, 0.0)), p, ne, 1, domain=(-1, 1, 0, h), limiter="lo", sparsify=sparsify)
    X, Y = pb.node_coords()
    U = np.sin(np.pi * X)[None]
    nsteps = int(np.ceil(T / pb.compute_dt(U)))
    for _ in range(nsteps):
        U, _ = pb.ssp_rk3_step(U, T / nsteps)
    return float(np.sum(pb.mass[None] * np.abs(U - np.sin(np.pi * (X - T))[None])) / h), float(U.max())


def test_sparsified_lo_does_not_degrade_with_p_unsparsified_does():
    res = {(p, sp): _sine_lo(p, sp) for p in (1, 3, 7) for sp in (True, False)}
    assert res[(1, True)] == res[(1, False)]
    for p in (3, 7):
        assert res[(p, False)][0] > 1.3 * res[(p, True)][0]
        assert res[(p, False)][1] < res[(p, True)][1]
    assert res[(7, False)][1] < 0.7 * res[(3, False)][1]          # the dense peak keeps collapsing
    assert res[(7, True)][1] > 0.8 * res[(3, True)][1]            # the sparse one does not
