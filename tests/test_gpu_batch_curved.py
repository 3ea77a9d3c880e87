"""Batches with instances on curved meshes (sidp_batch_set_geometry): every curved instance of a
mixed batch (Cartesian and curved instances, degrees 1..7, periodic, outflow and slip-wall sides,
ragged element blocks) against the FP64 curved-mesh oracle stage by stage (1e-12 for the
unlimited and low-order updates, the conditioning-aware comparator with the batch's captured
alpha-tilde for subcell limiting), and against the same instance advanced alone by a context
(the curved kernels: another instantiation of the same stage body, so equal to rounding); the
Cartesian instances of the batch stay equal to theirs bit for bit."""
import numpy as np
import pytest

import test_oracle_wall as tw
from fe_compare import euler_fe_check, scalar_fe_check
from oracle import laws, scheme
from oracle.curved import CurvedProblem
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu
G = 1.4

# (nx, ny, p, sides, mesh): mesh "warp" (periodic warp of the box), "wavy" (a wavy lower wall,
# Euler only), "cart" (left Cartesian); element counts that leave partial element blocks
SHAPES = [(5, 3, 1, ("periodic",) * 4, "warp"), (4, 4, 2, ("outflow",) * 4, "warp"),
          (3, 5, 3, ("periodic",) * 4, "warp"), (6, 2, 3, ("outflow",) * 4, "cart"),
          (4, 3, 3, ("periodic", "periodic", "wall", "wall"), "wavy"), (3, 3, 4, ("outflow",) * 4, "warp"),
          (2, 3, 5, ("periodic",) * 4, "warp"), (3, 2, 6, ("outflow",) * 4, "cart"),
          (2, 2, 7, ("periodic",) * 4, "warp")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def _law(name):
    return laws.Euler(G) if name == "euler" else laws.Burgers()


def _mesh(kind, X, Y, dom):
    if kind == "warp":
        return inputs.warped_coords(X, Y, 0.06, (dom[1], dom[3]))
    if kind == "wavy":
        return X, Y + 0.05 * (dom[3] - Y) * np.sin(2.0 * np.pi * X / dom[1])
    return X, Y


def _shapes(lawname):
    # slip walls are defined for the Euler equations only
    return [s for s in SHAPES if lawname == "euler" or s[4] != "wavy"]


def make_batch(lawname, limiter, precision="fp64"):
    """(oracles, batch, U0, meshes): one oracle per instance (CurvedProblem on curved instances,
    the Cartesian Problem otherwise) and the batch with the curved instances moved."""
    law = _law(lawname)
    cfgs, meta = [], []
    for nx, ny, p, bc, kind in _shapes(lawname):
        dom = (0.0, nx / max(nx, ny), 0.0, ny / max(nx, ny))
        cfgs.append(dict(law=lawname, p=p, nx=nx, ny=ny, precision=precision, domain=dom, bc=bc, limiter=limiter,
                         gamma=G))
        meta.append((nx, ny, p, bc, kind, dom))
    b = sidp.sidp_batch_create([sidp.make_config(**c) for c in cfgs])
    pbs, U0, meshes = [], [], []
    for i, (nx, ny, p, bc, kind, dom) in enumerate(meta):
        X, Y = scheme.Problem(law, p, nx, ny, domain=dom).node_coords()
        Xm, Ym = _mesh(kind, X, Y, dom)
        if kind == "cart":
            pb = scheme.Problem(law, p, nx, ny, domain=dom, bc=bc, limiter=limiter)
        else:
            pb = CurvedProblem(law, p, nx, ny, Xm, Ym, bc=bc, limiter=limiter)
            sidp.sidp_batch_set_geometry(b, i, Xm, Ym)
        U = law.prim_to_cons(*tw._data(Xm, Ym)) if lawname == "euler" else inputs.burgers_pulse(Xm, Ym)
        pbs.append(pb)
        U0.append(U)
        meshes.append((kind, Xm, Ym, cfgs[i]))
    return pbs, b, U0, meshes


def _rel(got, exp):
    nc = exp.shape[0]
    got, exp = got.reshape(nc, -1), exp.reshape(nc, -1)
    return np.max(np.abs(got - exp), axis=1) / np.max(np.abs(exp), axis=1)


def test_node_coords_and_mass_are_the_curved_ones():
    pbs, b, U0, meshes = make_batch("euler", "subcell")
    for i, (kind, X, Y, _) in enumerate(meshes):
        x, y = sidp.sidp_batch_node_coords(b, i)
        if kind == "cart":  # the library's Cartesian nodes (rounded in their own order)
            np.testing.assert_allclose(x, X.ravel(), rtol=0, atol=1e-15)
            np.testing.assert_allclose(y, Y.ravel(), rtol=0, atol=1e-15)
        else:  # the coordinates given
            np.testing.assert_array_equal(x, X.ravel())
            np.testing.assert_array_equal(y, Y.ravel())
        sidp.sidp_batch_set_state(b, i, U0[i].reshape(4, -1))
        np.testing.assert_allclose(sidp.sidp_batch_get_diag(b, i)["mass"], pbs[i].total_mass(U0[i]), rtol=1e-12)
    sidp.sidp_batch_destroy(b)


@pytest.mark.parametrize("lawname", ["euler", "burgers"])
@pytest.mark.parametrize("limiter", ["none", "lo"])
def test_curved_batch_stages_match_the_oracle(limiter, lawname):
    """The time step and stages 1, 2, 3 of every instance against its oracle, 1e-12 normwise."""
    pbs, b, U0, _ = make_batch(lawname, limiter)
    sidp.sidp_batch_set_stats(b, False)
    nc = U0[0].shape[0]
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(nc, -1))
    dts = np.array([pb.compute_dt(U) for pb, U in zip(pbs, U0)])
    cur = list(U0)
    for k in (1, 2, 3):
        sidp.sidp_batch_stage(b, k, dts)
        for i, pb in enumerate(pbs):
            exp = pb.stage(cur[i], U0[i], dts[i], k)
            err = _rel(sidp.sidp_batch_get_buffer(b, i, (1, 2, 0)[k - 1]), exp)
            assert np.all(err <= 1e-12), (i, k, err)
            cur[i] = exp
    # the device time step of every instance (one whole step from U0)
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(nc, -1))
    sidp.sidp_batch_step(b, 1)
    for i, pb in enumerate(pbs):
        assert abs(sidp.sidp_batch_get_diag(b, i)["last_dt"] - dts[i]) <= 1e-13 * dts[i], i
    sidp.sidp_batch_destroy(b)


@pytest.mark.parametrize("lawname", ["euler", "burgers"])
def test_curved_batch_limited_stage(lawname):
    """The subcell-limited forward-Euler stage of every instance with the conditioning-aware
    comparator, the alpha-tilde of each instance from the batch's debug capture."""
    pbs, b, U0, _ = make_batch(lawname, "subcell")
    sidp.sidp_batch_set_stats(b, False)
    sidp.sidp_batch_set_debug(b, True)
    nc = U0[0].shape[0]
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(nc, -1))
    dts = np.array([pb.compute_dt(U) for pb, U in zip(pbs, U0)])
    sidp.sidp_batch_stage(b, 1, dts)
    for i, pb in enumerate(pbs):
        got = sidp.sidp_batch_get_buffer(b, i, 1)
        alpha = sidp.sidp_batch_get_bounds(b, i)["alpha"]
        if lawname == "euler":
            euler_fe_check(pb, U0[i], dts[i], got, alpha)
        else:
            scalar_fe_check(pb, U0[i], dts[i], got, alpha)
    sidp.sidp_batch_destroy(b)


@pytest.mark.parametrize("limiter", ["subcell", "elementwise"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_curved_batch_equals_instances_alone(precision, limiter, monkeypatch):
    """Four whole steps of the batch (one graph: time steps, finalisation, stages) against each
    instance advanced alone; the violation statistics of the curved instances."""
    monkeypatch.setenv("SIDP_TILE", "0")  # the Cartesian instances: the same tile shape on both sides
    pbs, b, U0, meshes = make_batch("euler", limiter, precision)
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(4, -1))
    sidp.sidp_batch_step(b, 4)
    tol = 1e-13 if precision == "fp64" else 2e-5
    for i, (kind, X, Y, cfg) in enumerate(meshes):
        sv = sidp.Solver(**cfg)
        if kind != "cart":
            sv.set_geometry(X, Y)
        sv.set_state(U0[i].reshape(4, -1))
        sv.step(4)
        got, ref = sidp.sidp_batch_get_state(b, i), sv.get_state(0)
        if kind == "cart":
            np.testing.assert_array_equal(got, ref)
        else:
            assert np.all(_rel(got, ref) <= tol), (i, _rel(got, ref))
        d, ds = sidp.sidp_batch_get_diag(b, i), sv.diag()
        assert abs(d["t"] - ds["t"]) <= 1e-12 * ds["t"]
        assert d["rho_min"] > 0 and d["p_min"] > 0
        assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 0.0)
        assert d["max_entropy_violation"] <= (1e-12 if precision == "fp64" else 1e-6)
        sv.close()
    sidp.sidp_batch_destroy(b)


def test_curved_batch_conserves_mass():
    """Periodic and wall instances conserve mass over 20 limited steps (Sec. 3.1: the corrected
    metric keeps the low-order and the limited updates conservative on mapped elements)."""
    pbs, b, U0, meshes = make_batch("euler", "subcell")
    keep = [i for i, m in enumerate(meshes) if m[0] != "cart" and m[3]["bc"][0] == "periodic"]
    m0 = {}
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(4, -1))
        m0[i] = sidp.sidp_batch_get_diag(b, i)["mass"]
    sidp.sidp_batch_step(b, 20)
    for i in keep:
        m1 = sidp.sidp_batch_get_diag(b, i)["mass"]
        assert abs(m1[0] - m0[i][0]) <= 1e-12 * abs(m0[i][0]), i
        assert abs(m1[3] - m0[i][3]) <= 1e-12 * abs(m0[i][3]), i
    sidp.sidp_batch_destroy(b)


def test_batch_set_geometry_errors():
    X, Y = scheme.Problem(laws.Burgers(), 2, 3, 3).node_coords()
    b = sidp.sidp_batch_create([sidp.make_config(law="burgers", p=2, nx=3, ny=3, bc=("outflow",) * 4)])
    with pytest.raises(sidp.SidpError):
        sidp.sidp_batch_set_geometry(b, 0, -X, Y)  # det J < 0
    with pytest.raises(ValueError):
        sidp.sidp_batch_set_geometry(b, 0, X[:2], Y[:2])
    sidp.sidp_batch_destroy(b)
    v = inputs.SOLID_BODY_VELOCITY
    b = sidp.sidp_batch_create([sidp.make_config(law="advection_var", p=2, nx=3, ny=3, bc=("outflow",) * 4,
                                                 beta=(v[0], v[2]), grad=(v[1], v[3]))])
    with pytest.raises(sidp.SidpError):
        sidp.sidp_batch_set_geometry(b, 0, X, Y)
    sidp.sidp_batch_destroy(b)
