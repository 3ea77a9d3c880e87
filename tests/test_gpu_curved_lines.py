"""The line layout on curved meshes (tile candidate 4 on a mapped mesh: `k_stage_curved_lines`,
Euler, subcell limiting) against the FP64 curved-mesh oracle: limited stages through the
conditioning-aware comparator with the captured bounds, meshes spanning several CTAs with a
partial last one, slip walls, whole steps (conservation, free stream), the statistics variant,
mixed precision, and the full-size warped blast on sampled elements."""
import numpy as np
import pytest

import test_gpu_curved as tc
from fe_compare import euler_fe_check
from oracle import laws, scheme
from oracle.curved import CurvedProblem
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu
G = 1.4
LINE = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def make(p, nx, ny, bc=tc.PER, precision="fp64", eps=0.08):
    pb, sv, X, Y = tc.make("euler", p, nx, ny, "subcell", bc=bc, eps=eps, precision=precision)
    sv.set_tile(LINE)
    assert sv.tile()[2] == LINE
    return pb, sv, X, Y


@pytest.mark.parametrize("kind,max_relaxed", [("smooth", 0.25), ("quadrants", 1.0)])
@pytest.mark.parametrize("bc", [tc.PER, tc.OUT, tc.MIXED_BC])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7])
def test_line_curved_subcell_stage(p, bc, kind, max_relaxed):
    """One limited stage (Sec. 4.1.3, 4.3) on a warped mesh of 9 x 7 elements (several CTAs of the
    line layout, the last one partial), with the captured bounds against the oracle's.  "smooth":
    the density bump, contact and shear layer of the wall tests.  The nodes held to validity are
    flagged from the oracle's own stage alone (ill-conditioned entropy roots, rounding-level
    Zalesak 0/0 on density plateaus, where mapped elements give a constant state nonzero
    per-direction antidiffusive fluxes); with these data on 9 x 7 elements they are 3.6% of the
    nodes at p = 4 and 21% at p = 5 and 7 (the far-field plateau)."""
    pb, sv, X, Y = make(p, 9, 7, bc=bc)
    U = tc.data("euler", X, Y, seed=5) if kind == "quadrants" else pb.law.prim_to_cons(*tc.tw._data(X, Y))
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(4, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    sv.set_debug(True)
    sv.stage(1, dt)
    euler_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"], max_relaxed=max_relaxed)
    _, info = pb.fe_stage(U, dt, full=True)
    bd = sv.bounds()
    np.testing.assert_allclose(bd["lo"], info["lo"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(bd["hi"], info["hi"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(bd["K"], info["K"].ravel(), rtol=1e-12)


@pytest.mark.parametrize("mesh,max_relaxed", [("wavy", 0.15), ("rotated", 0.02)])
@pytest.mark.parametrize("p", [3, 4])
def test_line_curved_slip_walls(p, mesh, max_relaxed):
    """One limited stage next to curved slip walls (Sec. 5.7 on mapped faces)."""
    pb, sv, U = tc.wall_case(mesh, p, "subcell")
    sv.set_tile(LINE)
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(4, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    euler_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"], max_relaxed=max_relaxed)
    _, info = pb.fe_stage(U, dt, full=True)
    bd = sv.bounds()
    np.testing.assert_allclose(bd["lo"], info["lo"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(bd["hi"], info["hi"].ravel(), rtol=1e-12, atol=1e-13)


def test_line_curved_rk_stages():
    """Stages 2 and 3 (u^n read back): c0 u^n + c1 FE(u^(k-1)), FE from a second context on the
    same kernel, to float64 rounding."""
    pb, sv, X, Y = make(3, 9, 7)
    _, fe, _, _ = make(3, 9, 7)
    U0 = pb.law.prim_to_cons(*tc.tw._data(X, Y))
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(4, -1))
    sv.stage(1, dt)
    prev = sv.get_state(1)
    for k, (c0, c1), buf in ((2, (0.75, 0.25), 2), (3, (1.0 / 3.0, 2.0 / 3.0), 0)):
        sv.stage(k, dt)
        got = sv.get_state(buf)
        fe.set_state(prev)
        fe.stage(1, dt)
        expect = c0 * U0.reshape(4, -1) + c1 * fe.get_state(1)
        assert np.all(tc.rel(got, expect) <= 1e-14), (k, tc.rel(got, expect))
        prev = got


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_line_curved_conservation_and_free_stream(precision):
    """Periodic warped mesh, 20 whole steps: each conserved quantity's total (quadrature with the
    mesh's masses) is kept to rounding; a constant state stays constant."""
    pb, sv, X, Y = make(3, 12, 10, precision=precision)
    U = tc.data("euler", X, Y, seed=4)
    sv.set_state(U.reshape(4, -1))
    m0 = np.array(sv.diag()["mass"])
    sv.step(20)
    assert sv.tile()[2] == LINE
    m1 = np.array(sv.diag()["mass"])
    tol = 1e-13 if precision == "fp64" else 2e-6
    assert np.all(np.abs(m1 - m0) <= tol * np.maximum(1.0, np.abs(m0))), (m0, m1)
    c = pb.law.prim_to_cons(1.2 + 0 * X, 0.3 + 0 * X, -0.2 + 0 * X, 0.9 + 0 * X)
    sv.set_state(c.reshape(4, -1))
    sv.step(5)
    ftol = 1e-12 if precision == "fp64" else 1e-5
    assert np.all(tc.rel(sv.get_state(0), c.reshape(4, -1)) <= ftol)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_line_curved_statistics_variant(precision):
    """The statistics variant of the curved line kernel computes the same state as the timed one,
    and reports zero density-bound violations, the entropy minimum to 1e-6."""
    res = []
    for stats in (False, True):
        pb, sv, X, Y = make(3, 9, 7, bc=tc.OUT, precision=precision)
        sv.set_stats(stats)
        sv.set_state(tc.data("euler", X, Y, seed=2).reshape(4, -1))
        sv.step(8)
        res.append(sv.get_state(0))
        if stats:
            d = sv.diag()
            assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 0.0)
            assert d["max_entropy_violation"] <= (1e-12 if precision == "fp64" else 1e-6)
            assert d["rho_min"] > 0 and d["p_min"] > 0 and d["nonfinite"] == 0
    np.testing.assert_array_equal(res[0], res[1])


def test_line_curved_mixed_against_fp64_and_node_layout():
    """Mixed precision, 20 steps on the warped mesh with four-quadrant data: close to the FP64 form
    and to the node layout's mixed run, L1-relative per field (a discontinuity's nodes carry the
    limiter's rounding-decided coefficients, so the max norm is looser)."""
    out = {}
    for name, prec, tile in (("line", "mixed", LINE), ("node", "mixed", 0), ("fp64", "fp64", LINE)):
        pb, sv, X, Y = tc.make("euler", 3, 16, 16, "subcell", L=(1.0, 1.0), precision=prec)
        sv.set_tile(tile)
        sv.set_state(tc.data("euler", X, Y, seed=2).reshape(4, -1))
        sv.step(20)
        out[name] = sv.get_state(0)
        d = sv.diag()
        assert d["rho_min"] > 0 and d["p_min"] > 0 and d["nonfinite"] == 0
    a = out["line"]
    for other in ("node", "fp64"):
        b = out[other]
        l1 = np.abs(a - b).mean(axis=1) / np.abs(b).mean(axis=1)
        mx = tc.rel(a, b)
        assert np.all(l1 <= 1e-4) and np.all(mx <= 1e-2), (other, l1, mx)


def test_line_curved_full_size_blast_sampled():
    """The bench's curved workload at full size in FP64 on the line layout: the blast on the
    1024x1024 p=3 mesh warped by eps = 0.05 (periodic), one limited stage; the oracle recomputes a
    sample of elements (random, the corners across the periodic seams, the blast centre)."""
    nel, p = 1024, 3
    X, Y = scheme.Problem(laws.Euler(G), p, nel, nel).node_coords()
    Xw, Yw = inputs.warped_coords(X, Y, 0.05)
    del X, Y
    pb = CurvedProblem(laws.Euler(G), p, nel, nel, Xw, Yw)
    sv = sidp.Solver(law="euler", p=p, nx=nel, ny=nel, bc=tc.PER, limiter="subcell", gamma=G)
    sv.set_geometry(Xw, Yw)
    sv.set_tile(LINE)
    U = inputs.blast(Xw, Yw)
    del Xw, Yw
    sv.set_state(U.reshape(4, -1))
    dt = sv.compute_dt()
    sv.set_debug(True)
    sv.stage(1, dt)
    got = sv.get_state(1).reshape(4, pb.Ne, -1)
    rng = np.random.default_rng(2)
    c = nel // 2
    sample = np.unique(np.concatenate([
        rng.integers(0, pb.Ne, 48), [0, nel - 1, pb.Ne - nel, pb.Ne - 1],
        [(c + dy) * nel + c + dx for dy in range(-3, 3) for dx in range(-3, 3)]]))
    alpha = sv.bounds()["alpha"].reshape(pb.Ne, -1)[sample]
    # ambient plateau: a Zalesak 0/0 at every ambient node on mapped elements (as for the node layout)
    euler_fe_check(pb, U, dt, got[:, sample], alpha, elems=sample, max_relaxed=1.0)
    sv.close()


def test_curved_set_tile_rejections():
    pb, sv, X, Y = tc.make("euler", 3, 4, 3, "subcell")
    with pytest.raises(Exception):
        sv.set_tile(2)  # a curved mesh has the node layout (0) and the line layout (4)
    sv.set_tile(0)
    _, sb, _, _ = tc.make("burgers", 3, 4, 3, "subcell")
    with pytest.raises(Exception):
        sb.set_tile(4)
