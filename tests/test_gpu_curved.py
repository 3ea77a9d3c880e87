"""Curved (mapped) meshes on the GPU path against the FP64 oracle (Sec. 2.3 metric terms,
Sec. 3.1 conservative correction, with the limiting of Sec. 4): the time step, the unlimited and
low-order stages element by element, the limited stages through the conditioning-aware
comparators, whole steps, free-stream preservation, conservation, and the rotated Cartesian mesh
against the Cartesian kernels."""
import numpy as np
import pytest

import test_oracle_wall as tw
from fe_compare import elementwise_fe_check, euler_fe_check, scalar_fe_check
from oracle import laws, scheme
from oracle.curved import CurvedProblem
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu
G = 1.4
BETA = (1.0, 0.5)
PER = ("periodic",) * 4
OUT = ("outflow",) * 4
MIXED_BC = ("outflow", "outflow", "periodic", "periodic")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def _law(name):
    return {"euler": laws.Euler(G), "burgers": laws.Burgers(), "advection": laws.Advection(BETA)}[name]


def make(law, p, nx, ny, limiter, bc=PER, eps=0.08, L=None, precision="fp64", theta=None, smooth=None):
    lo = _law(law)
    L = (1.0, ny / nx) if L is None else L   # square elements
    X, Y = scheme.Problem(lo, p, nx, ny, domain=(0.0, L[0], 0.0, L[1])).node_coords()
    if theta is None:
        Xm, Ym = inputs.warped_coords(X, Y, eps, L)
    else:
        Xm, Ym = inputs.rotated_coords(X, Y, theta)
    pb = CurvedProblem(lo, p, nx, ny, Xm, Ym, bc=bc, limiter=limiter, smoothness=smooth)
    sv = sidp.Solver(law=law, p=p, nx=nx, ny=ny, domain=(0.0, L[0], 0.0, L[1]), bc=bc, limiter=limiter, gamma=G,
                     beta=BETA, precision=precision, smoothness=smooth)
    sv.set_geometry(Xm, Ym)
    return pb, sv, Xm, Ym


def data(law, X, Y, seed=3):
    if law == "euler":
        return inputs.four_quadrant(X, Y, seed)
    return inputs.burgers_pulse(X, Y)


def rel(a, b):
    a = a.reshape(b.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)


def test_node_coords_are_the_mapped_ones():
    pb, sv, X, Y = make("burgers", 3, 4, 3, "lo")
    x, y = sv.node_coords()
    np.testing.assert_array_equal(x, X.ravel())
    np.testing.assert_array_equal(y, Y.ravel())


@pytest.mark.parametrize("bc", [PER, OUT, MIXED_BC])
@pytest.mark.parametrize("limiter", ["none", "lo"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_euler_stages_match_the_oracle(p, limiter, bc):
    """dt (Eq. cfl-low) and the three SSP-RK3 stages, element by element, FP64."""
    pb, sv, X, Y = make("euler", p, 4, 3, limiter, bc=bc)
    U0 = data("euler", X, Y)
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(4, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    cur = U0
    for k in (1, 2, 3):
        expect = pb.stage(cur, U0, dt, k)
        sv.stage(k, dt)
        got = sv.get_state({1: 1, 2: 2, 3: 0}[k])
        assert np.all(rel(got, expect) <= 1e-12), (k, rel(got, expect))
        cur = expect


@pytest.mark.parametrize("law", ["burgers", "advection"])
@pytest.mark.parametrize("limiter", ["none", "lo"])
@pytest.mark.parametrize("p", [2, 4])
def test_scalar_stages_match_the_oracle(law, limiter, p):
    pb, sv, X, Y = make(law, p, 5, 4, limiter)
    U0 = data(law, X, Y)
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(1, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    cur = U0
    for k in (1, 2, 3):
        expect = pb.stage(cur, U0, dt, k)
        sv.stage(k, dt)
        got = sv.get_state({1: 1, 2: 2, 3: 0}[k])
        assert np.all(rel(got, expect) <= 1e-12), (k, rel(got, expect))
        cur = expect


@pytest.mark.parametrize("law", ["burgers", "advection"])
@pytest.mark.parametrize("p", [2, 3, 5])
def test_scalar_subcell_stage(law, p):
    """One limited forward-Euler stage (Zalesak, Sec. 4.1.3) with the conditioning-aware check."""
    pb, sv, X, Y = make(law, p, 5, 4, "subcell", bc=MIXED_BC)
    U = data(law, X, Y)
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(1, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    scalar_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"])


@pytest.mark.parametrize("kind,max_relaxed", [("smooth", 0.02), ("quadrants", 1.0)])
@pytest.mark.parametrize("bc", [PER, OUT])
@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_euler_subcell_stage(p, bc, kind, max_relaxed):
    """One limited stage with the density bounds and the entropy minimum (Sec. 4.3).  "smooth":
    a density bump, a contact and a shear layer (almost every node held to 1e-12).  "quadrants":
    four constant states; on mapped elements the per-direction antidiffusive fluxes of a constant
    state are not zero while its bounds collapse onto it, so Zalesak's ratio is a rounding-level
    0/0 on the plateaus and most nodes are held by validity (admissible, maximal alpha and the
    update rebuilt from it) rather than by the 1e-12 match."""
    pb, sv, X, Y = make("euler", p, 4, 3, "subcell", bc=bc)
    U = data("euler", X, Y, seed=5) if kind == "quadrants" else pb.law.prim_to_cons(*tw._data(X, Y))
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(4, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    euler_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"], max_relaxed=max_relaxed)
    # the bounds themselves (bar states of ordered pairs, element-face bars, K)
    _, info = pb.fe_stage(U, dt, full=True)
    bd = sv.bounds()
    lo, hi, K = bd["lo"], bd["hi"], bd["K"]
    np.testing.assert_allclose(lo, info["lo"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(hi, info["hi"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(K, info["K"].ravel(), rtol=1e-12)


@pytest.mark.parametrize("law,p", [("burgers", 3), ("advection", 2), ("euler", 3), ("euler", 5)])
def test_elementwise_stage(law, p):
    """Elementwise limiting (Sec. 4.1.2, 4.2.1) on the warped mesh: one stage against the oracle
    with the comparator that bounds the rounding interval of alpha_K."""
    pb, sv, X, Y = make(law, p, 6, 5, "elementwise")
    U = inputs.vortex(X, Y) if law == "euler" else data(law, X, Y)
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(pb.law.nc, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    elementwise_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"])


@pytest.mark.parametrize("law,limiter,p", [("burgers", "subcell", 3), ("advection", "subcell", 4),
                                            ("burgers", "elementwise", 3), ("advection", "elementwise", 2)])
def test_smoothness_indicator_stage(law, limiter, p):
    """Sec. 4.4 on mapped elements: the relaxed bounds (captured) and the limited stage."""
    smooth = dict(gmin=-0.5, gmax=2.5)
    pb, sv, X, Y = make(law, p, 6, 5, limiter, smooth=smooth)
    U = data(law, X, Y)
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(1, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    got = sv.get_state(1)
    _, info = pb.fe_stage(U, dt, full=True)
    eps, _ = pb.smoothness_factor(U, np.arange(pb.Ne))
    assert np.any(eps > 0.05) and np.any(eps < 0.95)   # the indicator is active and partial
    bd = sv.bounds()
    np.testing.assert_allclose(bd["lo"], info["lo"].ravel(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(bd["hi"], info["hi"].ravel(), rtol=1e-10, atol=1e-12)
    if limiter == "subcell":
        scalar_fe_check(pb, U, dt, got, bd["alpha"])
    else:
        elementwise_fe_check(pb, U, dt, got, bd["alpha"])


def test_whole_steps_burgers():
    pb, sv, X, Y = make("burgers", 3, 5, 4, "lo", bc=MIXED_BC)
    U = data("burgers", X, Y)
    sv.set_state(U.reshape(1, -1))
    for _ in range(5):
        U, dt = pb.ssp_rk3_step(U)
        sv.step()
        assert abs(sv.diag()["last_dt"] - dt) <= 1e-13 * dt
    assert np.all(rel(sv.get_state(0), U) <= 1e-11)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_free_stream_and_conservation(precision):
    """A constant state stays constant on the warped periodic mesh (Sec. 3.1: only with the
    corrected metric terms), and total mass is conserved on it with the limiter on."""
    tol = 1e-13 if precision == "fp64" else 2e-6
    pb, sv, X, Y = make("euler", 3, 6, 5, "subcell", precision=precision)
    Uc = inputs.constant_state(X, Y)
    sv.set_state(Uc.reshape(4, -1))
    sv.step(5)
    np.testing.assert_allclose(sv.get_state(0), Uc.reshape(4, -1), rtol=tol)
    U = data("euler", X, Y, seed=9)
    sv.set_state(U.reshape(4, -1))
    m0 = sv.diag()["mass"]
    # the mixed form stores the state in float32: its mass carries that rounding
    np.testing.assert_allclose(m0, pb.total_mass(U), rtol=1e-12 if precision == "fp64" else 1e-6)
    sv.step(10)
    d = sv.diag()
    np.testing.assert_allclose(d["mass"], m0, rtol=tol * 10, atol=tol * 10 * max(abs(v) for v in m0))
    assert d["rho_min"] > 0 and d["p_min"] > 0


@pytest.mark.parametrize("limiter", ["none", "lo"])
def test_rotated_mesh_equals_the_cartesian_kernels(limiter):
    """On the rotated image of a Cartesian mesh, with rotated momenta, the curved kernels give the
    rotated result of the Cartesian kernels (two independent kernel families on the GPU)."""
    th = 0.4
    pb, sv, X, Y = make("euler", 3, 5, 5, limiter, bc=OUT, L=(1.0, 1.0), theta=th)
    sc = sidp.Solver(law="euler", p=3, nx=5, ny=5, bc=OUT, limiter=limiter, gamma=G)
    x, y = sc.node_coords()
    U = inputs.four_quadrant(x, y, 4)
    c, s = np.cos(th), np.sin(th)
    Ur = U.copy()
    Ur[1], Ur[2] = c * U[1] - s * U[2], s * U[1] + c * U[2]
    sc.set_state(U)
    sv.set_state(Ur)
    for _ in range(3):
        sc.step()
        sv.step()
    a, b = sc.get_state(0), sv.get_state(0)
    ar = a.copy()
    ar[1], ar[2] = c * a[1] - s * a[2], s * a[1] + c * a[2]
    assert abs(sc.diag()["t"] - sv.diag()["t"]) <= 1e-12 * sc.diag()["t"]
    assert np.all(rel(b, ar) <= 1e-9), rel(b, ar)


def test_sampled_full_size_curved_blast_fp64():
    """The bench's curved workload at full size in FP64: the blast on the 1024x1024 p=3 mesh warped
    by eps = 0.05 (periodic), one limited stage on the GPU; the oracle recomputes a sample of
    elements (random, the four corners across the periodic seams, the blast centre) one by one."""
    nel, p = 1024, 3
    X, Y = scheme.Problem(laws.Euler(G), p, nel, nel).node_coords()
    Xw, Yw = inputs.warped_coords(X, Y, 0.05)
    del X, Y
    pb = CurvedProblem(laws.Euler(G), p, nel, nel, Xw, Yw)
    sv = sidp.Solver(law="euler", p=p, nx=nel, ny=nel, bc=PER, limiter="subcell", gamma=G)
    sv.set_geometry(Xw, Yw)
    U = inputs.blast(Xw, Yw)
    del Xw, Yw
    sv.set_state(U.reshape(4, -1))
    dt = sv.compute_dt()
    sv.set_debug(True)
    sv.stage(1, dt)
    got = sv.get_state(1).reshape(4, pb.Ne, -1)
    rng = np.random.default_rng(1)
    c = nel // 2
    sample = np.unique(np.concatenate([
        rng.integers(0, pb.Ne, 64), [0, nel - 1, pb.Ne - nel, pb.Ne - 1],
        [(c + dy) * nel + c + dx for dy in range(-3, 3) for dx in range(-3, 3)]]))
    alpha = sv.bounds()["alpha"].reshape(pb.Ne, -1)[sample]
    # the ambient gas is a density plateau with zero mass flux whose momentum has nonzero
    # per-direction antidiffusive fluxes on mapped elements: a Zalesak 0/0 at every ambient node,
    # held by validity (admissible, maximal alpha; the update rebuilt from it to 1e-12)
    euler_fe_check(pb, U, dt, got[:, sample], alpha, elems=sample, max_relaxed=1.0)
    sv.close()


def test_mixed_precision_warped_euler():
    """Mixed precision (float32 stages) on the warped mesh: positivity and agreement with FP64."""
    _, s64, X, Y = make("euler", 3, 8, 8, "subcell", L=(1.0, 1.0))
    _, s32, _, _ = make("euler", 3, 8, 8, "subcell", L=(1.0, 1.0), precision="mixed")
    U = data("euler", X, Y, seed=2)
    for sv in (s64, s32):
        sv.set_state(U.reshape(4, -1))
        sv.step(20)
    d = s32.diag()
    assert d["rho_min"] > 0 and d["p_min"] > 0 and d["nonfinite"] == 0
    assert np.all(rel(s32.get_state(0), s64.get_state(0)) <= 1e-3)


def test_set_geometry_errors():
    X, Y = scheme.Problem(laws.Burgers(), 2, 3, 3).node_coords()
    for kw in (dict(law="advection_var"), dict(bc=("exact",) + ("outflow",) * 3), dict(sparsify=False)):
        cfg = dict(law="burgers", p=2, nx=3, ny=3, bc=OUT, limiter="subcell")
        cfg.update(kw)
        sv = sidp.Solver(**cfg)
        with pytest.raises(sidp.SidpError):
            sv.set_geometry(X, Y)
    sv = sidp.Solver(law="burgers", p=2, nx=3, ny=3, bc=OUT)
    with pytest.raises(sidp.SidpError):
        sv.set_geometry(-X, Y)


# ---------------------------------------------------------------- slip walls on curved meshes
WALL_CHANNEL = ("periodic", "periodic", "wall", "wall")
ROT_WALLS = ("wall", "outflow", "wall", "wall")


def wavy_channel(p, nel, amp=0.06):
    """A channel periodic in x with a wavy lower wall y = amp sin(2 pi x) and a straight upper one:
    the nodes of the unit square moved by y += amp (1 - y) sin(2 pi x)."""
    X, Y = scheme.Problem(laws.Euler(G), p, nel, nel).node_coords()
    return X, Y + amp * (1.0 - Y) * np.sin(2.0 * np.pi * X)


def channel_data(X, Y):
    law = laws.Euler(G)
    rho = 1.0 + 0.3 * np.exp(-((X - 0.4) ** 2 + (Y - 0.5) ** 2) / 0.02)
    return law.prim_to_cons(rho, 0.5 + 0.2 * Y, 0.3 * np.sin(2 * np.pi * X), 1.0 + 0.2 * rho)


def wall_case(mesh, p, limiter, precision="fp64"):
    """(oracle, solver, U): the wavy channel (6x6) or the rotated square (4x4, theta = 0.3) with
    three walls and one outflow side, with smooth data."""
    law = laws.Euler(G)
    if mesh == "wavy":
        nel, bc = 6, WALL_CHANNEL
        X, Y = wavy_channel(p, nel)
        U = channel_data(X, Y)
    else:
        nel, bc = 4, ROT_WALLS
        X, Y = inputs.rotated_coords(*scheme.Problem(law, p, nel, nel).node_coords(), 0.3)
        U = law.prim_to_cons(*tw._data(X, Y))
    pb = CurvedProblem(law, p, nel, nel, X, Y, bc=bc, limiter=limiter)
    sv = sidp.Solver(law="euler", p=p, nx=nel, ny=nel, bc=bc, limiter=limiter, gamma=G, precision=precision)
    sv.set_geometry(X, Y)
    return pb, sv, U


@pytest.mark.parametrize("mesh", ["wavy", "rotated"])
@pytest.mark.parametrize("limiter", ["none", "lo"])
@pytest.mark.parametrize("p", [2, 3, 5])
def test_slip_wall_stages_match_the_oracle(p, limiter, mesh):
    """Slip walls on mapped faces (the ghost is the trace with its momentum reflected about the
    face's unit normal): dt and the three stages, element by element, FP64."""
    pb, sv, U0 = wall_case(mesh, p, limiter)
    dt = pb.compute_dt(U0)
    sv.set_state(U0.reshape(4, -1))
    assert abs(sv.compute_dt() - dt) <= 1e-13 * dt
    cur = U0
    for k in (1, 2, 3):
        expect = pb.stage(cur, U0, dt, k)
        sv.stage(k, dt)
        got = sv.get_state({1: 1, 2: 2, 3: 0}[k])
        assert np.all(rel(got, expect) <= 1e-12), (k, rel(got, expect))
        cur = expect


@pytest.mark.parametrize("mesh,max_relaxed", [("wavy", 0.15), ("rotated", 0.02)])
@pytest.mark.parametrize("p", [3, 4])
def test_slip_wall_subcell_stage(p, mesh, max_relaxed):
    """One limited stage next to curved walls, with the conditioning-aware comparator, and the
    bounds (bar states of the wall faces included) against the oracle's."""
    pb, sv, U = wall_case(mesh, p, "subcell")
    dt = pb.compute_dt(U)
    sv.set_state(U.reshape(4, -1))
    sv.set_debug(True)
    sv.stage(1, dt)
    euler_fe_check(pb, U, dt, sv.get_state(1), sv.bounds()["alpha"], max_relaxed=max_relaxed)
    _, info = pb.fe_stage(U, dt, full=True)
    bd = sv.bounds()
    np.testing.assert_allclose(bd["lo"], info["lo"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(bd["hi"], info["hi"].ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(bd["K"], info["K"].ravel(), rtol=1e-12)


def test_slip_wall_whole_steps_low_order():
    """Five whole steps (dt on the device) in the wavy channel against the oracle."""
    pb, sv, U = wall_case("wavy", 3, "lo")
    sv.set_state(U.reshape(4, -1))
    for _ in range(5):
        U, dt = pb.ssp_rk3_step(U)
        sv.step()
        assert abs(sv.diag()["last_dt"] - dt) <= 1e-13 * dt
    assert np.all(rel(sv.get_state(0), U) <= 1e-11)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wavy_channel_conservation_and_rest_state(precision):
    """No mass and no energy cross a curved wall: both conserved over 30 limited steps (the
    vertical momentum is not: the walls push), positivity, the violation statistics of the curved
    statistics kernel (density bounds held exactly, the entropy minimum to the float32 measure's
    rounding), and a gas at rest staying at rest to order sqrt(eps) of the stage precision: on
    mapped elements the per-direction momentum fluxes of a rest state are not zero, its u^L sits
    on the entropy bound to rounding, and kinetic energy is quadratic in the momentum, so the line
    search admits a coefficient of order sqrt(eps) (measured: 2.5e-8 in FP64, 1.8e-4 in float32
    after three steps, both below sqrt(eps))."""
    tol = 1e-12 if precision == "fp64" else 2e-6
    _, sv, U = wall_case("wavy", 3, "subcell", precision=precision)
    sv.set_state(U.reshape(4, -1))
    m0 = sv.diag()["mass"]
    sv.step(30)
    d = sv.diag()
    assert abs(d["mass"][0] - m0[0]) <= tol * abs(m0[0])
    assert abs(d["mass"][3] - m0[3]) <= tol * abs(m0[3])
    assert abs(d["mass"][2] - m0[2]) > 1e-5
    assert d["rho_min"] > 0 and d["p_min"] > 0 and d["nonfinite"] == 0
    assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 0.0)
    assert d["max_entropy_violation"] <= (1e-12 if precision == "fp64" else 1e-6)
    assert d["rootfind_max_iters"] > 0   # the statistics are collected (entropy root searches ran)
    X, Y = sv.node_coords()
    rest = laws.Euler(G).prim_to_cons(1.0 + 0.0 * X, 0.0 * X, 0.0 * X, 1.0 + 0.0 * X)
    sv.set_state(rest)
    sv.step(3)
    print(f"rest state, {precision}: max deviation {np.abs(sv.get_state(0) - rest).max():.3e}")
    eps = np.finfo(np.float64 if precision == "fp64" else np.float32).eps
    np.testing.assert_allclose(sv.get_state(0), rest, rtol=0, atol=4.0 * np.sqrt(eps))


@pytest.mark.parametrize("limiter", ["subcell", "elementwise"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_curved_statistics_kernel_computes_the_same_state(precision, limiter):
    """The statistics variant of the curved stage kernel (launched while statistics are on) gives
    the state of the timed variant (FP64: bit for bit; float32: to rounding, the compiler being
    free to contract the two variants' arithmetic differently), and reports the root-search
    counters and the violation maxima (zero density-bound excess; the entropy minimum to
    rounding)."""
    res = {}
    for on in (False, True):
        pb, sv, X, Y = make("euler", 3, 8, 8, limiter, L=(1.0, 1.0), precision=precision)
        sv.set_state(inputs.blast(X, Y).reshape(4, -1))
        sv.set_stats(on)
        sv.step(5)
        res[on] = (sv.get_state(0), sv.diag())
    if precision == "fp64":
        np.testing.assert_array_equal(res[True][0], res[False][0])
    else:
        assert np.all(rel(res[True][0], res[False][0]) <= 1e-6), rel(res[True][0], res[False][0])
    d = res[True][1]
    assert d["rootfind_max_iters"] > 0 and d["rootfind_cap_hits"] == 0
    assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 0.0)
    assert d["max_entropy_violation"] <= (1e-12 if precision == "fp64" else 1e-6)
    off = res[False][1]
    assert off["rootfind_max_iters"] == 0 and off["max_bound_violation"] == 0.0
