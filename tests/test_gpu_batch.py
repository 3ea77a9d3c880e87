"""Batched execution (many independent instances, task table per degree, one CUDA graph per
step): every instance of a mixed-degree batch against the FP64 oracle, stage by stage (the
strict 1e-12 bar for the unlimited and low-order updates, the conditioning-aware comparators
with the batch's captured alpha-tilde for subcell limiting), including a sample of the
512-instance benchmark mix; and every instance equal to the same instance advanced alone (bit
for bit with the degree-group launches, which run the same tile code on the same inputs; to
rounding with the single degree-switching launch, another instantiation)."""
import numpy as np
import pytest

import test_oracle_wall as tw
from fe_compare import euler_fe_check, scalar_fe_check
from oracle import laws, scheme
from paper_2004_08503_gb300 import build, inputs, sidp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sidp.load()


def _cfgs(law, precision):
    shapes = [(3, 2, 5), (5, 4, 3), (2, 7, 2), (4, 1, 7), (6, 3, 4), (3, 5, 1), (1, 6, 6)]
    cfgs = []
    for i, (nx, ny, p) in enumerate(shapes):
        h = 1.0 / max(nx, ny)
        bc = ("outflow",) * 4 if i % 2 else ("periodic",) * 4
        c = dict(law=law, p=p, nx=nx, ny=ny, precision=precision, domain=(0.0, nx * h, 0.0, ny * h), bc=bc,
                 cfl=0.4 if i % 3 else 0.5)
        if law == "advection_var":
            v = inputs.SOLID_BODY_VELOCITY
            c.update(beta=(v[0], v[2]), grad=(v[1], v[3]))
        cfgs.append(c)
    return cfgs


def _state(law, x, y, seed):
    if law == "euler":
        return inputs.four_quadrant(x, y, seed)
    if law == "advection_var":
        return inputs.solid_body(x, y)
    return inputs.burgers_pulse(x, y)


@pytest.mark.parametrize("law,precision", [("euler", "fp64"), ("euler", "mixed"), ("burgers", "fp64"),
                                           ("advection_var", "fp64"), ("advection_var", "mixed")])
@pytest.mark.parametrize("mode", ["groups", "single"])
def test_batch_equals_instances_alone(law, precision, mode, monkeypatch):
    # the same tile shape on both sides: different shapes are different instantiations whose
    # float roundings may differ in the last bit (checked to a tolerance below)
    monkeypatch.setenv("SIDP_TILE", "0")
    monkeypatch.setenv("SIDP_BATCH_LAUNCH", mode)
    cfgs = _cfgs(law, precision)
    b = sidp.sidp_batch_create([sidp.make_config(**c) for c in cfgs])
    states = []
    for i, c in enumerate(cfgs):
        x, y = sidp.sidp_batch_node_coords(b, i)
        U = _state(law, x, y, i)
        states.append(U)
        sidp.sidp_batch_set_state(b, i, U)
    if mode == "single":  # the single launch runs the timed kernels (statistics off)
        sidp.sidp_batch_set_stats(b, False)
    sidp.sidp_batch_step(b, 4)
    for i, c in enumerate(cfgs):
        sv = sidp.Solver(**c)
        x, y = sv.node_coords()
        sx, sy = sidp.sidp_batch_node_coords(b, i)
        np.testing.assert_array_equal(x, sx)
        sv.set_state(states[i])
        sv.step(4)
        if mode == "groups":
            np.testing.assert_array_equal(sidp.sidp_batch_get_state(b, i), sv.get_state(0))
        else:  # another kernel instantiation: equal to rounding
            got, ref = sidp.sidp_batch_get_state(b, i), sv.get_state(0)
            err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
            assert np.all(err <= (1e-12 if precision == "fp64" else 2e-5)), err
        d = sidp.sidp_batch_get_diag(b, i)
        assert d["steps"] == 4 and d["t"] > 0
        if mode == "groups":
            assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 0.0)
        sv.close()
    assert sidp.sidp_batch_total_nodes(b) == sum(c["nx"] * c["ny"] * (c["p"] + 1) ** 2 for c in cfgs)
    sidp.sidp_batch_destroy(b)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_tile_shapes_agree(precision, tol, monkeypatch):
    """Every tile-shape candidate gives the same update up to rounding."""
    res = []
    for t in range(4):
        monkeypatch.setenv("SIDP_TILE", str(t))
        sv = sidp.Solver(law="euler", p=3, nx=13, ny=9, precision=precision, domain=(0.0, 1.0, 0.0, 9.0 / 13.0),
                         bc=("outflow",) * 4)
        x, y = sv.node_coords()
        sv.set_state(inputs.four_quadrant(x, y, 7))
        sv.step(3)
        res.append(sv.get_state(0))
        sv.close()
    for r in res[1:]:
        err = np.max(np.abs(r - res[0]), axis=1) / np.max(np.abs(res[0]), axis=1)
        assert np.all(err <= tol), err


def test_batch_rejects_mixed_laws():
    a = sidp.make_config(law="euler", p=3, nx=2, ny=2)
    c = sidp.make_config(law="burgers", p=3, nx=2, ny=2)
    with pytest.raises(sidp.SidpError):
        sidp.sidp_batch_create([a, c])


# p = 1..7, ragged meshes (partial element tiles), periodic and outflow sides, two instances of
# p = 3 so that one degree group holds several instances
ORACLE_SHAPES = [(5, 3, 1, "periodic"), (4, 4, 2, "outflow"), (3, 5, 3, "periodic"), (6, 2, 3, "outflow"),
                 (3, 3, 4, "outflow"), (2, 3, 5, "periodic"), (3, 2, 6, "outflow"), (2, 2, 7, "periodic")]


def _oracle_batch(lawname, limiter):
    law = laws.Euler(1.4) if lawname == "euler" else laws.Burgers()
    pbs, cfgs, U0 = [], [], []
    for i, (nx, ny, p, bc) in enumerate(ORACLE_SHAPES):
        dom = (0.0, nx / max(nx, ny), 0.0, ny / max(nx, ny))
        pb = scheme.Problem(law, p, nx, ny, domain=dom, bc=(bc,) * 4, limiter=limiter)
        pbs.append(pb)
        cfgs.append(dict(law=lawname, p=p, nx=nx, ny=ny, precision="fp64", domain=dom, bc=(bc,) * 4,
                         limiter=limiter))
        X, Y = pb.node_coords()
        if lawname == "euler":  # a density bump, a contact and a shear layer with a pressure jump
            U = law.prim_to_cons(*tw._data(X, Y))
        else:
            U = inputs.burgers_pulse(X, Y)
        U0.append(U)
    b = sidp.sidp_batch_create([sidp.make_config(**c) for c in cfgs])
    sidp.sidp_batch_set_stats(b, False)  # the timed kernels
    return pbs, b, U0


@pytest.mark.parametrize("limiter", ["none", "lo"])
def test_batch_stages_match_oracle_strict(limiter):
    """Stages 1, 2, 3 of every instance of a mixed-degree Euler batch (FP64) against the oracle's
    SSP-RK3 stages, 1e-12 normwise per field."""
    pbs, b, U0 = _oracle_batch("euler", limiter)
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(4, -1))
    dts = np.array([pb.compute_dt(U) for pb, U in zip(pbs, U0)])
    cur = list(U0)
    for k in (1, 2, 3):
        sidp.sidp_batch_stage(b, k, dts)
        for i, pb in enumerate(pbs):
            exp = pb.stage(cur[i], U0[i], dts[i], k)
            got = sidp.sidp_batch_get_buffer(b, i, (1, 2, 0)[k - 1])
            err = np.max(np.abs(got - exp.reshape(4, -1)), axis=1) / np.max(np.abs(exp), axis=(1, 2))
            assert np.all(err <= 1e-12), (i, k, err)
            cur[i] = exp
    sidp.sidp_batch_destroy(b)


@pytest.mark.parametrize("mode", ["groups", "single", "groups-line"])
@pytest.mark.parametrize("lawname", ["euler", "burgers"])
def test_batch_limited_stages_match_oracle(lawname, mode, monkeypatch):
    """The subcell-limited forward-Euler operator of every instance, from the oracle's SSP-RK3
    stage-k input, against the oracle with the conditioning-aware comparators (the alpha-tilde
    of each instance from the batch's debug capture); with the concurrent degree-group launches,
    with the single degree-switching launch, and with the line kernel in every degree group
    (Euler: tile candidate 4)."""
    if mode == "groups-line":
        if lawname != "euler":
            pytest.skip("the line kernel is an Euler kernel")
        monkeypatch.setenv("SIDP_TILE", "4")
        mode = "groups"
    monkeypatch.setenv("SIDP_BATCH_LAUNCH", mode)
    pbs, b, U0 = _oracle_batch(lawname, "subcell")
    nc = U0[0].shape[0]
    sidp.sidp_batch_set_debug(b, True)
    dts = np.array([pb.compute_dt(U) for pb, U in zip(pbs, U0)])
    cur = list(U0)
    for k in (1, 2, 3):
        for i, U in enumerate(cur):
            sidp.sidp_batch_set_state(b, i, U.reshape(nc, -1))
        sidp.sidp_batch_stage(b, 1, dts)
        for i, pb in enumerate(pbs):
            got = sidp.sidp_batch_get_buffer(b, i, 1)
            alpha = sidp.sidp_batch_get_bounds(b, i)["alpha"]
            if lawname == "euler":
                euler_fe_check(pb, cur[i], dts[i], got, alpha)
            else:
                scalar_fe_check(pb, cur[i], dts[i], got, alpha)
        cur = [pb.stage(cur[i], U0[i], dts[i], k) for i, pb in enumerate(pbs)]
    # the RK combinations of stages 2 and 3 through the batch, from the same inputs
    for i, U in enumerate(U0):
        sidp.sidp_batch_set_state(b, i, U.reshape(nc, -1))
    sidp.sidp_batch_stage(b, 1, dts)
    sidp.sidp_batch_stage(b, 2, dts)
    for i, pb in enumerate(pbs):
        u1 = sidp.sidp_batch_get_buffer(b, i, 1).reshape(U0[i].shape)
        exp = 0.75 * U0[i] + 0.25 * pb.fe_stage(u1, dts[i])
        got = sidp.sidp_batch_get_buffer(b, i, 2).reshape(U0[i].shape)
        fe_part = (got - 0.75 * U0[i]) / 0.25
        alpha = sidp.sidp_batch_get_bounds(b, i)["alpha"]
        check = euler_fe_check if lawname == "euler" else scalar_fe_check
        check(pb, u1, dts[i], fe_part, alpha, tol=1e-11)
        assert np.max(np.abs(got - exp)) <= 1e-3 * np.max(np.abs(exp))
    sidp.sidp_batch_destroy(b)


def test_benchmark_batch_mix_sampled_against_oracle():
    """The 512-instance benchmark mix (elements per side in {8,16,32,64}, p in 2..7, seeded
    four-quadrant data) in FP64: one limited stage of the whole batch on the GPU; for two
    instances of every degree, the oracle recomputes a sample of elements (random, corners)."""
    shapes = inputs.batch_shapes(0, 512)
    cfgs = [sidp.make_config(law="euler", p=p, nx=nel, ny=nel, precision="fp64", bc=("outflow",) * 4)
            for nel, p in shapes]
    b = sidp.sidp_batch_create(cfgs)
    sidp.sidp_batch_set_stats(b, False)
    sidp.sidp_batch_set_debug(b, True)
    states = []
    for i in range(len(shapes)):
        x, y = sidp.sidp_batch_node_coords(b, i)
        states.append(inputs.four_quadrant(x, y, 100003 * 0 + i))
        sidp.sidp_batch_set_state(b, i, states[i])
    law = laws.Euler(1.4)
    picks = []
    for p in range(2, 8):
        picks += [i for i, (nel, q) in enumerate(shapes) if q == p][:2]
    pbs = {i: scheme.Problem(law, shapes[i][1], shapes[i][0], shapes[i][0], bc=("outflow",) * 4) for i in picks}
    # the sampled instances take their CFL time step; the others a step far below theirs
    dts = np.array([pbs[i].compute_dt(states[i].reshape(4, shapes[i][0] ** 2, -1)) if i in pbs else 1e-6
                    for i in range(len(shapes))])
    sidp.sidp_batch_stage(b, 1, dts)
    rng = np.random.default_rng(3)
    for i in picks:
        pb = pbs[i]
        nel = shapes[i][0]
        U = states[i].reshape(4, pb.Ne, -1)
        sample = np.unique(np.concatenate([rng.integers(0, pb.Ne, 12), [0, nel - 1, pb.Ne - nel, pb.Ne - 1]]))
        got = sidp.sidp_batch_get_buffer(b, i, 1).reshape(4, pb.Ne, -1)[:, sample]
        alpha = sidp.sidp_batch_get_bounds(b, i)["alpha"].reshape(pb.Ne, -1)[sample]
        euler_fe_check(pb, U, dts[i], got, alpha, elems=sample)
    sidp.sidp_batch_destroy(b)
