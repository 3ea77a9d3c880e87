"""Batched execution (many independent instances, task table per degree, one CUDA graph per
step): every instance must equal the same instance advanced alone (bit for bit: the batched
launch runs the same tile code on the same inputs)."""
import numpy as np
import pytest

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
def test_batch_equals_instances_alone(law, precision, monkeypatch):
    # the same tile shape on both sides: different shapes are different instantiations whose
    # float roundings may differ in the last bit (checked to a tolerance below)
    monkeypatch.setenv("SIDP_TILE", "0")
    cfgs = _cfgs(law, precision)
    b = sidp.sidp_batch_create([sidp.make_config(**c) for c in cfgs])
    states = []
    for i, c in enumerate(cfgs):
        x, y = sidp.sidp_batch_node_coords(b, i)
        U = _state(law, x, y, i)
        states.append(U)
        sidp.sidp_batch_set_state(b, i, U)
    sidp.sidp_batch_step(b, 4)
    for i, c in enumerate(cfgs):
        sv = sidp.Solver(**c)
        x, y = sv.node_coords()
        sx, sy = sidp.sidp_batch_node_coords(b, i)
        np.testing.assert_array_equal(x, sx)
        sv.set_state(states[i])
        sv.step(4)
        np.testing.assert_array_equal(sidp.sidp_batch_get_state(b, i), sv.get_state(0))
        d = sidp.sidp_batch_get_diag(b, i)
        assert d["steps"] == 4 and d["t"] > 0
        assert d["max_bound_violation"] <= (1e-12 if precision == "fp64" else 1e-5)
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
