"""The seeded input generators against the workloads they stand in for (no
GPU): sizes, materials, grids, loading and the statistics of the random
inputs (the Cam-Clay preconsolidation, the slope's property fields, the
serving stream's draws), and that a seed fixes every array."""
import numpy as np
import pytest

from paper_2507_09435_gb300 import scenes as S


def _lattice_ok(sc, ppc):
    """Every particle sits at a Gauss-like lattice offset inside its cell."""
    xi = sc.x[:, :sc.dim] / sc.h
    frac = xi - np.floor(xi)
    offs = (np.arange(ppc) + 0.5) / ppc
    return np.abs(frac[..., None] - offs).min(-1).max() < 1e-9


def test_block_compression_workload():
    sc = S.block_compression()
    assert sc.dim == 2 and sc.n[:2] == (32, 32) and sc.h == 1.0 / 32
    assert sc.x.shape[0] == 1024 and _lattice_ok(sc, 2)
    m = sc.materials[0]
    assert m.model == S.MODEL_NH and m.E == 1e6 and m.nu == 0.3
    assert len(sc.steps) == 5 and sc.meta["strain_per_step"] == 1e-3


def test_footing_workload():
    sc = S.footing()
    assert sc.dim == 2 and sc.n[:2] == (256, 128) and sc.h == 0.1
    assert sc.x.shape[0] == 128016 and _lattice_ok(sc, 2)
    m = sc.materials[0]
    assert (m.model, m.phi, m.psi, m.c, m.E, m.nu) == (S.MODEL_NH_DP, 30.0, 0.0, 5e3, 1e7, 0.3)
    assert len(sc.steps) == 51                     # geostatic step + 50 footing increments
    assert all(np.allclose(st.gravity, (0.0, -9.81, 0.0)) for st in sc.steps)
    # 4 mm per step on the footing nodes (0.1 B over 50 steps), nothing else moves
    moved = np.unique(sc.steps[1].value[sc.steps[1].value != 0])
    assert np.allclose(moved, [-0.1 * 2.0 / 50])
    assert np.all(sc.steps[0].value == 0)


@pytest.mark.parametrize("col,count", [((32, 32, 48), 393216), ((72, 72, 48), 1990656)])
def test_column_3d_workloads(col, count):
    sc = S.column_collapse_3d(col=col)
    assert sc.dim == 3 and sc.n == (128, 128, 64)
    assert sc.x.shape[0] == count and _lattice_ok(sc, 2)
    m = sc.materials[0]
    assert (m.model, m.M, m.lambda_cc, m.kappa_cc) == (S.MODEL_NH_MCC, 1.2, 0.1, 0.02)
    # pc0 lognormal about -100 kPa with sigma 0.1
    z = np.log(sc.pc0_p / -1e5)
    assert np.all(sc.pc0_p < 0)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 0.1) < 5e-3
    # gravity ramps 0 -> g over 20 steps
    gz = np.array([st.gravity[2] for st in sc.steps])
    assert len(gz) == 20 and np.allclose(gz, -9.81 * np.arange(1, 21) / 20)


def test_slope_workload_random_fields():
    sc = S.slope()
    assert sc.dim == 2 and sc.n[:2] == (192, 96)
    assert sc.x.shape[0] == 70704 and _lattice_ok(sc, 3)
    rel_E = sc.E_p / 1e7 - 1.0
    rel_phi = sc.phi_p / 30.0 - 1.0
    # 10 % standard deviation about E = 1e7 Pa and phi = 30 deg (standardised
    # over the whole grid; the particles sample part of it)
    for r in (rel_E, rel_phi):
        assert abs(r.mean()) < 0.05 and 0.06 < r.std() < 0.14
    # correlated over about 10 cells: neighbouring cells nearly equal, far ones not
    c = np.floor(sc.x[:, :2] / sc.h).astype(int)
    key = c[:, 0] * 1000 + c[:, 1]
    _, first = np.unique(key, return_index=True)
    cell_E = dict(zip(key[first], rel_E[first]))
    near = [(cell_E[k], cell_E[k + 1000]) for k in cell_E if k + 1000 in cell_E]
    far = [(cell_E[k], cell_E[k + 40000]) for k in cell_E if k + 40000 in cell_E]
    assert np.corrcoef(np.array(near).T)[0, 1] > 0.9
    assert abs(np.corrcoef(np.array(far).T)[0, 1]) < 0.5
    assert len(sc.steps) == 20


def test_serving_stream_draws():
    d = S.serving_draws(512)
    assert len(d) == 512
    kinds = [x["kind"] for x in d]
    for k in S.SERVING_KINDS:
        assert 0.25 < kinds.count(k) / 512 < 0.42        # uniform over three kinds
    cells = np.array([x["cells"] for x in d])
    assert cells.min() >= 1e3 and cells.max() <= 6e4
    lc = np.log(cells)
    assert abs(lc.mean() - 0.5 * (np.log(1e3) + np.log(6e4))) < 0.2   # log-uniform
    steps = np.array([x["nsteps"] for x in d])
    assert steps.min() >= 10 and steps.max() <= 40 and len(np.unique(steps)) > 20
    for x in d[:12]:
        sc, st = S.serving_scene(x, consolidation="full")
        assert len(st) == x["nsteps"]
        if x["kind"] == "up_terzaghi":
            N = sc.n[1] - 2
            assert 64 <= N <= 512 and sc.formulation == "up"
            T_end = sc.meta["cv"] * sc.dt * len(st) / sc.meta["H"] ** 2
            assert abs(T_end - 1.0) < 1e-9


def test_seed_fixes_every_array():
    a, b = S.slope(), S.slope()
    for f in ("x", "E_p", "phi_p", "vol0", "mass"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    a, b = S.column_collapse_3d(), S.column_collapse_3d()
    assert np.array_equal(a.pc0_p, b.pc0_p)
    assert S.serving_draws(64) == S.serving_draws(64)
    c = S.tiny_scene(2, S.MODEL_NH_DP, seed=5)
    assert np.array_equal(c.x, S.tiny_scene(2, S.MODEL_NH_DP, seed=5).x)
    assert not np.array_equal(c.x, S.tiny_scene(2, S.MODEL_NH_DP, seed=6).x)
