"""Pins of the CPU oracle against values the paper prints (fixtures under
tests/golden/, each citing its table or section; no GPU).

* Table 1: block size b = 2w - 1 of the seed pattern for a shape function of
  support w.  The quadratic B-spline of the oracle has support w = 3, the
  coloured difference Jacobian with the table's b = 5 equals one-DOF-at-a-time
  differences bit for bit, and one colour fewer per axis (b = 4) mixes
  columns (a wrong stencil reach or a wrong colouring fails one of these).
* Sec. 4.3: the sparse (coloured) and dense difference Jacobians agree below
  the printed relative Frobenius bound of 1e-15.
* Sec. 4.2: on the bar under self-weight every load step reaches a relative
  residual of 1e-11 within four Newton iterations (a wrong tangent term
  slows Newton to a linear rate and fails this).
* Sec. 4.4: the consolidation column's printed data give the printed
  coefficient of consolidation and duration, and at the paper's own
  discretisation (100 cells, 2x2 particles per cell, dt = 1e5 s) the pore
  pressure follows Terzaghi's series up to T = 1.
"""
import os

import numpy as np
import pytest

from paper_2507_09435_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def _kv(name):
    return {k: float(v) for k, v in _rows(name)}


# ---------------------------------------------------------------- Table 1
def test_table1_block_size_rule():
    rows = _rows("table1_block_size.txt")
    assert len(rows) == 4
    for _, w, b in rows:
        assert int(b) == 2 * int(w) - 1


def test_quadratic_bspline_support_is_table1_w(oracle):
    w_tab = {r[0]: int(r[1]) for r in _rows("table1_block_size.txt")}["quadratic_bspline"]
    h, n, o = 0.25, (12, 12, 0), (0.0, 0.0, 0.0)
    rng = np.random.default_rng(42)
    for _ in range(40):
        xp = np.array([h * rng.uniform(3, 8), h * rng.uniform(3, 8), 0.0])
        node, wgt, _ = oracle.stencil(2, n, h, o, xp)
        ix = node % (n[0] + 1)
        # nodes that carry weight along x: exactly w consecutive ones
        on = np.unique(ix[wgt > 0])
        assert len(on) == w_tab and (np.diff(on) == 1).all()
    # a node exactly w/2 cells away carries none: the support is w cells wide
    xp = np.array([5.5 * h, 5.25 * h, 0.0])
    node, wgt, _ = oracle.stencil(2, n, h, o, xp)
    ix = node % (n[0] + 1)
    far = np.abs(ix * h - xp[0]) >= 0.5 * w_tab * h - 1e-12
    assert far.any() and np.abs(wgt[far]).max() == 0.0


def test_table1_block_size_is_the_smallest_collision_free_colouring(oracle):
    b_tab = {r[0]: int(r[2]) for r in _rows("table1_block_size.txt")}["quadratic_bspline"]
    sc = S.tiny_scene(2, S.MODEL_NH_DP, seed=11, ncell=5)
    orc = oracle.OracleScene.from_scene(sc)
    du = S.random_increment(sc, 0.02, seed=12)
    eps = 1e-6 * sc.h
    _, M = orc.residual(du)
    act = np.nonzero(orc.active_dofs(M))[0]
    Jp = oracle.fd_jacobian_plain(orc, du, eps, act)
    Jb = oracle.fd_jacobian_colored(orc, du, eps, b=b_tab)
    assert np.array_equal(Jb[:, act], Jp)
    # Sec. 4.3: sparse and dense Jacobians agree to below 1e-15 in relative
    # Frobenius norm (here they agree bit for bit)
    bound = _kv("sec43_sparse_dense_jacobian.txt")["relative_frobenius_error_below"]
    assert np.linalg.norm(Jb[:, act] - Jp) / np.linalg.norm(Jp) < bound
    Jless = oracle.fd_jacobian_colored(orc, du, eps, b=b_tab - 1)
    scale = np.abs(Jp).max()
    assert np.abs(Jless[:, act] - Jp).max() > 1e-3 * scale


# ---------------------------------------------------------------- Sec. 4.2
@pytest.mark.parametrize("ncell", [4, 16])
def test_self_weight_bar_newton_count(oracle, ncell):
    g = _kv("sec42_self_weight_newton.txt")
    sc = S.self_weight_column(ncell)
    orc = oracle.OracleScene.from_scene(sc)
    for st in sc.steps:
        # the paper's plain Newton (full steps), whose count Sec. 4.2 reports
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=g["residual_tol"], globalise=False)
        assert out["converged"] and out["iters"] <= int(g["max_newton_iterations"])
        assert out["hist"][-1] <= g["residual_tol"]


# ---------------------------------------------------------------- Sec. 4.4
def _terzaghi_series(z, T, H, nterms=400):
    s = np.zeros_like(z)
    for m in range(nterms):
        M = np.pi * (2 * m + 1) / 2
        s += 2.0 / M * np.sin(M * z / H) * np.exp(-M * M * T)
    return s


def test_consolidation_printed_coefficient_and_duration():
    g = _kv("sec44_consolidation.txt")
    # Darcy: hydraulic conductivity = k rho_f g / viscosity (water, 1e-3 Pa s);
    # c_v = conductivity / (rho_f g) * constrained modulus (lambda + 2 mu)
    mobility = g["intrinsic_permeability_m2"] / 1e-3
    cv = mobility * (g["lame_lambda_pa"] + 2 * g["lame_mu_pa"])
    assert abs(cv - g["coefficient_of_consolidation_m2_s"]) < 0.05 * g["coefficient_of_consolidation_m2_s"]
    days = g["final_time_factor"] * g["column_height_m"] ** 2 / cv / 86400.0
    assert abs(days - g["final_time_days"]) < 0.01 * g["final_time_days"]
    sc = S.terzaghi()
    assert abs(sc.meta["cv"] - cv) < 1e-9 * cv
    assert abs(sc.meta["H"] - g["column_height_m"]) < 1e-12
    assert abs(sc.meta["dt"] - g["time_step_s"]) < 1e-9
    assert abs(sc.meta["t_load"] - g["surface_load_pa"]) < 1e-12
    assert sc.n[1] - 2 == int(g["vertical_cells"]) and sc.n[0] - 2 == int(g["horizontal_cells"])
    ppa = int(g["particles_per_cell_axis"])
    assert sc.x.shape[0] == int(g["vertical_cells"] * g["horizontal_cells"]) * ppa ** 2


@pytest.mark.slow
def test_consolidation_at_the_printed_discretisation_follows_the_series(oracle):
    g = _kv("sec44_consolidation.txt")
    H, t_load, dt = g["column_height_m"], g["surface_load_pa"], g["time_step_s"]
    cv = g["coefficient_of_consolidation_m2_s"]
    nsteps = int(round(g["final_time_factor"] * H * H / cv / dt))
    sc = S.terzaghi(ncell=int(g["vertical_cells"]), dt=dt, nsteps=nsteps)
    orc = oracle.OracleScene.from_scene(sc)
    y0 = orc.x[:, 1].copy()
    checks = {int(round(T * H * H / cv / dt)): T for T in (0.1, 0.2, 0.5, g["final_time_factor"])}
    errs = {}
    for k, st in enumerate(sc.steps, start=1):
        # as the pressure decays, r^0 shrinks and the rounding floor of the
        # relative residual rises to about 1e-10 near T = 1: solve to 1e-9
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-9)
        assert out["converged"]
        if k in checks:
            T = sc.meta["cv"] * k * dt / H ** 2
            p_ref = t_load * _terzaghi_series(sc.meta["y_top"] - y0, T, H)
            errs[checks[k]] = np.abs(orc.pp - p_ref).max() / t_load
    assert len(errs) == 4
    # within 1 % of the load at every checked time factor
    assert max(errs.values()) < 0.01, errs
