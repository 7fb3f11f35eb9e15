"""Parity of the CUDA u-p path (coupled displacement / pore pressure, paper
Sec. 2.2 remark and Sec. 4.4) with the FP64 CPU oracle, through the C ABI:
residual and Jacobian at random states (elastic and Drucker-Prager
skeletons), the Terzaghi column step by step (converged displacement and
pressure, committed particles, particle pore pressure), and the mixed
precision path on the same column with its stated error."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2507_09435_gb300 import mpm, scenes as S

from parity_util import (DU_TOL, JAC_TOL_FP64, JAC_TOL_MIXED, RES_TOL, du_error, fixed_mask, jacobian_error,
                         residual_error)

pytestmark = pytest.mark.gpu


def _up_tiny(model, seed):
    sc = S.tiny_scene(2, model, seed=seed, ncell=3, ppc=3)
    sc.formulation = "up"
    sc.dt = 1e4
    sc.materials[0].k_hyd = 9.81e-9
    return sc


@pytest.mark.parametrize("model", [S.MODEL_NH, S.MODEL_NH_DP])
@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
def test_up_random_states(model, precision):
    sc = _up_tiny(model, seed=31 + model)
    B = sc.B
    nx1, ny1 = sc.n[0] + 1, sc.n[1] + 1
    nodes = np.arange(sc.nnode)
    iy = (nodes // nx1) % ny1
    dof = np.concatenate([nodes[iy <= 3] * B + a for a in range(2)] + [nodes[iy >= 6] * B + 2])
    step = S.LoadStep(np.sort(dof).astype(np.int64), np.zeros(dof.size), (0.0, -9.81, 0.0))
    fixed = fixed_mask(sc, step)
    orc = O.OracleScene.from_scene(sc)
    orc.gravity = np.array(step.gravity)
    gs = mpm.GpuScene(sc, precision=precision)
    gs.begin(step)
    _, M = orc.residual(np.zeros(sc.nnode * B))
    act = orc.active_dofs(M)
    rng = np.random.default_rng(7)
    U = np.zeros(sc.nnode * B)
    U[0::B] = rng.standard_normal(sc.nnode) * 0.03 * sc.h
    U[1::B] = rng.standard_normal(sc.nnode) * 0.03 * sc.h
    U[2::B] = rng.standard_normal(sc.nnode) * 1e4
    U[~act] = 0.0
    U[fixed] = 0.0
    gs.set_du(U)
    assert np.abs(gs.du() - U).max() <= 1e-9 * np.abs(U).max()
    _, _, modes = orc.residual(U, with_mode=True)
    if model != S.MODEL_NH:
        assert (modes > 0).sum() >= 3
    assert residual_error(gs, orc, U, fixed) < RES_TOL
    gs.assemble()
    ej, ng, no = jacobian_error(gs, orc, U, fixed)
    assert ng == no
    assert ej < (JAC_TOL_FP64 if precision == mpm.MPM_FP64 else JAC_TOL_MIXED), ej
    gs.close()


def test_terzaghi_parity_fp64():
    """A 20-cell Terzaghi column (80 particles), six consolidation steps, each
    driven to a relative residual of 1e-11 on both sides (about the rounding
    floor of this system: with u_x fixed everywhere, lateral pressure modes
    are held only by the Darcy term); GMRES(30) with row-segment
    block-Jacobi (the u-p default)."""
    h = 0.5
    sc = S.terzaghi(ncell=20, dt=0.5 * h * h / 1.8e-6, nsteps=6)
    B = sc.B
    orc = O.OracleScene.from_scene(sc)
    gs = mpm.GpuScene(sc, newton_tol=1e-12, newton_maxit=30, forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13,
                      krylov=mpm.MPM_GMRES)
    for k, st in enumerate(sc.steps):
        fixed = fixed_mask(sc, st)
        gs.begin(st)
        U0 = gs.du()
        assert residual_error(gs, orc, U0, fixed) < RES_TOL
        gs.assemble()
        ej, ng, no = jacobian_error(gs, orc, U0, fixed)
        assert ej < JAC_TOL_FP64 and ng == no, (k, ej)
        rel, best, it = 1.0, 1.0, 0
        while rel > 1e-13 and it < 30:
            rel = gs.newton().rel_residual
            it += 1
            assert residual_error(gs, orc, gs.du(), fixed) < RES_TOL
            if it >= 3 and rel > 0.5 * best:
                break
            best = min(best, rel)
        assert min(rel, best) <= 1e-11, (k, rel)
        U = gs.du()
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-13, maxit=30)
        assert out["hist"][-1] <= 1e-11
        assert du_error(U, out["du"], B, 2) < DU_TOL, (k, du_error(U, out["du"], B, 2))
        gs.commit()
        part = gs.particles()
        assert np.abs(part["x"] - orc.x).max() < 1e-12 * np.abs(orc.x).max() + DU_TOL * np.abs(out["du"][0::3]).max()
        assert np.abs(part["F"] - orc.F.reshape(-1, 3, 3)).max() < 1e-9
        pp = gs.pressure()
        assert np.abs(pp - orc.pp).max() <= DU_TOL * np.abs(orc.pp).max()
    gs.close()


def test_terzaghi_mixed_precision_states_its_error():
    """Mixed precision (FP32 Jacobian and Krylov, FP64 residual) on the same
    column to a relative residual of 1e-10: the particle pore pressures agree
    with the FP64 oracle to 1e-7 of the load."""
    h = 0.5
    sc = S.terzaghi(ncell=20, dt=0.5 * h * h / 1.8e-6, nsteps=6)
    orc = O.OracleScene.from_scene(sc)
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-10, newton_maxit=30, krylov=mpm.MPM_GMRES)
    for st in sc.steps:
        rep = gs.solve_step(st)
        assert rep.converged
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-11)
        assert out["converged"]
    err = np.abs(gs.pressure() - orc.pp).max() / sc.meta["t_load"]
    assert err < 1e-7, err
    gs.close()


def test_up_desc_validation():
    sc = S.terzaghi(ncell=10, nsteps=1)
    with pytest.raises(mpm.MPMError):
        mpm.GpuScene(sc, dt=0.0)
