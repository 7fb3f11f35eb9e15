"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs: residual, Jacobian blocks, converged increments and the
committed particle state.  Sizes span several cells/tiles with ragged cell
occupancy; plastic, apex and repeated-eigenvalue states are exercised through
random increments set with mpm_set_du."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2507_09435_gb300 import mpm, scenes as S

from parity_util import (DU_TOL, JAC_TOL_FP64, JAC_TOL_MIXED, RES_TOL, du_error, fixed_mask, jacobian_error,
                         residual_error)

pytestmark = pytest.mark.gpu


def _run_parity(sc, nsteps, precision=mpm.MPM_FP64, jac_every_step=True, expect_plastic=False,
                expect_globalised=False, **kw):
    orc = O.OracleScene.from_scene(sc)
    gs = mpm.GpuScene(sc, precision=precision, newton_tol=1e-12, newton_maxit=30,
                      forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13 if precision == mpm.MPM_FP64 else 1e-6,
                      krylov_maxit=20000, **kw)
    saw_plastic = False
    jtol = JAC_TOL_FP64 if precision == mpm.MPM_FP64 else JAC_TOL_MIXED
    for k, st in enumerate(sc.steps[:nsteps]):
        fixed = fixed_mask(sc, st)
        orc.gravity = np.asarray(st.gravity, dtype=np.float64)
        rep = gs.begin(st)
        du = gs.du()
        assert residual_error(gs, orc, du, fixed) < RES_TOL
        if jac_every_step or k == 0:
            gs.assemble()
            ej, ng, no = jacobian_error(gs, orc, du, fixed)
            assert ej < jtol, (k, ej)
            assert ng == no
        # both sides are driven to a relative residual of 1e-13 (or the GPU's
        # rounding floor) so that the increment comparison is not limited by
        # kappa(J) times the stopping tolerance
        it = 0
        rel, best = 1.0, 1.0
        floor = False
        while rel > 1e-13 and it < 40:
            nr = gs.newton()
            it += 1
            rel = nr.rel_residual
            saw_plastic |= nr.n_plastic > 0
            assert residual_error(gs, orc, gs.du(), fixed) < RES_TOL
            if rel < 1e-10 and rel > 0.5 * best:
                floor = True
                break   # at the rounding floor
            best = min(best, rel)
        # 1e-12, or a rounding floor just above it (the first steps of a
        # gravity ramp carry loads small against the stresses' rounding)
        assert rel <= 1e-12 or (floor and best <= 2e-12), (k, rel, best)
        du_g = gs.du()
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-13, maxit=40)
        assert out["hist"][-1] <= 1e-12, out["hist"]   # 1e-13 or the oracle's own rounding floor
        assert du_error(du_g, out["du"]) < DU_TOL, (k, du_error(du_g, out["du"]))
        gs.commit()
        part = gs.particles()
        scale_x = np.abs(orc.x).max()
        assert np.abs(part["x"] - orc.x).max() < 1e-12 * scale_x + DU_TOL * np.abs(out["du"]).max()
        assert np.abs(part["F"] - orc.F.reshape(-1, 3, 3)).max() < 1e-6
        assert np.abs(part["be"] - orc.be).max() < 1e-6
        if sc.materials[0].model == S.MODEL_NH_MCC:
            assert np.abs(part["pc"] - orc.pc).max() < 1e-6 * np.abs(orc.pc).max()
    if expect_plastic:
        assert saw_plastic
    if expect_globalised:
        limited, halvings = mpm.mpm_get_newton_counters(gs.h)
        assert limited + halvings > 0, (limited, halvings)
    gs.close()


def test_block_compression_fp64():
    """1,024-particle Neo-Hookean block, 5 load steps (32x32 grid)."""
    _run_parity(S.block_compression(), 5)


def test_block_compression_matches_homogeneous_closed_form():
    sc = S.block_compression()
    gs = mpm.GpuScene(sc, newton_tol=1e-12, krylov_rtol=1e-13)
    mu, lam = 1e6 / 2.6, 1e6 * 0.3 / (1.3 * 0.4)
    for k, st in enumerate(sc.steps):
        rep = gs.solve_step(st)
        assert rep.converged
        l2 = 0.999 ** (k + 1)
        l1 = 1.0
        for _ in range(50):
            g = mu * (l1 * l1 - 1) + lam * np.log(l1 * l2)
            l1 -= g / (2 * mu * l1 + lam / l1)
        F = gs.particles()["F"]
        assert np.abs(F - np.diag([l1, l2, 1.0])[None]).max() < 1e-10
    gs.close()


def test_footing_coarse_fp64_plastic():
    """Coarsened footing (46x22 soil cells, 4,048 particles): geostatic step
    plus footing steps of 0.5 cm that drive Drucker-Prager particles plastic."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    _run_parity(sc, 4, jac_every_step=True, expect_plastic=True)


def test_footing_coarse_fp64_large_increments():
    """The coarse footing pushed 4 cm per step (8 % of a cell), geostatic step
    plus three increments.  The first increment takes about two dozen Newton
    iterations on both sides, most of them scaled by the step-length limit or
    halved: the globalised, strongly plastic regime, compared iterate by
    iterate (residual) and at convergence (Jacobian, increment, state).  The
    fourth increment (16 cm in all) meets the bearing-failure mechanism: there
    neither side converges, and the GPU reports it without committing."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=5, settle_frac=0.1)
    _run_parity(sc, 4, jac_every_step=True, expect_plastic=True, expect_globalised=True)
    orc = O.OracleScene.from_scene(sc)
    for st in sc.steps[:4]:
        assert orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, maxit=40)["converged"]
    st = sc.steps[4]
    assert not orc.solve_step(st.dof, st.value, st.gravity, tol=1e-8, maxit=30, commit=False)["converged"]
    gs = mpm.GpuScene(sc, precision=mpm.MPM_FP64, newton_tol=1e-8, newton_maxit=30)
    for s_ in sc.steps[:4]:
        assert gs.solve_step(s_).converged
    x_before = gs.particles(be=False, pc=False, F=False, tau=False)["x"]
    gs.set_step(st)
    rep = mpm.mpm_solve_step(gs.h, check=False)
    assert rep.status != 0 and not rep.converged
    assert np.array_equal(gs.particles(be=False, pc=False, F=False, tau=False)["x"], x_before)
    gs.close()


@pytest.mark.parametrize("krylov", [mpm.MPM_BICGSTAB, mpm.MPM_GMRES])
def test_segment_preconditioner_footing_fp64(krylov):
    """Row-segment block-Jacobi (4 consecutive active nodes per block) on the
    coarse footing: the converged steps match the oracle as with node blocks."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    _run_parity(sc, 3, jac_every_step=False, expect_plastic=True, precond=mpm.MPM_PC_SEG4, krylov=krylov)


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
def test_modified_newton_reaches_the_newton_increment(precision):
    """Jacobian reuse (modified Newton, reassembled every second iteration):
    the plastic coarse footing and the 3D Cam-Clay column converge to the
    increments of full Newton, with fewer assemblies than iterations, and
    the converged increment matches the oracle's."""
    cases = [(S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1), 3),
             (S.column_collapse_3d(nx=12, ny=12, nz=12, h=0.1, col=(4, 4, 6), nsteps=6, pc_mean=-1.2e4, E=1e6), 3)]
    for sc, nsteps in cases:
        # mixed: driven to 1e-10, so that the increment comparison is not
        # limited by kappa(J) times the stopping tolerance
        tol = 1e-12 if precision == mpm.MPM_FP64 else 1e-10
        kw = dict(precision=precision, newton_tol=tol, newton_maxit=32)
        full = mpm.GpuScene(sc, **kw)
        mod = mpm.GpuScene(sc, jacobian_reuse=2, **kw)
        orc = O.OracleScene.from_scene(sc)
        for st in sc.steps[:nsteps]:
            rf = full.solve_step(st)
            rm = mod.solve_step(st)
            assert rf.converged and rm.converged
            assert rm.newton_iters >= rf.newton_iters
            out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, maxit=40)
            assert out["converged"]
            du_o = np.asarray(out["du"])
            fixed = fixed_mask(sc, st)
            scale = max(np.abs(du_o[~fixed]).max(), 1e-300)
            bar = DU_TOL if precision == mpm.MPM_FP64 else 1e-5
            assert np.abs(mod.du() - du_o)[~fixed].max() / scale < bar
            assert np.abs(mod.du() - full.du())[~fixed].max() / scale < bar
        full.close()
        mod.close()


def test_segment_preconditioner_column_3d_fp64():
    sc = S.column_collapse_3d(nx=12, ny=12, nz=12, h=0.1, col=(4, 4, 6), nsteps=3, pc_mean=-8e3, E=1e6)
    _run_parity(sc, 1, jac_every_step=False, expect_plastic=True, precond=mpm.MPM_PC_SEG4)


@pytest.mark.parametrize("dim,model,amp", [(2, S.MODEL_NH, 0.03), (2, S.MODEL_NH_DP, 0.03),
                                           (3, S.MODEL_NH_MCC, 0.01), (3, S.MODEL_NH_DP, 0.02),
                                           (3, S.MODEL_NH, 0.03), (2, S.MODEL_NH_MCC, 0.02)])
@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
def test_random_states(dim, model, amp, precision):
    """Residual and Jacobian at random increments (plastic and apex branches,
    jittered particles, ragged cell occupancy)."""
    sc = S.tiny_scene(dim, model, seed=11 + dim + model, ncell=3 if dim == 2 else 2, ppc=3 if dim == 2 else 2)
    # fix the bottom layer so that J is non-singular
    n = sc.n
    nx1, ny1 = n[0] + 1, n[1] + 1
    nodes = np.arange(sc.nnode)
    iy = (nodes // nx1) % ny1
    dof = np.concatenate([nodes[iy <= 3] * dim + a for a in range(dim)])
    step = S.LoadStep(np.sort(dof).astype(np.int64), np.zeros(dof.size), (0.0, -9.81, 0.0))
    fixed = fixed_mask(sc, step)
    orc = O.OracleScene.from_scene(sc)
    orc.gravity = np.array(step.gravity)
    gs = mpm.GpuScene(sc, precision=precision)
    gs.begin(step)
    _, M = orc.residual(np.zeros(sc.nnode * dim))
    act = orc.active_dofs(M)
    du = S.random_increment(sc, amp, seed=5)
    du[~act] = 0.0
    du[fixed] = 0.0
    gs.set_du(du)
    _, _, modes = orc.residual(du, with_mode=True)
    if model != S.MODEL_NH:
        assert (modes > 0).sum() >= 3
    assert residual_error(gs, orc, du, fixed) < RES_TOL
    gs.assemble()
    ej, ng, no = jacobian_error(gs, orc, du, fixed)
    assert ej < (JAC_TOL_FP64 if precision == mpm.MPM_FP64 else JAC_TOL_MIXED), ej
    gs.close()


def test_column_3d_mcc_fp64():
    """Small 3D modified Cam-Clay column (4x4x6 cells, 768 particles): the
    first three steps of a six-step gravity ramp with a low preconsolidation,
    so that the plastic zone grows from 1 to 22 to about 150 particles.  (The
    same column under 20 g, or carried past half of g, has no equilibrium:
    the unconfined Cam-Clay column collapses and Newton stalls on both
    sides.)"""
    sc = S.column_collapse_3d(nx=12, ny=12, nz=12, h=0.1, col=(4, 4, 6), nsteps=6, pc_mean=-1.2e4, E=1e6)
    _run_parity(sc, 3, jac_every_step=True, expect_plastic=True)


def test_oedometer_3d_mcc_fp64():
    """3D oedometric compression of a normally consolidated Cam-Clay cube
    (512 particles, prestressed): every particle plastic, four load steps."""
    _run_parity(S.oedometer_3d(), 4, jac_every_step=True, expect_plastic=True)


def test_oedometer_3d_dp_fp64():
    """The same oedometer with Drucker-Prager soil (3D spectral DP return)."""
    _run_parity(S.oedometer_3d(model=S.MODEL_NH_DP, strain_per_step=5e-3, phi=5.0, c=0.0), 3,
                jac_every_step=True, expect_plastic=True)


def test_mixed_precision_footing_converges_and_states_error():
    """Mixed mode (FP32 Jacobian and Krylov, FP64 residual/return map/check)
    reaches the 1e-8 Newton tolerance; its increment is within the stated
    error of the FP64 oracle's."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    orc = O.OracleScene.from_scene(sc)
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
    for k, st in enumerate(sc.steps[:3]):
        gs.set_step(st)
        rep = mpm.mpm_solve_step(gs.h, check=False)
        assert rep.converged, (rep.status, mpm.lib().mpm_last_error(gs.h).decode(),
                               [rep.hist[i] for i in range(rep.newton_iters + 1)])
        assert rep.rel_residual <= 1e-8
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12)
        part = gs.particles()
        # stated error of the mixed form against the FP64 oracle
        ex = np.abs(part["x"] - orc.x).max() / np.abs(out["du"]).max()
        assert ex < 1e-5, ex
    gs.close()


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
def test_persistent_krylov_path_matches_graph_path(precision, monkeypatch):
    """The single cooperative BiCGStab kernel (MPM_KRYLOV_PERSISTENT=1)
    converges to the same step as the default CUDA-graph form."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    out = []
    for persistent in ("0", "1"):
        monkeypatch.setenv("MPM_KRYLOV_PERSISTENT", persistent)
        gs = mpm.GpuScene(sc, precision=precision, newton_tol=1e-10, forcing=mpm.MPM_FORCING_FIXED,
                          krylov_rtol=1e-12 if precision == mpm.MPM_FP64 else 1e-6)
        for st in sc.steps[:2]:
            rep = gs.solve_step(st)
            assert rep.converged
        out.append(gs.particles()["x"])
        gs.close()
    scale = np.abs(out[0] - sc.x).max()
    assert np.abs(out[0] - out[1]).max() < (1e-8 if precision == mpm.MPM_FP64 else 1e-5) * scale


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
@pytest.mark.parametrize("restart", [30, 8])
def test_gmres_matches_oracle_step(precision, restart):
    """GMRES(m) with block-Jacobi (CGS2) converges each load step to the
    oracle's solution: FP64 to the increment parity bar, mixed within the
    stated mixed-mode error."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    orc = O.OracleScene.from_scene(sc)
    tight = precision == mpm.MPM_FP64
    gs = mpm.GpuScene(sc, precision=precision, krylov=mpm.MPM_GMRES, gmres_restart=restart,
                      newton_tol=1e-12 if tight else 1e-8, newton_maxit=30, forcing=mpm.MPM_FORCING_FIXED,
                      krylov_rtol=1e-13 if tight else 1e-6)
    for st in sc.steps[:2]:
        gs.set_step(st)
        rep = mpm.mpm_solve_step(gs.h, check=False)
        assert rep.converged, (rep.status, mpm.lib().mpm_last_error(gs.h).decode())
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12)
        part = gs.particles()
        err = np.abs(part["x"] - orc.x).max() / np.abs(out["du"]).max()
        assert err < (DU_TOL if tight else 1e-5), err
    gs.close()


def test_empty_scene_and_state_errors():
    sc = S.block_compression()
    d = mpm.make_desc(2, sc.n, sc.h)
    h = mpm.mpm_create_scene(d, np.zeros((0, 2)), np.zeros(0), np.zeros(0), np.zeros(0, np.int32),
                             mpm.materials_of(sc))
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_newton_step(h)
    assert e.value.status == 11
    rep = mpm.mpm_solve_step(h)
    assert rep.converged and rep.newton_iters == 0
    mpm.mpm_destroy_scene(h)


def test_particle_leaving_grid_is_reported():
    """A prescribed increment that pushes particles out of the grid makes the
    next load step fail with MPM_ERR_BOUNDS (flag raised in the kernels)."""
    sc = S.block_compression()
    gs = mpm.GpuScene(sc, newton_maxit=3)
    nodes = np.arange(sc.nnode)
    dof = np.concatenate([nodes * 2, nodes * 2 + 1])
    val = np.concatenate([np.full(sc.nnode, -2.5 * sc.h), np.zeros(sc.nnode)])
    step = S.LoadStep(dof.astype(np.int64), val, (0.0, 0.0, 0.0))
    gs.set_step(step)
    rep = mpm.mpm_solve_step(gs.h, check=False)
    assert rep.status == 0
    with pytest.raises(mpm.MPMError) as e:
        gs.begin(step)
    assert e.value.status == 9
    gs.close()
