"""Device-pointer variants of the boundary, determinism, and failures made on
the host (no GPU fault):

* mpm_get_du_dev / mpm_get_residual_dev / mpm_get_positions_dev write into
  caller-owned CUDA tensors exactly what the host getters return (u-p
  pressure in physical units), and mpm_set_dirichlet_dev stages the same step
  as mpm_set_dirichlet;
* the residual and the Jacobian at a given increment are reproducible bit
  for bit (every sum is taken in a fixed order), and so is a whole 3D load
  step with its Krylov iteration counts;
* an infinite Young's modulus injected into one particle is reported as
  MPM_ERR_NONFINITE (or MPM_ERR_RETURN_MAP), a Newton limit of one iteration as
  MPM_ERR_NOT_CONVERGED with the particles left uncommitted, and the scene
  stays usable afterwards.
"""
import numpy as np
import pytest

from paper_2507_09435_gb300 import mpm, scenes as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scenes():
    return [S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1), S.terzaghi(ncell=20, dt=5e4, nsteps=3)]


def _kw(sc):
    # the u-p column is solved with GMRES(30), as in its parity tests
    return dict(precision=mpm.MPM_FP64, newton_tol=1e-10, newton_maxit=30,
                krylov=mpm.MPM_GMRES if sc.formulation == "up" else mpm.MPM_BICGSTAB)


@pytest.mark.parametrize("k", [0, 1])
def test_device_getters_match_host(k):
    sc = _scenes()[k]
    gs = mpm.GpuScene(sc, **_kw(sc))
    gs.solve_step(sc.steps[0])
    gs.begin(sc.steps[1])
    gs.newton()
    dev = torch.device("cuda:0")
    du_t = torch.full((gs.ndof,), np.nan, dtype=torch.float64, device=dev)
    r_t = torch.full((gs.ndof,), np.nan, dtype=torch.float64, device=dev)
    x_t = torch.full((gs.np * 3,), np.nan, dtype=torch.float64, device=dev)
    gs.du_into(du_t)
    gs.residual_into(r_t)
    gs.positions_into(x_t)
    torch.cuda.synchronize()
    assert np.array_equal(du_t.cpu().numpy(), gs.du())
    assert np.array_equal(r_t.cpu().numpy(), gs.residual())
    assert np.array_equal(x_t.cpu().numpy().reshape(-1, 3), gs.particles()["x"])
    with pytest.raises(ValueError):
        gs.du_into(torch.zeros(gs.ndof, dtype=torch.float32, device=dev))
    gs.close()


@pytest.mark.parametrize("k", [0, 1])
def test_dirichlet_dev_stages_the_same_step(k):
    sc = _scenes()[k]
    out = []
    for use_dev in (False, True):
        gs = mpm.GpuScene(sc, **_kw(sc))
        for st in sc.steps[:2]:
            if use_dev:
                gs.set_dirichlet_dev(torch.as_tensor(np.asarray(st.dof, dtype=np.int64), device="cuda:0"),
                                     torch.as_tensor(np.asarray(st.value, dtype=np.float64), device="cuda:0"))
                mpm.mpm_set_gravity(gs.h, st.gravity)
                rep = mpm.mpm_solve_step(gs.h)
            else:
                rep = gs.solve_step(st)
            assert rep.converged
        out.append(gs.particles()["x"])
        gs.close()
    # the u-p column's GMRES(30) dot products still sum with atomics, which
    # the Newton iterations carry to about their tolerance (hence a bound)
    x0 = np.zeros_like(out[0])
    x0[:, :sc.dim] = sc.x[:, :sc.dim]
    assert np.abs(out[0] - out[1]).max() <= 1e-8 * np.abs(out[0] - x0).max()


def test_dirichlet_dev_rejects_out_of_range_index():
    sc = _scenes()[0]
    gs = mpm.GpuScene(sc, precision=mpm.MPM_FP64)
    bad = torch.tensor([0, gs.ndof + 5], dtype=torch.int64, device="cuda:0")
    val = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(mpm.MPMError) as e:
        gs.set_dirichlet_dev(bad, val)
    assert "out of range" in str(e.value)
    # the scene is still usable with a valid step
    assert gs.solve_step(sc.steps[0]).converged
    gs.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_residual_and_assembly_reproducible(dim):
    """Two scenes in the same state, the same increment: the residuals agree
    bit for bit (the cells' particles in source order, each node's
    contributions added in cell and particle order), and so do the assembled
    FP32 Jacobians (3D: cell block products, then each row's 27 cells in a
    fixed order; 2D: one warp per node row of a tile, its cells in order)."""
    if dim == 2:
        sc, st = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1), 1
    else:
        sc, st = S.column_collapse_3d(nx=12, ny=12, nz=12, h=0.1, col=(4, 4, 6), nsteps=6, pc_mean=-1.2e4, E=1e6), 0
    res = []
    for _ in range(2):
        gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
        gs.begin(sc.steps[st])
        rng = np.random.default_rng(7)
        du = gs.du()
        du = du + 1e-5 * rng.standard_normal(du.shape)
        gs.set_du(du)
        gs.assemble()
        res.append((gs.residual(), gs.jacobian_bsr()))
        gs.close()
    (r0, J0), (r1, J1) = res
    assert np.array_equal(r0, r1)
    for a, b in zip(J0[:3], J1[:3]):
        assert np.array_equal(a, b)     # the same pattern
    assert np.array_equal(J0[3], J1[3])


def test_3d_load_steps_reproducible():
    """Three load steps of a 3D Cam-Clay column in mixed precision, solved
    twice on fresh scenes: the same Newton and BiCGStab iteration counts and
    the same increments bit for bit (the residual, the assembly and the
    Krylov dot products are all summed in fixed orders)."""
    sc = S.column_collapse_3d(nx=12, ny=12, nz=12, h=0.1, col=(4, 4, 6), nsteps=6, pc_mean=-1.2e4, E=1e6)
    runs = []
    for _ in range(2):
        gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
        counts = []
        for stp in sc.steps[:3]:
            rep = gs.solve_step(stp)
            assert rep.converged
            counts.append([rep.krylov_iters[i] for i in range(rep.newton_iters)])
        runs.append((counts, gs.du(), gs.particles(be=False, pc=False, F=False, tau=False)["x"]))
        gs.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])


def test_injected_infinite_modulus_is_reported():
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
    assert gs.solve_step(sc.steps[0]).converged
    E = np.full(sc.np, sc.materials[0].E)
    E[sc.np // 2] = np.inf
    gs.set_params(E_p=E)
    with pytest.raises(mpm.MPMError) as e:
        gs.solve_step(sc.steps[1])
    # the particle's stress is non-finite; its return map, which sees it first,
    # may report the failure instead
    assert str(e.value).split(":")[0] in ("MPM_ERR_NONFINITE", "MPM_ERR_RETURN_MAP"), str(e.value)
    # restoring the modulus makes the scene usable again
    E[sc.np // 2] = sc.materials[0].E
    gs.set_params(E_p=E)
    assert gs.solve_step(sc.steps[1]).converged
    gs.close()


def test_newton_limit_reports_not_converged_and_does_not_commit():
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-12, newton_maxit=1)
    x0 = gs.particles()["x"]
    rep = gs.solve_step(sc.steps[0], check=False)
    assert rep.status == 4 and not rep.converged   # MPM_ERR_NOT_CONVERGED
    assert np.array_equal(gs.particles()["x"], x0)
    gs.close()


def test_multigrid_load_steps_reproducible():
    """The coarse plastic footing with the multigrid V-cycle in mixed
    precision, solved twice on fresh scenes: the same iteration counts and
    the same increments bit for bit (the smoother's damping estimate, the
    nodal mass and every other sum in a fixed order)."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    runs = []
    for _ in range(2):
        gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8, precond=mpm.MPM_PC_MG)
        counts = []
        for stp in sc.steps[:3]:
            rep = gs.solve_step(stp)
            assert rep.converged
            counts.append([rep.krylov_iters[i] for i in range(rep.newton_iters)])
        runs.append((counts, gs.du(), gs.particles(be=False, pc=False, F=False, tau=False)["x"]))
        gs.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])
