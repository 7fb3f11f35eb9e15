"""Adjoint of implicit steps (mpm_adjoint, mpm_adjoint_step) against the
oracle's gradient by its definition: central differences of the oracle's
converged solves, per parameter and along random directions (one step, three
steps, the coarse random-field slope), the conductivity of a u-p column, and
through the torch.autograd wrappers.  No test uses the GPU's own solve as
its reference."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2507_09435_gb300 import mpm, scenes as S

pytestmark = pytest.mark.gpu


def _dp_scene():
    """A small Drucker-Prager block on a fixed base, compressed from the top
    by 1 % so that part of it yields."""
    sc = S.tiny_scene(2, S.MODEL_NH_DP, seed=41, ncell=3, ppc=2, jitter=0.1)
    nx1, ny1 = sc.n[0] + 1, sc.n[1] + 1
    nodes = np.arange(sc.nnode)
    ix, iy = nodes % nx1, (nodes // nx1) % ny1
    base = nodes[iy <= 3]
    top = nodes[iy >= 6]
    dof = np.concatenate([base * 2, base * 2 + 1, top * 2, top * 2 + 1])
    val = np.concatenate([np.zeros(2 * base.size), np.zeros(top.size), np.full(top.size, -3e-3)])
    order = np.argsort(dof)
    step = S.LoadStep(dof[order].astype(np.int64), val[order], (0.0, -9.81, 0.0))
    return sc, step


def test_adjoint_matches_oracle_gradient_fp64():
    sc, step = _dp_scene()
    rng = np.random.default_rng(5)
    c = rng.standard_normal((sc.np, 3))
    c[:, 2] = 0.0

    def loss(du, dup):
        return float(np.sum(c * dup))

    gs = mpm.GpuScene(sc, newton_tol=1e-12, newton_maxit=30, forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13)
    gs.solve_staged(step)
    gE, gP, _ = gs.adjoint(dL_dx=c)
    dup = gs.particle_increment()
    # the loss on the GPU's increments equals the oracle's at the same state
    make = lambda: O.OracleScene.from_scene(sc)
    out = make().solve_step(step.dof, step.value, step.gravity, tol=1e-13, commit=False)
    orc = make()
    assert np.abs(dup - O.particle_increments(orc, out["du"])).max() < 1e-9 * np.abs(dup).max()
    _, _, modes = orc.residual(out["du"], with_mode=True)
    assert (modes > 0).sum() >= 3, "the step should drive particles plastic"
    idx = list(range(0, sc.np, max(1, sc.np // 12)))
    fdE = np.array([O.step_gradient_fd(make, step, loss, "E", p) for p in idx])
    fdP = np.array([O.step_gradient_fd(make, step, loss, "phi", p) for p in idx])
    assert np.abs(gE[idx] - fdE).max() <= 1e-5 * np.abs(fdE).max(), (gE[idx], fdE)
    assert np.abs(gP[idx] - fdP).max() <= 1e-5 * max(np.abs(fdP).max(), 1e-300), (gP[idx], fdP)
    gs.close()


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_MIXED])
def test_adjoint_directional_derivative_footing(precision):
    """Coarse footing, first settlement step after the geostatic step: the
    adjoint's directional derivative along random E and phi directions
    against central differences of the oracle's FP64 solve of the same two
    steps (eps = 1e-6 relative along the direction)."""
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    rng = np.random.default_rng(9)
    c = rng.standard_normal((sc.np, 3))
    c[:, 2] = 0.0
    E0 = np.full(sc.np, sc.materials[0].E)
    P0 = np.full(sc.np, sc.materials[0].phi)
    vE = rng.standard_normal(sc.np) * E0
    vP = rng.standard_normal(sc.np)

    gs = mpm.GpuScene(sc, precision=precision, newton_tol=1e-12 if precision == mpm.MPM_FP64 else 1e-9,
                      newton_maxit=32, forcing=mpm.MPM_FORCING_FIXED,
                      krylov_rtol=1e-13 if precision == mpm.MPM_FP64 else 1e-7)
    gs.solve_step(sc.steps[0])          # geostatic step (committed)
    gs.set_params(E_p=E0, phi_p=P0)
    gs.solve_staged(sc.steps[1])
    gE, gP, _ = gs.adjoint(dL_dx=c)
    gs.close()

    def oracle_loss(E, P, modes=None):
        orc = O.OracleScene.from_scene(sc)
        st = sc.steps[0]
        assert orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, maxit=40)["converged"]
        orc.params[:, 0] = E
        orc.params[:, 2] = P
        st = sc.steps[1]
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, maxit=40, commit=False)
        assert out["converged"]
        if modes is not None:
            modes.append(orc.residual(out["du"], with_mode=True)[2])
        return float(np.sum(c * O.particle_increments(orc, out["du"])))

    modes = []
    oracle_loss(E0, P0, modes)
    assert (modes[0] > 0).sum() >= 10, "the settlement step should drive particles plastic"
    eps = 1e-6
    for v, g, which in ((vE, gE, "E"), (vP, gP, "phi")):
        Ls = []
        for sgn in (1.0, -1.0):
            E = E0 + sgn * eps * vE if which == "E" else E0
            P = P0 + sgn * eps * vP if which == "phi" else P0
            Ls.append(oracle_loss(E, P))
        fd = (Ls[0] - Ls[1]) / (2 * eps)
        ad = float(np.dot(g, v))
        tol = 1e-4 if precision == mpm.MPM_FP64 else 1e-3
        assert abs(ad - fd) <= tol * abs(fd), (which, ad, fd)


def test_adjoint_conductivity_terzaghi():
    """u-p column: dL/dk (per material) for a loss on the nodal pressures and
    displacements, against the oracle's central difference in log k."""
    h = 0.5
    sc = S.terzaghi(ncell=20, dt=0.5 * h * h / 1.8e-6, nsteps=2)
    B = sc.B
    rng = np.random.default_rng(3)
    cU = rng.standard_normal(sc.nnode * B)
    cU[2::3] *= 1e-3      # pressure entries on the scale of 1/Pa vs 1/m

    def loss(du, dup):
        return float(np.dot(cU, du))

    gs = mpm.GpuScene(sc, krylov=mpm.MPM_GMRES, newton_tol=1e-11, newton_maxit=30,
                      forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13)
    gs.solve_staged(sc.steps[0], tol=1e-11)
    _, _, gK = gs.adjoint(dL_dU=cU, want_E=False, want_phi=False, want_k=True)
    make = lambda: O.OracleScene.from_scene(sc)
    fd = O.step_gradient_fd(make, sc.steps[0], loss, "k", 0, rel=1e-5, tol=1e-12)
    k = sc.materials[0].k_hyd
    assert abs(gK[0] * k - fd) <= 1e-4 * abs(fd), (gK[0] * k, fd)
    gs.close()


def test_autograd_function_matches_adjoint():
    import torch
    from paper_2507_09435_gb300.autograd import ImplicitStep
    sc, step = _dp_scene()
    gs = mpm.GpuScene(sc, newton_tol=1e-12, newton_maxit=30, forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13)
    E = torch.full((sc.np,), sc.materials[0].E, dtype=torch.float64, requires_grad=True)
    P = torch.full((sc.np,), sc.materials[0].phi, dtype=torch.float64, requires_grad=True)
    du = ImplicitStep.apply(gs, step, E, P)
    w = torch.linspace(-1.0, 1.0, du.numel(), dtype=torch.float64).reshape(du.shape)
    (du * w).sum().backward()
    c = np.zeros((sc.np, 3))
    c[:, :2] = w.numpy()
    gE, gP, _ = gs.adjoint(dL_dx=c)
    # two adjoint solves agree to their tolerance (atomic summation order differs)
    assert np.abs(E.grad.numpy() - gE).max() <= 1e-8 * np.abs(gE).max()
    assert np.abs(P.grad.numpy() - gP).max() <= 1e-8 * np.abs(gP).max()
    gs.commit()
    gs.close()


def _oracle_multistep_loss(sc, steps, c, which=None, index=None, delta=0.0):
    orc = O.OracleScene.from_scene(sc)
    if which == "E":
        orc.params[index, 0] += delta
    elif which == "phi":
        orc.params[index, 2] += delta
    for st in steps:
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-13, maxit=40)
        assert out["converged"]
    return float(np.sum(c * orc.x))


def test_multistep_adjoint_matches_oracle_gradient_fp64():
    """Three load steps of the plastic Drucker-Prager block; loss on the final
    particle positions.  The reverse chain through the committed states
    (positions, elastic strain, deformation gradient) against central
    differences of the oracle's three-step solve."""
    import torch
    from paper_2507_09435_gb300.autograd import ImplicitSteps
    sc, step = _dp_scene()
    steps = [step, step, step]
    rng = np.random.default_rng(17)
    c = np.zeros((sc.np, 3))
    c[:, :2] = rng.standard_normal((sc.np, 2))
    gs = mpm.GpuScene(sc, newton_tol=1e-12, newton_maxit=30, forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13)
    E = torch.full((sc.np,), sc.materials[0].E, dtype=torch.float64, requires_grad=True)
    P = torch.full((sc.np,), sc.materials[0].phi, dtype=torch.float64, requires_grad=True)
    xN = ImplicitSteps.apply(gs, steps, E, P)
    (xN * torch.from_numpy(c[:, :2])).sum().backward()
    gE, gP = E.grad.numpy(), P.grad.numpy()
    idx = list(range(0, sc.np, max(1, sc.np // 8)))
    for which, g, scale in (("E", gE, sc.materials[0].E), ("phi", gP, max(sc.materials[0].phi, 1.0))):
        fd = []
        for p in idx:
            d = 1e-5 * scale
            fd.append((_oracle_multistep_loss(sc, steps, c, which, p, d) -
                       _oracle_multistep_loss(sc, steps, c, which, p, -d)) / (2 * d))
        fd = np.array(fd)
        assert np.abs(g[idx] - fd).max() <= 1e-4 * np.abs(fd).max(), (which, g[idx], fd)
    # the scene is back at its final committed state
    part = gs.particles()
    assert np.abs(part["x"][:, :2] - xN.detach().numpy()).max() == 0.0
    gs.close()


def test_slope_multistep_directional_derivative():
    """Coarse Drucker-Prager slope with per-particle E and phi random fields
    (the inverse-analysis workload's shape, 4,284 particles, cohesion 2 kPa):
    the first three steps of a six-step gravity ramp, over which the plastic
    zone grows to about 1,300 particles; loss on the final positions of the
    surface particles.  The adjoint's directional derivatives along random
    field perturbations against central differences of the oracle's FP64
    three-step solve (eps = 1e-6 relative), each within 1e-4 of its own
    size."""
    import torch
    from paper_2507_09435_gb300.autograd import ImplicitSteps
    sc = S.slope(nx=48, ny=24, h=0.5, ppc=3, nsteps=6, found_h=6, body_h=8, crest=20, toe=32, c=2e3)
    steps = sc.steps[:3]
    ytop = sc.x[:, 1].max()
    surf = sc.x[:, 1] > ytop - 0.5 * sc.h
    rng = np.random.default_rng(23)
    c = np.zeros((sc.np, 2))
    c[surf] = rng.standard_normal((surf.sum(), 2))
    E0, P0 = sc.E_p.copy(), sc.phi_p.copy()
    vE = 0.1 * E0 * rng.standard_normal(sc.np)
    vP = 0.1 * P0 * rng.standard_normal(sc.np)

    def oracle_loss(E, P, modes=None):
        orc = O.OracleScene.from_scene(sc)
        orc.params[:, 0] = E
        orc.params[:, 2] = P
        for st in steps:
            out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, maxit=40, commit=False)
            assert out["converged"]
            if modes is not None:
                modes.append(orc.residual(out["du"], with_mode=True)[2])
            orc.commit(out["du"])
        return float(np.sum(c * orc.x[:, :2]))

    kw = dict(newton_tol=1e-11, newton_maxit=32, forcing=mpm.MPM_FORCING_FIXED, krylov_rtol=1e-13)
    gs = mpm.GpuScene(sc, **kw)
    Et = torch.tensor(E0, requires_grad=True)
    Pt = torch.tensor(P0, requires_grad=True)
    xN = ImplicitSteps.apply(gs, steps, Et, Pt)
    (xN * torch.from_numpy(c)).sum().backward()
    gs.close()
    modes = []
    L0 = oracle_loss(E0, P0, modes)
    assert abs(L0 - float(np.sum(c * xN.detach().numpy()))) <= 1e-9 * abs(L0)
    assert (modes[-1] > 0).sum() >= 500, "the ramp should drive a plastic zone"
    eps = 1e-6
    fdE = (oracle_loss(E0 + eps * vE, P0) - oracle_loss(E0 - eps * vE, P0)) / (2 * eps)
    adE = float(np.dot(Et.grad.numpy(), vE))
    assert abs(adE - fdE) <= 1e-4 * abs(fdE), (adE, fdE)
    fdP = (oracle_loss(E0, P0 + eps * vP) - oracle_loss(E0, P0 - eps * vP)) / (2 * eps)
    adP = float(np.dot(Pt.grad.numpy(), vP))
    assert abs(adP - fdP) <= 1e-4 * abs(fdP), (adP, fdP)
