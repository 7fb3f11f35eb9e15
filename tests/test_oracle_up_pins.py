"""Pins of the CPU oracle's coupled u-p formulation (paper Sec. 2.2 remark;
Sec. 4.4 one-dimensional consolidation), no GPU.

* With zero pore pressure and zero mobility the momentum rows are those of
  the single-phase residual (a wrong sign or factor on the pressure term of
  the total stress cannot hide behind the solid part).
* The exact u-p Jacobian equals central differences of the oracle's own
  residual (coupling blocks, the flux term's dependence on dF and the
  pressure-pressure block).
* Discrete flux energy: with du = 0, sum_i p_i r_p,i = sum_p kdt V_p |grad p_p|^2
  >= 0 (the sign and the quadratic form of the Darcy term).
* Pore-pressure term: under a uniform dilation a uniform pressure p0 adds
  momentum rows with zero sum and virial -p0 (current volume) 1.
* Volume change: under a uniform dilation with zero pressure the mass-balance
  rows sum to (J - 1) sum_p V_p.
* Finite strain: the Darcy rows are unchanged by a superposed rigid rotation
  and scale by s1 / s2 under a stretch s1 across and s2 along the flow.
* Terzaghi (Sec. 4.4): pore pressure and settlement converge to the series
  solution p/p0 = sum 2/M sin(M z/H) exp(-M^2 T) and s = s_inf U(T) as the
  column is refined (time step proportional to h^2).
"""
import numpy as np
import pytest

from paper_2507_09435_gb300 import scenes as S


def _up_tiny(model, seed, kdt_scale=1.0):
    sc = S.tiny_scene(2, model, seed=seed, ncell=3)
    sc.formulation = "up"
    sc.dt = 1e4 * kdt_scale
    sc.materials[0].k_hyd = 9.81e-9
    return sc


def _random_U(sc, amp, p_amp, seed):
    rng = np.random.default_rng(seed)
    B = sc.B
    U = np.zeros(sc.nnode * B)
    U[0::B] = rng.standard_normal(sc.nnode) * amp * sc.h
    U[1::B] = rng.standard_normal(sc.nnode) * amp * sc.h
    U[2::B] = rng.standard_normal(sc.nnode) * p_amp
    return U


def test_up_momentum_rows_reduce_to_single_phase(oracle):
    sc = _up_tiny(S.MODEL_NH_DP, seed=3, kdt_scale=0.0)
    up = oracle.OracleScene.from_scene(sc)
    sc.formulation = "solid"
    so = oracle.OracleScene.from_scene(sc)
    g = np.array([0.0, -9.81, 0.0])
    up.gravity = g
    so.gravity = g
    du = S.random_increment(sc, 0.02, seed=4)
    U = np.zeros(sc.nnode * 3)
    U[0::3] = du[0::2]
    U[1::3] = du[1::2]
    ru, Mu = up.residual(U)
    rs, Ms = so.residual(du)
    assert np.array_equal(Mu, Ms)
    scale = np.abs(rs).max()
    assert np.abs(ru[0::3] - rs[0::2]).max() <= 1e-14 * scale
    assert np.abs(ru[1::3] - rs[1::2]).max() <= 1e-14 * scale


@pytest.mark.parametrize("model", [S.MODEL_NH, S.MODEL_NH_DP])
def test_up_jacobian_matches_colored_central_differences(oracle, model):
    sc = _up_tiny(model, seed=11)
    orc = oracle.OracleScene.from_scene(sc)
    orc.gravity = np.array([0.0, -9.81, 0.0])
    U = _random_U(sc, 0.02, 1e4, seed=12)
    r, M, modes = orc.residual(U, with_mode=True)
    if model != S.MODEL_NH:
        assert (modes > 0).sum() >= 4
    J = orc.jacobian(U).toarray()
    Jfd = oracle.fd_jacobian_colored(orc, U, eps=[1e-6 * sc.h, 1e-6 * sc.h, 1e-2])
    act = orc.active_dofs(M)
    Ja, Jf = J[np.ix_(act, act)], Jfd[np.ix_(act, act)]
    # compare each (row kind, column kind) block on its own scale
    B = 3
    kind = np.arange(J.shape[0])[act] % B
    for a in range(B):
        for b in range(B):
            blk = np.ix_(kind == a, kind == b)
            ref = np.abs(Ja[blk]).max()
            assert ref > 0
            assert np.abs(Ja[blk] - Jf[blk]).max() < 1e-6 * ref, (a, b)


def test_up_flux_energy_identity(oracle):
    sc = _up_tiny(S.MODEL_NH, seed=21)
    orc = oracle.OracleScene.from_scene(sc)
    U = _random_U(sc, 0.0, 1e4, seed=22)
    r, _ = orc.residual(U)
    kdt = sc.particle_kdt()
    lhs = np.dot(U[2::3], r[2::3])
    rhs = 0.0
    for p in range(sc.np):
        node, w, g = oracle.stencil(2, sc.n, sc.h, sc.origin, orc.x[p])
        G = (U[node * 3 + 2][:, None] * g).sum(axis=0)
        rhs += kdt[p] * orc.V0[p] * float(G @ G)
    assert rhs > 0
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_up_pore_pressure_virial(oracle):
    """A uniform pore pressure p0 in a body under a uniform dilation
    (1 + e) adds the momentum rows of the total-stress term -p J dF^-T; their
    virial sum_i x_i (x) dr_i over the current node positions is
    -p0 times the current volume times the identity (positive pressure in
    compression, scaled by J, pushed forward by dF^-T: a sign, a dropped J or
    a missing dF^-T fails it)."""
    sc = _up_tiny(S.MODEL_NH, seed=41)
    orc = oracle.OracleScene.from_scene(sc)
    X = sc.node_coords()[:, :2]
    e, p0 = 0.02, 3e4
    U = np.zeros(sc.nnode * 3)
    U[0::3], U[1::3] = e * X[:, 0], e * X[:, 1]
    r0, _ = orc.residual(U)
    U[2::3] = p0
    r1, _ = orc.residual(U)
    dr = (r1 - r0).reshape(-1, 3)[:, :2]
    x = (1 + e) * X
    vir = x.T @ dr
    ref = -p0 * (1 + e) ** 2 * sc.vol0.sum()
    assert np.abs(vir - ref * np.eye(2)).max() <= 1e-12 * abs(ref)
    assert np.abs(dr.sum(axis=0)).max() <= 1e-12 * np.abs(dr).sum()


def _flux_rows(orc, sc, dF, pnode):
    """Mass-balance rows of the Darcy term alone at a uniform deformation dF
    (an affine nodal increment, which G2P reproduces exactly) and nodal
    pressures pnode: the rows at pnode minus the rows at zero pressure (the
    volume-change part does not depend on the pressure)."""
    X = sc.node_coords()[:, :2]
    U = np.zeros(sc.nnode * 3)
    u = X @ (dF - np.eye(2)).T
    U[0::3], U[1::3] = u[:, 0], u[:, 1]
    r0, _ = orc.residual(U)
    U[2::3] = pnode
    r1, M = orc.residual(U)
    return (r1 - r0)[2::3], M


def test_up_darcy_flux_is_objective_and_scales_with_the_deformed_geometry(oracle):
    """Darcy's law holds in the deformed configuration.  (1) A superposed
    rigid rotation leaves every flux row unchanged.  (2) Stretching the body by
    s1 across and s2 along a uniform reference pressure gradient widens the
    flow section by s1 and lengthens the flow path by s2, so every flux row
    scales by s1 / s2 (a dropped volume ratio, a single inverse deformation
    gradient in place of dF^-1 dF^-T, or the gradient pushed the wrong way
    fails one of these)."""
    sc = _up_tiny(S.MODEL_NH, seed=31)
    orc = oracle.OracleScene.from_scene(sc)
    X = sc.node_coords()[:, :2]
    rng = np.random.default_rng(32)
    p_rand = rng.standard_normal(sc.nnode) * 1e4
    F_ref, M = _flux_rows(orc, sc, np.eye(2), p_rand)
    act = M > 0
    scale = np.abs(F_ref[act]).max()
    assert scale > 0
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    F_rot, _ = _flux_rows(orc, sc, R, p_rand)
    assert np.abs(F_rot - F_ref)[act].max() <= 1e-12 * scale
    # the volume-change part of the mass balance: with zero pressure and a
    # uniform dilation the rows sum (partition of unity) to (J - 1) sum_p V_p
    e = 0.01
    Xd = sc.node_coords()[:, :2]
    U = np.zeros(sc.nnode * 3)
    U[0::3], U[1::3] = e * Xd[:, 0], e * Xd[:, 1]
    r_vol, _ = orc.residual(U)
    J = (1 + e) ** 2
    assert abs(r_vol[2::3].sum() - (J - 1) * sc.vol0.sum()) <= 1e-13 * (J - 1) * sc.vol0.sum() * 10
    s1, s2 = 1.1, 0.9
    for axis in (0, 1):
        g = 1e4 / sc.h
        p_lin = g * X[:, axis]
        F0, _ = _flux_rows(orc, sc, np.eye(2), p_lin)
        dF = np.diag([s2, s1]) if axis == 0 else np.diag([s1, s2])   # s2 along the gradient
        F1, _ = _flux_rows(orc, sc, dF, p_lin)
        ref = np.abs(F0[act]).max()
        assert ref > 0
        assert np.abs(F1 - (s1 / s2) * F0)[act].max() <= 1e-12 * ref


def _terzaghi_series(z, T, H, nterms=400):
    s = np.zeros_like(z)
    U = 1.0
    for m in range(nterms):
        M = np.pi * (2 * m + 1) / 2
        s += 2.0 / M * np.sin(M * z / H) * np.exp(-M * M * T)
        U -= 2.0 / (M * M) * np.exp(-M * M * T)
    return s, U


@pytest.mark.slow
def test_terzaghi_consolidation_converges_to_series(oracle):
    """Sec. 4.4: H = 10 m, lambda = mu = 600 kPa, c_v = 1.8e-6 m^2/s, load
    1 kPa, drained top.  At T = 0.2 the pore pressure at the particles and the
    settlement of the loaded face approach the Terzaghi series at first order
    in h (the drained boundary sits on a node and its ghost, a boundary layer
    of one cell), with c_v dt / h^2 = 1/2 held fixed."""
    H, cv, t_load, T_end = 10.0, 1.8e-6, 1e3, 0.2
    M_c = 600e3 + 2 * 600e3
    perr, serr = [], []
    for N in (10, 20, 40):
        h = H / N
        dt = 0.5 * h * h / cv
        nsteps = int(round(T_end * H * H / cv / dt))
        sc = S.terzaghi(ncell=N, dt=dt, nsteps=nsteps)
        assert abs(sc.meta["cv"] - cv) < 1e-9 * cv
        orc = oracle.OracleScene.from_scene(sc)
        y0 = orc.x[:, 1].copy()
        for st in sc.steps:
            out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-10)
            assert out["converged"] and out["iters"] <= 4
        T = cv * nsteps * dt / H ** 2
        shape, Udeg = _terzaghi_series(sc.meta["y_top"] - y0, T, H)
        perr.append(np.abs(orc.pp - t_load * shape).max() / t_load)
        top = y0 > y0.max() - 1e-9
        s_num = -(orc.x[top, 1] - y0[top]).mean()
        s_ref = t_load * H / M_c * Udeg
        serr.append(abs(s_num - s_ref) / s_ref)
    perr, serr = np.array(perr), np.array(serr)
    for e in (perr, serr):
        assert (np.diff(e) < 0).all()
        assert (np.log2(e[:-1] / e[1:]) > 0.8).all()
    assert perr[-1] < 0.015 and serr[-1] < 0.025
