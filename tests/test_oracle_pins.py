"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test names what it checks and why a plausible mistake in the
oracle would fail it.

* B-spline: partition of unity, zero gradient sum, linear reproduction
  (a wrong node offset, a dropped 1/h or a sign error fails these).
* Eigen-decomposition against LAPACK (an independent library routine).
* G2P patch test: an affine nodal field gives dF = 1 + A exactly.
* Zero-strain tangent equals the isotropic elasticity tensor (closed form).
* Per-particle tangent against central differences of the oracle's own
  stress, elastic, plastic, apex and repeated-eigenvalue states.
* Return maps: consistency f = 0, flow rule, hardening law; at small strain
  both tend, at first order, to the textbook returns of linear elasticity
  (Drucker-Prager radial return, Cam-Clay in p-q invariants).
* P2G: linear and angular momentum balance of the internal force; gravity
  sums to the total weight; particle forces keep their sum and moment (a
  transposed dF^-T breaks the angular balance).
* Residual of a Neo-Hookean body = gradient of its total potential (energy
  density and B-spline kinematics written again in the test).
* Global Jacobian against the coloured central-difference Jacobian, and the
  coloured difference equal, bit for bit, to one-DOF-at-a-time differences
  (the paper's sparse = dense Jacobian check, Sec. 4.3).
* Newton converges quadratically (paper Sec. 4.2/4.1 observation).
* Block compression: exact homogeneous closed form at every load step.
* Bar under self-weight (paper Sec. 4.2): error against
  sigma_yy = -rho0 g (l0 - Y) decreases monotonically with refinement and the
  height tends to the closed-form height.
"""
import numpy as np
import pytest

from paper_2507_09435_gb300 import scenes as S

RNG = np.random.default_rng(20250709)


def _mat(model, **kw):
    base = dict(E=1e6, nu=0.3, phi=30.0, psi=0.0, c=2e3, M=1.2, lambda_cc=0.1, kappa_cc=0.02)
    base.update(kw)
    return np.array([base[k] for k in ("E", "nu", "phi", "psi", "c", "M", "lambda_cc", "kappa_cc")])


def _lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


# ---------------------------------------------------------------- B-splines
@pytest.mark.parametrize("dim", [2, 3])
def test_bspline_reproduction(oracle, dim):
    n = (10, 9, 8 if dim == 3 else 0)
    h, o = 0.37, (0.3, -0.2, 0.1)
    for _ in range(50):
        xp = np.array([o[a] + h * RNG.uniform(0.5, n[a] - 0.5) if a < dim else 0.0 for a in range(3)])
        node, w, g = oracle.stencil(dim, n, h, o, xp)
        assert len(node) == 3 ** dim
        nx1, ny1 = n[0] + 1, n[1] + 1
        xi = np.stack([node % nx1, (node // nx1) % ny1, node // (nx1 * ny1)], 1) * h + np.array(o)
        assert abs(w.sum() - 1) < 1e-14
        assert np.abs(g.sum(0)).max() < 1e-12
        assert np.abs((w[:, None] * xi).sum(0)[:dim] - xp[:dim]).max() < 1e-13
        G = xi[:, :dim].T @ g[:, :dim]
        assert np.abs(G - np.eye(dim)).max() < 1e-13
        assert (w >= 0).all()


def test_bspline_outside_grid_is_rejected(oracle):
    with pytest.raises(oracle.OracleError):
        oracle.stencil(2, (4, 4, 0), 1.0, (0, 0, 0), np.array([0.4, 2.0, 0.0]))
    with pytest.raises(oracle.OracleError):
        oracle.stencil(2, (4, 4, 0), 1.0, (0, 0, 0), np.array([2.0, 3.6, 0.0]))


# ---------------------------------------------------------------- eigen
def test_eig_matches_lapack(oracle):
    cases = []
    for _ in range(30):
        a = RNG.standard_normal((3, 3))
        cases.append(a + a.T)
    cases.append(np.eye(3))
    cases.append(np.diag([2.0, 2.0, 1.0]))
    q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    cases.append(q @ np.diag([1.5, 1.5, 0.7]) @ q.T)
    cases.append(np.array([[1.0, 1e-9, 0.0], [1e-9, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    for a in cases:
        lam, Q = oracle.eig(a)
        assert np.abs(np.sort(lam) - np.linalg.eigvalsh(a)).max() < 1e-13 * max(1, np.abs(a).max())
        assert np.abs(Q @ np.diag(lam) @ Q.T - a).max() < 1e-13 * max(1, np.abs(a).max())
        assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-14


# ---------------------------------------------------------------- G2P patch
@pytest.mark.parametrize("dim", [2, 3])
def test_g2p_patch_affine_field(oracle, dim):
    sc = S.tiny_scene(dim, S.MODEL_NH, seed=1, ncell=2)
    orc = oracle.OracleScene.from_scene(sc)
    A = np.zeros((3, 3))
    A[:dim, :dim] = 1e-3 * RNG.standard_normal((dim, dim))
    X = sc.node_coords()
    du = (X @ A.T)[:, :dim].ravel()
    x0 = orc.x.copy()
    orc.commit(du)
    F = orc.F.reshape(-1, 3, 3)
    assert np.abs(F - (np.eye(3) + A)[None]).max() < 1e-15
    assert np.abs(orc.x - (x0 + x0 @ A.T)).max() < 1e-15


# ---------------------------------------------------------------- tangents
def test_zero_strain_tangent_is_isotropic_elasticity(oracle):
    for model in (S.MODEL_NH, S.MODEL_NH_DP, S.MODEL_NH_MCC):
        p = _mat(model, E=2e6, nu=0.25)
        o = oracle.particle(model, p, [1, 1, 1, 0, 0, 0], -1e5, np.eye(3), V0=0.5)
        assert np.abs(o["tau"]).max() < 1e-9
        mu, lam = _lame(2e6, 0.25)
        d = np.eye(3)
        C = 0.5 * (mu * (np.einsum("ab,ce->acbe", d, d) + np.einsum("ae,cb->acbe", d, d))
                   + lam * np.einsum("ac,be->acbe", d, d))
        assert np.abs(o["A"] - C).max() < 1e-9 * mu  # C already carries V0 = 0.5


def _fd_A(oracle, model, p, be6, pcn, dF, V0, delta=1e-6):
    A = np.zeros((3, 3, 3, 3))
    for b in range(3):
        for e in range(3):
            dp = dF.copy(); dp[b, e] += delta
            dm = dF.copy(); dm[b, e] -= delta
            Pp = oracle.particle(model, p, be6, pcn, dp, V0, tangent=False)["P"]
            Pm = oracle.particle(model, p, be6, pcn, dm, V0, tangent=False)["P"]
            A[:, :, b, e] = (Pp - Pm) / (2 * delta)
    return A


def _spd6(scale):
    a = RNG.standard_normal((3, 3)) * scale
    s = 0.5 * (a + a.T)
    w, V = np.linalg.eigh(s)
    B = V @ np.diag(np.exp(2 * w)) @ V.T
    return np.array([B[0, 0], B[1, 1], B[2, 2], B[0, 1], B[1, 2], B[0, 2]])


TANGENT_CASES = [
    # (model, params, be6, pcn, dF, expected mode)
    ("nh_random", S.MODEL_NH, {}, "spd", -1e5, "rand0.05", 0),
    ("nh_zero", S.MODEL_NH, {}, "eye", -1e5, np.eye(3), 0),
    ("nh_repeated", S.MODEL_NH, {}, "eye", -1e5, np.diag([1.01, 1.01, 1.0]), 0),
    ("dp_elastic", S.MODEL_NH_DP, dict(c=2e5), "eye", -1e5, "rand0.01", 0),
    ("dp_plastic", S.MODEL_NH_DP, {}, "eye", -1e5, "shear", 1),
    ("dp_plastic_dilatant", S.MODEL_NH_DP, dict(psi=10.0), "eye", -1e5, "shear", 1),
    ("dp_plastic_repeated", S.MODEL_NH_DP, {}, "eye", -1e5, np.diag([0.97, 1.015, 1.015]), 1),
    ("dp_plastic_prestrained", S.MODEL_NH_DP, {}, "spd", -1e5, "shear", 1),
    ("dp_apex", S.MODEL_NH_DP, {}, "eye", -1e5, np.diag([1.02, 1.02, 1.01]), 2),
    ("mcc_elastic", S.MODEL_NH_MCC, {}, "eye", -1e6, "rand0.001c", 0),
    ("mcc_compaction", S.MODEL_NH_MCC, {}, "eye", -2e4, "compress", 1),
    ("mcc_repeated", S.MODEL_NH_MCC, {}, "eye", -2e4, np.diag([0.96, 0.99, 0.99]), 1),
    ("mcc_prestrained", S.MODEL_NH_MCC, {}, "spd", -2e4, "compress", 1),
]


def _make_dF(spec):
    if isinstance(spec, np.ndarray):
        return spec.copy()
    if spec == "rand0.05":
        return np.eye(3) + 0.05 * RNG.standard_normal((3, 3))
    if spec == "rand0.01":
        return np.eye(3) + 0.01 * RNG.standard_normal((3, 3))
    if spec == "rand0.001c":
        return np.eye(3) * 0.999 + 0.001 * RNG.standard_normal((3, 3))
    if spec == "shear":
        return np.eye(3) + np.array([[0.01, 0.04, 0], [0.01, -0.02, 0.0], [0, 0.005, 0.0]]) \
            + 0.003 * RNG.standard_normal((3, 3))
    if spec == "compress":
        return np.eye(3) * 0.97 + np.array([[0, 0.03, 0], [0.0, -0.01, 0.0], [0, 0, 0]]) \
            + 0.003 * RNG.standard_normal((3, 3))
    raise ValueError(spec)


@pytest.mark.parametrize("case", TANGENT_CASES, ids=[c[0] for c in TANGENT_CASES])
def test_particle_tangent_matches_central_differences(oracle, case):
    _, model, kw, be_spec, pcn, dF_spec, mode = case
    p = _mat(model, **kw)
    be6 = np.array([1, 1, 1, 0, 0, 0.0]) if be_spec == "eye" else _spd6(0.01)
    dF = _make_dF(dF_spec)
    o = oracle.particle(model, p, be6, pcn, dF, V0=0.3)
    assert o["mode"] == mode
    Afd = _fd_A(oracle, model, p, be6, pcn, dF, 0.3)
    scale = np.abs(o["A"]).max()
    assert np.abs(o["A"] - Afd).max() < 2e-7 * scale


@pytest.mark.parametrize("model", [S.MODEL_NH_DP, S.MODEL_NH_MCC])
def test_committed_plastic_state_is_elastic_at_zero_increment(oracle, model):
    """A state returned to the yield surface, re-evaluated with dF = 1, takes
    the elastic branch (yield tolerance reading) and keeps its stress."""
    p = _mat(model)
    pcn = -2e4
    dF = _make_dF("shear" if model == S.MODEL_NH_DP else "compress")
    o = oracle.particle(model, p, [1, 1, 1, 0, 0, 0], pcn, dF)
    assert o["mode"] == 1
    o2 = oracle.particle(model, p, o["be"], o["pc"], np.eye(3))
    assert o2["mode"] == 0
    assert np.abs(o2["tau"] - o["tau"]).max() < 1e-9 * np.abs(o["tau"]).max()


# ---------------------------------------------------------------- return maps
def test_dp_return_consistency_and_flow(oracle):
    for psi in (0.0, 8.0):
        p = _mat(S.MODEL_NH_DP, psi=psi)
        mu, lam = _lame(p[0], p[1])
        tp, ts = np.tan(np.radians(30.0)), np.tan(np.radians(psi))
        eta, xi = 3 * tp / np.sqrt(9 + 12 * tp ** 2), 3 / np.sqrt(9 + 12 * tp ** 2)
        etab = 3 * ts / np.sqrt(9 + 12 * ts ** 2)
        for _ in range(20):
            etr = RNG.standard_normal(3) * 0.02 - 0.01
            eps, pc, mode, _, dg = oracle.return_map(S.MODEL_NH_DP, p, etr)
            tau = mu * (np.exp(2 * eps) - 1) + lam * eps.sum()
            pr = tau.mean()
            s = tau - pr
            rJ2 = np.sqrt(0.5 * (s ** 2).sum())
            f = rJ2 + eta * pr - xi * 2e3
            if mode == 0:
                assert f <= 1e-9 * mu and np.array_equal(eps, etr)
            elif mode == 1:
                assert abs(f) < 1e-9 * 2e3
                assert dg > 0
                flow = s / (2 * rJ2) + etab / 3
                assert np.abs((etr - eps) - dg * flow).max() < 1e-13
                if psi == 0.0:
                    assert abs(eps.sum() - etr.sum()) < 1e-15
            else:
                assert np.abs(tau - xi * 2e3 / eta).max() < 1e-8 * 2e3


def test_mcc_return_consistency_flow_and_hardening(oracle):
    p = _mat(S.MODEL_NH_MCC)
    mu, lam = _lame(p[0], p[1])
    M, lmk = 1.2, 0.08
    nplastic = 0
    for _ in range(30):
        pcn = -2e4 * np.exp(0.2 * RNG.standard_normal())
        etr = RNG.standard_normal(3) * 0.01 - 0.01
        eps, pc, mode, _, dg = oracle.return_map(S.MODEL_NH_MCC, p, etr, pcn)
        tau = mu * (np.exp(2 * eps) - 1) + lam * eps.sum()
        pr = tau.mean()
        s = tau - pr
        q2 = 1.5 * (s ** 2).sum()
        f = q2 / M ** 2 + pr * (pr - pc)
        if mode == 0:
            assert f <= 0 and pc == pcn
        else:
            nplastic += 1
            assert abs(f) < 1e-9 * pcn ** 2
            assert abs(pc - pcn * np.exp(-(etr - eps).sum() / lmk)) < 1e-12 * abs(pcn)
            flow = 3 * s / M ** 2 + (2 * pr - pc) / 3
            assert np.abs((etr - eps) - dg * flow).max() < 1e-13
    assert nplastic > 5


# ---------------------------------------------------------------- P2G balances
@pytest.mark.parametrize("dim,model", [(2, S.MODEL_NH), (2, S.MODEL_NH_DP), (3, S.MODEL_NH_MCC)])
def test_internal_force_momentum_balance(oracle, dim, model):
    sc = S.tiny_scene(dim, model, seed=3, ncell=3)
    orc = oracle.OracleScene.from_scene(sc)
    du = S.random_increment(sc, 0.01, seed=4)
    orc.gravity = np.zeros(3)
    r, M = orc.residual(du)
    f = r.reshape(-1, dim)
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-12 * scale * len(f)
    y = sc.node_coords()[:, :dim] + du.reshape(-1, dim)
    if dim == 2:
        mom = (y[:, 0] * f[:, 1] - y[:, 1] * f[:, 0]).sum()
        assert abs(mom) < 1e-12 * scale * np.abs(y).max() * len(f)
    else:
        mom = np.cross(y, f).sum(0)
        assert np.abs(mom).max() < 1e-12 * scale * np.abs(y).max() * len(f)
    g = np.array([0.3, -9.81, 1.2])
    orc.gravity = g
    r2, M2 = orc.residual(du)
    fg = (r2 - r).reshape(-1, dim).sum(0)
    assert np.allclose(-fg, sc.mass.sum() * g[:dim], rtol=1e-13)
    assert abs(M2.sum() - sc.mass.sum()) < 1e-13 * sc.mass.sum()
    # particle forces (the traction reading): spread by w_ip, they sum to the
    # total applied force and carry its moment about the origin (the B-spline
    # weights reproduce linear fields)
    orc.gravity = np.zeros(3)
    fp = np.zeros((sc.np, 3))
    fp[:, :dim] = RNG.standard_normal((sc.np, dim)) * 1e3
    orc.fext[:] = fp
    r3, _ = orc.residual(du)
    ft = -(r3 - r).reshape(-1, dim)
    assert np.allclose(ft.sum(0), fp[:, :dim].sum(0), rtol=1e-12, atol=1e-12 * np.abs(fp).sum())
    X = sc.node_coords()[:, :dim]
    xp = sc.x[:, :dim]
    if dim == 2:
        m_nodes = (X[:, 0] * ft[:, 1] - X[:, 1] * ft[:, 0]).sum()
        m_parts = (xp[:, 0] * fp[:, 1] - xp[:, 1] * fp[:, 0]).sum()
    else:
        m_nodes = np.cross(X, ft).sum(0)
        m_parts = np.cross(xp, fp[:, :3]).sum(0)
    assert np.allclose(m_nodes, m_parts, rtol=1e-11, atol=1e-11 * np.abs(fp).sum() * np.abs(xp).max())


# ---------------------------------------------------------------- global Jacobian
JAC_CASES = [(2, S.MODEL_NH, 0.02), (2, S.MODEL_NH_DP, 0.03), (3, S.MODEL_NH, 0.02), (3, S.MODEL_NH_DP, 0.03),
             (3, S.MODEL_NH_MCC, 0.01)]


@pytest.mark.parametrize("dim,model,amp", JAC_CASES)
def test_jacobian_matches_colored_central_differences(oracle, dim, model, amp):
    sc = S.tiny_scene(dim, model, seed=7, ncell=3 if dim == 2 else 2)
    orc = oracle.OracleScene.from_scene(sc)
    orc.gravity = np.array([0.0, -9.81, 0.0])
    du = S.random_increment(sc, amp, seed=8)
    r, M, modes = orc.residual(du, with_mode=True)
    if model != S.MODEL_NH:
        assert (modes > 0).sum() >= 4, "case should drive particles plastic"
    J = orc.jacobian(du).toarray()
    Jfd = oracle.fd_jacobian_colored(orc, du, eps=1e-6 * sc.h)
    act = orc.active_dofs(M)
    Ja, Jf = J[np.ix_(act, act)], Jfd[np.ix_(act, act)]
    assert np.abs(Ja - Jf).max() < 1e-6 * np.abs(Ja).max()
    # nodes no particle reaches have empty rows and columns
    empty = np.repeat(M == 0.0, orc.B)
    assert np.abs(J[empty]).max() == 0 and np.abs(J[:, empty]).max() == 0


def test_colored_fd_equals_plain_fd_bitwise(oracle):
    sc = S.tiny_scene(2, S.MODEL_NH_DP, seed=9, ncell=3)
    orc = oracle.OracleScene.from_scene(sc)
    du = S.random_increment(sc, 0.02, seed=10)
    eps = 1e-6 * sc.h
    Jc = oracle.fd_jacobian_colored(orc, du, eps)
    _, M = orc.residual(du)
    act = np.nonzero(orc.active_dofs(M))[0]
    cols = act[:: max(1, len(act) // 12)]
    Jp = oracle.fd_jacobian_plain(orc, du, eps, cols)
    for k, j in enumerate(cols):
        nz = Jc[:, j] != 0
        assert np.array_equal(Jc[nz, j], Jp[nz, k])
        assert np.abs(Jp[~nz, k]).max() == 0.0


# ---------------------------------------------------------------- Newton and closed forms
def test_block_compression_homogeneous_closed_form_and_quadratic_newton(oracle):
    sc = S.block_compression()
    orc = oracle.OracleScene.from_scene(sc)
    mu, lam = _lame(1e6, 0.3)
    for k, st in enumerate(sc.steps):
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-12, globalise=False)
        assert out["converged"] and out["iters"] <= 4
        h = out["hist"]
        for a, b in zip(h[1:-1], h[2:]):
            assert b <= 50 * a * a + 1e-13
        l2 = (1 - sc.meta["strain_per_step"]) ** (k + 1)
        l1 = 1.0
        for _ in range(50):
            g = mu * (l1 * l1 - 1) + lam * np.log(l1 * l2)
            l1 -= g / (2 * mu * l1 + lam / l1)
        F = orc.F.reshape(-1, 3, 3)
        assert np.abs(F - np.diag([l1, l2, 1.0])[None]).max() < 1e-11
        tau, _ = orc.stresses()
        assert np.abs(tau[:, 0, 0]).max() < 1e-9 * mu
        J = l1 * l2
        assert np.abs(tau[:, 1, 1] - (mu * (l2 * l2 - 1) + lam * np.log(J))).max() < 1e-9 * mu


def test_self_weight_bar_converges_to_closed_form(oracle):
    """Paper Sec. 4.2: sigma_yy(Y) = -rho0 g (l0 - Y) for the bar under
    self-weight; error metric of the paper (volume-weighted |sigma_yy -
    sigma_a| over rho0 g l0).  With quadratic B-splines and fixed ghost nodes
    at the base the error has a first-order boundary layer, so the pin is
    monotone decrease at a rate of at least 0.6 per halving, plus convergence
    of the bar height to the closed-form height."""
    rho0, g, l0, mu = 80.0, 9.81, 50.0, 5e3
    Yq = np.linspace(0, l0, 20001)
    q = rho0 * g * (l0 - Yq)
    lam_q = (-q + np.sqrt(q * q + 4 * mu * mu)) / (2 * mu)
    H = np.trapezoid(lam_q, Yq)
    errs, herr = [], []
    for nc in (4, 8, 16, 32):
        sc = S.self_weight_column(nc)
        orc = oracle.OracleScene.from_scene(sc)
        Y = sc.x[:, 1] - sc.meta["y_base"]
        for st in sc.steps:
            out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-11, globalise=False)
            assert out["converged"] and out["iters"] <= 6
        tau, _ = orc.stresses()
        J = np.linalg.det(orc.F.reshape(-1, 3, 3))
        sig = tau[:, 1, 1] / J
        sa = -rho0 * g * (l0 - Y)
        errs.append(np.sum(np.abs(sig - sa) * orc.V0) / (g * rho0 * l0 * orc.V0.sum()))
        top = orc.x[:, 1].max() - sc.meta["y_base"] + 0.25 * sc.h * lam_q[-1]
        herr.append(abs(top - H) / H)
    errs = np.array(errs)
    assert (np.diff(errs) < 0).all()
    assert (np.log2(errs[:-1] / errs[1:]) > 0.6).all()
    assert errs[-1] < 0.04
    assert herr[-1] < 0.06 and herr[-1] < herr[0]


# ---------------------------------------------------------------- small-strain limits
# At strains of size d, Neo-Hookean principal Kirchhoff stresses
# mu (exp(2 eps) - 1) + lam tr eps differ from linear (Hencky) ones
# 2 mu eps + lam tr eps by O(d) relative, so the log-strain return maps must
# approach the textbook small-strain returns of linear elasticity at first
# order in d.  Those are written here from their own derivation in stress
# invariants (no principal-space local Newton), so a sign, a factor of the
# invariants or the direction of hardening that is wrong in the oracle shows
# up as an O(1) difference.

def _hencky_dp_return(etr, mu, lam, eta, etab, xi, c):
    """Radial return for Drucker-Prager with linear elasticity: the deviatoric
    direction is kept, sqrt(J2) drops by mu dg, p by K etab dg, and
    f_tr - (mu + K eta etab) dg = 0 (de Souza Neto et al., Sec. 8.3)."""
    K = lam + 2.0 * mu / 3.0
    ev = etr.sum()
    e_dev = etr - ev / 3.0
    s_tr = 2.0 * mu * e_dev
    rJ2 = np.sqrt(0.5 * (s_tr ** 2).sum())
    p_tr = K * ev
    f_tr = rJ2 + eta * p_tr - xi * c
    dg = f_tr / (mu + K * eta * etab)
    eps = etr - dg * (s_tr / (2.0 * rJ2) + etab / 3.0)
    return eps, dg


def _small_strain_mcc_return(etr, mu, lam, M, lmk, pcn):
    """Modified Cam-Clay return with linear elasticity in (p, q): q scales by
    1 / (1 + 6 mu dg / M^2), p = p_tr - K dg (2p - pc), pc = pcn
    exp(-dg (2p - pc) / (lambda - kappa)), f(p, q, pc) = 0 (Borja and Lee
    1990, invariant form), solved with a library root finder."""
    from scipy.optimize import fsolve
    K = lam + 2.0 * mu / 3.0
    ev = etr.sum()
    e_dev = etr - ev / 3.0
    s_tr = 2.0 * mu * e_dev
    q_tr = np.sqrt(1.5 * (s_tr ** 2).sum())
    p_tr = K * ev

    def eqs(z):
        dg, p, pc = z[0] / abs(pcn), z[1] * abs(pcn), z[2] * abs(pcn)
        q = q_tr / (1.0 + 6.0 * mu * dg / M ** 2)
        return [(q * q / M ** 2 + p * (p - pc)) / pcn ** 2,
                (p - p_tr + K * dg * (2 * p - pc)) / abs(pcn),
                (pc - pcn * np.exp(-dg * (2 * p - pc) / lmk)) / abs(pcn)]

    z, _, ok, msg = fsolve(eqs, [1e-12, p_tr / abs(pcn), pcn / abs(pcn)], xtol=1e-14, full_output=True)
    assert ok == 1, msg
    dg, p, pc = z[0] / abs(pcn), z[1] * abs(pcn), z[2] * abs(pcn)
    s = s_tr / (1.0 + 6.0 * mu * dg / M ** 2)
    eps = etr - dg * (3.0 * s / M ** 2 + (2.0 * p - pc) / 3.0)
    return eps, dg, pc


def test_dp_return_tends_to_the_small_strain_radial_return(oracle):
    E, nu = 1e6, 0.3
    mu, lam = _lame(E, nu)
    tp = np.tan(np.radians(30.0))
    eta, xi = 3 * tp / np.sqrt(9 + 12 * tp ** 2), 3 / np.sqrt(9 + 12 * tp ** 2)
    direction = np.array([0.8, -1.0, 0.1])          # mostly deviatoric, slight dilation
    for psi in (0.0, 10.0):
        ts = np.tan(np.radians(psi))
        etab = 3 * ts / np.sqrt(9 + 12 * ts ** 2)
        errs = []
        for d in (1e-3, 1e-4, 1e-5):
            etr = d * direction
            K = lam + 2 * mu / 3
            rJ2 = np.sqrt(0.5 * ((2 * mu * (etr - etr.sum() / 3)) ** 2).sum())
            c = (0.5 * rJ2 + eta * K * etr.sum()) / xi     # trial f = half of sqrt(J2)
            p = _mat(S.MODEL_NH_DP, E=E, nu=nu, c=c, psi=psi)
            eps, _, mode, _, dg = oracle.return_map(S.MODEL_NH_DP, p, etr)
            assert mode == 1
            eps_l, dg_l = _hencky_dp_return(etr, mu, lam, eta, etab, xi, c)
            errs.append(max(abs(dg - dg_l) / dg_l, np.abs(eps - eps_l).max() / d))
        errs = np.array(errs)
        assert errs[0] < 0.01
        assert (errs[1:] < 0.2 * errs[:-1]).all()        # first order in d


def test_mcc_return_tends_to_the_small_strain_invariant_return(oracle):
    E, nu, M, lmk = 1e6, 0.3, 1.2, 0.08
    mu, lam = _lame(E, nu)
    direction = np.array([-1.0, -0.4, -0.2])         # compression with shear
    errs = []
    for d in (1e-3, 1e-4, 1e-5):
        etr = d * direction
        pcn = -0.4 * E * d                            # on the scale of the trial stress: plastic
        p = _mat(S.MODEL_NH_MCC, E=E, nu=nu, M=M, lambda_cc=0.1, kappa_cc=0.1 - lmk)
        eps, pc, mode, _, dg = oracle.return_map(S.MODEL_NH_MCC, p, etr, pcn)
        assert mode == 1
        eps_l, dg_l, pc_l = _small_strain_mcc_return(etr, mu, lam, M, lmk, pcn)
        errs.append(max(abs(dg - dg_l) / dg_l, np.abs(eps - eps_l).max() / d, abs(pc - pc_l) / abs(pcn)))
    errs = np.array(errs)
    assert errs[0] < 0.01
    assert (errs[1:] < 0.2 * errs[:-1]).all()


# ---------------------------------------------------------------- residual as an energy gradient
def _bspline_1d(x, h):
    """Textbook quadratic B-spline on a uniform grid: the three node indices
    from floor(x/h - 1/2), their weights N(xi) and derivatives dN/dx."""
    base = int(np.floor(x / h - 0.5))
    idx = np.arange(base, base + 3)
    xi = x / h - idx
    a = np.abs(xi)
    N = np.where(a < 0.5, 0.75 - xi * xi, 0.5 * (1.5 - a) ** 2)
    dN = np.where(a < 0.5, -2.0 * xi, -(1.5 - a) * np.sign(xi)) / h
    return idx, N, dN


def _nh_total_potential(sc, du, grav):
    """Total potential of a fresh Neo-Hookean body (b_e = 1 at the start of
    the step): sum_p V0_p psi(dF_p) - sum_p m_p g . u(x_p), with
    psi = mu/2 (tr b - 3) - mu ln J + lam/2 (ln J)^2 and dF_p from the
    textbook B-spline gradients (plane strain: dF_zz = 1)."""
    _, params, _ = sc.particle_params()
    d = sc.dim
    U = du.reshape(-1, d)
    nx1, ny1 = sc.n[0] + 1, sc.n[1] + 1
    total = 0.0
    for p in range(sc.np):
        E, nu = params[p, 0], params[p, 1]
        mu, lam = _lame(E, nu)
        ax = [_bspline_1d(sc.x[p, a] - sc.origin[a], sc.h) for a in range(d)]
        dF = np.eye(3)
        up = np.zeros(d)
        for combo in np.ndindex(*(3,) * d):
            node = ax[0][0][combo[0]] + nx1 * ax[1][0][combo[1]]
            if d == 3:
                node += nx1 * ny1 * ax[2][0][combo[2]]
            w = np.prod([ax[a][1][combo[a]] for a in range(d)])
            gw = np.array([ax[a][2][combo[a]] * np.prod([ax[b][1][combo[b]] for b in range(d) if b != a])
                           for a in range(d)])
            dF[:d, :d] += np.outer(U[node], gw)
            up += w * U[node]
        J = np.linalg.det(dF)
        b = dF @ dF.T
        psi = 0.5 * mu * (np.trace(b) - 3.0) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
        total += sc.vol0[p] * psi - sc.mass[p] * float(grav[:d] @ up)
    return total


@pytest.mark.parametrize("dim", [2, 3])
def test_neo_hookean_residual_is_the_gradient_of_the_total_potential(oracle, dim):
    """For a hyperelastic body the discrete residual is the gradient of the
    total potential (stored energy minus the work of gravity), computed here
    from the energy density with its own B-spline kinematics: a transposed
    dF^-T, a wrong stress formula, a dropped volume or a wrong gravity sign
    breaks it."""
    sc = S.tiny_scene(dim, S.MODEL_NH, seed=41, ncell=3 if dim == 2 else 2)
    orc = oracle.OracleScene.from_scene(sc)
    g = np.array([0.4, -9.81, 0.7 if dim == 3 else 0.0])
    orc.gravity = g
    du = S.random_increment(sc, 0.03, seed=42)
    r, M = orc.residual(du)
    rng = np.random.default_rng(43)
    for _ in range(3):
        v = rng.standard_normal(du.size) * sc.h
        eps = 1e-6
        dPi = (_nh_total_potential(sc, du + eps * v, g) - _nh_total_potential(sc, du - eps * v, g)) / (2 * eps)
        assert abs(dPi - r @ v) <= 1e-7 * np.abs(r).max() * np.abs(v).sum() / np.sqrt(v.size)
    # the Jacobian is then the Hessian of that potential: symmetric
    J = orc.jacobian(du).toarray()
    assert np.abs(J - J.T).max() <= 1e-12 * np.abs(J).max()
    # one DOF at a time on the busiest node
    i = int(np.argmax(M))
    for a in range(dim):
        e = np.zeros(du.size)
        e[i * dim + a] = sc.h
        dPi = (_nh_total_potential(sc, du + 1e-6 * e, g) - _nh_total_potential(sc, du - 1e-6 * e, g)) / 2e-6
        assert abs(dPi - r[i * dim + a] * sc.h) <= 1e-7 * abs(r[i * dim + a] * sc.h) + 1e-9 * np.abs(r).max() * sc.h


@pytest.mark.parametrize("model,kw", [(S.MODEL_NH_MCC, {}), (S.MODEL_NH_DP, dict(c=100.0, nu=0.2, prestrain=0.0))],
                         ids=["cam_clay", "drucker_prager"])
def test_plastic_newton_converges_quadratically_once_yielding(oracle, model, kw):
    """The consistent tangent makes Newton quadratic once the plastic set is
    fixed (the paper's observation for its plastic examples, Sec. 4.1-4.2):
    on oedometers whose particles all yield (Cam-Clay after the first steps;
    Drucker-Prager with a low Poisson ratio and no pre-compression),
    e_{k+1} <= e_k^2 until the rounding floor.  A continuum (non-consistent)
    tangent gives a linear rate and fails this."""
    sc = S.oedometer_3d(model=model, **kw)
    orc = oracle.OracleScene.from_scene(sc)
    checked = 0
    for k, st in enumerate(sc.steps):
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-13, commit=False, globalise=False)
        assert out["converged"] and out["iters"] <= 5
        _, _, modes = orc.residual(out["du"], with_mode=True)
        if (modes > 0).mean() == 1.0:
            h = out["hist"]
            for a, b in zip(h[1:], h[2:]):
                if a * a > 1e-12:      # above the rounding floor of about 5e-14
                    assert b <= 1.0 * a * a, (k, h)
                    checked += 1
        orc.commit(out["du"])
    assert checked >= 4


@pytest.mark.parametrize("dim", [2, 3])
def test_associative_drucker_prager_jacobian_is_symmetric(oracle, dim):
    """With associative flow (psi = phi), no hardening and an elastic law with
    a potential in principal log strain, the return map is the stationarity
    condition of an incremental potential, so the consistent tangent, and the
    global Jacobian, is symmetric, apex states included (Simo 1992).  The
    non-associative case (psi = 0) is not: a wrong flow direction or a
    transposed term of the spectral tangent breaks the first, the second
    shows the check can fail."""
    sc = S.tiny_scene(dim, S.MODEL_NH_DP, seed=7, ncell=3 if dim == 2 else 2)
    du = S.random_increment(sc, 0.03, seed=8)
    sc.materials[0].psi = sc.materials[0].phi
    orc = oracle.OracleScene.from_scene(sc)
    _, _, modes = orc.residual(du, with_mode=True)
    assert (modes == 1).sum() >= 10 and (modes == 2).sum() >= 10
    J = orc.jacobian(du).toarray()
    assert np.abs(J - J.T).max() <= 1e-13 * np.abs(J).max()
    sc.materials[0].psi = 0.0
    J0 = oracle.OracleScene.from_scene(sc).jacobian(du).toarray()
    assert np.abs(J0 - J0.T).max() > 1e-2 * np.abs(J0).max()


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("case", [c for c in TANGENT_CASES if c[0] in
                                  ("nh_random", "dp_plastic", "dp_apex", "dp_plastic_prestrained",
                                   "mcc_compaction", "mcc_prestrained")], ids=lambda c: c[0])
def test_constitutive_update_is_objective(oracle, case):
    """A rigid rotation R superposed on the increment (dF -> R dF) rotates
    the Kirchhoff stress and the elastic left Cauchy-Green tensor (R . R^T),
    leaves the mode and the hardening variable unchanged, and transforms
    P = V0 tau dF^-T to R P and the tangent dP/d(dF) to
    R_ai A_icje R_bj.  A frame-dependent step anywhere in the spectral return
    map or its tangent fails this."""
    _, model, kw, be_spec, pcn, dF_spec, _ = case
    rng = np.random.default_rng(77)
    p = _mat(model, **kw)
    be6 = np.array([1, 1, 1, 0, 0, 0.0]) if be_spec == "eye" else _spd6(0.01)
    dF = _make_dF(dF_spec)
    R = _rotation(rng)
    o = oracle.particle(model, p, be6, pcn, dF, V0=0.3)
    oR = oracle.particle(model, p, be6, pcn, R @ dF, V0=0.3)
    assert oR["mode"] == o["mode"]
    s = np.abs(o["tau"]).max()
    assert np.abs(oR["tau"] - R @ o["tau"] @ R.T).max() <= 1e-10 * s
    assert np.abs(oR["P"] - R @ o["P"]).max() <= 1e-10 * np.abs(o["P"]).max()

    def full(b6):
        return np.array([[b6[0], b6[3], b6[5]], [b6[3], b6[1], b6[4]], [b6[5], b6[4], b6[2]]])
    assert np.abs(full(oR["be"]) - R @ full(o["be"]) @ R.T).max() <= 1e-12
    assert abs(oR["pc"] - o["pc"]) <= 1e-12 * abs(o["pc"]) + 1e-300
    A_rot = np.einsum("ai,icje,bj->acbe", R, o["A"], R)
    assert np.abs(oR["A"] - A_rot).max() <= 1e-9 * np.abs(o["A"]).max()


@pytest.mark.parametrize("dim,model", [(2, S.MODEL_NH), (2, S.MODEL_NH_DP), (3, S.MODEL_NH_MCC)])
def test_internal_force_virial_equals_the_kirchhoff_stress_sum(oracle, dim, model):
    """For any increment, sum_i (X_i + du_i) (x) f_int,i = sum_p V0_p tau_p:
    the B-spline gradients reproduce dF exactly, and P = V0 tau dF^-T.  It
    ties the residual to the stress the update reports (a wrong sign, scale or
    transposition of P between the two fails it)."""
    sc = S.tiny_scene(dim, model, seed=51, ncell=3 if dim == 2 else 2)
    orc = oracle.OracleScene.from_scene(sc)
    orc.gravity = np.zeros(3)
    du = S.random_increment(sc, 0.02, seed=52)
    r, _ = orc.residual(du)
    x = sc.node_coords()[:, :dim] + du.reshape(-1, dim)
    vir = x.T @ r.reshape(-1, dim)
    tau, modes = orc.stresses(du)
    ref = np.einsum("p,pab->ab", orc.V0, tau)[:dim, :dim]
    assert np.abs(vir - ref).max() <= 1e-11 * np.abs(ref).max()
    if model != S.MODEL_NH:
        assert (modes > 0).any()


def test_globalised_newton_reaches_the_plain_newton_root(oracle):
    """The step-length limit and the step halving change the Newton path, not
    its end point: on the bar under self-weight (large compaction, where the
    limit is active) both forms converge to the same increment, and on the
    block both take the same full steps."""
    for sc in (S.self_weight_column(4), S.block_compression()):
        a = oracle.OracleScene.from_scene(sc)
        b = oracle.OracleScene.from_scene(sc)
        for st in sc.steps[:3]:
            oa = a.solve_step(st.dof, st.value, st.gravity, tol=1e-12, globalise=False)
            ob = b.solve_step(st.dof, st.value, st.gravity, tol=1e-12, globalise=True)
            assert oa["converged"] and ob["converged"]
            scale = np.abs(oa["du"]).max()
            assert np.abs(oa["du"] - ob["du"]).max() <= 1e-9 * scale


def test_slope_ramp_converges_with_the_active_node_threshold(oracle):
    """Reading of the active set: a node reached only by the far tail of a
    particle's B-spline (a distance t inside its support edge: mass ~ t^2 m/2,
    stiffness ~ t^2, but an O(1) lever on the particle's dF) is left out
    below 1e-4 of a particle's mass.  On a 96 x 48 random-field slope (3 x 3
    particles per cell, whose middle particles start on support edges) every
    step of the 20-step gravity ramp then converges; with a threshold of
    1e-12 Newton stalls at about three quarters of g."""
    sc = S.slope(nx=96, ny=48, h=1.0, ppc=3, nsteps=20, found_h=12, body_h=16, crest=40, toe=64)
    orc = oracle.OracleScene.from_scene(sc)
    assert oracle.ACTIVE_REL == 1e-4
    for st in sc.steps:
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=1e-8, maxit=32)
        assert out["converged"] and out["iters"] <= 8, out["hist"]
