"""Parity at the benchmark sizes, in the launch configuration the bench times
(mixed precision, BiCGStab, CUDA-graph chunks): the 256x128 footing (128,016
particles) and the 2M-particle 3D Cam-Clay column.  The oracle cannot build
these whole Jacobians quickly, so rows are sampled: the residual and the
Jacobian blocks of a node depend only on the particles whose B-spline support
contains it, and the oracle evaluates exactly those particles."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2507_09435_gb300 import mpm, scenes as S

from parity_util import JAC_TOL_MIXED, RES_TOL, fixed_mask, _bc_blocks

pytestmark = pytest.mark.gpu


def _sub_oracle(sc, nodes):
    """Oracle scene of the particles whose support contains one of `nodes`."""
    nx1, ny1 = sc.n[0] + 1, sc.n[1] + 1
    ix, iy, iz = nodes % nx1, (nodes // nx1) % ny1, nodes // (nx1 * ny1)
    s = (sc.x[:, :sc.dim] - np.asarray(sc.origin[:sc.dim])) / sc.h
    base = np.floor(s - 0.5).astype(np.int64)
    # a particle reaches nodes base..base+2 per axis
    cand = np.ones((sc.np, len(nodes)), dtype=bool)
    for a, ia in enumerate((ix, iy, iz)[:sc.dim]):
        d = ia[None, :] - base[:, a][:, None]
        cand &= (d >= 0) & (d <= 2)
    keep = cand.any(axis=1)
    model, params, pc0 = sc.particle_params()
    orc = O.OracleScene(sc.dim, sc.n, sc.h, sc.origin, sc.x[keep], sc.vol0[keep], sc.mass[keep], model[keep],
                        params[keep], pc0[keep])
    if sc.be0 is not None:
        orc.be[:] = sc.be0[keep]
    return orc


def _check_sampled(sc, gs, step, nodes, jac_tol=JAC_TOL_MIXED):
    fixed = fixed_mask(sc, step)
    d = sc.dim
    orc = _sub_oracle(sc, nodes)
    orc.gravity = np.asarray(step.gravity, dtype=np.float64)
    du = gs.du()
    r_g = gs.residual()
    r_o, M, rabs = orc.residual(du, with_scale=True)
    Mg = gs.mass()
    act = Mg[nodes] > O.ACTIVE_REL * sc.mass.max()
    nodes = nodes[act]
    dofs = (nodes[:, None] * d + np.arange(d)[None, :]).ravel()
    free = dofs[~fixed[dofs]]
    scale = rabs[free].max()
    assert np.abs(r_g[free] - r_o[free]).max() <= RES_TOL * scale
    # Jacobian rows of the sampled nodes
    gs.assemble()
    row_node, row_ptr, col_node, val = gs.jacobian_bsr()
    rows = {int(n): r for r, n in enumerate(row_node)}
    bi, bj, bv = orc.jacobian_blocks(du)
    want = set(int(n) for n in nodes)
    Ob = {(int(i), int(j)): v for i, j, v in zip(bi, bj, bv) if int(i) in want and Mg[int(j)] > O.ACTIVE_REL * sc.mass.max()}
    Ob = _bc_blocks(Ob, fixed, d)
    worst = 0.0
    for n in nodes:
        r = rows[int(n)]
        G = {int(col_node[k]): val[k] for k in range(row_ptr[r], row_ptr[r + 1])}
        Orow = {j: v for (i, j), v in Ob.items() if i == int(n)}
        sc_row = max(float(np.abs(v).max()) for v in Orow.values())
        assert set(G) == set(Orow), int(n)
        for j, v in Orow.items():
            worst = max(worst, float(np.abs(G[j] - v).max()) / sc_row)
    assert worst < jac_tol, worst
    return len(nodes)


def test_footing_full_size_sampled_parity():
    sc = S.footing(nx=256, ny=128, h=0.1, ppc=2, nsteps=50)
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
    rng = np.random.default_rng(2)
    st = sc.steps[0]
    gs.begin(st)
    M = gs.mass()
    active = np.nonzero(M > O.ACTIVE_REL * sc.mass.max())[0]
    nodes = rng.choice(active, size=48, replace=False)
    assert _check_sampled(sc, gs, st, nodes) >= 40
    gs.newton()
    assert _check_sampled(sc, gs, st, nodes) >= 40
    gs.close()


def test_column3d_2M_sampled_parity():
    sc = S.column_collapse_3d(col=(72, 72, 48))
    assert sc.np == 1_990_656
    gs = mpm.GpuScene(sc, precision=mpm.MPM_MIXED, newton_tol=1e-8)
    rng = np.random.default_rng(3)
    st = sc.steps[0]
    gs.begin(st)
    M = gs.mass()
    active = np.nonzero(M > O.ACTIVE_REL * sc.mass.max())[0]
    nodes = rng.choice(active, size=24, replace=False)
    assert _check_sampled(sc, gs, st, nodes, JAC_TOL_MIXED) >= 20
    gs.newton()
    assert _check_sampled(sc, gs, st, nodes, JAC_TOL_MIXED) >= 20
    gs.close()
