"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (the parity bar of the CUDA path, written out here so the tests
state them):
* residual: max |r_gpu - r_oracle| over free DOFs divided by the largest
  per-DOF sum of absolute particle contributions (the scale at which the
  summation rounds): 1e-10;
* Jacobian: per block, max |K_gpu - K_oracle| divided by the largest entry of
  the oracle's blocks in that block row (the row's scale; rows of nodes at the
  edge of the particle cloud have a tiny diagonal block next to larger
  off-diagonal ones): 1e-10 in FP64 mode, 1e-5 in mixed mode (FP32 blocks);
* converged increment: max |du_gpu - du_oracle| / max |du_oracle| <= 1e-7
  with both sides converged to a relative residual of 1e-12.
For the coupled u-p formulation the momentum and mass-balance rows, and the
displacement and pressure unknowns, carry different units, so every scale
above is taken per kind: residual scales per row kind, Jacobian scales per
(block row, row component, column kind), increment scales per unknown kind.
"""
import numpy as np

from oracle import mpm_oracle as O

RES_TOL = 1e-10
JAC_TOL_FP64 = 1e-10
JAC_TOL_MIXED = 1e-5
DU_TOL = 1e-7


def _B(x):
    return getattr(x, "B", x.dim)


def kinds(B, dim):
    """Kind of each node component: 0 displacement, 1 pore pressure."""
    return np.array([0] * dim + [1] * (B - dim))


def fixed_mask(scene, step):
    f = np.zeros(scene.nnode * _B(scene), dtype=bool)
    f[np.asarray(step.dof, dtype=np.int64)] = True
    return f


def residual_error(gs, orc, du, fixed):
    r_g = gs.residual()
    r_o, M, rabs = orc.residual(du, with_scale=True)
    act = orc.active_dofs(M)
    free = act & ~fixed
    if not free.any():
        return 0.0
    # the GPU reports zeros on prescribed and inactive DOFs
    assert np.all(r_g[~free] == 0.0)
    B = _B(orc)
    kind = np.tile(kinds(B, orc.dim), orc.nnode)
    worst = 0.0
    for k in np.unique(kind):
        sel = free & (kind == k)
        if not sel.any():
            continue
        scale = max(rabs[sel].max(), 1e-300)
        worst = max(worst, float(np.abs(r_g[sel] - r_o[sel]).max() / scale))
    return worst


def _bc_blocks(blocks, fixed, dim):
    """Apply the identity rows/columns of prescribed DOFs to a block dict."""
    out = {}
    for (i, j), B in blocks.items():
        B = B.copy()
        for a in range(dim):
            if fixed[i * dim + a]:
                B[a, :] = 0.0
                if i == j:
                    B[a, a] = 1.0
            for b in range(dim):
                if fixed[j * dim + b] and not (i == j and a == b and fixed[i * dim + a]):
                    B[a, b] = 0.0
        out[(i, j)] = B
    return out


def jacobian_error(gs, orc, du, fixed):
    dim = _B(orc)
    row_node, row_ptr, col_node, val = gs.jacobian_bsr()
    G = {}
    for r in range(len(row_node)):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            G[(int(row_node[r]), int(col_node[k]))] = val[k]
    bi, bj, bv = orc.jacobian_blocks(du)
    _, M = orc.residual(du)
    act_node = M > O.ACTIVE_REL * orc.m.max()
    Ob = {(int(i), int(j)): v for i, j, v in zip(bi, bj, bv) if act_node[i] and act_node[j]}
    Ob = _bc_blocks(Ob, fixed, dim)
    keys = set(G) | set(Ob)
    zero = np.zeros((dim, dim))
    worst = 0.0
    if dim == orc.dim:
        row_scale = {}
        for (i, j), B in Ob.items():
            row_scale[i] = max(row_scale.get(i, 0.0), float(np.abs(B).max()))
        for key in keys:
            i = key[0]
            g = G.get(key, zero)
            o = Ob.get(key, zero)
            sc = row_scale.get(i, 1.0)
            worst = max(worst, float(np.abs(g - o).max() / sc))
        return worst, len(G), len(Ob)
    # u-p: scale per (block row, row component, column kind)
    kd = kinds(dim, orc.dim)
    row_scale = {}
    for (i, j), B in Ob.items():
        for a in range(dim):
            for kb in (0, 1):
                v = float(np.abs(B[a, kd == kb]).max())
                row_scale[(i, a, kb)] = max(row_scale.get((i, a, kb), 0.0), v)
    for key in keys:
        i = key[0]
        g = G.get(key, zero)
        o = Ob.get(key, zero)
        for a in range(dim):
            for b in range(dim):
                sc = row_scale.get((i, a, kd[b]), 0.0)
                d = abs(g[a, b] - o[a, b])
                if sc > 0:
                    worst = max(worst, d / sc)
                elif d > 0:
                    worst = np.inf
    return worst, len(G), len(Ob)


def du_error(du_g, du_o, B=None, dim=None):
    if B is None or B == dim:
        return float(np.abs(du_g - du_o).max() / max(np.abs(du_o).max(), 1e-300))
    kind = np.tile(kinds(B, dim), du_o.size // B)
    worst = 0.0
    for k in (0, 1):
        sel = kind == k
        worst = max(worst, float(np.abs(du_g[sel] - du_o[sel]).max() / max(np.abs(du_o[sel]).max(), 1e-300)))
    return worst
