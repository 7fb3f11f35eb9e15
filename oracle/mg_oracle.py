"""Plain FP64 reference of the geometric multigrid V-cycle preconditioner.

TEST INFRASTRUCTURE ONLY.  Only tests/ may import this module.  It does not
import the CUDA package, and the CUDA package never imports it.

The preconditioner is not the paper's (it solves its linear systems with AMG
or a direct solver on the host, Sec. 2.2 remark, and names stronger block
preconditioning as future work, Sec. 5).  This module writes out, with SciPy
sparse matrices and NumPy, the V-cycle the solver applies, from its
definition:

* hierarchy on the background grid: level l+1 holds every second node of
  level l (n1 // 2 + 1 nodes per axis), down to the first level with at most
  ``dense_max`` unknowns on its active nodes, which is solved exactly;
* prolongation P: per-axis linear interpolation (weight 1 at a coincident
  node, 1/2 at an odd fine node), per node component, with the rows of
  inactive or prescribed fine DOFs zero; restriction P^T;
* coarse operator P^T A P, plus 1 on the diagonal of prescribed coarse DOFs
  (those with no free fine DOF under them); a coarse node is active when a
  fine node it interpolates to is active;
* smoother: damped node-block Jacobi, z <- z + w D^-1 (b - A z), D the
  node's B x B diagonal block, w = damp / lambda with lambda the estimate of
  lambda_max(D^-1 A) after ``power_it`` power iterations from a fixed
  start vector (component d: the SplitMix64 output of d mapped to [-1, 1),
  zero on prescribed DOFs; Steele, Lea and Flood 2014), w = 1/2 when the
  estimate is unusable;
* cycle: ``nu0`` sweeps before and after the coarse correction on the
  finest level (the first from zero), one on every coarse level (the first
  from zero, after the restriction), the coarsest level solved exactly.

Vectors live on a level's dense DOF space (node index x B + component);
entries of inactive nodes are zero.  Parity of the oracle itself:
``tests/test_mg_oracle.py``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_M64 = (1 << 64) - 1


GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state):
    """The output of SplitMix64 for generator state `state`: the state
    advanced by the golden gamma, then the finaliser (xor-shift 30, multiply,
    xor-shift 27, multiply, xor-shift 31; Steele, Lea and Flood 2014)."""
    x = (int(state) + GAMMA) & _M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
    return x ^ (x >> 31)


def splitmix_unit(d):
    """splitmix64(d) for each integer of the array d, top 53 bits mapped to
    [-1, 1)."""
    return np.array([(splitmix64(v) >> 11) * (1.0 / 4503599627370496.0) - 1.0
                     for v in np.asarray(d, dtype=np.int64).tolist()])


def prolongation(fine_dims, coarse_dims, B, keep):
    """P (fine DOFs x coarse DOFs) of the per-axis linear interpolation, x
    fastest; rows where ``keep`` is False are zero."""
    mats = []
    for n1, nc in zip(fine_dims, coarse_dims):
        rows, cols, vals = [], [], []
        for i in range(n1):
            parents = (i // 2, (i + 1) // 2) if i % 2 else (i // 2,)
            for J in parents:
                rows.append(i)
                cols.append(J)
                vals.append(1.0 if i % 2 == 0 else 0.5)
        mats.append(sp.csr_matrix((vals, (rows, cols)), shape=(n1, nc)))
    P = mats[0]
    for m in mats[1:]:
        P = sp.kron(m, P)
    P = sp.kron(P, sp.eye(B)).tocsr()
    return (sp.diags(np.asarray(keep, dtype=float)) @ P).tocsr()


def _block_inverses(A, act, B):
    """Inverse of each active node's B x B diagonal block (zero elsewhere)."""
    nn = len(act)
    Dinv = np.zeros((nn, B, B))
    Ad = A.tocsr()
    for n in np.nonzero(act)[0]:
        idx = n * B + np.arange(B)
        Dinv[n] = np.linalg.inv(Ad[idx][:, idx].toarray())
    return Dinv


def _apply_blocks(Dinv, v, B):
    return np.einsum("nab,nb->na", Dinv, v.reshape(-1, B)).ravel()


def power_lambda(A, Dinv, act, fix, B, iters):
    """lambda_max(D^-1 A) estimate: v_0 the SplitMix64 start vector on the
    active free DOFs, v_{k+1} = D^-1 A v_k / ||v_k||, lambda = ||v_iters||."""
    N = A.shape[0]
    dofs = np.arange(N)
    on = np.repeat(act, B) & ~fix
    v = np.where(on, splitmix_unit(dofs), 0.0)
    v[~np.repeat(act, B)] = 0.0
    n2 = float(v @ v)
    for _ in range(iters):
        sc = 1.0 / np.sqrt(n2) if 0.0 < n2 < 1e300 else 0.0
        v = _apply_blocks(Dinv, A @ v, B) * sc
        n2 = float(v @ v)
    return float(np.sqrt(n2))


class Hierarchy:
    """The levels of the V-cycle for the level-0 operator A0 (CSR over the
    dense DOF space, prescribed rows and columns already the identity),
    active node mask ``act0``, prescribed DOF mask ``fix0``, grid node
    counts per axis ``dims``."""

    def __init__(self, A0, act0, fix0, dims, B, dense_max=128, power_it=8, damp=1.2):
        self.B = B
        self.dims = [list(dims)]
        act0 = np.asarray(act0, dtype=bool)
        on0 = np.repeat(act0, B)
        A0 = sp.csr_matrix(A0)
        # inactive nodes have no rows or columns
        A0 = (sp.diags(on0.astype(float)) @ A0 @ sp.diags(on0.astype(float))).tocsr()
        self.A, self.act, self.fix, self.P = [A0], [act0], [np.asarray(fix0, dtype=bool)], []
        while int(self.act[-1].sum()) * B > dense_max:
            fd = self.dims[-1]
            cd = [n // 2 + 1 for n in fd]
            keep = np.repeat(self.act[-1], B) & ~self.fix[-1]
            P = prolongation(fd, cd, B, keep)
            Pn = prolongation(fd, cd, 1, self.act[-1])
            act_c = np.asarray((abs(Pn).T @ np.ones(Pn.shape[0])) > 0).ravel()
            fix_c = ~np.asarray((abs(P).T @ keep.astype(float)) > 0).ravel()
            Ac = (P.T @ self.A[-1] @ P).tocsr()
            Ac = (Ac + sp.diags((fix_c & np.repeat(act_c, B)).astype(float))).tocsr()
            self.P.append(P)
            self.A.append(Ac)
            self.act.append(act_c)
            self.fix.append(fix_c)
            self.dims.append(cd)
        self.L = len(self.A)
        # smoother of every level but the dense one
        self.Dinv, self.lam = [], []
        for l in range(self.L - 1):
            Dl = _block_inverses(self.A[l], self.act[l], B)
            lam = power_lambda(self.A[l], Dl, self.act[l], self.fix[l], B, power_it)
            w = damp / lam if 1e-3 <= lam < 1e30 else 0.5
            self.lam.append(lam)
            self.Dinv.append(Dl * w)
        # the dense level: its active DOFs and the inverse there
        on = np.repeat(self.act[-1], B)
        self.dense_idx = np.nonzero(on)[0]
        Ad = self.A[-1][self.dense_idx][:, self.dense_idx].toarray()
        self.dense_inv = np.linalg.inv(Ad) if len(self.dense_idx) else np.zeros((0, 0))

    def _sweep(self, l, b, z):
        return z + _apply_blocks(self.Dinv[l], b - self.A[l] @ z, self.B)

    def _mask(self, l, v):
        return np.where(np.repeat(self.act[l], self.B), v, 0.0)

    def down(self, b0, nu0=2):
        """Right-hand sides and smoothed iterates of the down leg (lists per
        level; the dense level's b only)."""
        L = self.L
        bs, zs = [np.asarray(b0, dtype=float)], []
        z = _apply_blocks(self.Dinv[0], bs[0], self.B)   # first sweep from zero
        for _ in range(1, nu0):
            z = self._sweep(0, bs[0], z)
        zs.append(self._mask(0, z))
        for l in range(L - 1):
            r = self._mask(l, bs[l] - self.A[l] @ zs[l])
            bc = self._mask(l + 1, self.P[l].T @ r)
            bs.append(bc)
            if l + 2 < L:
                zs.append(self._mask(l + 1, _apply_blocks(self.Dinv[l + 1], bc, self.B)))
        return bs, zs

    def dense_solve(self, b):
        z = np.zeros_like(b)
        z[self.dense_idx] = self.dense_inv @ b[self.dense_idx]
        return z

    def up(self, bs, zs, zc, nu0=2):
        """Up leg from the dense level's solution zc: prolongation, then one
        sweep per coarse level and nu0 on the finest."""
        for l in range(self.L - 2, -1, -1):
            r = self._mask(l, zs[l] + self.P[l] @ zc)
            z = r
            for _ in range(nu0 if l == 0 else 1):
                z = self._mask(l, self._sweep(l, bs[l], z))
            zc = z
        return zc

    def up_linear(self, zc, nu0=2):
        """The linear part of the up leg (b terms dropped), applied to a
        change zc of the dense level's solution."""
        for l in range(self.L - 2, -1, -1):
            z = self._mask(l, self.P[l] @ zc)
            for _ in range(nu0 if l == 0 else 1):
                z = self._mask(l, z - _apply_blocks(self.Dinv[l], self.A[l] @ z, self.B))
            zc = z
        return zc

    def vcycle(self, b0, nu0=2):
        """z = M^-1 b0, one V-cycle (the exact inverse when there is one level)."""
        if self.L == 1:
            return self.dense_solve(np.asarray(b0, dtype=float))
        bs, zs = self.down(b0, nu0)
        return self.up(bs, zs, self.dense_solve(bs[-1]), nu0)
