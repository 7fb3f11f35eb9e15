"""Plain FP64 CPU oracle driver for the implicit-MPM Newton step.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
does not import the CUDA package, and the CUDA package never imports it.

The per-particle and per-node arithmetic is in ``oracle.cpp`` (compiled to
``oracle/_build/liboracle.so`` by :func:`build`).  This module holds the
Newton loop of the paper's Sec. 2.2:

* residual r(u^{n+1,k}) = assembled f_int - f_ext;
* Newton update  -J du = r  with J = dr/du (exact, from the oracle's tangent),
  solved by a sparse direct factorisation (SciPy's SuperLU, a library step);
* stop when ||r^k|| / ||r^0|| <= tol (paper's convergence criterion), with
  r^0 taken after the prescribed boundary increment is applied;
* the correction is globalised (a reading: the paper takes full steps):
  limited to one cell width h per node, halved up to four times when the
  residual cannot be evaluated or does not decrease (``_globalised_update``);
* commit of the particle state after convergence.

Readings (the paper is silent on these):
* active DOFs are those of nodes with nodal mass M_i > ACTIVE_REL * max_p m_p;
* a prescribed DOF takes its increment at k = 0; its row and column of J are
  replaced by the identity and its residual entry is excluded from the norm;
* a prescribed DOF on an inactive node is ignored;
* u-p: the pressure DOF holds the pore pressure at the end of the step (a
  prescribed pressure is its value, not an increment) and starts each step
  at zero; the Newton norm weighs the mass-balance rows by ``p_scale``.

It also provides the coloured central finite-difference Jacobian used to pin
the exact tangent: the seeding pattern of the paper's sparse differentiation
(Algorithm 2, block size b = 5 for quadratic B-splines, Table 1) with a
central difference in place of a reverse-mode pass.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "liboracle.so")
ACTIVE_REL = 1e-4

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile oracle.cpp with g++ (-O2, no FMA contraction)."""
    src = os.path.join(HERE, "oracle.cpp")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(src):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, src])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.orc_stencil.argtypes = [_I, _D, _D, _L, _D, _D]
        L.orc_eig.argtypes = [_D, _D, _D]
        L.orc_return_map.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, _D, _D, _I, _D, _D]
        L.orc_particle.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, _D, ctypes.c_double,
                                   _D, _D, _D, _I, _D, _D]
        L.orc_residual.argtypes = [_I, _D, _D, ctypes.c_int, _D, _D, _D, _I, _D, _D, _D, _D, _D,
                                   _D, _D, _I, _D]
        L.orc_jacobian.argtypes = [_I, _D, ctypes.c_int, _D, _D, _I, _D, _D, _D, _D,
                                   ctypes.c_long, _L, _L, _D]
        L.orc_commit.argtypes = [_I, _D, ctypes.c_int, _D, _D, _I, _D, _D, _D, _D, _D]
        L.orc_residual_up.argtypes = [_I, _D, _D, ctypes.c_int, _D, _D, _D, _D, _I, _D, _D, _D, _D,
                                      _D, _D, _D, _D, _I, _D]
        L.orc_jacobian_up.argtypes = [_I, _D, ctypes.c_int, _D, _D, _D, _I, _D, _D, _D, _D, _D,
                                      ctypes.c_long, _L, _L, _D]
        L.orc_commit_up.argtypes = [_I, _D, ctypes.c_int, _D, _D, _I, _D, _D, _D, _D, _D, _D]
        _lib = L
    return _lib


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


# --------------------------------------------------------------------------
# single-particle entry points (used by the pins)
# --------------------------------------------------------------------------

def stencil(dim, n, h, origin, xp):
    gi = np.array([dim, n[0], n[1], n[2] if dim == 3 else 0], dtype=np.int32)
    gd = _f64([h, origin[0], origin[1], origin[2]])
    node = np.zeros(27, dtype=np.int64)
    w = np.zeros(27)
    g = np.zeros(81)
    c = lib().orc_stencil(_p(gi, _I), _p(gd), _p(_f64(xp)), _p(node, _L), _p(w), _p(g))
    if c < 0:
        raise OracleError("particle outside the grid")
    return node[:c], w[:c], g[:3 * c].reshape(c, 3)


def eig(a):
    a = _f64(a).reshape(9)
    lam = np.zeros(3)
    Q = np.zeros(9)
    lib().orc_eig(_p(a), _p(lam), _p(Q))
    return lam, Q.reshape(3, 3)


def return_map(model, params, etr, pcn=-1e5):
    eps = np.zeros(3)
    pc = np.zeros(1)
    mode = np.zeros(1, dtype=np.int32)
    deps = np.zeros(9)
    dg = np.zeros(1)
    rc = lib().orc_return_map(int(model), _p(_f64(params)), _p(_f64(etr)), float(pcn), _p(eps),
                              _p(pc), _p(mode, _I), _p(deps), _p(dg))
    if rc:
        raise OracleError(f"return map failed ({rc})")
    return eps, float(pc[0]), int(mode[0]), deps.reshape(3, 3), float(dg[0])


def particle(model, params, be6, pcn, dF, V0=1.0, tangent=True):
    """Stress update of one particle. Returns dict(tau, be, pc, mode, P, A)
    with A[a,c,b,e] = dP[a,c]/d dF[b,e]."""
    tau = np.zeros(9)
    be = np.zeros(6)
    pc = np.zeros(1)
    mode = np.zeros(1, dtype=np.int32)
    P = np.zeros(9)
    A = np.zeros(81) if tangent else None
    rc = lib().orc_particle(int(model), _p(_f64(params)), _p(_f64(be6)), float(pcn),
                            _p(_f64(np.asarray(dF).reshape(9))), float(V0), _p(tau), _p(be),
                            _p(pc), _p(mode, _I), _p(P), _p(A) if tangent else None)
    if rc:
        raise OracleError(f"particle update failed ({rc})")
    return dict(tau=tau.reshape(3, 3), be=be, pc=float(pc[0]), mode=int(mode[0]),
                P=P.reshape(3, 3), A=A.reshape(3, 3, 3, 3) if tangent else None)


# --------------------------------------------------------------------------
# scene-level oracle
# --------------------------------------------------------------------------

class OracleScene:
    """Particle state plus grid, evolved load step by load step.

    ``formulation`` is ``"solid"`` (dim displacement DOFs per node) or
    ``"up"`` (dim displacements and the pore pressure per node, the coupled
    formulation of the paper's Sec. 2.2 remark).  For u-p, ``kdt`` is the
    mobility times the time step per particle, ``p_scale`` the factor that
    puts the mass-balance rows and pressure unknowns on the scale of the
    momentum rows in the Newton norm (default max mu / h)."""

    def __init__(self, dim, n, h, origin, x, vol0, mass, model, params, pc0, formulation="solid",
                 kdt=None, p_scale=None):
        self.dim = int(dim)
        self.n = (int(n[0]), int(n[1]), int(n[2]) if dim == 3 else 0)
        self.h = float(h)
        self.origin = tuple(float(o) for o in origin)
        self.gi = np.array([self.dim, *self.n], dtype=np.int32)
        self.gd = _f64([self.h, *self.origin])
        self.x = _f64(x).copy()
        self.V0 = _f64(vol0).copy()
        self.m = _f64(mass).copy()
        self.model = np.ascontiguousarray(model, dtype=np.int32).copy()
        self.params = _f64(params).copy()
        self.np = self.x.shape[0]
        self.be = np.zeros((self.np, 6))
        self.be[:, :3] = 1.0
        self.pc = _f64(pc0).copy()
        self.F = np.tile(np.eye(3).reshape(9), (self.np, 1))
        self.gravity = np.zeros(3)
        self.formulation = formulation
        self.B = self.dim + (1 if formulation == "up" else 0)
        self.kdt = np.zeros(self.np) if kdt is None else _f64(kdt).copy()
        self.fext = np.zeros((self.np, 3))
        self.pp = np.zeros(self.np)
        if p_scale is None:
            mu = self.params[:, 0] / (2.0 * (1.0 + self.params[:, 1])) if self.np else np.zeros(1)
            p_scale = float(mu.max()) / self.h if self.np else 1.0
        self.p_scale = float(p_scale)
        nn = 1
        for a in range(self.dim):
            nn *= self.n[a] + 1
        self.nnode = nn

    @classmethod
    def from_scene(cls, sc):
        model, params, pc0 = sc.particle_params()
        form = getattr(sc, "formulation", "solid")
        kdt = sc.particle_kdt() if form == "up" else None
        o = cls(sc.dim, sc.n, sc.h, sc.origin, sc.x, sc.vol0, sc.mass, model, params, pc0,
                formulation=form, kdt=kdt)
        if getattr(sc, "be0", None) is not None:
            o.be[:] = sc.be0
        if getattr(sc, "fext", None) is not None:
            o.fext[:] = sc.fext
        return o

    @property
    def ndof(self):
        return self.nnode * self.B

    # ---- residual / Jacobian -------------------------------------------
    def residual(self, du, with_mode=False, with_scale=False):
        """r(du) on the dense DOF grid and the nodal mass; optionally the
        per-particle modes and the per-DOF sum of absolute contributions."""
        du = _f64(du)
        r = np.zeros(self.ndof)
        M = np.zeros(self.nnode)
        mode = np.zeros(self.np, dtype=np.int32)
        rabs = np.zeros(self.ndof) if with_scale else None
        if self.formulation == "up":
            rc = lib().orc_residual_up(_p(self.gi, _I), _p(self.gd), _p(_f64(self.gravity)), self.np,
                                       _p(self.x), _p(self.V0), _p(self.F), _p(self.m),
                                       _p(self.model, _I), _p(self.params), _p(self.be), _p(self.pc),
                                       _p(self.kdt), _p(self.fext), _p(du), _p(r), _p(M),
                                       _p(mode, _I), _p(rabs) if with_scale else None)
        else:
            rc = lib().orc_residual(_p(self.gi, _I), _p(self.gd), _p(_f64(self.gravity)), self.np,
                                    _p(self.x), _p(self.V0), _p(self.m), _p(self.model, _I),
                                    _p(self.params), _p(self.be), _p(self.pc), _p(self.fext), _p(du), _p(r),
                                    _p(M), _p(mode, _I), _p(rabs) if with_scale else None)
        if rc:
            raise OracleError(f"residual failed ({rc})")
        out = (r, M)
        if with_mode:
            out = out + (mode,)
        if with_scale:
            out = out + (rabs,)
        return out

    def jacobian_blocks(self, du):
        """Node-pair blocks (bi, bj, val[nb, d, d]) of J = dr/du, summed."""
        d = self.B
        cap = self.nnode * (5 ** self.dim)
        bi = np.zeros(cap, dtype=np.int64)
        bj = np.zeros(cap, dtype=np.int64)
        val = np.zeros(cap * d * d)
        if self.formulation == "up":
            nb = lib().orc_jacobian_up(_p(self.gi, _I), _p(self.gd), self.np, _p(self.x), _p(self.V0),
                                       _p(self.F), _p(self.model, _I), _p(self.params), _p(self.be),
                                       _p(self.pc), _p(self.kdt), _p(_f64(du)), cap, _p(bi, _L),
                                       _p(bj, _L), _p(val))
        else:
            nb = lib().orc_jacobian(_p(self.gi, _I), _p(self.gd), self.np, _p(self.x), _p(self.V0),
                                    _p(self.model, _I), _p(self.params), _p(self.be), _p(self.pc),
                                    _p(_f64(du)), cap, _p(bi, _L), _p(bj, _L), _p(val))
        if nb < 0:
            raise OracleError(f"jacobian failed ({nb})")
        return bi[:nb], bj[:nb], val[:nb * d * d].reshape(nb, d, d)

    def jacobian(self, du):
        """J over the dense DOF space as a scipy CSR matrix."""
        d = self.B
        bi, bj, val = self.jacobian_blocks(du)
        rows = (bi[:, None, None] * d + np.arange(d)[None, :, None]) + 0 * np.arange(d)[None, None, :]
        cols = (bj[:, None, None] * d + np.arange(d)[None, None, :]) + 0 * np.arange(d)[None, :, None]
        N = self.nnode * d
        return sp.csr_matrix((val.ravel(), (rows.ravel(), cols.ravel())), shape=(N, N))

    def active_dofs(self, M):
        act = M > ACTIVE_REL * self.m.max()
        return np.repeat(act, self.B)

    def norm_weights(self):
        """Per-DOF weights of the Newton norm: 1 for displacement rows,
        p_scale for the u-p mass-balance rows."""
        w = np.ones(self.ndof)
        if self.formulation == "up":
            w[self.dim::self.B] = self.p_scale
        return w

    # ---- Newton (paper Sec. 2.2) ------------------------------------------
    def solve_step(self, dof, value, gravity, tol=1e-12, maxit=25, commit=True, globalise=True):
        """One load step.  Returns dict(du, hist, iters, converged, r0).
        ``globalise=False`` takes the paper's plain full Newton steps."""
        self.gravity = _f64(gravity).copy()
        N = self.ndof
        wn = self.norm_weights()
        du = np.zeros(N)
        r, M = self.residual(du)
        act = self.active_dofs(M)
        fixed = np.zeros(N, dtype=bool)
        dof = np.asarray(dof, dtype=np.int64)
        keep = act[dof]
        fixed[dof[keep]] = True
        du[dof[keep]] = np.asarray(value, dtype=np.float64)[keep]
        free = act & ~fixed
        fidx = np.nonzero(free)[0]
        r, M = self.residual(du)
        r0 = np.linalg.norm((wn * r)[free])
        hist = [1.0]
        it = 0
        conv = r0 == 0.0
        disp = np.tile(np.arange(self.B) < self.dim, self.nnode)[fidx]
        rk = r0
        while not conv and it < maxit:
            J = self.jacobian(du)[fidx][:, fidx].tocsc()
            delta = spla.spsolve(J, -r[fidx])
            if globalise:
                du, r, M = self._globalised_update(du, fidx, delta, disp, rk, r0, tol, wn, free)
            else:
                du[fidx] += delta
                r, M = self.residual(du)
            it += 1
            rk = np.linalg.norm((wn * r)[free])
            rel = rk / r0
            hist.append(rel)
            conv = rel <= tol
        out = dict(du=du, hist=np.array(hist), iters=it, converged=bool(conv), r0=r0,
                   free=free, fixed=fixed, active=act, r=r, mass=M)
        if commit:
            self.commit(du)
        return out

    def _globalised_update(self, du, fidx, delta, disp, rk, r0, tol, wn, free):
        """Apply the Newton correction `delta` (over the free DOFs `fidx`) with
        the globalisation reading (the paper's Newton of Sec. 2.2 takes full
        steps; it states no safeguard):
        * step-length limit: when the largest displacement component of the
          correction exceeds one cell width h, the correction is scaled so
          that it equals h (a non-finite correction becomes zero);
        * a step whose residual cannot be evaluated because a return map
          leaves its domain or a particle's deformation stops being
          invertible, or whose residual norm is not below (1 - 1e-4) times the
          current one while that is above 10 tol ||r0||, is halved, at most
          four times; the fourth halving is taken whatever its residual.
        Returns the new increment, its residual and the nodal mass."""
        xmax = float(np.abs(delta[disp]).max()) if disp.any() else 0.0
        lim = 0.0 if not np.isfinite(xmax) else (self.h / xmax if xmax > self.h else 1.0)
        base = du.copy()

        def trial(alpha):
            d = base.copy()
            d[fidx] += (alpha * lim) * delta
            try:
                r, M = self.residual(d)
            except OracleError as e:
                if "(-1)" in str(e):
                    raise           # a particle's support left the grid
                return d, None, None
            return d, r, M

        d, r, M = trial(1.0)
        for half in range(1, 5):
            if r is not None:
                rnew = np.linalg.norm((wn * r)[free])
                if rnew < (1.0 - 1e-4) * rk or rk <= 10.0 * tol * r0:
                    break
            d, r, M = trial(2.0 ** -half)
        if r is None:
            raise OracleError("residual failed after four step halvings")
        return d, r, M

    def commit(self, du):
        if self.formulation == "up":
            rc = lib().orc_commit_up(_p(self.gi, _I), _p(self.gd), self.np, _p(self.x), _p(self.V0),
                                     _p(self.model, _I), _p(self.params), _p(self.be), _p(self.pc),
                                     _p(self.F), _p(_f64(du)), _p(self.pp))
            if rc:
                raise OracleError(f"commit failed ({rc})")
            return
        rc = lib().orc_commit(_p(self.gi, _I), _p(self.gd), self.np, _p(self.x), _p(self.V0),
                              _p(self.model, _I), _p(self.params), _p(self.be), _p(self.pc),
                              _p(self.F), _p(_f64(du)))
        if rc:
            raise OracleError(f"commit failed ({rc})")

    # ---- state helpers -----------------------------------------------------
    def stresses(self, du=None):
        """Kirchhoff stress (np,3,3) and mode of each particle at increment du
        (zero increment by default: the committed state)."""
        if du is None:
            du = np.zeros(self.ndof)
        out = np.zeros((self.np, 3, 3))
        modes = np.zeros(self.np, dtype=np.int32)
        for p in range(self.np):
            node, w, g = stencil(self.dim, self.n, self.h, self.origin, self.x[p])
            dF = np.eye(3)
            for l in range(len(node)):
                for a in range(self.dim):
                    for c in range(self.dim):
                        dF[a, c] += du[node[l] * self.B + a] * g[l, c]
            o = particle(self.model[p], self.params[p], self.be[p], self.pc[p], dF,
                         self.V0[p], tangent=False)
            out[p] = o["tau"]
            modes[p] = o["mode"]
        return out, modes

    def snapshot(self):
        return dict(x=self.x.copy(), be=self.be.copy(), pc=self.pc.copy(), F=self.F.copy(),
                    pp=self.pp.copy())

    def restore(self, s):
        self.x[:] = s["x"]
        self.be[:] = s["be"]
        self.pc[:] = s["pc"]
        self.F[:] = s["F"]
        self.pp[:] = s["pp"]


def node_ijk(sc: OracleScene, node):
    nx1 = sc.n[0] + 1
    ny1 = sc.n[1] + 1
    ix = node % nx1
    iy = (node // nx1) % ny1
    iz = node // (nx1 * ny1)
    return ix, iy, iz


def fd_jacobian_colored(sc: OracleScene, du, eps, b=5):
    """Central-difference Jacobian with the sparse-differentiation colouring:
    one colour per (local_x, local_y[, local_z], component) with block size b,
    seeding every DOF of that colour at once; each seeded column is read off
    the rows within +-2 nodes of its node.  ``eps`` is one step for every
    DOF or one step per node component.  Returns a dense (N, N) array."""
    d = sc.dim
    B = sc.B
    N = sc.nnode * B
    nodes = np.arange(sc.nnode)
    ix, iy, iz = node_ijk(sc, nodes)
    J = np.zeros((N, N))
    locs = [(lx, ly, lz) for lz in (range(b) if d == 3 else [0]) for ly in range(b) for lx in range(b)]
    for (lx, ly, lz) in locs:
        sel = (ix % b == lx) & (iy % b == ly) & ((iz % b == lz) if d == 3 else True)
        seeded = nodes[sel]
        for comp in range(B):
            ec = float(np.broadcast_to(np.asarray(eps, dtype=np.float64), (B,))[comp])
            e = np.zeros(N)
            e[seeded * B + comp] = 1.0
            rp, _ = sc.residual(du + ec * e)
            rm, _ = sc.residual(du - ec * e)
            col = (rp - rm) / (2 * ec)
            for j in seeded:
                jx, jy, jz = ix[j], iy[j], iz[j]
                near = (np.abs(ix - jx) <= 2) & (np.abs(iy - jy) <= 2)
                if d == 3:
                    near &= np.abs(iz - jz) <= 2
                rows = nodes[near]
                for a in range(B):
                    J[rows * B + a, j * B + comp] = col[rows * B + a]
    return J


def fd_jacobian_plain(sc: OracleScene, du, eps, cols):
    """Central-difference columns of J, one DOF at a time (the dense
    differentiation of the paper's Algorithm 1 with a difference in place of a
    reverse pass).  Returns (N, len(cols))."""
    N = sc.ndof
    out = np.zeros((N, len(cols)))
    for k, j in enumerate(cols):
        e = np.zeros(N)
        e[j] = 1.0
        rp, _ = sc.residual(du + eps * e)
        rm, _ = sc.residual(du - eps * e)
        out[:, k] = (rp - rm) / (2 * eps)
    return out


# --------------------------------------------------------------------------
# gradient of a load step's loss by its definition (the adjoint's oracle)
# --------------------------------------------------------------------------

def particle_increments(sc: OracleScene, du):
    """du_p = sum_i w_ip du_i for every particle (np, 3), from the start-of-step
    positions (the G2P of the increment, Sec. 2.2)."""
    out = np.zeros((sc.np, 3))
    for p in range(sc.np):
        node, w, g = stencil(sc.dim, sc.n, sc.h, sc.origin, sc.x[p])
        for a in range(sc.dim):
            out[p, a] = float(np.dot(w, du[node * sc.B + a]))
    return out


def step_gradient_fd(make_scene, step, loss, which, index, rel=1e-5, tol=1e-13):
    """Central difference of loss(converged du, particle increments) with
    respect to one parameter: which = "E" or "phi" (per particle `index`) or
    "k" (the conductivity of every particle scaled by 1 +- rel, i.e. the
    derivative with respect to log k).  `make_scene()` returns a fresh
    OracleScene at the start of the step."""
    vals = []
    for sgn in (1.0, -1.0):
        sc = make_scene()
        if which == "E":
            h_ = rel * sc.params[index, 0]
            sc.params[index, 0] += sgn * h_
        elif which == "phi":
            h_ = rel * max(abs(sc.params[index, 2]), 1.0)
            sc.params[index, 2] += sgn * h_
        elif which == "k":
            h_ = rel
            sc.kdt = sc.kdt * (1.0 + sgn * rel)
        else:
            raise ValueError(which)
        out = sc.solve_step(step.dof, step.value, step.gravity, tol=tol, maxit=40, commit=False)
        if not out["converged"]:
            raise OracleError("finite-difference solve did not converge")
        vals.append(loss(out["du"], particle_increments(sc, out["du"])))
    return (vals[0] - vals[1]) / (2.0 * h_)
