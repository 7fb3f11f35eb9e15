"""Seeded synthetic scene generators for the implicit-MPM Newton step.

This module holds data only: particle lattices, material tables, random
material fields and the per-load-step boundary schedules of the test and
benchmark workloads.  It contains none of the method's arithmetic (no shape
functions, kinematics, stresses or solver steps), so that the CUDA path and
the CPU oracle can both consume the same inputs without sharing code.

Geometry follows the paper's statement of the problem (Sec. 2.1: a body on a
background grid with Dirichlet and Neumann parts of the boundary) and its
workloads (Sec. 4.2 bar under self-weight; Sec. 4.5 footing indentation);
the sizes are those of the synthetic footing, column-collapse, slope and
block-compression problems this library is measured on.

Conventions
-----------
* Grid: ``n = (nx, ny, nz)`` cells (``nz = 0`` in 2D), spacing ``h``, nodes at
  ``origin + i*h`` for ``0 <= i <= n``.  Node linear index is x-fastest:
  ``ix + (nx+1)*(iy + (ny+1)*iz)``; a DOF index is ``node*dim + comp``.
* Particles sit on a regular lattice, ``ppc`` per axis per cell, at offsets
  ``(k + 1/2)/ppc`` inside the cell (1/4, 3/4 for two; 1/6, 1/2, 5/6 for three).
* A 2D scene is plane strain with unit thickness: a particle volume is
  ``h**2 / ppc**2``.
* Material models: 0 = Neo-Hookean, 1 = Neo-Hookean + Drucker-Prager,
  2 = Neo-Hookean + modified Cam-Clay.  Angles are in degrees, stresses in Pa,
  ``pc0`` is negative (compression negative).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

SEED_BASE = 2507_09435

MODEL_NH = 0
MODEL_NH_DP = 1
MODEL_NH_MCC = 2


@dataclass
class Material:
    model: int = MODEL_NH
    E: float = 1e6
    nu: float = 0.3
    rho: float = 1000.0
    phi: float = 0.0        # friction angle, degrees
    psi: float = 0.0        # dilation angle, degrees
    c: float = 0.0          # cohesion, Pa
    M: float = 1.0          # critical-state slope
    lambda_cc: float = 0.1  # virgin compression index
    kappa_cc: float = 0.02  # swelling index
    pc0: float = -1e5       # initial preconsolidation pressure, Pa
    k_hyd: float = 0.0      # hydraulic conductivity, m/s (u-p only)
    gamma_w: float = 9810.0  # unit weight of the pore fluid, N/m^3 (u-p only)

    def params8(self) -> np.ndarray:
        """The eight per-particle parameters in the order both sides read them:
        E, nu, phi, psi, c, M, lambda_cc, kappa_cc."""
        return np.array([self.E, self.nu, self.phi, self.psi, self.c, self.M,
                         self.lambda_cc, self.kappa_cc], dtype=np.float64)


@dataclass
class LoadStep:
    """Boundary data of one load step: prescribed displacement increments on
    node DOFs and the gravity vector in force during the step."""
    dof: np.ndarray             # int64 DOF indices on the dense node grid
    value: np.ndarray           # float64 increments, same length
    gravity: Tuple[float, float, float] = (0.0, 0.0, 0.0)


@dataclass
class Scene:
    name: str
    dim: int
    n: Tuple[int, int, int]
    h: float
    origin: Tuple[float, float, float]
    x: np.ndarray               # (np, 3) float64; z = 0 in 2D
    vol0: np.ndarray            # (np,)
    mass: np.ndarray            # (np,)
    mat_id: np.ndarray          # (np,) int32
    materials: List[Material]
    E_p: Optional[np.ndarray] = None     # per-particle Young's modulus override
    phi_p: Optional[np.ndarray] = None   # per-particle friction angle override
    pc0_p: Optional[np.ndarray] = None   # per-particle initial preconsolidation
    be0: Optional[np.ndarray] = None     # (np, 6) initial elastic left Cauchy-Green, default identity
    steps: List[LoadStep] = field(default_factory=list)
    meta: dict = field(default_factory=dict)
    formulation: str = "solid"           # "solid" or "up" (displacement + pore pressure per node)
    dt: float = 0.0                      # time step of a u-p load step, s
    fext: Optional[np.ndarray] = None    # (np, 3) external force carried by each particle, N

    @property
    def B(self) -> int:
        """DOFs per node: dim, plus the pore pressure for u-p."""
        return self.dim + (1 if self.formulation == "up" else 0)

    def particle_kdt(self) -> np.ndarray:
        """Per-particle mobility times time step, k_hyd / gamma_w * dt (u-p)."""
        k = np.array([self.materials[m].k_hyd / self.materials[m].gamma_w for m in self.mat_id])
        return k * self.dt

    @property
    def np(self) -> int:
        return int(self.x.shape[0])

    @property
    def nnode(self) -> int:
        c = 1
        for a in range(self.dim):
            c *= self.n[a] + 1
        return c

    def node_index(self, ix, iy, iz=0):
        nx1 = self.n[0] + 1
        ny1 = self.n[1] + 1
        return ix + nx1 * (iy + ny1 * iz)

    def node_coords(self) -> np.ndarray:
        """(nnode, 3) node positions, x-fastest."""
        axes = [self.origin[a] + self.h * np.arange(self.n[a] + 1) for a in range(self.dim)]
        if self.dim == 2:
            yy, xx = np.meshgrid(axes[1], axes[0], indexing="ij")
            return np.stack([xx.ravel(), yy.ravel(), np.zeros(xx.size)], axis=1)
        zz, yy, xx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)

    def particle_params(self):
        """Per-particle (model, params[np,8], pc0[np]) with overrides applied.
        Pure table lookup, used to hand the same numbers to both sides."""
        model = np.array([self.materials[m].model for m in self.mat_id], dtype=np.int32)
        params = np.stack([self.materials[m].params8() for m in range(len(self.materials))])[self.mat_id]
        params = np.ascontiguousarray(params)
        if self.E_p is not None:
            params[:, 0] = self.E_p
        if self.phi_p is not None:
            params[:, 2] = self.phi_p
        pc0 = np.array([self.materials[m].pc0 for m in self.mat_id], dtype=np.float64)
        if self.pc0_p is not None:
            pc0 = np.array(self.pc0_p, dtype=np.float64)
        return model, params, pc0


# --------------------------------------------------------------------------
# lattice helpers
# --------------------------------------------------------------------------

def lattice(cells: np.ndarray, h: float, ppc: int, dim: int, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Particles of the occupied ``cells`` (k, dim) int array, ``ppc`` per axis,
    ordered cell by cell.  Returns (np, 3) positions."""
    off = (np.arange(ppc) + 0.5) / ppc
    if dim == 2:
        oy, ox = np.meshgrid(off, off, indexing="ij")
        sub = np.stack([ox.ravel(), oy.ravel()], axis=1)
    else:
        oz, oy, ox = np.meshgrid(off, off, off, indexing="ij")
        sub = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1)
    pts = (cells[:, None, :].astype(np.float64) + sub[None, :, :]) * h
    pts = pts.reshape(-1, dim)
    out = np.zeros((pts.shape[0], 3))
    out[:, :dim] = pts + np.asarray(origin[:dim])[None, :]
    return out


def box_cells(lo, hi) -> np.ndarray:
    """All integer cells with lo <= c < hi per axis (x-fastest order)."""
    rng = [np.arange(l, u) for l, u in zip(lo, hi)]
    mesh = np.meshgrid(*rng[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def _dofs(scene_like, nodes_mask_fn, comp, dim, n, stride=None):
    """DOF indices of nodes selected by a predicate on integer node coords
    (``stride`` DOFs per node, default ``dim``)."""
    axes = [np.arange(n[a] + 1) for a in range(dim)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    coords = [m.ravel() for m in mesh[::-1]]          # x-fastest enumeration
    sel = nodes_mask_fn(*coords)
    nx1, ny1 = n[0] + 1, n[1] + 1
    if dim == 2:
        lin = coords[0] + nx1 * coords[1]
    else:
        lin = coords[0] + nx1 * (coords[1] + ny1 * coords[2])
    lin = lin[sel]
    stride = dim if stride is None else stride
    return lin.astype(np.int64) * stride + comp, [c[sel] for c in coords]


def _merge(*pairs):
    """Concatenate (dof, value) pairs; a later pair overrides an earlier one
    on the same DOF."""
    d = {}
    for dof, val in pairs:
        for k, v in zip(dof.tolist(), np.broadcast_to(val, dof.shape).tolist()):
            d[k] = v
    keys = np.array(sorted(d), dtype=np.int64)
    return keys, np.array([d[k] for k in keys.tolist()], dtype=np.float64)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def block_compression(nsteps: int = 5, strain_per_step: float = 1e-3, ppc: int = 2,
                      E: float = 1e6, nu: float = 0.3, ngrid: int = 32) -> Scene:
    """2D plane-strain Neo-Hookean block, 32x32 grid (h = 1/32), block on cells
    [2,18)^2 with 2x2 particles per cell (1024 particles), top face displaced
    0.1 % of the height per step.  ``ngrid`` scales the grid (block on cells
    [o, o + ngrid/2)^2, o = ngrid/16, h = 1/ngrid).

    Boundary reading: the affine increment du_y = -eps*(y - y_bottom) is
    prescribed on every node within one cell of the bottom (y <= 3h) or top
    (y >= 17h) face or beyond it; du_x = 0 on the left wall node column x = 2h.
    With this node set and particles at the 1/4, 3/4 offsets the first load
    step has the homogeneous solution F = diag(l1, 1-eps, 1) as its exact
    discrete solution (the quadrature of grad w over a full column vanishes)."""
    n = (ngrid, ngrid, 0)
    h = 1.0 / ngrid
    o, L = max(ngrid // 16, 2), ngrid // 2
    cells = box_cells((o, o), (o + L, o + L))
    x = lattice(cells, h, ppc, 2)
    mat = Material(model=MODEL_NH, E=E, nu=nu, rho=1000.0)
    vol = np.full(x.shape[0], h * h / ppc ** 2)
    sc = Scene("block_compression", 2, n, h, (0.0, 0.0, 0.0), x, vol, vol * mat.rho,
               np.zeros(x.shape[0], np.int32), [mat])
    yb = o * h
    dy, (ix, iy) = _dofs(sc, lambda ix, iy: (iy <= o + 1) | (iy >= o + L - 1), 1, 2, n)
    vy = -strain_per_step * (iy * h - yb)
    dx, _ = _dofs(sc, lambda ix, iy: ix == o, 0, 2, n)
    dof, val = _merge((dy, vy), (dx, np.zeros(dx.shape)))
    sc.steps = [LoadStep(dof, val, (0.0, 0.0, 0.0)) for _ in range(nsteps)]
    sc.meta = dict(strain_per_step=strain_per_step, y_bottom=yb, x_left=o * h)
    return sc


def footing(nx: int = 256, ny: int = 128, h: float = 0.1, ppc: int = 2, nsteps: int = 50,
            B: float = 2.0, settle_frac: float = 0.1, geostatic: bool = True,
            E: float = 1e7, nu: float = 0.3, phi: float = 30.0, psi: float = 0.0,
            c: float = 5e3, rho: float = 2000.0, g: float = 9.81, prestress: bool = False) -> Scene:
    """2D plane-strain rigid-footing bearing capacity: Neo-Hookean +
    non-associative Drucker-Prager soil filling cells [1,nx-1) x [1,ny-1)
    (256 x 128 grid, h = 0.1 m, 2x2 particles per cell: 128,016 particles).

    Readings (the workload statement leaves them open): rollers on the side
    walls (u_x = 0 on nodes x <= h and x >= (nx-1)h), fixed base (u = 0 on nodes
    y <= h); a rough rigid footing of width B centred on the surface pushes the
    surface nodes under it (y >= (ny-1)h, |x - xc| <= B/2) down by
    settle_frac*B over nsteps steps with u_x = 0.  Load step 0 is a geostatic
    step (gravity on, footing free) when ``geostatic`` is set.

    ``prestress`` starts the soil from the linear-elastic at-rest state of a
    laterally confined layer instead of from b_e = 1: a particle at depth d
    below the surface carries the vertical log strain eps_y = -rho g d /
    (lam + 2 mu) (one-dimensional compression, eps_x = eps_z = 0), i.e.
    b_e = diag(1, exp(2 eps_y), 1).  Without it a deep layer settles under
    its own weight by rho g H^2 / (2 (lam + 2 mu)) (0.12 m for the 12.7 m
    layer above), which can leave the prescribed surface nodes outside
    every particle's stencil; with it the geostatic step only removes the
    small nonlinear remainder."""
    n = (nx, ny, 0)
    cells = box_cells((1, 1), (nx - 1, ny - 1))
    x = lattice(cells, h, ppc, 2)
    mat = Material(model=MODEL_NH_DP, E=E, nu=nu, rho=rho, phi=phi, psi=psi, c=c)
    vol = np.full(x.shape[0], h * h / ppc ** 2)
    be0 = None
    if prestress:
        lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        mu = E / (2.0 * (1.0 + nu))
        depth = (ny - 1) * h - x[:, 1]
        be0 = np.zeros((x.shape[0], 6))
        be0[:, 0] = 1.0
        be0[:, 1] = np.exp(-2.0 * rho * g * depth / (lam + 2.0 * mu))
        be0[:, 2] = 1.0
    sc = Scene("footing", 2, n, h, (0.0, 0.0, 0.0), x, vol, vol * rho,
               np.zeros(x.shape[0], np.int32), [mat], be0=be0)
    grav = (0.0, -g, 0.0)
    lx, _ = _dofs(sc, lambda ix, iy: (ix <= 1) | (ix >= nx - 1), 0, 2, n)
    bx, _ = _dofs(sc, lambda ix, iy: iy <= 1, 0, 2, n)
    by, _ = _dofs(sc, lambda ix, iy: iy <= 1, 1, 2, n)
    walls = _merge((lx, np.zeros(lx.shape)), (bx, np.zeros(bx.shape)), (by, np.zeros(by.shape)))
    xc = 0.5 * nx * h
    under = lambda ix, iy: (iy >= ny - 1) & (np.abs(ix * h - xc) <= 0.5 * B + 1e-9 * h)
    fx, _ = _dofs(sc, under, 0, 2, n)
    fy, _ = _dofs(sc, under, 1, 2, n)
    du = -settle_frac * B / nsteps
    steps = []
    if geostatic:
        steps.append(LoadStep(walls[0], walls[1], grav))
    fdof, fval = _merge(walls, (fx, np.zeros(fx.shape)), (fy, np.full(fy.shape, du)))
    steps += [LoadStep(fdof, fval, grav) for _ in range(nsteps)]
    sc.steps = steps
    sc.meta = dict(B=B, settle_per_step=-du, xc=xc, surface_y=(ny - 1) * h)
    return sc


def column_collapse_3d(nx: int = 128, ny: int = 128, nz: int = 64, h: float = 0.1,
                       col: Tuple[int, int, int] = (32, 32, 48), ppc: int = 2,
                       nsteps: int = 20, rho: float = 2000.0, g: float = 9.81,
                       E: float = 1e7, nu: float = 0.3, M: float = 1.2,
                       lambda_cc: float = 0.1, kappa_cc: float = 0.02,
                       pc_mean: float = -1e5, pc_sigma: float = 0.1,
                       seed: int = SEED_BASE + 3) -> Scene:
    """3D granular column under a gravity ramp, modified Cam-Clay with
    Neo-Hookean elasticity, 8 particles per cell.  The column of ``col`` cells
    stands centred on a rough floor (u = 0 on nodes z <= h); rollers on the
    far side walls.  Gravity ramps 0 -> g over ``nsteps`` load steps.
    Initial preconsolidation is lognormal: pc0 = pc_mean*exp(pc_sigma*Z).

    ``col=(32,32,48)`` is the stated column (393,216 particles);
    ``col=(72,72,48)`` the ~2M-particle variant."""
    n = (nx, ny, nz)
    cx0 = (nx - col[0]) // 2
    cy0 = (ny - col[1]) // 2
    cells = box_cells((cx0, cy0, 1), (cx0 + col[0], cy0 + col[1], 1 + col[2]))
    x = lattice(cells, h, ppc, 3)
    mat = Material(model=MODEL_NH_MCC, E=E, nu=nu, rho=rho, M=M, lambda_cc=lambda_cc,
                   kappa_cc=kappa_cc, pc0=pc_mean)
    vol = np.full(x.shape[0], h ** 3 / ppc ** 3)
    rng = np.random.default_rng(seed)
    pc0 = pc_mean * np.exp(pc_sigma * rng.standard_normal(x.shape[0]))
    sc = Scene("column_collapse_3d", 3, n, h, (0.0, 0.0, 0.0), x, vol, vol * rho,
               np.zeros(x.shape[0], np.int32), [mat], pc0_p=pc0)
    pairs = []
    for comp in range(3):
        d, _ = _dofs(sc, lambda ix, iy, iz: iz <= 1, comp, 3, n)
        pairs.append((d, np.zeros(d.shape)))
    d, _ = _dofs(sc, lambda ix, iy, iz: (ix <= 1) | (ix >= nx - 1), 0, 3, n)
    pairs.append((d, np.zeros(d.shape)))
    d, _ = _dofs(sc, lambda ix, iy, iz: (iy <= 1) | (iy >= ny - 1), 1, 3, n)
    pairs.append((d, np.zeros(d.shape)))
    dof, val = _merge(*pairs)
    sc.steps = [LoadStep(dof, val, (0.0, 0.0, -g * (k + 1) / nsteps)) for k in range(nsteps)]
    sc.meta = dict(col=col, ppc=ppc)
    return sc


def oedometer_3d(ncell: int = 4, h: float = 0.1, ppc: int = 2, nsteps: int = 4, strain_per_step: float = 2e-3,
                 model: int = MODEL_NH_MCC, E: float = 1e6, nu: float = 0.3, pc0: float = -26e3,
                 pc_sigma: float = 0.05, prestrain: float = 0.01, phi: float = 30.0, c: float = 2e3,
                 seed: int = SEED_BASE + 13) -> Scene:
    """3D oedometric compression of a cube of ``ncell``^3 cells: the affine
    increment du_z = -eps (z - z_bottom) on every node within one cell of the
    bottom or top face (or beyond), rollers (u_x = 0 / u_y = 0) on the nodes
    within one cell of the side faces (or beyond).  The particles start from
    an isotropic elastic pre-compression b_e = (1 - prestrain)^2 1 and a
    preconsolidation near the corresponding pressure, so that loading is
    plastic from the first step while every particle stays in compression
    (where the modified Cam-Clay return map is defined)."""
    ng = ncell + 4
    n = (ng, ng, ng)
    lo, hi = 2, 2 + ncell
    cells = box_cells((lo, lo, lo), (hi, hi, hi))
    x = lattice(cells, h, ppc, 3)
    mat = Material(model=model, E=E, nu=nu, rho=1000.0, M=1.2, lambda_cc=0.1, kappa_cc=0.02, pc0=pc0,
                   phi=phi, psi=0.0, c=c)
    vol = np.full(x.shape[0], h ** 3 / ppc ** 3)
    rng = np.random.default_rng(seed)
    pc = pc0 * np.exp(pc_sigma * rng.standard_normal(x.shape[0]))
    be0 = np.zeros((x.shape[0], 6))
    be0[:, :3] = (1.0 - prestrain) ** 2
    sc = Scene("oedometer_3d", 3, n, h, (0.0, 0.0, 0.0), x, vol, vol * mat.rho,
               np.zeros(x.shape[0], np.int32), [mat], pc0_p=pc, be0=be0)
    zb = lo * h
    dz, (ix, iy, iz) = _dofs(sc, lambda ix, iy, iz: (iz <= lo + 1) | (iz >= hi - 1), 2, 3, n)
    vz = -strain_per_step * (iz * h - zb)
    dx, _ = _dofs(sc, lambda ix, iy, iz: (ix <= lo + 1) | (ix >= hi - 1), 0, 3, n)
    dy, _ = _dofs(sc, lambda ix, iy, iz: (iy <= lo + 1) | (iy >= hi - 1), 1, 3, n)
    dof, val = _merge((dz, vz), (dx, np.zeros(dx.shape)), (dy, np.zeros(dy.shape)))
    sc.steps = [LoadStep(dof, val, (0.0, 0.0, 0.0)) for _ in range(nsteps)]
    sc.meta = dict(strain_per_step=strain_per_step)
    return sc


def gaussian_field(shape, corr_cells: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean unit-variance stationary Gaussian random field on a cell
    lattice: white noise filtered in Fourier space by a Gaussian kernel of
    correlation length ``corr_cells``, then standardised."""
    w = rng.standard_normal(shape)
    k = [np.fft.fftfreq(s) for s in shape]
    kk = np.meshgrid(*k, indexing="ij")
    k2 = sum(ki ** 2 for ki in kk)
    filt = np.exp(-0.5 * (2 * np.pi) ** 2 * k2 * corr_cells ** 2)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    f -= f.mean()
    return f / f.std()


def slope(nx: int = 192, ny: int = 96, h: float = 0.5, ppc: int = 3, nsteps: int = 20,
          found_h: int = 24, body_h: int = 32, crest: int = 80, toe: int = 128,
          E: float = 1e7, nu: float = 0.3, phi: float = 30.0, c: float = 20e3,
          rho: float = 2000.0, g: float = 9.81, std: float = 0.1, corr: float = 10.0,
          seed: int = SEED_BASE + 5) -> Scene:
    """2D Drucker-Prager slope with per-particle E and friction angle drawn
    from seeded Gaussian random fields (10 % std, correlation 10 cells):
    a foundation layer of ``found_h`` cells plus a slope body ``body_h`` cells
    high whose face runs from x = toe (bottom) to x = crest (top).  Gravity
    ramps 0 -> g over ``nsteps`` steps; rollers on the sides, fixed base.
    3x3 particles per cell (about 71k particles for the default sizes).
    Cohesion 20 kPa keeps the 16 m, 34 degree face stable under full gravity
    (with 5 kPa it fails part-way up the ramp and Newton has no solution)."""
    n = (nx, ny, 0)
    cl = []
    for iy in range(1, 1 + found_h + body_h):
        if iy < 1 + found_h:
            xmax = nx - 1
        else:
            t = (iy - (1 + found_h) + 0.5) / body_h
            xmax = int(round(toe + (crest - toe) * t))
        for ix in range(1, xmax):
            cl.append((ix, iy))
    cells = np.array(cl, dtype=np.int64)
    x = lattice(cells, h, ppc, 2)
    rng = np.random.default_rng(seed)
    zE = gaussian_field((nx, ny), corr, rng)
    zphi = gaussian_field((nx, ny), corr, rng)
    cidx = np.repeat(cells, ppc * ppc, axis=0)
    E_p = E * (1.0 + std * zE[cidx[:, 0], cidx[:, 1]])
    phi_p = phi * (1.0 + std * zphi[cidx[:, 0], cidx[:, 1]])
    mat = Material(model=MODEL_NH_DP, E=E, nu=nu, rho=rho, phi=phi, psi=0.0, c=c)
    vol = np.full(x.shape[0], h * h / ppc ** 2)
    sc = Scene("slope", 2, n, h, (0.0, 0.0, 0.0), x, vol, vol * rho,
               np.zeros(x.shape[0], np.int32), [mat], E_p=E_p, phi_p=phi_p)
    lx, _ = _dofs(sc, lambda ix, iy: (ix <= 1) | (ix >= nx - 1), 0, 2, n)
    bx, _ = _dofs(sc, lambda ix, iy: iy <= 1, 0, 2, n)
    by, _ = _dofs(sc, lambda ix, iy: iy <= 1, 1, 2, n)
    dof, val = _merge((lx, np.zeros(lx.shape)), (bx, np.zeros(bx.shape)), (by, np.zeros(by.shape)))
    sc.steps = [LoadStep(dof, val, (0.0, -g * (k + 1) / nsteps, 0.0)) for k in range(nsteps)]
    sc.meta = dict(crest=crest, toe=toe, found_h=found_h, body_h=body_h)
    return sc


def self_weight_column(ncell: int, l0: float = 50.0, rho0: float = 80.0, E: float = 1e4,
                       nsteps: int = 40, g: float = 9.81, ppc: int = 2) -> Scene:
    """Vertical bar under self-weight (paper Sec. 4.2): height l0 = 50 m,
    rho0 = 80 kg/m^3, E = 10 kPa, nu = 0, gravity applied over 40 load steps.
    One cell wide, ``ncell`` cells high, 2x2 particles per cell (16 to 2048
    particles for 2^2 .. 2^9 cells).  Lateral confinement: u_x = 0 on every
    node; the base (nodes y <= 2h) is fixed.  Neo-Hookean elasticity is used
    in place of the paper's Hencky law; the equilibrium closed form
    sigma_yy(Y) = -rho0*g*(l0 - Y) does not depend on the elastic law."""
    h = l0 / ncell
    n = (5, ncell + 4, 0)
    cells = box_cells((2, 2), (3, 2 + ncell))
    x = lattice(cells, h, ppc, 2)
    mat = Material(model=MODEL_NH, E=E, nu=0.0, rho=rho0)
    vol = np.full(x.shape[0], h * h / ppc ** 2)
    sc = Scene("self_weight_column", 2, n, h, (0.0, 0.0, 0.0), x, vol, vol * rho0,
               np.zeros(x.shape[0], np.int32), [mat])
    ax, _ = _dofs(sc, lambda ix, iy: ix >= 0, 0, 2, n)
    by, _ = _dofs(sc, lambda ix, iy: iy <= 2, 1, 2, n)
    dof, val = _merge((ax, np.zeros(ax.shape)), (by, np.zeros(by.shape)))
    sc.steps = [LoadStep(dof, val, (0.0, -g * (k + 1) / nsteps, 0.0)) for k in range(nsteps)]
    sc.meta = dict(l0=l0, rho0=rho0, g=g, y_base=2 * h)
    return sc


def terzaghi(ncell: int = 100, H: float = 10.0, ppc: int = 2, lam: float = 600e3, mu: float = 600e3,
             k_hyd: float = 9.81e-9, t_load: float = 1e3, dt: float = 1e5, nsteps: int = 40,
             ncell_x: int = 1) -> Scene:
    """One-dimensional consolidation (paper Sec. 4.4): a column H = 10 m tall,
    one cell wide and ``ncell`` cells high (100 in the paper) with 2x2
    particles per cell, Neo-Hookean skeleton with lambda = mu = 600 kPa,
    a surface load t = 1 kPa on the top, which is also the only drained
    boundary, time step 1e5 s.  The paper's intrinsic permeability 1e-15 m^2
    with a fluid of density 1 t/m^3 (and water's viscosity 1e-3 Pa s) is the
    hydraulic conductivity 9.81e-9 m/s, giving c_v = k/gamma_w (lambda + 2 mu)
    = 1.8e-6 m^2/s as the paper states.

    u-p scene: DOFs (u_x, u_y, p) per node.  u_x = 0 on every node (rollers
    on both sides of a one-cell column), u_y = 0 on the base nodes (y <= base),
    p = 0 on the top nodes (y >= top); no gravity (p is the excess pressure).
    The load is a force of t * h / ppc on each particle of the top lattice row
    (its share of the loaded face).  ``ncell_x`` > 1 gives a wider column
    (rollers on its two side walls only, u_x free inside)."""
    h = H / ncell
    n = (ncell_x + 2, ncell + 2, 0)
    cells = box_cells((1, 1), (1 + ncell_x, 1 + ncell))
    x = lattice(cells, h, ppc, 2)
    E = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    mat = Material(model=MODEL_NH, E=E, nu=nu, rho=2000.0, k_hyd=k_hyd)
    vol = np.full(x.shape[0], h * h / ppc ** 2)
    sc = Scene("terzaghi", 2, n, h, (0.0, 0.0, 0.0), x, vol, vol * mat.rho,
               np.zeros(x.shape[0], np.int32), [mat], formulation="up", dt=dt)
    y_top = (1 + ncell) * h
    fext = np.zeros((x.shape[0], 3))
    top_row = x[:, 1] > y_top - h / ppc
    fext[top_row, 1] = -t_load * h / ppc
    sc.fext = fext
    B = 3
    if ncell_x == 1:
        ax, _ = _dofs(sc, lambda ix, iy: ix >= 0, 0, 2, n, B)
    else:
        ax, _ = _dofs(sc, lambda ix, iy: (ix <= 1) | (ix >= 1 + ncell_x), 0, 2, n, B)
    by, _ = _dofs(sc, lambda ix, iy: iy <= 1, 1, 2, n, B)
    pt, _ = _dofs(sc, lambda ix, iy: iy >= 1 + ncell, 2, 2, n, B)
    dof, val = _merge((ax, np.zeros(ax.shape)), (by, np.zeros(by.shape)), (pt, np.zeros(pt.shape)))
    sc.steps = [LoadStep(dof, val, (0.0, 0.0, 0.0)) for _ in range(nsteps)]
    cv = k_hyd / mat.gamma_w * (lam + 2 * mu)
    sc.meta = dict(H=H, y_top=y_top, y_base=h, t_load=t_load, cv=cv, dt=dt)
    return sc


# --------------------------------------------------------------------------
# serving stream
# --------------------------------------------------------------------------

SERVING_KINDS = ("elastic_block", "dp_footing", "up_terzaghi")


def serving_draws(n: int, seed: int = SEED_BASE + 4, cells_lo: float = 1e3, cells_hi: float = 6e4,
                  steps_lo: int = 10, steps_hi: int = 40):
    """Seeded request descriptors of the serving stream: kind uniform over the
    three kinds, grid cells log-uniform in [cells_lo, cells_hi], load steps
    uniform in [steps_lo, steps_hi]."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, len(SERVING_KINDS), size=n)
    cells = np.exp(rng.uniform(np.log(cells_lo), np.log(cells_hi), size=n))
    steps = rng.integers(steps_lo, steps_hi + 1, size=n)
    return [dict(kind=SERVING_KINDS[k], cells=float(c), nsteps=int(s)) for k, c, s in zip(kinds, cells, steps)]


# Newton tolerance of each serving kind: the footing requests stop at 1e-7
# (their small footing increments leave the residual's rounding floor at
# 5e-8 to 9e-8 of r0 on the largest requests, in FP64 as well)
SERVING_NEWTON_TOL = {"elastic_block": 1e-8, "dp_footing": 1e-7, "up_terzaghi": 1e-8}


def serving_scene(d, consolidation: str = "layer") -> Tuple[Scene, list]:
    """The scene and load steps of one serving request descriptor.
    elastic block: square grid of ~cells cells, block on a quarter of it,
    1 % strain over the steps; footing: nx = 2 ny with nx*ny ~ cells, h = 0.1,
    B = nx h / 12.8, nu = 0.35, at-rest prestress, settlement 0.0003 B per step after the geostatic step; Terzaghi: a
    column 16 cells wide, k = 1e-9 m/s, and
    * consolidation="full": N = cells/16 clipped to [64, 512] cells high, the
      load steps spanning T = c_v t / H^2 in [0, 1] (c_v dt / h^2 = N^2 /
      nsteps, up to about 17,000; solved with the multigrid V-cycle);
    * consolidation="layer": N clipped to [64, 256], c_v dt / h^2 = 10 (the
      early, boundary-layer part of the consolidation, which block-Jacobi
      Krylov solves reliably)."""
    kind, cells, ns = d["kind"], d["cells"], d["nsteps"]
    if kind == "elastic_block":
        ng = max(32, int(round(np.sqrt(cells) / 16)) * 16)
        sc = block_compression(nsteps=ns, strain_per_step=0.01 / ns, ngrid=ng)
        return sc, sc.steps
    if kind == "dp_footing":
        # footing width in the proportions of the 256 x 128 footing
        # (B = domain width / 12.8); 0.0003 B per step keeps the 40-step
        # requests short of the bearing-capacity plateau (at 0.001 B per step
        # the narrower footings reach it after about 30 steps, at 0.0005 B a
        # few of the larger ones after 14 to 23 steps, and Newton stalls
        # there on the GPU and in the oracle alike).  nu = 0.35: with
        # nu = 0.3 the at-rest state (K0 = nu / (1 - nu) = 0.43) lies outside
        # the Drucker-Prager cone below about 6.5 m, so the geostatic step
        # leaves half of a deep request plastic, and the first footing
        # increments unload it: Newton then stalls near 1e-6 on the GPU and in
        # the oracle alike; with K0 = 0.54 the geostatic state is elastic.
        # The soil starts from the at-rest prestress: from b_e = 1 a 17 m
        # layer settles by 0.2 m (two cells) in the geostatic step, and the
        # prescribed surface nodes of the footing fall outside every
        # particle's stencil
        ny = max(16, int(round(np.sqrt(cells / 2.0))))
        B = 2 * ny * 0.1 / 12.8
        sc = footing(nx=2 * ny, ny=ny, h=0.1, nsteps=ns - 1, B=B, settle_frac=0.0003 * (ns - 1), nu=0.35,
                     prestress=True)
        return sc, sc.steps
    full = consolidation == "full"
    N = int(np.clip(round(cells / 16.0), 64, 512 if full else 256))
    lam = mu = 600e3
    k_hyd = 1e-9
    cv = k_hyd / 9810.0 * (lam + 2 * mu)
    hh = 10.0 / N
    dt = (10.0 * 10.0 / (cv * ns)) if full else 10.0 * hh * hh / cv
    sc = terzaghi(ncell=N, ncell_x=16, k_hyd=k_hyd, dt=dt, nsteps=ns)
    return sc, sc.steps


def tiny_scene(dim: int, model: int, seed: int, ncell: int = 4, ppc: int = 2,
               jitter: float = 0.15) -> Scene:
    """A few cells of jittered particles in the middle of a small grid, for
    finite-difference and parity checks on random states.  Materials are
    chosen so that a modest random increment drives part of the particles
    plastic."""
    rng = np.random.default_rng(seed)
    ng = ncell + 6
    n = (ng, ng, ng if dim == 3 else 0)
    h = 0.1
    lo = (3,) * dim
    hi = (3 + ncell,) * dim
    cells = box_cells(lo, hi)
    x = lattice(cells, h, ppc, dim)
    x[:, :dim] += rng.uniform(-jitter, jitter, size=(x.shape[0], dim)) * h / ppc
    if model == MODEL_NH:
        mat = Material(model=MODEL_NH, E=1e6, nu=0.3, rho=1000.0)
    elif model == MODEL_NH_DP:
        mat = Material(model=MODEL_NH_DP, E=1e6, nu=0.3, rho=1000.0, phi=30.0, psi=0.0, c=2e3)
    else:
        mat = Material(model=MODEL_NH_MCC, E=1e6, nu=0.3, rho=1000.0, M=1.2, lambda_cc=0.1,
                       kappa_cc=0.02, pc0=-2e4)
    vol = np.full(x.shape[0], h ** dim / ppc ** dim)
    sc = Scene(f"tiny{dim}d_m{model}", dim, n, h, (0.0, 0.0, 0.0), x, vol, vol * mat.rho,
               np.zeros(x.shape[0], np.int32), [mat])
    return sc


def random_increment(scene: Scene, amplitude: float, seed: int) -> np.ndarray:
    """A smooth-ish random nodal displacement increment (nnode*dim), scaled so
    that the increment's gradient is about ``amplitude``."""
    rng = np.random.default_rng(seed)
    du = rng.standard_normal(scene.nnode * scene.dim) * amplitude * scene.h
    return du
