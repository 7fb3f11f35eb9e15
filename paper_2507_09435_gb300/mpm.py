"""Thin Python binding of the C ABI in include/mpm.h (argument marshalling
only; every step of the Newton path runs in libmpm's CUDA kernels).

Function names match the C symbols.  Arrays are NumPy host arrays (or
anything ``np.ascontiguousarray`` accepts, e.g. a CPU/pinned torch tensor's
``.numpy()``).  There is no CPU fallback: if ``libmpm.so`` cannot be built or
loaded, or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MPM_OK = 0
MPM_NH, MPM_NH_DP, MPM_NH_MCC = 0, 1, 2
MPM_FP64, MPM_MIXED = 0, 1
MPM_BICGSTAB, MPM_GMRES = 0, 1
MPM_FORCING_FIXED, MPM_FORCING_EW = 0, 1
MPM_SOLID, MPM_UP = 0, 1
MPM_PC_AUTO, MPM_PC_NODE, MPM_PC_SEG4, MPM_PC_MG = 0, 1, 2, 3

STATUS = {
    0: "MPM_OK", 1: "MPM_ERR_INVALID_ARG", 2: "MPM_ERR_OOM", 3: "MPM_ERR_CUDA",
    4: "MPM_ERR_NOT_CONVERGED", 5: "MPM_ERR_KRYLOV_MAXIT", 6: "MPM_ERR_KRYLOV_BREAKDOWN",
    7: "MPM_ERR_NONFINITE", 8: "MPM_ERR_TIMEOUT", 9: "MPM_ERR_BOUNDS", 10: "MPM_ERR_RETURN_MAP",
    11: "MPM_ERR_STATE",
}


class mpm_scene_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("precision", ctypes.c_int), ("krylov", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("newton_tol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int), ("forcing", ctypes.c_int), ("krylov_rtol", ctypes.c_double),
                ("krylov_maxit", ctypes.c_int), ("formulation", ctypes.c_int), ("dt", ctypes.c_double),
                ("p_scale", ctypes.c_double), ("precond", ctypes.c_int), ("jacobian_reuse", ctypes.c_int)]


class mpm_material(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho", ctypes.c_double), ("phi", ctypes.c_double), ("psi", ctypes.c_double),
                ("c", ctypes.c_double), ("M", ctypes.c_double), ("lambda_cc", ctypes.c_double),
                ("kappa_cc", ctypes.c_double), ("pc0", ctypes.c_double), ("k_hyd", ctypes.c_double),
                ("gamma_w", ctypes.c_double)]


class mpm_newton_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("krylov_iters", ctypes.c_int), ("krylov_rel", ctypes.c_double),
                ("krylov_rtol", ctypes.c_double), ("r_norm", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("n_plastic", ctypes.c_int)]


class mpm_step_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("krylov_iters_total", ctypes.c_int), ("r0_norm", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("hist", ctypes.c_double * 33),
                ("krylov_iters", ctypes.c_int * 32), ("n_active_nodes", ctypes.c_int),
                ("nnzb", ctypes.c_longlong), ("t_setup_ms", ctypes.c_double),
                ("t_residual_ms", ctypes.c_double), ("t_assembly_ms", ctypes.c_double),
                ("t_krylov_ms", ctypes.c_double), ("t_commit_ms", ctypes.c_double)]


class mpm_request(ctypes.Structure):
    _fields_ = [("desc", ctypes.POINTER(mpm_scene_desc)), ("np", ctypes.c_int),
                ("x", ctypes.POINTER(ctypes.c_double)), ("vol0", ctypes.POINTER(ctypes.c_double)),
                ("mass", ctypes.POINTER(ctypes.c_double)), ("mat_id", ctypes.POINTER(ctypes.c_int)),
                ("E_p", ctypes.POINTER(ctypes.c_double)), ("phi_p", ctypes.POINTER(ctypes.c_double)),
                ("pc0_p", ctypes.POINTER(ctypes.c_double)), ("be0", ctypes.POINTER(ctypes.c_double)),
                ("mats", ctypes.POINTER(mpm_material)), ("nmat", ctypes.c_int),
                ("ntraction", ctypes.c_int), ("traction_particle", ctypes.POINTER(ctypes.c_int)),
                ("traction_force", ctypes.POINTER(ctypes.c_double)), ("nsteps", ctypes.c_int),
                ("step_ndof", ctypes.POINTER(ctypes.c_int)), ("step_dof", ctypes.POINTER(ctypes.c_longlong)),
                ("step_value", ctypes.POINTER(ctypes.c_double)), ("step_gravity", ctypes.POINTER(ctypes.c_double))]


class mpm_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("krylov_iters", ctypes.c_int), ("t_queue_ms", ctypes.c_double), ("t_service_ms", ctypes.c_double),
                ("t_latency_ms", ctypes.c_double), ("footprint", ctypes.c_size_t), ("slot", ctypes.c_int)]


class mpm_server_stats(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("budget", ctypes.c_size_t), ("in_use", ctypes.c_size_t),
                ("peak_in_use", ctypes.c_size_t), ("running", ctypes.c_int), ("peak_running", ctypes.c_int),
                ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong)]


class MPMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_LL = ctypes.POINTER(ctypes.c_longlong)
_P = ctypes.c_void_p
_lib = None

# every symbol declared in include/mpm.h
EXPORTS = ["mpm_create_scene", "mpm_set_gravity", "mpm_set_dirichlet", "mpm_begin_step", "mpm_newton_step",
           "mpm_set_du", "mpm_assemble", "mpm_commit_step", "mpm_solve_step", "mpm_get_residual", "mpm_get_du", "mpm_get_mass",
           "mpm_get_counts", "mpm_get_jacobian_bsr", "mpm_get_mg_level", "mpm_mg_apply", "mpm_get_particles", "mpm_get_pressure",
           "mpm_get_du_dev", "mpm_get_residual_dev", "mpm_get_positions_dev", "mpm_set_dirichlet_dev",
           "mpm_set_traction", "mpm_kernel_launches", "mpm_get_newton_counters", "mpm_fma_peak", "mpm_set_params", "mpm_get_particle_increment",
           "mpm_adjoint", "mpm_adjoint_step", "mpm_set_state",
           "mpm_time_spmv", "mpm_set_particles", "mpm_residual_norm_noalloc", "mpm_noalloc_last_error",
           "mpm_footprint_bytes",
           "mpm_destroy_scene", "mpm_status_string", "mpm_last_error",
           # include/mpm_serve.h
           "mpm_server_create", "mpm_server_submit", "mpm_server_wait", "mpm_server_result_particles",
           "mpm_server_release", "mpm_server_get_stats", "mpm_server_destroy"]


def lib(build: bool = True):
    """Load libmpm.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmpm.so not found at {path}")
    L = ctypes.CDLL(path)
    L.mpm_create_scene.argtypes = [ctypes.POINTER(mpm_scene_desc), ctypes.c_int, _D, _D, _D, _I, _D, _D, _D,
                                   ctypes.POINTER(mpm_material), ctypes.c_int, _P, ctypes.POINTER(_P)]
    L.mpm_set_gravity.argtypes = [_P, _D]
    L.mpm_set_dirichlet.argtypes = [_P, ctypes.c_int, _LL, _D]
    L.mpm_begin_step.argtypes = [_P, ctypes.POINTER(mpm_newton_report)]
    L.mpm_newton_step.argtypes = [_P, ctypes.POINTER(mpm_newton_report)]
    L.mpm_set_du.argtypes = [_P, _D]
    L.mpm_assemble.argtypes = [_P]
    L.mpm_commit_step.argtypes = [_P]
    L.mpm_solve_step.argtypes = [_P, ctypes.POINTER(mpm_step_report)]
    L.mpm_get_residual.argtypes = [_P, _D]
    L.mpm_get_du.argtypes = [_P, _D]
    L.mpm_get_mass.argtypes = [_P, _D]
    L.mpm_get_counts.argtypes = [_P, _I, _LL]
    L.mpm_get_jacobian_bsr.argtypes = [_P, ctypes.c_longlong, _I, _LL, _I, _D]
    L.mpm_mg_apply.argtypes = [_P, _D, _D]
    L.mpm_get_mg_level.argtypes = [_P, ctypes.c_int, _I, _I, _I, ctypes.c_int, _I, _D,
                                   ctypes.POINTER(ctypes.c_ubyte), _D]
    L.mpm_get_particles.argtypes = [_P, _D, _D, _D, _D, _D]
    L.mpm_get_du_dev.argtypes = [_P, _P]
    L.mpm_get_residual_dev.argtypes = [_P, _P]
    L.mpm_get_positions_dev.argtypes = [_P, _P]
    L.mpm_set_dirichlet_dev.argtypes = [_P, ctypes.c_int, _P, _P]
    L.mpm_get_pressure.argtypes = [_P, _D]
    L.mpm_set_traction.argtypes = [_P, ctypes.c_int, _I, _D]
    L.mpm_set_params.argtypes = [_P, _D, _D, _D]
    L.mpm_get_particle_increment.argtypes = [_P, _D]
    L.mpm_adjoint.argtypes = [_P, _D, _D, _D, _D, _D]
    L.mpm_adjoint_step.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _D, _D]
    L.mpm_set_state.argtypes = [_P, _D, _D, _D, _D]
    L.mpm_kernel_launches.argtypes = [_P, _LL]
    L.mpm_get_newton_counters.argtypes = [_P, _LL, _LL]
    L.mpm_fma_peak.argtypes = [ctypes.c_int, _D]
    L.mpm_set_particles.argtypes = [_P, _D, _D, _D]
    L.mpm_residual_norm_noalloc.argtypes = [_P, _P, ctypes.c_int, _P, ctypes.c_int, _D, _P]
    L.mpm_noalloc_last_error.argtypes = []
    L.mpm_noalloc_last_error.restype = ctypes.c_char_p
    L.mpm_time_spmv.argtypes = [_P, ctypes.c_int, _D, _D]
    L.mpm_footprint_bytes.argtypes = [ctypes.POINTER(mpm_scene_desc), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_size_t)]
    L.mpm_destroy_scene.argtypes = [_P]
    L.mpm_destroy_scene.restype = None
    L.mpm_status_string.argtypes = [ctypes.c_int]
    L.mpm_status_string.restype = ctypes.c_char_p
    L.mpm_last_error.argtypes = [_P]
    L.mpm_last_error.restype = ctypes.c_char_p
    L.mpm_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)]
    L.mpm_server_submit.argtypes = [_P, ctypes.POINTER(mpm_request), _LL]
    L.mpm_server_wait.argtypes = [_P, ctypes.c_longlong, ctypes.POINTER(mpm_request_result)]
    L.mpm_server_result_particles.argtypes = [_P, ctypes.c_longlong, _D, _D]
    L.mpm_server_release.argtypes = [_P, ctypes.c_longlong]
    L.mpm_server_get_stats.argtypes = [_P, ctypes.POINTER(mpm_server_stats)]
    L.mpm_server_destroy.argtypes = [_P]
    L.mpm_server_destroy.restype = None
    for name in EXPORTS:
        if name not in ("mpm_destroy_scene", "mpm_status_string", "mpm_last_error", "mpm_noalloc_last_error",
                        "mpm_server_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _p(a, t=_D):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, handle=None):
    if rc != MPM_OK:
        msg = lib().mpm_last_error(handle).decode() if handle is not None or rc else ""
        raise MPMError(rc, msg)


def make_desc(dim, n, h, origin=(0.0, 0.0, 0.0), precision=MPM_FP64, krylov=MPM_BICGSTAB, gmres_restart=30,
              newton_tol=1e-8, newton_maxit=25, forcing=None, krylov_rtol=None, krylov_maxit=20000,
              formulation=MPM_SOLID, dt=0.0, p_scale=0.0, precond=MPM_PC_AUTO, jacobian_reuse=0):
    d = mpm_scene_desc()
    d.dim = dim
    for a in range(3):
        d.n[a] = int(n[a]) if a < len(n) else 0
        d.origin[a] = float(origin[a]) if a < len(origin) else 0.0
    d.h = float(h)
    d.precision = precision
    d.krylov = krylov
    d.gmres_restart = gmres_restart
    d.newton_tol = newton_tol
    d.newton_maxit = newton_maxit
    if forcing is None:
        forcing = MPM_FORCING_EW if precision == MPM_MIXED else MPM_FORCING_FIXED
    if krylov_rtol is None:
        krylov_rtol = 1e-6 if precision == MPM_MIXED else 1e-10
    d.forcing = forcing
    d.krylov_rtol = krylov_rtol
    d.krylov_maxit = krylov_maxit
    d.formulation = formulation
    d.dt = float(dt)
    d.p_scale = float(p_scale)
    d.precond = int(precond)
    d.jacobian_reuse = int(jacobian_reuse)
    return d


def mpm_footprint_bytes(desc, np_):
    out = ctypes.c_size_t(0)
    _check(lib().mpm_footprint_bytes(ctypes.byref(desc), int(np_), ctypes.byref(out)))
    return int(out.value)


def mpm_create_scene(desc, x, vol0, mass, mat_id, mats, E_p=None, phi_p=None, pc0_p=None, stream=None):
    x = _f64(x)
    np_ = x.shape[0]
    x3 = np.zeros((np_, 3))
    x3[:, :x.shape[1]] = x
    mat_id = np.ascontiguousarray(mat_id, dtype=np.int32)
    marr = (mpm_material * len(mats))(*mats)
    h = _P()
    L = lib()
    rc = L.mpm_create_scene(ctypes.byref(desc), np_, _p(x3), _p(_f64(vol0)), _p(_f64(mass)), _p(mat_id, _I),
                            _p(_f64(E_p)), _p(_f64(phi_p)), _p(_f64(pc0_p)), marr, len(mats),
                            _P(stream) if stream else None, ctypes.byref(h))
    if rc != MPM_OK:
        raise MPMError(rc, L.mpm_last_error(None).decode())
    return h


def mpm_destroy_scene(h):
    lib().mpm_destroy_scene(h)


def mpm_set_gravity(h, g):
    _check(lib().mpm_set_gravity(h, _p(_f64(np.asarray(g, dtype=np.float64).reshape(3)))), h)


def mpm_set_dirichlet(h, dof, value):
    dof = np.ascontiguousarray(dof, dtype=np.int64)
    value = _f64(value)
    _check(lib().mpm_set_dirichlet(h, int(dof.size), _p(dof, _LL), _p(value)), h)


def mpm_begin_step(h):
    rep = mpm_newton_report()
    _check(lib().mpm_begin_step(h, ctypes.byref(rep)), h)
    return rep


def mpm_newton_step(h):
    rep = mpm_newton_report()
    _check(lib().mpm_newton_step(h, ctypes.byref(rep)), h)
    return rep


def mpm_set_du(h, du):
    _check(lib().mpm_set_du(h, _p(_f64(du))), h)


def mpm_assemble(h):
    _check(lib().mpm_assemble(h), h)


def mpm_commit_step(h):
    _check(lib().mpm_commit_step(h), h)


def mpm_solve_step(h, check=True):
    rep = mpm_step_report()
    rc = lib().mpm_solve_step(h, ctypes.byref(rep))
    if check:
        _check(rc, h)
    return rep


def mpm_get_residual(h, ndof):
    r = np.zeros(ndof)
    _check(lib().mpm_get_residual(h, _p(r)), h)
    return r


def mpm_get_du(h, ndof):
    r = np.zeros(ndof)
    _check(lib().mpm_get_du(h, _p(r)), h)
    return r


def mpm_get_mass(h, nnode):
    r = np.zeros(nnode)
    _check(lib().mpm_get_mass(h, _p(r)), h)
    return r


def mpm_get_counts(h):
    na = ctypes.c_int(0)
    nb = ctypes.c_longlong(0)
    _check(lib().mpm_get_counts(h, ctypes.byref(na), ctypes.byref(nb)), h)
    return na.value, nb.value


def _dev_ptr(t, n, dtype):
    """Data pointer of a contiguous CUDA tensor of `n` elements of `dtype`."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == dtype and t.numel() >= n):
        raise ValueError(f"need a contiguous CUDA {dtype} tensor of at least {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def mpm_get_du_dev(h, out, ndof):
    import torch
    _check(lib().mpm_get_du_dev(h, _dev_ptr(out, ndof, torch.float64)), h)
    return out


def mpm_get_residual_dev(h, out, ndof):
    import torch
    _check(lib().mpm_get_residual_dev(h, _dev_ptr(out, ndof, torch.float64)), h)
    return out


def mpm_get_positions_dev(h, out, np_):
    import torch
    _check(lib().mpm_get_positions_dev(h, _dev_ptr(out, 3 * np_, torch.float64)), h)
    return out


def mpm_set_dirichlet_dev(h, dof, value):
    import torch
    n = int(dof.numel())
    if int(value.numel()) != n:
        raise ValueError("dof and value lengths differ")
    _check(lib().mpm_set_dirichlet_dev(h, n, _dev_ptr(dof, n, torch.int64), _dev_ptr(value, n, torch.float64)), h)


def mpm_get_mg_level(h, level, dim, B):
    """Coarse level `level` >= 1 of the multigrid hierarchy: dict with levels,
    dims, nodes, vals[nrow, 5**dim, B, B], fixed[nnode*B], lambda_max."""
    levels = ctypes.c_int(0)
    if level == 0:
        lam = ctypes.c_double(0.0)
        _check(lib().mpm_get_mg_level(h, 0, ctypes.byref(levels), None, None, 0, None, None, None,
                                      ctypes.byref(lam)), h)
        return dict(levels=levels.value, lambda_max=lam.value)
    dims = np.zeros(3, dtype=np.int32)
    nrow = ctypes.c_int(0)
    _check(lib().mpm_get_mg_level(h, level, ctypes.byref(levels), _p(dims, _I), ctypes.byref(nrow), 0, None,
                                  None, None, None), h)
    n = nrow.value
    S = 5 ** dim
    nodes = np.zeros(max(n, 1), dtype=np.int32)
    vals = np.zeros(max(n, 1) * S * B * B)
    fixed = np.zeros(int(np.prod(dims)) * B, dtype=np.uint8)
    lam = ctypes.c_double(0.0)
    _check(lib().mpm_get_mg_level(h, level, ctypes.byref(levels), _p(dims, _I), ctypes.byref(nrow), n,
                                  _p(nodes, _I), _p(vals), fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                  ctypes.byref(lam)), h)
    return dict(levels=levels.value, dims=dims, nodes=nodes[:n], vals=vals[:n * S * B * B].reshape(n, S, B, B),
                fixed=fixed.astype(bool), lambda_max=lam.value)


def mpm_mg_apply(h, b):
    """z = M^-1 b, one V-cycle of the last assembly's multigrid hierarchy
    (b: nnode*B doubles; z the same)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    z = np.zeros_like(b)
    _check(lib().mpm_mg_apply(h, _p(b), _p(z)), h)
    return z


def mpm_get_jacobian_bsr(h, dim):
    na, nb = mpm_get_counts(h)
    row_node = np.zeros(na, dtype=np.int32)
    row_ptr = np.zeros(na + 1, dtype=np.int64)
    col_node = np.zeros(max(nb, 1), dtype=np.int32)
    val = np.zeros(max(nb, 1) * dim * dim)
    _check(lib().mpm_get_jacobian_bsr(h, nb, _p(row_node, _I), _p(row_ptr, _LL), _p(col_node, _I), _p(val)), h)
    return row_node, row_ptr, col_node[:nb], val[:nb * dim * dim].reshape(nb, dim, dim)


def mpm_get_particles(h, np_, x=True, be=True, pc=True, F=True, tau=True):
    out = {}
    bufs = {}
    for k, sz, want in (("x", 3, x), ("be", 6, be), ("pc", 1, pc), ("F", 9, F), ("tau", 9, tau)):
        bufs[k] = np.zeros(np_ * sz) if want else None
    _check(lib().mpm_get_particles(h, _p(bufs["x"]), _p(bufs["be"]), _p(bufs["pc"]), _p(bufs["F"]),
                                   _p(bufs["tau"])), h)
    if x:
        out["x"] = bufs["x"].reshape(np_, 3)
    if be:
        out["be"] = bufs["be"].reshape(np_, 6)
    if pc:
        out["pc"] = bufs["pc"]
    if F:
        out["F"] = bufs["F"].reshape(np_, 3, 3)
    if tau:
        out["tau"] = bufs["tau"].reshape(np_, 3, 3)
    return out


def mpm_get_pressure(h, np_):
    out = np.zeros(np_)
    _check(lib().mpm_get_pressure(h, _p(out)), h)
    return out


def mpm_set_traction(h, particle, f):
    particle = np.ascontiguousarray(particle, dtype=np.int32)
    f = _f64(np.asarray(f, dtype=np.float64).reshape(-1, 3))
    _check(lib().mpm_set_traction(h, int(particle.size), _p(particle, _I), _p(f)), h)


def mpm_set_params(h, E_p=None, phi_p=None, k_p=None):
    _check(lib().mpm_set_params(h, _p(_f64(E_p)), _p(_f64(phi_p)), _p(_f64(k_p))), h)


def mpm_get_particle_increment(h, np_):
    out = np.zeros(np_ * 3)
    _check(lib().mpm_get_particle_increment(h, _p(out)), h)
    return out.reshape(np_, 3)


def mpm_adjoint(h, np_, nmat, dL_dU=None, dL_dx=None, want_E=True, want_phi=True, want_k=False):
    """dL/dE_p, dL/dphi_p (np each) and dL/dk per material of the staged,
    converged step (see include/mpm.h)."""
    gE = np.zeros(max(np_, 1)) if want_E else None
    gP = np.zeros(max(np_, 1)) if want_phi else None
    gK = np.zeros(nmat) if want_k else None
    x = None if dL_dx is None else _f64(np.asarray(dL_dx, dtype=np.float64).reshape(np_, 3))
    _check(lib().mpm_adjoint(h, _p(_f64(dL_dU)), _p(x), _p(gE), _p(gP), _p(gK)), h)
    return (gE[:np_] if gE is not None else None, gP[:np_] if gP is not None else None, gK)


def mpm_adjoint_step(h, np_, sbar, dL_dU=None, dL_dx=None, grads=None):
    """One step of the reverse chain (include/mpm.h).  `sbar` is a dict of
    x (np,3), be (np,6), pc (np,), F (np,3,3) arrays, updated in place from
    dL/ds_n to dL/ds_{n-1}; `grads` a dict of E, phi (np,) and k (nmat,)
    arrays that the gradients are added to."""
    for k in ("x", "be", "pc", "F"):
        sbar[k] = np.ascontiguousarray(sbar[k], dtype=np.float64)
    x = None if dL_dx is None else _f64(np.asarray(dL_dx, dtype=np.float64).reshape(np_, 3))
    g = grads or {}
    _check(lib().mpm_adjoint_step(h, _p(_f64(dL_dU)), _p(x), _p(sbar["x"]), _p(sbar["be"]), _p(sbar["pc"]),
                                  _p(sbar["F"]), _p(g.get("E")), _p(g.get("phi")), _p(g.get("k"))), h)
    return sbar


def mpm_set_state(h, x=None, be=None, pc=None, F=None):
    _check(lib().mpm_set_state(h, _p(_f64(x)), _p(_f64(be)), _p(_f64(pc)), _p(_f64(F))), h)


def mpm_set_particles(h, be=None, pc=None, F=None):
    _check(lib().mpm_set_particles(h, _p(_f64(be)), _p(_f64(pc)), _p(_f64(F))), h)


def mpm_residual_norm_noalloc(r_dev, rows_dev, nrow, fixed_dev, dim, stream=None):
    """Free-DOF residual norm from caller-owned device buffers (integer device
    addresses), using no device allocation; see include/mpm.h."""
    out = ctypes.c_double(0)
    rc = lib().mpm_residual_norm_noalloc(_P(r_dev), _P(rows_dev), int(nrow), _P(fixed_dev), int(dim),
                                         ctypes.byref(out), _P(stream) if stream else None)
    if rc != MPM_OK:
        raise MPMError(rc, lib().mpm_noalloc_last_error().decode())
    return out.value


def mpm_kernel_launches(h):
    out = ctypes.c_longlong(0)
    _check(lib().mpm_kernel_launches(h, ctypes.byref(out)), h)
    return int(out.value)


def mpm_get_newton_counters(h):
    """(limited, halvings): Newton corrections scaled by the step-length
    limit and halved steps, counted since the scene was created."""
    lim = ctypes.c_longlong(0)
    hal = ctypes.c_longlong(0)
    _check(lib().mpm_get_newton_counters(h, ctypes.byref(lim), ctypes.byref(hal)), h)
    return int(lim.value), int(hal.value)


def mpm_fma_peak(precision):
    """Measured FMA throughput of the current device in TFLOP/s (MPM_FP64 or
    MPM_MIXED for FP32)."""
    out = ctypes.c_double(0)
    rc = lib().mpm_fma_peak(int(precision), ctypes.byref(out))
    if rc != MPM_OK:
        raise MPMError(rc, "mpm_fma_peak failed")
    return out.value


def mpm_time_spmv(h, reps):
    ms = ctypes.c_double(0)
    by = ctypes.c_double(0)
    _check(lib().mpm_time_spmv(h, int(reps), ctypes.byref(ms), ctypes.byref(by)), h)
    return ms.value, by.value


# --------------------------------------------------------------------------
# convenience wrapper over a generated scene (see scenes.py)
# --------------------------------------------------------------------------

def materials_of(scene):
    out = []
    for m in scene.materials:
        q = mpm_material()
        q.model, q.E, q.nu, q.rho = m.model, m.E, m.nu, m.rho
        q.phi, q.psi, q.c = m.phi, m.psi, m.c
        q.M, q.lambda_cc, q.kappa_cc, q.pc0 = m.M, m.lambda_cc, m.kappa_cc, m.pc0
        q.k_hyd, q.gamma_w = getattr(m, "k_hyd", 0.0), getattr(m, "gamma_w", 9810.0)
        out.append(q)
    return out


class GpuScene:
    """A scene resident on the GPU, driven load step by load step."""

    def __init__(self, scene, precision=MPM_FP64, krylov=MPM_BICGSTAB, stream=None, **kw):
        self.scene = scene
        self.dim = scene.dim
        up = getattr(scene, "formulation", "solid") == "up"
        self.B = scene.dim + (1 if up else 0)
        if up:
            kw.setdefault("formulation", MPM_UP)
            kw.setdefault("dt", scene.dt)
        self.desc = make_desc(scene.dim, scene.n, scene.h, scene.origin, precision=precision, krylov=krylov,
                              **kw)
        self.h = mpm_create_scene(self.desc, scene.x[:, :scene.dim], scene.vol0, scene.mass, scene.mat_id,
                                  materials_of(scene), E_p=scene.E_p, phi_p=scene.phi_p, pc0_p=scene.pc0_p,
                                  stream=stream)
        self.nnode = scene.nnode
        self.ndof = scene.nnode * self.B
        self.np = scene.np
        if getattr(scene, "be0", None) is not None:
            mpm_set_particles(self.h, be=scene.be0)
        fext = getattr(scene, "fext", None)
        if fext is not None:
            idx = np.nonzero(np.abs(fext).sum(axis=1) > 0)[0]
            mpm_set_traction(self.h, idx, fext[idx])

    def close(self):
        if self.h is not None:
            mpm_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_step(self, step):
        mpm_set_dirichlet(self.h, step.dof, step.value)
        mpm_set_gravity(self.h, step.gravity)

    def solve_step(self, step, check=True):
        self.set_step(step)
        return mpm_solve_step(self.h, check=check)

    def begin(self, step):
        self.set_step(step)
        return mpm_begin_step(self.h)

    def newton(self):
        return mpm_newton_step(self.h)

    def commit(self):
        mpm_commit_step(self.h)

    def set_du(self, du):
        mpm_set_du(self.h, du)

    def assemble(self):
        mpm_assemble(self.h)

    def residual(self):
        return mpm_get_residual(self.h, self.ndof)

    def du(self):
        return mpm_get_du(self.h, self.ndof)

    def mass(self):
        return mpm_get_mass(self.h, self.nnode)

    def jacobian_bsr(self):
        return mpm_get_jacobian_bsr(self.h, self.B)

    def mg_level(self, level):
        return mpm_get_mg_level(self.h, level, self.dim, self.B)

    def mg_apply(self, b):
        if len(b) != self.ndof:
            raise ValueError(f"b has {len(b)} entries, the scene {self.ndof} DOFs")
        return mpm_mg_apply(self.h, b)

    # device-tensor variants (work on the scene's stream, no host sync)
    def du_into(self, out):
        return mpm_get_du_dev(self.h, out, self.ndof)

    def residual_into(self, out):
        return mpm_get_residual_dev(self.h, out, self.ndof)

    def positions_into(self, out):
        return mpm_get_positions_dev(self.h, out, self.np)

    def set_dirichlet_dev(self, dof, value):
        mpm_set_dirichlet_dev(self.h, dof, value)

    def pressure(self):
        return mpm_get_pressure(self.h, self.np)

    def particle_increment(self):
        return mpm_get_particle_increment(self.h, self.np)

    def set_params(self, E_p=None, phi_p=None, k_p=None):
        mpm_set_params(self.h, E_p, phi_p, k_p)

    def solve_staged(self, step, tol=None, maxit=None):
        """Begin the step and run Newton iterations to the scene's tolerance
        without committing (for the adjoint).  Returns the relative residual
        history."""
        tol = self.desc.newton_tol if tol is None else tol
        maxit = self.desc.newton_maxit if maxit is None else maxit
        self.begin(step)
        hist = [1.0]
        for _ in range(maxit):
            rel = self.newton().rel_residual
            hist.append(rel)
            if rel <= tol:
                return hist
        raise MPMError(4, f"Newton did not reach {tol} (last {hist[-1]:.3e})")

    def adjoint(self, dL_dU=None, dL_dx=None, want_E=True, want_phi=True, want_k=False):
        return mpm_adjoint(self.h, self.np, len(self.scene.materials), dL_dU=dL_dU, dL_dx=dL_dx,
                           want_E=want_E, want_phi=want_phi, want_k=want_k)

    def particles(self, **kw):
        return mpm_get_particles(self.h, self.np, **kw)


# --------------------------------------------------------------------------
# serving loop (include/mpm_serve.h)
# --------------------------------------------------------------------------

def scene_desc(scene, precision=MPM_MIXED, krylov=None, **kw):
    """The scene descriptor a generated scene is solved with (u-p scenes get
    their time step)."""
    up = getattr(scene, "formulation", "solid") == "up"
    if up:
        kw.setdefault("formulation", MPM_UP)
        kw.setdefault("dt", scene.dt)
    if krylov is None:
        krylov = MPM_BICGSTAB
    return make_desc(scene.dim, scene.n, scene.h, scene.origin, precision=precision, krylov=krylov, **kw)


class Server:
    """Continuous-batching server: ``slots`` worker threads with their own
    CUDA streams, admission by device footprint within ``budget`` bytes."""

    def __init__(self, slots=4, budget=0):
        h = _P()
        rc = lib().mpm_server_create(int(slots), int(budget), ctypes.byref(h))
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_server_create failed")
        self.h = h
        self._np = {}

    def submit(self, scene, steps=None, desc=None, **kw):
        """Queue the scene with its load steps (all by default); returns the
        ticket.  The arrays are copied by the call."""
        steps = scene.steps if steps is None else steps
        desc = desc if desc is not None else scene_desc(scene, **kw)
        np_ = scene.np
        x = np.zeros((np_, 3))
        x[:, :scene.dim] = scene.x[:, :scene.dim]
        keep = dict(x=x, vol0=_f64(scene.vol0), mass=_f64(scene.mass),
                    mat_id=np.ascontiguousarray(scene.mat_id, dtype=np.int32),
                    E_p=_f64(scene.E_p), phi_p=_f64(scene.phi_p), pc0_p=_f64(scene.pc0_p),
                    be0=_f64(getattr(scene, "be0", None)))
        mats = materials_of(scene)
        marr = (mpm_material * len(mats))(*mats)
        ndof = np.array([len(s.dof) for s in steps], dtype=np.int32)
        dof = np.ascontiguousarray(np.concatenate([np.asarray(s.dof, dtype=np.int64) for s in steps])
                                   if steps else np.zeros(0, np.int64))
        val = _f64(np.concatenate([np.asarray(s.value, dtype=np.float64) for s in steps])
                   if steps else np.zeros(0))
        grav = _f64(np.array([s.gravity for s in steps], dtype=np.float64).reshape(-1))
        fext = getattr(scene, "fext", None)
        if fext is not None:
            tp = np.ascontiguousarray(np.nonzero(np.abs(fext).sum(axis=1) > 0)[0], dtype=np.int32)
            tf = _f64(fext[tp])
        else:
            tp, tf = np.zeros(0, np.int32), np.zeros((0, 3))
        q = mpm_request()
        q.desc = ctypes.pointer(desc)
        q.np = np_
        q.x, q.vol0, q.mass = _p(keep["x"]), _p(keep["vol0"]), _p(keep["mass"])
        q.mat_id = _p(keep["mat_id"], _I)
        q.E_p, q.phi_p, q.pc0_p, q.be0 = _p(keep["E_p"]), _p(keep["phi_p"]), _p(keep["pc0_p"]), _p(keep["be0"])
        q.mats = ctypes.cast(marr, ctypes.POINTER(mpm_material))
        q.nmat = len(mats)
        q.ntraction = int(tp.size)
        q.traction_particle = _p(tp, _I) if tp.size else None
        q.traction_force = _p(tf) if tp.size else None
        q.nsteps = len(steps)
        q.step_ndof = _p(ndof, _I)
        q.step_dof = _p(dof, _LL) if dof.size else None
        q.step_value = _p(val) if val.size else None
        q.step_gravity = _p(grav)
        t = ctypes.c_longlong(0)
        rc = lib().mpm_server_submit(self.h, ctypes.byref(q), ctypes.byref(t))
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_server_submit rejected the request")
        self._np[t.value] = (np_, desc.formulation == MPM_UP)
        return t.value

    def wait(self, ticket):
        r = mpm_request_result()
        rc = lib().mpm_server_wait(self.h, int(ticket), ctypes.byref(r))
        if rc != MPM_OK:
            raise MPMError(rc, "unknown ticket")
        return r

    def particles(self, ticket):
        """(x[np,3], pore pressure[np] or None) of a finished request."""
        np_, up = self._np[ticket]
        x = np.zeros(np_ * 3)
        pp = np.zeros(np_) if up else None
        rc = lib().mpm_server_result_particles(self.h, int(ticket), _p(x), _p(pp))
        if rc != MPM_OK:
            raise MPMError(rc, "no particles for this ticket")
        return x.reshape(np_, 3), pp

    def release(self, ticket):
        lib().mpm_server_release(self.h, int(ticket))
        self._np.pop(ticket, None)

    def stats(self):
        st = mpm_server_stats()
        _check(lib().mpm_server_get_stats(self.h, ctypes.byref(st)))
        return st

    def close(self):
        if self.h is not None:
            lib().mpm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
