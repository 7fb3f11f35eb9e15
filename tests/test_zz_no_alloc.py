"""The allocation-free residual norm, mpm_residual_norm_noalloc, for callers
that cannot call cudaMalloc where they check Newton convergence (a host
framework owns all device memory, or allocation is forbidden after start-up).

It is compared, through the C ABI, with the free-DOF residual norm that the
scene's own Newton driver reports (mpm_begin_step / mpm_newton_step), within
the residual parity tolerance of the other GPU tests, on two calls in a row
at each of two iterates.  The test allocates its input buffers itself (with
torch); the entry point allocates nothing.  This file is collected last."""
import numpy as np
import pytest

from parity_util import RES_TOL

pytestmark = pytest.mark.gpu


def _inputs(gs, sc, step, rng):
    import torch
    dim = sc.dim
    fixed = np.zeros(sc.nnode * dim, dtype=np.uint8)
    fixed[np.asarray(step.dof)] = 1
    M = gs.mass()
    rows = np.nonzero(M > 1e-12 * sc.mass.max())[0].astype(np.int32)
    r = gs.residual()
    # values on prescribed DOFs must be skipped by the norm
    r[fixed == 1] = rng.standard_normal(int(fixed.sum())) * 1e6
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(r).to(dev), torch.from_numpy(rows).to(dev), torch.from_numpy(fixed).to(dev),
            len(rows))


def test_noalloc_norm_matches_the_scene_norm_on_two_calls_in_a_row():
    import torch
    from paper_2507_09435_gb300 import mpm, scenes as S
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    gs = mpm.GpuScene(sc, newton_tol=1e-8)
    step = sc.steps[0]
    ref = gs.begin(step).r_norm
    for stage in range(2):
        r_t, rows_t, fixed_t, nrow = _inputs(gs, sc, step, rng)
        torch.cuda.synchronize()
        for _ in range(2):
            got = mpm.mpm_residual_norm_noalloc(r_t.data_ptr(), rows_t.data_ptr(), nrow, fixed_t.data_ptr(),
                                                sc.dim)
            assert abs(got - ref) <= RES_TOL * ref, (stage, got, ref)
        ref = gs.newton().r_norm
    gs.close()


def test_noalloc_norm_smaller_call_after_larger_empty_call_and_own_stream():
    """The shared scratch keeps the last call's partial sums: a call over a
    prefix of the rows right after the full call must not see the full
    call's extra partials; nrow = 0 gives 0; a caller's stream works."""
    import torch
    from paper_2507_09435_gb300 import mpm, scenes as S
    torch.cuda.set_device(0)
    rng = np.random.default_rng(11)
    sc = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    gs = mpm.GpuScene(sc, newton_tol=1e-8)
    step = sc.steps[0]
    gs.begin(step)
    r_t, rows_t, fixed_t, nrow = _inputs(gs, sc, step, rng)
    gs.close()
    r = r_t.cpu().numpy()
    rows = rows_t.cpu().numpy()
    fixed = fixed_t.cpu().numpy()
    dim = sc.dim

    def numpy_norm(n):
        d = (rows[:n, None].astype(np.int64) * dim + np.arange(dim)[None, :]).ravel()
        d = d[fixed[d] == 0]
        return float(np.sqrt(np.sum(r[d] ** 2)))

    torch.cuda.synchronize()
    full = mpm.mpm_residual_norm_noalloc(r_t.data_ptr(), rows_t.data_ptr(), nrow, fixed_t.data_ptr(), dim)
    assert abs(full - numpy_norm(nrow)) <= RES_TOL * numpy_norm(nrow)
    # a prefix ending inside the first block, then one spanning a few blocks
    for n in (100, 3 * 256 + 17):
        assert n < nrow
        got = mpm.mpm_residual_norm_noalloc(r_t.data_ptr(), rows_t.data_ptr(), n, fixed_t.data_ptr(), dim)
        assert abs(got - numpy_norm(n)) <= RES_TOL * numpy_norm(n), (n, got, numpy_norm(n))
    assert mpm.mpm_residual_norm_noalloc(r_t.data_ptr(), rows_t.data_ptr(), 0, fixed_t.data_ptr(), dim) == 0.0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    got = mpm.mpm_residual_norm_noalloc(r_t.data_ptr(), rows_t.data_ptr(), nrow, fixed_t.data_ptr(), dim,
                                        stream=s.cuda_stream)
    assert abs(got - full) <= RES_TOL * full


def test_noalloc_norm_rejects_sizes_beyond_its_limit():
    from paper_2507_09435_gb300 import mpm
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_residual_norm_noalloc(0, 0, 8192 * 256 + 1, 0, 2)
    assert e.value.status == 1 and "limit" in str(e.value)
