"""Serving loop (include/mpm_serve.h) on the GPU: each request's result is the
same alone and in a concurrent mix (within the Newton tolerance) and matches
the FP64 oracle solved step by step, requests overlap on the device,
admission keeps the running footprint within the budget, and a failing
request is reported without stopping the others."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2507_09435_gb300 import mpm, scenes as S

from parity_util import DU_TOL

pytestmark = pytest.mark.gpu


def _mix():
    """Small requests of the serving kinds: elastic block, Drucker-Prager
    footing, u-p Terzaghi column; different sizes and materials."""
    out = []
    out.append((S.block_compression(nsteps=4), None))
    blk = S.block_compression(nsteps=3, strain_per_step=2e-3)
    blk.materials[0].E = 3e6
    out.append((blk, None))
    fo = S.footing(nx=48, ny=24, h=0.5, nsteps=20, settle_frac=0.1)
    out.append((fo, fo.steps[:3]))
    fo2 = S.footing(nx=64, ny=32, h=0.4, nsteps=20, settle_frac=0.1)
    out.append((fo2, fo2.steps[:2]))
    out.append((S.terzaghi(ncell=24, dt=2e5, nsteps=4), None))
    out.append((S.terzaghi(ncell=40, dt=5e4, nsteps=3), None))
    return out


KW = dict(precision=mpm.MPM_FP64, newton_tol=1e-11, newton_maxit=30)


def _tol(sc):
    # the u-p columns' rounding floor is about 1.2e-12 (lateral pressure
    # modes are held only by the Darcy term), the solid requests reach 1e-12
    return 1e-11 if getattr(sc, "formulation", "solid") == "up" else 1e-12


def _oracle_result(sc, steps):
    """The request solved by the FP64 oracle, load step by load step, to the
    same relative residual as the served request."""
    orc = O.OracleScene.from_scene(sc)
    for st in (sc.steps if steps is None else steps):
        out = orc.solve_step(st.dof, st.value, st.gravity, tol=_tol(sc), maxit=40)
        assert out["converged"], (sc.name, out["hist"][-3:])
    return orc.x.copy(), (orc.pp.copy() if orc.formulation == "up" else None)


def _run_alone(sc, steps):
    sv = mpm.Server(slots=1)
    t = sv.submit(sc, steps=steps, **dict(KW, newton_tol=_tol(sc)))
    r = sv.wait(t)
    assert r.status == mpm.MPM_OK, mpm.STATUS.get(r.status)
    x, pp = sv.particles(t)
    sv.close()
    return x, pp


def test_same_alone_and_in_the_mix_and_as_the_oracle():
    """Every request of a concurrent FP64 mix: the same as when served alone,
    and the oracle's result (particle positions within 1e-7 of the request's
    displacement scale, u-p particle pressures within 1e-7 of their largest
    value: the converged-increment parity bar, both sides at the same
    relative residual)."""
    mix = _mix()
    alone = [_run_alone(sc, st) for sc, st in mix]
    sv = mpm.Server(slots=4)
    tickets = [sv.submit(sc, steps=st, **dict(KW, newton_tol=_tol(sc))) for sc, st in mix]
    res = [sv.wait(t) for t in tickets]
    stats = sv.stats()
    assert stats.peak_running >= 2, "requests should overlap on the device"
    for (sc, st), t, r, (xa, pa) in zip(mix, tickets, res, alone):
        assert r.status == mpm.MPM_OK, (sc.name, mpm.STATUS.get(r.status))
        x, pp = sv.particles(t)
        x0 = np.zeros_like(x)
        x0[:, :sc.dim] = sc.x[:, :sc.dim]
        disp = max(np.abs(xa - x0).max(), 1e-300)
        assert np.abs(x - xa).max() <= 1e-7 * disp + 1e-13 * np.abs(xa).max(), sc.name
        if pa is not None:
            assert np.abs(pp - pa).max() <= 1e-7 * np.abs(pa).max(), sc.name
        xo, po = _oracle_result(sc, st)
        x_o = np.zeros_like(x)
        x_o[:, :sc.dim] = xo[:, :sc.dim]
        disp_o = max(np.abs(x_o - x0).max(), 1e-300)
        err = np.abs(x - x_o).max() / disp_o
        assert err <= DU_TOL, (sc.name, err)
        if po is not None:
            errp = np.abs(pp - po).max() / np.abs(po).max()
            assert errp <= DU_TOL, (sc.name, errp)
    sv.close()


def test_admission_keeps_footprint_within_budget():
    mix = _mix()
    fps = [mpm.mpm_footprint_bytes(mpm.scene_desc(sc, **KW), sc.np) for sc, _ in mix]
    budget = int(1.5 * max(fps))
    sv = mpm.Server(slots=4, budget=budget)
    tickets = [sv.submit(sc, steps=st, **KW) for sc, st in mix]
    for t in tickets:
        assert sv.wait(t).status == mpm.MPM_OK
    st = sv.stats()
    assert st.completed == len(mix) and st.failed == 0
    assert st.peak_in_use <= budget
    assert st.in_use == 0 and st.running == 0
    sv.close()


def test_failed_request_does_not_stop_the_server():
    sv = mpm.Server(slots=2)
    bad = S.block_compression(nsteps=2)
    # a prescribed increment of several cells pushes particles off the grid
    bad.steps = [S.LoadStep(st.dof, st.value * 4000.0, st.gravity) for st in bad.steps]
    good = S.block_compression(nsteps=2)
    tb = sv.submit(bad, **KW)
    tg = sv.submit(good, **KW)
    rb, rg = sv.wait(tb), sv.wait(tg)
    assert rb.status != mpm.MPM_OK
    assert rg.status == mpm.MPM_OK and rg.steps_done == 2
    st = sv.stats()
    assert st.failed == 1 and st.completed == 2
    sv.close()


def test_multigrid_requests_same_alone_and_in_the_mix():
    """Requests preconditioned by the multigrid V-cycle (the bench's serving
    setting), mixed precision: every request converges, concurrently on
    several streams (CUDA graphs captured per worker thread, cluster launches
    on each stream) as alone, to within the Newton tolerance."""
    kw = dict(precision=mpm.MPM_MIXED, newton_tol=1e-8, newton_maxit=32, precond=mpm.MPM_PC_MG)
    # the solid requests of the mix, and u-p columns as the serving stream
    # draws them (16 cells wide; a one-cell-wide column coarsens to two nodes
    # across, where the V-cycle's coarse levels carry little of the problem)
    mix = _mix()[:4] + [S.serving_scene(dict(kind="up_terzaghi", cells=c, nsteps=3)) for c in (1024, 2048)]
    alone = []
    for sc, st in mix:
        sv = mpm.Server(slots=1)
        t = sv.submit(sc, steps=st, **kw)
        r = sv.wait(t)
        assert r.status == mpm.MPM_OK, (sc.name, mpm.STATUS.get(r.status))
        alone.append(sv.particles(t)[0])
        sv.close()
    sv = mpm.Server(slots=4)
    tickets = [sv.submit(sc, steps=st, **kw) for sc, st in mix]
    res = [sv.wait(t) for t in tickets]
    assert sv.stats().peak_running >= 2
    for (sc, st), t, r, xa in zip(mix, tickets, res, alone):
        assert r.status == mpm.MPM_OK, (sc.name, mpm.STATUS.get(r.status))
        x = sv.particles(t)[0]
        x0 = np.zeros_like(x)
        x0[:, :sc.dim] = sc.x[:, :sc.dim]
        disp = max(np.abs(xa - x0).max(), 1e-300)
        assert np.abs(x - xa).max() <= 1e-5 * disp, sc.name
    sv.close()
