"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports exactly the symbols include/*.h declare; host-only calls work;
compute calls fail loudly without a GPU (there is no CPU fallback)."""
import os
import re
import subprocess

import pytest

from paper_2507_09435_gb300 import build, mpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    out = set()
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not name.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", name)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        out |= set(re.findall(r"^\s*(?:mpm_status|void|const char\s*\*)\s*(mpm_\w+)\s*\(", txt, flags=re.M))
    return out


def test_header_and_binding_agree():
    assert header_functions() == set(mpm.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mpm_\w+)$", out, flags=re.M))
    assert header_functions() <= exported
    L = mpm.lib()
    for name in header_functions():
        assert hasattr(L, name)


def test_host_only_calls():
    d = mpm.make_desc(2, (32, 32), 1 / 32)
    fp = mpm.mpm_footprint_bytes(d, 1024)
    assert fp > 1024 * 100
    d3 = mpm.make_desc(3, (16, 16, 16), 0.1, precision=mpm.MPM_MIXED)
    assert mpm.mpm_footprint_bytes(d3, 10000) > mpm.mpm_footprint_bytes(d3, 1000)
    assert mpm.lib().mpm_status_string(4).decode() == "Newton did not converge"
    bad = mpm.make_desc(2, (2, 32), 1 / 32)
    with pytest.raises(mpm.MPMError):
        mpm.mpm_footprint_bytes(bad, 10)
    with pytest.raises(mpm.MPMError):
        mpm.mpm_footprint_bytes(mpm.make_desc(2, (32, 32), 1 / 32, jacobian_reuse=-1), 10)
    assert mpm.mpm_footprint_bytes(mpm.make_desc(2, (32, 32), 1 / 32, jacobian_reuse=3), 1024) == fp


def test_footprint_counts_the_krylov_and_preconditioner_storage():
    """Admission footprint: the GMRES(m) basis (m + 3 vectors beside the nine
    BiCGStab ones) and the 4-row-segment block inverses of u-p scenes are
    counted; FP32 Jacobian and vectors take less than FP64."""
    n, B = (64, 64), 2
    nn = 65 * 65
    pad = 2 + 2 * 65
    bi = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precision=mpm.MPM_MIXED), 4096)
    for m in (10, 30):
        gm = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precision=mpm.MPM_MIXED, krylov=mpm.MPM_GMRES,
                                                   gmres_restart=m), 4096)
        assert gm - bi == (m + 3) * (nn + 2 * pad) * B * 4
    f64 = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precision=mpm.MPM_FP64), 4096)
    assert f64 > bi
    up = dict(precision=mpm.MPM_MIXED, formulation=mpm.MPM_UP, dt=1.0)
    seg = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precond=mpm.MPM_PC_SEG4, **up), 4096)
    node = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precond=mpm.MPM_PC_NODE, **up), 4096)
    auto = mpm.mpm_footprint_bytes(mpm.make_desc(2, n, 0.1, precond=mpm.MPM_PC_AUTO, **up), 4096)
    assert seg - node == nn * 3 * 9 * 4 and auto == seg


def test_compute_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2507_09435_gb300 import scenes
    sc = scenes.block_compression()
    with pytest.raises(mpm.MPMError):
        mpm.GpuScene(sc)


def test_create_rejects_bad_input_before_touching_the_gpu():
    from paper_2507_09435_gb300 import scenes
    sc = scenes.block_compression()
    d = mpm.make_desc(2, sc.n, sc.h)
    x = sc.x[:, :2].copy()
    x[0, 0] = 0.2 * sc.h          # support would leave the grid
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_create_scene(d, x, sc.vol0, sc.mass, sc.mat_id, mpm.materials_of(sc))
    assert e.value.status == 1 and "outside" in str(e.value)
    m = sc.mass.copy()
    m[3] = 0.0
    with pytest.raises(mpm.MPMError):
        mpm.mpm_create_scene(d, sc.x[:, :2], sc.vol0, m, sc.mat_id, mpm.materials_of(sc))
