"""The C-ABI library builds for sm_103a, loads, and exports what include/zeitlin.h declares (CPU only)."""
import ctypes
import subprocess

import pytest

from paper_2206_05466_gb300 import build as B
from paper_2206_05466_gb300 import zeitlin as z


def test_header_declares_the_boundary():
    names = set(z.declared_functions())
    for want in ("zeitlin_laplacian_apply", "zeitlin_stream_solve", "isomp_step", "isomp_run",
                 "zt_plan_create", "zt_plan_destroy", "zt_last_error", "zt_zgemm_skew"):
        assert want in names, want


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    for name in z.declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(z.declared_functions()), exported ^ set(z.declared_functions())


def test_no_compute_without_gpu_reports_an_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    L = z.load()
    h = ctypes.c_void_p()
    rc = L.zt_plan_create(8, 0, None, ctypes.byref(h))
    assert rc < 0 and not h.value
    assert len(L.zt_last_error()) > 0


def test_argument_validation_on_host():
    L = z.load()
    h = ctypes.c_void_p()
    assert L.zt_plan_create(0, 0, None, ctypes.byref(h)) == z.ZT_EINVAL
    assert L.zt_plan_create(8, 7, None, ctypes.byref(h)) == z.ZT_EINVAL
    assert L.zt_plan_create(8, 0, None, None) == z.ZT_EINVAL
    assert L.zeitlin_stream_solve(None, None, None, None) == z.ZT_EINVAL
    assert L.isomp_step(None, None, 0.01, 1e-12, 50, None, None) == z.ZT_EINVAL
    assert L.zeitlin_casimirs(None, None, None, None) == z.ZT_EINVAL
    assert L.zeitlin_energy_spectrum(None, None, None, None) == z.ZT_EINVAL
    assert L.zt_basis_create(None, 3, ctypes.byref(h)) == z.ZT_EINVAL and not h.value
    assert L.zt_basis_create(None, 3, None) == z.ZT_EINVAL
    assert L.zt_basis_vector(None, 0, 0, None) == z.ZT_EINVAL
    assert L.zeitlin_w_from_omega(None, None, None, None) == z.ZT_EINVAL
    assert L.zeitlin_omega_from_w(None, None, None, None) == z.ZT_EINVAL
    L.zt_basis_destroy(None)   # no-op


@pytest.mark.parametrize("bad", [dict(slices=2), dict(slices=9), dict(digit_bits=5), dict(digit_bits=9),
                                 dict(slices=4, exact_groups=5), dict(slices=8, digit_bits=8),
                                 dict(tile_order=7), dict(tile_order=-1), dict(sweeps_per_sync=65), dict(sweeps_per_sync=-1),
                                 dict(final_mode=7), dict(no_persistent=2), dict(wait_us=-1),
                                 dict(wait_us=60000001), dict(debug_stall_loads=-1), dict(slices2=1),
                                 dict(slices=6, slices2=7), dict(slices2=-1),
                                 dict(first_iterate=2), dict(first_iterate=-1),
                                 dict(second_form=3), dict(second_form=-1)])
def test_split_tuning_validation_on_host(bad):
    # rejected before any device work, so this runs without a GPU
    L = z.load()
    t = z.Tuning()
    for k, v in bad.items():
        setattr(t, k, v)
    h = ctypes.c_void_p()
    assert L.zt_plan_create(64, z.PRECISION_SPLIT, ctypes.byref(t), ctypes.byref(h)) == z.ZT_EINVAL
    assert not h.value
