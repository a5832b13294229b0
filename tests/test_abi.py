"""Host-side checks of the C-ABI library (no GPU needed).

The library builds, loads, exports every function include/boltz.h declares,
rejects bad arguments before touching CUDA, and its own host quadrature (an
independent implementation) agrees with the oracle's.
"""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2112_02695_gb300 import build
    build.build()
    from paper_2112_02695_gb300 import boltz
    return boltz


def declared_functions():
    src = open(os.path.join(ROOT, "include", "boltz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(boltz_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("boltz_grid_init", "boltz_collide_batched", "boltz_project", "boltz_grid_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(B):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert set(B.EXPORTED) == set(declared_functions())


def test_abi_version_and_status_strings(B):
    assert B.boltz_abi_version() == 1
    assert B.status_string(B.BOLTZ_EINVAL) == "invalid argument"
    assert B.status_string(99) == "unknown status"


@pytest.mark.parametrize("args", [
    (33, 3, 8.0, 8.0, 1.0, 32, 38),      # odd N
    (32, 4, 8.0, 8.0, 1.0, 32, 38),      # d_v
    (32, 3, -1.0, 8.0, 1.0, 32, 38),     # L
    (32, 3, 8.0, 0.0, 1.0, 32, 38),      # R
    (32, 3, 8.0, 8.0, -3.5, 32, 38),     # gamma <= -d
    (32, 3, 8.0, 8.0, 1.0, 0, 38),       # N_rho
    (32, 3, 8.0, 8.0, 1.0, 32, 40),      # no octahedral rule with 40 points
    (32, 2, 8.0, 8.0, 1.0, 16, 15),      # odd circle rule
    (32, 3, float("nan"), 8.0, 1.0, 16, 38),
])
def test_grid_init_rejects_bad_arguments(B, args):
    with pytest.raises(B.BoltzError) as ei:
        B.boltz_grid_init(*args)
    assert ei.value.status == B.BOLTZ_EINVAL


def test_grid_init_reports_unbuilt_shapes(B):
    with pytest.raises(B.BoltzError) as ei:
        B.boltz_grid_init(128, 3, 10.0, 10.0, 1.0, 32, 86)
    assert ei.value.status == B.BOLTZ_EUNSUPPORTED


def test_null_handles_are_rejected(B):
    import ctypes
    lib = B._lib
    assert lib.boltz_grid_destroy(None) == B.BOLTZ_OK
    assert lib.boltz_spectrum(None, None, 1, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_project(None, None, 4, None, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_grid_init(None, 32, 3, 8.0, 8.0, 1.0, 32, 38, None) == B.BOLTZ_EINVAL
    z = ctypes.c_size_t()
    assert lib.boltz_workspace_size(None, 1, None, None, 0, 0, ctypes.byref(z)) == B.BOLTZ_EINVAL
    assert lib.boltz_spectrum_f64(None, None, 1, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_collide_batched_f64(None, None, 1, None, None, 1, None, 0, None) == B.BOLTZ_EINVAL
    assert lib.boltz_project_f64(None, None, 4, None, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_kstep_collision(None, 4, None, 10, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_kstep_collision(None, 65, None, 10, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_lstep_collision(None, 0, None, 10, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_qr_f64(None, 4, 100, 0.5, None, None, None, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_svd_truncate_f64(None, 4, 1e-6, None, None, None, None, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_basis_rotate_f64(None, 4, 10, None, 5, None, None) == B.BOLTZ_EINVAL
    assert lib.boltz_qr_f64_workspace(4, 3, ctypes.byref(z)) == B.BOLTZ_EINVAL      # n < r
    assert lib.boltz_qr_f64_workspace(16, 32768, ctypes.byref(z)) == B.BOLTZ_OK and z.value > 0
    h = ctypes.c_void_p()
    assert lib.boltz_shock_create(None, 16, 6.0, None, None, 16, 0, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert lib.boltz_shock_destroy(None) == B.BOLTZ_OK
    assert lib.boltz_shock_full_step(None, None, 1, 0.01, None) == B.BOLTZ_EINVAL
    r = ctypes.c_int(4)
    assert lib.boltz_shock_lowrank_step(None, None, None, None, ctypes.byref(r), 0.01, 1e-6, None,
                                        None) == B.BOLTZ_EINVAL
    assert lib.boltz_shock_reconstruct(None, None, None, None, 4, None, None) == B.BOLTZ_EINVAL


@pytest.mark.parametrize("d,M", [(2, 16), (2, 64), (3, 6), (3, 14), (3, 26), (3, 38), (3, 50), (3, 86)])
def test_library_quadrature_matches_oracle(B, d, M):
    from oracle import quadrature as Q
    rho, wr, sig, ws = B.boltz_host_quadrature(d, 32, M, 8.0)
    r2, w2 = Q.radial_rule(32, 8.0)
    s2, ww2 = Q.direction_rule(d, M)
    assert np.max(np.abs(rho - r2)) < 1e-13 and np.max(np.abs(wr - w2)) < 1e-13
    o1 = np.lexsort(np.round(sig, 10).T)
    o2 = np.lexsort(np.round(s2, 10).T)
    assert np.max(np.abs(sig[o1] - s2[o2])) < 1e-12
    assert np.max(np.abs(ws[o1] - ww2[o2])) < 1e-12


def test_host_quadrature_rejects_bad_rules(B):
    with pytest.raises(B.BoltzError):
        B.boltz_host_quadrature(3, 16, 40, 8.0)
    with pytest.raises(B.BoltzError):
        B.boltz_host_quadrature(2, 0, 16, 8.0)
