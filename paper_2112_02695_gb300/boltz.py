"""Thin ctypes binding of libboltz.so (include/boltz.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device pointers on the
caller's current CUDA stream; every computation runs in the library's
kernels.  There is no fallback: if the shared library cannot be loaded the
import of this module raises, and every status other than BOLTZ_OK raises
BoltzError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

BOLTZ_OK = 0
BOLTZ_EINVAL = 1
BOLTZ_ENOMEM = 2
BOLTZ_ECUDA = 3
BOLTZ_ETIMEOUT = 4
BOLTZ_EUNSUPPORTED = 5
BOLTZ_ENONFINITE = 6

BOLTZ_FORM_BATCHED = 0
BOLTZ_FORM_PLAIN = 1
BOLTZ_FORM_SPLIT_BF16 = 2
BOLTZ_FORM_CARLEMAN = 3

EXPORTED = (
    "boltz_abi_version", "boltz_status_string", "boltz_grid_init", "boltz_grid_destroy",
    "boltz_spectrum", "boltz_collide_batched", "boltz_project", "boltz_lowrank_step_host",
    "boltz_host_quadrature", "boltz_workspace_size", "boltz_profile_enable", "boltz_profile_read",
    "boltz_project_noalloc", "boltz_sync_status", "boltz_selftest", "boltz_moments",
    "boltz_batch_plan", "boltz_batch_run", "boltz_batch_kernel_count", "boltz_batch_destroy",
    "boltz_autotune", "boltz_spectrum_f64", "boltz_collide_batched_f64", "boltz_project_f64",
    "boltz_kstep_collision", "boltz_lstep_collision", "boltz_qr_f64_workspace", "boltz_qr_f64",
    "boltz_svd_truncate_f64", "boltz_basis_rotate_f64", "boltz_lowrank_coupling", "boltz_mott_smith",
    "boltz_shock_create", "boltz_shock_destroy", "boltz_shock_full_step", "boltz_shock_lowrank_step",
    "boltz_shock_reconstruct",
)

KERNEL_CLASSES = ("spectrum", "prep", "shift", "contract", "radial", "output", "project", "pipeline")

BOLTZ_SCHEDULE_AUTO = 0
BOLTZ_SCHEDULE_NODE_BLOCKS = 1
BOLTZ_LOSS_EXACT = 0
BOLTZ_LOSS_MASS_CONSISTENT = 1


class BoltzError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class _Options(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double), ("workspace_max", ctypes.c_size_t), ("field_budget_mb", ctypes.c_int),
                ("schedule", ctypes.c_int), ("loss", ctypes.c_int)]


class _Work(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("fields", ctypes.c_void_p), ("spectra", ctypes.c_void_p),
                ("n_inputs", ctypes.c_int), ("pair_j", ctypes.POINTER(ctypes.c_int32)),
                ("pair_l", ctypes.POINTER(ctypes.c_int32)), ("n_pairs", ctypes.c_int),
                ("Q_out", ctypes.c_void_p), ("V", ctypes.c_void_p), ("r", ctypes.c_int),
                ("T_out", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    path = os.environ.get("BOLTZ_LIB") or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libboltz.so not built ({path}); run python -m paper_2112_02695_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i32p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    sig = {
        "boltz_abi_version": ([], ctypes.c_int),
        "boltz_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "boltz_grid_init": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Options)], ctypes.c_int),
        "boltz_grid_destroy": ([vp], ctypes.c_int),
        "boltz_spectrum": ([vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_collide_batched": ([vp, vp, ctypes.c_int, i32p, i32p, ctypes.c_int, vp, ctypes.c_int, vp],
                                  ctypes.c_int),
        "boltz_project": ([vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "boltz_lowrank_step_host": ([vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "boltz_host_quadrature": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, f64p, f64p, f64p,
                                   f64p], ctypes.c_int),
        "boltz_workspace_size": ([vp, ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "boltz_profile_enable": ([vp, ctypes.c_int], ctypes.c_int),
        "boltz_sync_status": ([vp, vp], ctypes.c_int),
        "boltz_moments": ([vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_batch_plan": ([ctypes.POINTER(vp), ctypes.POINTER(_Work), ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "boltz_batch_run": ([vp, vp], ctypes.c_int),
        "boltz_autotune": ([vp, vp, ctypes.c_int, i32p, i32p, ctypes.c_int, vp, ctypes.c_int, ctypes.c_char_p, vp,
                            ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "boltz_batch_kernel_count": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "boltz_batch_destroy": ([vp], ctypes.c_int),
        "boltz_selftest": ([vp, ctypes.c_int, vp], ctypes.c_int),
        "boltz_project_noalloc": ([vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "boltz_profile_read": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "boltz_spectrum_f64": ([vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_collide_batched_f64": ([vp, vp, ctypes.c_int, i32p, i32p, ctypes.c_int, vp, ctypes.c_int, vp],
                                      ctypes.c_int),
        "boltz_project_f64": ([vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "boltz_kstep_collision": ([vp, ctypes.c_int, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_lstep_collision": ([vp, ctypes.c_int, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_qr_f64_workspace": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "boltz_qr_f64": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp, vp, vp, vp], ctypes.c_int),
        "boltz_svd_truncate_f64": ([vp, ctypes.c_int, ctypes.c_double, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "boltz_basis_rotate_f64": ([vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "boltz_lowrank_coupling": ([vp, vp, ctypes.c_int, vp, vp, vp, vp], ctypes.c_int),
        "boltz_mott_smith": ([vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              vp], ctypes.c_int),
        "boltz_shock_create": ([vp, ctypes.c_int, ctypes.c_double, vp, vp, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(vp)], ctypes.c_int),
        "boltz_shock_destroy": ([vp], ctypes.c_int),
        "boltz_shock_full_step": ([vp, vp, ctypes.c_int, ctypes.c_double, vp], ctypes.c_int),
        "boltz_shock_lowrank_step": ([vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp], ctypes.c_int),
        "boltz_shock_reconstruct": ([vp, vp, vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()
LIB_PATH = _lib._name


def status_string(status: int) -> str:
    return _lib.boltz_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != BOLTZ_OK:
        raise BoltzError(status, what)


def boltz_abi_version() -> int:
    return _lib.boltz_abi_version()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype_name: str, what: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{what} must be {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Owning wrapper of a boltz_grid handle."""

    def __init__(self, handle, N, d_v, L, R, gamma, N_rho, M, b):
        self.handle = handle
        self.N, self.d_v, self.L, self.R, self.gamma, self.N_rho, self.M, self.b = N, d_v, L, R, gamma, N_rho, M, b
        self.n = N ** d_v
        self.half = N ** (d_v - 1) * (N // 2 + 1)

    @property
    def shape(self):
        return (self.N,) * self.d_v

    @property
    def half_shape(self):
        return (self.N,) * (self.d_v - 1) + (self.N // 2 + 1,)

    def close(self):
        if self.handle:
            _lib.boltz_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boltz_grid_init(N: int, d_v: int, L: float, R: float, gamma: float, N_rho: int, M: int,
                    b: float | None = None, workspace_max: int = 0, field_budget_mb: int = 0,
                    schedule: int = BOLTZ_SCHEDULE_AUTO, loss: int = BOLTZ_LOSS_EXACT) -> Grid:
    h = ctypes.c_void_p()
    opt = _Options(b if b is not None else 0.0, workspace_max, field_budget_mb, schedule, loss)
    _check(_lib.boltz_grid_init(ctypes.byref(h), N, d_v, L, R, gamma, N_rho, M, ctypes.byref(opt)),
           "boltz_grid_init")
    area = 2 * np.pi if d_v == 2 else 4 * np.pi
    return Grid(h, N, d_v, L, R, gamma, N_rho, M, b if b is not None else 1.0 / area)


def boltz_grid_destroy(grid: Grid):
    grid.close()


def boltz_spectrum(grid: Grid, f, out=None, stream=None):
    """Half spectra (complex64 [n_inputs, *half_shape]) of real fields f [n_inputs, *shape]."""
    import torch
    n_in = f.shape[0]
    if out is None:
        out = torch.empty((n_in,) + grid.half_shape, dtype=torch.complex64, device=f.device)
    _check(_lib.boltz_spectrum(grid.handle, _dev_ptr(f, "float32", "f"), n_in,
                               _dev_ptr(out, "complex64", "out"), _stream_ptr(stream)), "boltz_spectrum")
    return out


def _pairs(pair_j, pair_l):
    pj = np.ascontiguousarray(np.asarray(pair_j, dtype=np.int32))
    pl = np.ascontiguousarray(np.asarray(pair_l, dtype=np.int32))
    if pj.shape != pl.shape or pj.ndim != 1:
        raise ValueError("pair_j and pair_l must be 1-D of equal length")
    return pj, pl


def boltz_collide_batched(grid: Grid, spectra, pair_j, pair_l, form: int = BOLTZ_FORM_BATCHED, out=None,
                          stream=None):
    """Q(g = input pair_j[e], f = input pair_l[e]) for every e: float32 [n_pairs, *shape]."""
    import torch
    pj, pl = _pairs(pair_j, pair_l)
    if out is None:
        out = torch.empty((len(pj),) + grid.shape, dtype=torch.float32, device=spectra.device)
    i32p = ctypes.POINTER(ctypes.c_int32)
    _check(_lib.boltz_collide_batched(grid.handle, _dev_ptr(spectra, "complex64", "spectra"), spectra.shape[0],
                                      pj.ctypes.data_as(i32p), pl.ctypes.data_as(i32p), len(pj),
                                      _dev_ptr(out, "float32", "out"), int(form), _stream_ptr(stream)),
           "boltz_collide_batched")
    return out


def boltz_project(grid: Grid, V, Q, out=None, stream=None):
    """T[k, j, l] = dv^d sum_v V_k Q_{j*r+l}: float32 [r, r, r]."""
    import torch
    r = V.shape[0]
    if Q.shape[0] != r * r:
        raise ValueError("Q must hold r*r fields")
    if out is None:
        out = torch.empty((r, r, r), dtype=torch.float32, device=V.device)
    _check(_lib.boltz_project(grid.handle, _dev_ptr(V, "float32", "V"), r, _dev_ptr(Q, "float32", "Q"),
                              _dev_ptr(out, "float32", "out"), _stream_ptr(stream)), "boltz_project")
    return out


def boltz_spectrum_f64(grid: Grid, f, out=None, stream=None):
    """FP64 check build of boltz_spectrum: complex128 half spectra of float64 fields."""
    import torch
    n_in = f.shape[0]
    if out is None:
        out = torch.empty((n_in,) + grid.half_shape, dtype=torch.complex128, device=f.device)
    _check(_lib.boltz_spectrum_f64(grid.handle, _dev_ptr(f, "float64", "f"), n_in,
                                   _dev_ptr(out, "complex128", "out"), _stream_ptr(stream)), "boltz_spectrum_f64")
    return out


def boltz_collide_batched_f64(grid: Grid, spectra, pair_j, pair_l, form: int = BOLTZ_FORM_BATCHED, out=None,
                              stream=None):
    """FP64 check build of boltz_collide_batched: float64 [n_pairs, *shape]."""
    import torch
    pj, pl = _pairs(pair_j, pair_l)
    if out is None:
        out = torch.empty((len(pj),) + grid.shape, dtype=torch.float64, device=spectra.device)
    i32p = ctypes.POINTER(ctypes.c_int32)
    _check(_lib.boltz_collide_batched_f64(grid.handle, _dev_ptr(spectra, "complex128", "spectra"),
                                          spectra.shape[0], pj.ctypes.data_as(i32p), pl.ctypes.data_as(i32p),
                                          len(pj), _dev_ptr(out, "float64", "out"), int(form),
                                          _stream_ptr(stream)), "boltz_collide_batched_f64")
    return out


def boltz_project_f64(grid: Grid, V, Q, out=None, stream=None):
    """FP64 check build of boltz_project: float64 [r, r, r]."""
    import torch
    r = V.shape[0]
    if Q.shape[0] != r * r:
        raise ValueError("Q must hold r*r fields")
    if out is None:
        out = torch.empty((r, r, r), dtype=torch.float64, device=V.device)
    _check(_lib.boltz_project_f64(grid.handle, _dev_ptr(V, "float64", "V"), r, _dev_ptr(Q, "float64", "Q"),
                                  _dev_ptr(out, "float64", "out"), _stream_ptr(stream)), "boltz_project_f64")
    return out


def boltz_project_noalloc(grid: Grid, V, Q, out, stream=None):
    """Like boltz_project, but the library allocates no device memory for it:
    the partial sums use a fixed 2 MiB device array inside the library, so
    callers that must not allocate (a solver loop that cannot afford the
    device-wide synchronisation of cudaMalloc/cudaFree, or a process whose
    device memory is reserved up front) can still project.  `out` must be
    given (float32 [r, r, r]); r <= 64.  Calls that may overlap on the GPU
    share the array and must be serialised by the caller."""
    r = V.shape[0]
    if Q.shape[0] != r * r:
        raise ValueError("Q must hold r*r fields")
    _check(_lib.boltz_project_noalloc(grid.handle, _dev_ptr(V, "float32", "V"), r, _dev_ptr(Q, "float32", "Q"),
                                      _dev_ptr(out, "float32", "out"), _stream_ptr(stream)),
           "boltz_project_noalloc")
    return out


def boltz_lowrank_step_host(grid: Grid, V_host, Q_host=None, T_host=None, stream=None):
    """Host-memory end-to-end step: V (host float32 [r, *shape]) -> Q (host, optional), T (host)."""
    import torch
    r = V_host.shape[0]
    if T_host is None:
        T_host = torch.empty((r, r, r), dtype=torch.float32)
    for name, t in (("V_host", V_host), ("Q_host", Q_host), ("T_host", T_host)):
        if t is not None and (t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CPU tensor")
    qp = ctypes.c_void_p(Q_host.data_ptr()) if Q_host is not None else None
    _check(_lib.boltz_lowrank_step_host(grid.handle, ctypes.c_void_p(V_host.data_ptr()), r, qp,
                                        ctypes.c_void_p(T_host.data_ptr()), _stream_ptr(stream)),
           "boltz_lowrank_step_host")
    return Q_host, T_host


def boltz_host_quadrature(d_v: int, N_rho: int, M: int, R: float):
    """(rho, w_rho, sigma [M, d_v], w_sigma) as the library computes them (no GPU needed)."""
    rho = np.zeros(N_rho)
    wr = np.zeros(N_rho)
    sig = np.zeros(M * d_v)
    ws = np.zeros(M)
    f64p = ctypes.POINTER(ctypes.c_double)
    _check(_lib.boltz_host_quadrature(d_v, N_rho, M, R, rho.ctypes.data_as(f64p), wr.ctypes.data_as(f64p),
                                      sig.ctypes.data_as(f64p), ws.ctypes.data_as(f64p)), "boltz_host_quadrature")
    return rho, wr, sig.reshape(M, d_v), ws


def boltz_workspace_size(grid: Grid, n_inputs: int, pair_j, pair_l, form: int = BOLTZ_FORM_BATCHED) -> int:
    pj, pl = _pairs(pair_j, pair_l)
    out = ctypes.c_size_t()
    i32p = ctypes.POINTER(ctypes.c_int32)
    _check(_lib.boltz_workspace_size(grid.handle, n_inputs, pj.ctypes.data_as(i32p), pl.ctypes.data_as(i32p),
                                     len(pj), int(form), ctypes.byref(out)), "boltz_workspace_size")
    return out.value


def boltz_moments(grid: Grid, Q, out=None, stream=None):
    """FP64 [n_fields, d+2]: mass, momentum (d components), energy moments of each field."""
    import torch
    nf = Q.shape[0]
    if out is None:
        out = torch.empty((nf, grid.d_v + 2), dtype=torch.float64, device=Q.device)
    _check(_lib.boltz_moments(grid.handle, _dev_ptr(Q, "float32", "Q"), nf, _dev_ptr(out, "float64", "out"),
                              _stream_ptr(stream)), "boltz_moments")
    return out


def boltz_sync_status(grid: Grid, stream=None):
    """Wait for the stream and raise if a kernel reported a device error (e.g. a timed-out wait)."""
    _check(_lib.boltz_sync_status(grid.handle, _stream_ptr(stream)), "boltz_sync_status")


def boltz_selftest(grid: Grid, which: int = 0, stream=None) -> int:
    """Run a failure-path self-test; returns the raw status (BOLTZ_ETIMEOUT expected for which=0)."""
    return _lib.boltz_selftest(grid.handle, int(which), _stream_ptr(stream))


def boltz_profile_enable(grid: Grid, enable: bool = True):
    _check(_lib.boltz_profile_enable(grid.handle, int(bool(enable))), "boltz_profile_enable")


def boltz_profile_read(grid: Grid, reset: bool = True):
    """{class: (launches, total_ms)} since the last reset (see KERNEL_CLASSES)."""
    n = len(KERNEL_CLASSES)
    la = (ctypes.c_longlong * n)()
    ms = (ctypes.c_double * n)()
    _check(_lib.boltz_profile_read(grid.handle, int(bool(reset)), la, ms), "boltz_profile_read")
    return {name: (int(la[i]), float(ms[i])) for i, name in enumerate(KERNEL_CLASSES)}


def boltz_autotune(grid: Grid, spectra, pair_j, pair_l, Q_scratch=None, form: int = BOLTZ_FORM_BATCHED,
                   cache_path: str | None = None, stream=None) -> int:
    """Time the shifted-field budget candidates for this batch, keep the fastest
    in the grid and return it (MB); with cache_path, reuse/record the choice."""
    import torch
    pj, pl = _pairs(pair_j, pair_l)
    if Q_scratch is None:
        Q_scratch = torch.empty((len(pj),) + grid.shape, dtype=torch.float32, device=spectra.device)
    mb = ctypes.c_int()
    i32p = ctypes.POINTER(ctypes.c_int32)
    _check(_lib.boltz_autotune(grid.handle, _dev_ptr(spectra, "complex64", "spectra"), spectra.shape[0],
                               pj.ctypes.data_as(i32p), pl.ctypes.data_as(i32p), len(pj),
                               _dev_ptr(Q_scratch, "float32", "Q_scratch"), int(form),
                               cache_path.encode() if cache_path else None, _stream_ptr(stream), ctypes.byref(mb)),
           "boltz_autotune")
    return mb.value


class Batch:
    """Owning wrapper of a boltz_batch (a captured CUDA graph over several grids).
    Keeps references to every tensor and pair array the graph uses."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            _lib.boltz_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boltz_batch_plan(items, form: int = BOLTZ_FORM_BATCHED) -> Batch:
    """items: list of dicts with keys grid, spectra, pair_j, pair_l, Q_out and
    optionally fields, V, T_out (torch CUDA tensors; V/T_out for the projection)."""
    n = len(items)
    arr = (_Work * n)()
    keep = []
    i32p = ctypes.POINTER(ctypes.c_int32)
    for i, it in enumerate(items):
        pj, pl = _pairs(it["pair_j"], it["pair_l"])
        keep += [pj, pl, it]
        w = arr[i]
        w.grid = it["grid"].handle
        w.fields = _dev_ptr(it["fields"], "float32", "fields") if it.get("fields") is not None else None
        w.spectra = _dev_ptr(it["spectra"], "complex64", "spectra")
        w.n_inputs = it["spectra"].shape[0]
        w.pair_j = pj.ctypes.data_as(i32p)
        w.pair_l = pl.ctypes.data_as(i32p)
        w.n_pairs = len(pj)
        w.Q_out = _dev_ptr(it["Q_out"], "float32", "Q_out")
        if it.get("V") is not None:
            w.V = _dev_ptr(it["V"], "float32", "V")
            w.r = it["V"].shape[0]
            w.T_out = _dev_ptr(it["T_out"], "float32", "T_out")
    h = ctypes.c_void_p()
    _check(_lib.boltz_batch_plan(ctypes.byref(h), arr, n, int(form)), "boltz_batch_plan")
    return Batch(h, keep)


def boltz_batch_run(batch: Batch, stream=None):
    _check(_lib.boltz_batch_run(batch.handle, _stream_ptr(stream)), "boltz_batch_run")


def boltz_batch_kernel_count(batch: Batch) -> int:
    k = ctypes.c_int()
    _check(_lib.boltz_batch_kernel_count(batch.handle, ctypes.byref(k)), "boltz_batch_kernel_count")
    return k.value


def boltz_batch_destroy(batch: Batch):
    batch.close()


# ----------------------------------------------------------------------------- low-rank step consumers

def boltz_kstep_collision(T, K, out=None, stream=None):
    """C[j, x] = sum_{m,n} T[j, m, n] K[m, x] K[n, x]: float32 [r, n_x]."""
    import torch
    r, n_x = K.shape
    if tuple(T.shape) != (r, r, r):
        raise ValueError("T must be [r, r, r] for K [r, n_x]")
    if out is None:
        out = torch.empty((r, n_x), dtype=torch.float32, device=K.device)
    _check(_lib.boltz_kstep_collision(_dev_ptr(T, "float32", "T"), r, _dev_ptr(K, "float32", "K"), n_x,
                                      _dev_ptr(out, "float32", "out"), _stream_ptr(stream)), "boltz_kstep_collision")
    return out


def boltz_lstep_collision(Q, C, out=None, stream=None):
    """G[i, v] = sum_{p,q} C[i, p, q] Q[p*r + q, v]: float32 [r, n_v]."""
    import torch
    r = C.shape[0]
    Q2 = Q.reshape(Q.shape[0], -1)
    if Q2.shape[0] != r * r or tuple(C.shape) != (r, r, r):
        raise ValueError("Q must hold r*r fields and C be [r, r, r]")
    n_v = Q2.shape[1]
    if out is None:
        out = torch.empty((r, n_v), dtype=torch.float32, device=Q.device)
    _check(_lib.boltz_lstep_collision(_dev_ptr(Q2, "float32", "Q"), r, _dev_ptr(C, "float32", "C"), n_v,
                                      _dev_ptr(out, "float32", "out"), _stream_ptr(stream)), "boltz_lstep_collision")
    return out


def boltz_qr_f64(W, w: float, Y=None, stream=None):
    """W [r, n] float64 -> (Y [r, n], R [r, r], info int32 tensor [1]) with
    W_j = sum_i Y_i R[i, j] and w Y Y^T = I."""
    import torch
    r, n = W.shape
    ws = ctypes.c_size_t()
    _check(_lib.boltz_qr_f64_workspace(r, n, ctypes.byref(ws)), "boltz_qr_f64_workspace")
    work = torch.empty(ws.value, dtype=torch.uint8, device=W.device)
    if Y is None:
        Y = torch.empty_like(W)
    R = torch.empty((r, r), dtype=torch.float64, device=W.device)
    info = torch.empty(1, dtype=torch.int32, device=W.device)
    _check(_lib.boltz_qr_f64(_dev_ptr(W, "float64", "W"), r, n, float(w), _dev_ptr(Y, "float64", "Y"),
                             _dev_ptr(R, "float64", "R"), ctypes.c_void_p(work.data_ptr()),
                             _dev_ptr(info, "int32", "info"), _stream_ptr(stream)), "boltz_qr_f64")
    return Y, R, info


def boltz_svd_truncate_f64(S, drop_tol: float, stream=None):
    """S [r, r] float64 -> (U, sigma, Q, r_keep, info); r_keep and info are
    int32 device tensors [1]."""
    import torch
    r = S.shape[0]
    dev = S.device
    U = torch.empty((r, r), dtype=torch.float64, device=dev)
    Qm = torch.empty((r, r), dtype=torch.float64, device=dev)
    sigma = torch.empty(r, dtype=torch.float64, device=dev)
    rk = torch.empty(1, dtype=torch.int32, device=dev)
    info = torch.empty(1, dtype=torch.int32, device=dev)
    _check(_lib.boltz_svd_truncate_f64(_dev_ptr(S, "float64", "S"), r, float(drop_tol), _dev_ptr(U, "float64", "U"),
                                       _dev_ptr(sigma, "float64", "sigma"), _dev_ptr(Qm, "float64", "Q"),
                                       _dev_ptr(rk, "int32", "r_keep"), _dev_ptr(info, "int32", "info"),
                                       _stream_ptr(stream)), "boltz_svd_truncate_f64")
    return U, sigma, Qm, rk, info


def boltz_basis_rotate_f64(X, U, r_new: int, out=None, stream=None):
    """X_out[k] = sum_i X[i] U[i, k] for k < r_new: float64 [r_new, n]."""
    import torch
    r, n = X.shape
    if out is None:
        out = torch.empty((r_new, n), dtype=torch.float64, device=X.device)
    _check(_lib.boltz_basis_rotate_f64(_dev_ptr(X, "float64", "X"), r, n, _dev_ptr(U, "float64", "U"), int(r_new),
                                       _dev_ptr(out, "float64", "out"), _stream_ptr(stream)),
           "boltz_basis_rotate_f64")
    return out


def boltz_lowrank_coupling(E, S, T=None, stream=None):
    """C [r, r, r] (the L-step coupling) and, with T, D [r, r] (the S-step
    collision term), both float32."""
    import torch
    r = S.shape[0]
    C = torch.empty((r, r, r), dtype=torch.float32, device=S.device)
    D = torch.empty((r, r), dtype=torch.float32, device=S.device) if T is not None else None
    _check(_lib.boltz_lowrank_coupling(_dev_ptr(E, "float32", "E"), _dev_ptr(S, "float32", "S"), r,
                                       _dev_ptr(T, "float32", "T") if T is not None else None,
                                       _dev_ptr(C, "float32", "C"),
                                       _dev_ptr(D, "float32", "D") if D is not None else None,
                                       _stream_ptr(stream)), "boltz_lowrank_coupling")
    return C, D


def boltz_mott_smith(grid: Grid, spectra, rho_L: float, u_L: float, T_L: float, T_R: float, R_gas: float = 1.0,
                     Q_scratch=None, stream=None):
    """(alpha, beta, Q) of the Mott-Smith closure; spectra = [f_L, f_R]."""
    import torch
    if spectra.shape[0] != 2:
        raise ValueError("spectra must hold f_L and f_R")
    if Q_scratch is None:
        Q_scratch = torch.empty((2,) + grid.shape, dtype=torch.float32, device=spectra.device)
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.boltz_mott_smith(grid.handle, _dev_ptr(spectra, "complex64", "spectra"), float(rho_L), float(u_L),
                                 float(T_L), float(T_R), float(R_gas), _dev_ptr(Q_scratch, "float32", "Q_scratch"),
                                 ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)), "boltz_mott_smith")
    return a.value, b.value, Q_scratch


class Shock:
    """Owning wrapper of a boltz_shock handle (1D normal shock solver)."""

    def __init__(self, handle, grid, n_x, L_x, r_max):
        self.handle, self.grid, self.n_x, self.L_x, self.r_max = handle, grid, n_x, L_x, r_max

    def close(self):
        if self.handle:
            _lib.boltz_shock_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boltz_shock_create(grid: Grid, n_x: int, L_x: float, f_L, f_R, r_max: int, form: int = BOLTZ_FORM_BATCHED):
    """f_L, f_R: host float64 arrays of N^d values (the inflow Maxwellians on the grid)."""
    import numpy as np
    fl = np.ascontiguousarray(f_L, dtype=np.float64).reshape(-1)
    fr = np.ascontiguousarray(f_R, dtype=np.float64).reshape(-1)
    if fl.size != grid.n or fr.size != grid.n:
        raise ValueError("f_L and f_R must hold N^d values")
    h = ctypes.c_void_p()
    _check(_lib.boltz_shock_create(grid.handle, int(n_x), float(L_x), fl.ctypes.data_as(ctypes.c_void_p),
                                   fr.ctypes.data_as(ctypes.c_void_p), int(r_max), int(form), ctypes.byref(h)),
           "boltz_shock_create")
    return Shock(h, grid, n_x, L_x, r_max)


def boltz_shock_full_step(shock: Shock, f, n_steps: int, dt: float, stream=None):
    """f: device float64 [n_x, N^d], advanced n_steps full-tensor steps in place."""
    _check(_lib.boltz_shock_full_step(shock.handle, _dev_ptr(f, "float64", "f"), int(n_steps), float(dt),
                                      _stream_ptr(stream)), "boltz_shock_full_step")
    return f


def boltz_shock_lowrank_step(shock: Shock, X, S, V, r: int, dt: float, drop_tol: float, stream=None):
    """One adaptive low-rank step on device float64 factors X [r_max, n_x],
    S [r_max * r_max] (packed [r][r]), V [r_max, N^d]; returns (new rank,
    ||f^{n+1} - f^n|| of the step)."""
    rr = ctypes.c_int(int(r))
    err = ctypes.c_double()
    _check(_lib.boltz_shock_lowrank_step(shock.handle, _dev_ptr(X, "float64", "X"), _dev_ptr(S, "float64", "S"),
                                         _dev_ptr(V, "float64", "V"), ctypes.byref(rr), float(dt), float(drop_tol),
                                         ctypes.byref(err), _stream_ptr(stream)), "boltz_shock_lowrank_step")
    return rr.value, err.value


def boltz_shock_reconstruct(shock: Shock, X, S, V, r: int, f, stream=None):
    """f [n_x, N^d] = X^T S V (device float64)."""
    _check(_lib.boltz_shock_reconstruct(shock.handle, _dev_ptr(X, "float64", "X"), _dev_ptr(S, "float64", "S"),
                                        _dev_ptr(V, "float64", "V"), int(r), _dev_ptr(f, "float64", "f"),
                                        _stream_ptr(stream)), "boltz_shock_reconstruct")
    return f
