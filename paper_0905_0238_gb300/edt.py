"""Thin ctypes binding of the C ABI in ``include/edt.h`` (argument marshalling only).

Every computation runs in ``_lib/libedt.so``; torch is used here only to own device
memory (the workspace and the caller's tensors) and to supply CUDA streams.  Loading
fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libedt.so")

EDT_OK, EDT_EINVAL, EDT_ENOMEM_WS, EDT_ENOTPD = 0, -1, -2, -3
EDT_ETIMEOUT, EDT_ENONFINITE, EDT_ECUDA, EDT_EUNSUPPORTED = -4, -5, -6, -7
EDT_FP64, EDT_MIXED = 0, 1
EDT_GEOM_LINE, EDT_GEOM_WINDOW = 0, 1
EDT_SOLVE_DAMPED, EDT_SOLVE_TSVD = 0, 1
EDT_C64, EDT_C128, EDT_F32, EDT_F64 = 0, 1, 2, 3


class edt_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("dx", C.c_double),
        ("nz", C.c_int), ("dz", C.c_double), ("z0", C.c_double),
        ("nfreq", C.c_int), ("freq_hz", C.POINTER(C.c_double)), ("eps", C.c_double),
        ("nlayer", C.c_int), ("layer_top_m", C.POINTER(C.c_double)),
        ("layer_vel_mps", C.POINTER(C.c_double)),
        ("precision", C.c_int), ("passes", C.c_int), ("refine", C.c_int),
        ("alpha", C.c_double), ("cutoff", C.c_double), ("fold", C.c_int),
        ("chol_df", C.c_int), ("freq_chunk", C.c_int),
        ("geometry", C.c_int), ("ny", C.c_int), ("dy", C.c_double), ("wx", C.c_int), ("wy", C.c_int),
        ("solver", C.c_int), ("tsvd_tol", C.c_double), ("kz_disk", C.c_double),
        ("gram_seg_rows", C.c_int), ("resid", C.c_int), ("sub_begin", C.c_int), ("sub_end", C.c_int),
    ]


class edt_stats(C.Structure):
    _fields_ = [
        ("n_sub", C.c_int), ("rows_total", C.c_longlong), ("rows_solved", C.c_longlong),
        ("rows_min", C.c_int), ("rows_max", C.c_int), ("workspace_bytes", C.c_size_t),
        ("gram_flop", C.c_double), ("n_notpd", C.c_int), ("n_nonfinite", C.c_int),
        ("last_status", C.c_int), ("launches_per_invert", C.c_int),
        ("gram_rows_padded", C.c_longlong), ("freq_chunk", C.c_int),
        ("launches_per_grad", C.c_int), ("gram_timeouts", C.c_int),
    ]


class edt_tuning(C.Structure):
    _fields_ = [
        ("band_budget_mb", C.c_int), ("band_cols", C.c_int), ("refine_shape", C.c_int),
        ("window_ztile", C.c_int), ("overlap", C.c_int), ("invert_ms", C.c_double),
    ]


class edt_sub1d(C.Structure):
    _fields_ = [
        ("nz", C.c_int), ("dz", C.c_double), ("z0", C.c_double),
        ("eps", C.c_double), ("alpha", C.c_double), ("dx", C.c_double),
        ("nlayer", C.c_int), ("layer_top_m", C.POINTER(C.c_double)),
        ("layer_vel_mps", C.POINTER(C.c_double)),
        ("nfreq", C.c_int), ("freq_hz", C.POINTER(C.c_double)),
        ("nk", C.c_int), ("kval", C.POINTER(C.c_double)),
        ("nrow", C.c_int), ("rows", C.POINTER(C.c_int)), ("data", C.POINTER(C.c_float)),
    ]


class edt_stream_stats(C.Structure):
    _fields_ = [
        ("requests", C.c_longlong), ("batches", C.c_longlong), ("compute_ms", C.c_double),
        ("busy_ms", C.c_double),
        ("bytes_in", C.c_longlong), ("bytes_out", C.c_longlong), ("launches", C.c_longlong),
        ("launches_per_batch", C.c_int), ("arena_bytes", C.c_size_t), ("max_batch", C.c_int),
    ]


class EdtError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib().edt_strerror(code).decode()
        if code == EDT_ECUDA:
            msg += ": " + _lib().edt_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


_LIB: Optional[C.CDLL] = None


def _lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_0905_0238_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        vp, i, sz = C.c_void_p, C.c_int, C.c_size_t
        L.edt_create.argtypes = [C.POINTER(vp), C.POINTER(edt_config), C.POINTER(sz)]
        L.edt_set_workspace.argtypes = [vp, vp, sz]
        L.edt_invert.argtypes = [vp, vp, i, vp, i, vp]
        L.edt_invert_host.argtypes = [vp, vp, i, vp, i, vp]
        L.edt_forward.argtypes = [vp, vp, i, vp, i, vp]
        L.edt_adjoint.argtypes = [vp, vp, i, vp, i, vp]
        L.edt_green.argtypes = [vp, vp, vp]
        L.edt_get_vhat.argtypes = [vp, vp, vp]
        L.edt_get_factor.argtypes = [vp, vp, vp]
        L.edt_row_offsets.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.edt_row_offsets.restype = i
        L.edt_export_rhs.argtypes = [vp, vp, i, vp, vp]
        L.edt_import_rhs.argtypes = [vp, vp, C.c_longlong, i, i, vp]
        L.edt_solve_imported.argtypes = [vp, vp, vp]
        L.edt_inverse_vhat.argtypes = [vp, vp, vp, i, vp]
        L.edt_row_counts.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.edt_gram.argtypes = [vp, vp, i, vp, vp, vp, vp]
        d = C.c_double
        L.edt_green_noalloc.argtypes = [i, d, i, d, d, i, C.POINTER(d), d, i, C.POINTER(d),
                                        C.POINTER(d), vp, vp]
        L.edt_get_stats.argtypes = [vp, C.POINTER(edt_stats)]
        L.edt_set_profiling.argtypes = [vp, i]
        L.edt_set_graph.argtypes = [vp, i]
        L.edt_autotune.argtypes = [vp, vp, i, vp, i, vp, i]
        L.edt_get_tuning.argtypes = [vp, C.POINTER(edt_tuning)]
        L.edt_set_tuning.argtypes = [vp, C.POINTER(edt_tuning)]
        L.edt_read_profile.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_char_p), i,
                                       C.POINTER(i)]
        L.edt_misfit_grad.argtypes = [vp, vp, i, vp, i, vp, vp, vp, vp]
        L.edt_invert_adjoint.argtypes = [vp, vp, i, vp, i, vp]
        L.edt_invert_vjp.argtypes = [vp, vp, i, vp, i, vp, vp]
        L.edt_set_host_pipeline.argtypes = [vp, i]
        L.edt_set_wait_test.argtypes = [vp, C.c_longlong, i]
        L.edt_set_reference.argtypes = [vp, C.POINTER(d), vp]
        L.edt_strerror.argtypes = [i]
        L.edt_strerror.restype = C.c_char_p
        L.edt_last_cuda_error.restype = C.c_char_p
        L.edt_destroy.argtypes = [vp]
        L.edt_destroy.restype = None
        for name in ("edt_create", "edt_set_workspace", "edt_invert", "edt_invert_host",
                     "edt_forward", "edt_adjoint", "edt_green", "edt_get_vhat", "edt_get_factor", "edt_export_rhs",
                     "edt_import_rhs", "edt_solve_imported", "edt_inverse_vhat", "edt_row_counts", "edt_gram",
                     "edt_get_stats", "edt_set_profiling", "edt_read_profile", "edt_green_noalloc",
                     "edt_set_graph", "edt_autotune", "edt_get_tuning", "edt_set_tuning",
                     "edt_misfit_grad", "edt_set_reference", "edt_invert_adjoint", "edt_invert_vjp",
                     "edt_set_host_pipeline", "edt_set_wait_test"):
            getattr(L, name).restype = i
        ll = C.c_longlong
        L.edt_measure_fma_rates.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.edt_measure_fma_rates.restype = i
        L.edt_kz_disk_columns.argtypes = [vp, C.POINTER(i)]
        L.edt_kz_disk_columns.restype = i
        L.edt_stream_request_bytes.argtypes = [C.POINTER(edt_sub1d)]
        L.edt_stream_request_bytes.restype = ll
        L.edt_stream_plan.argtypes = [i, C.POINTER(ll), ll, i, C.POINTER(i)]
        L.edt_stream_create.argtypes = [C.POINTER(vp), i, vp, C.POINTER(sz)]
        L.edt_stream_set_workspace.argtypes = [vp, vp, sz]
        L.edt_stream_submit.argtypes = [vp, i, C.POINTER(edt_sub1d), vp, vp, C.POINTER(ll)]
        L.edt_stream_wait.argtypes = [vp, ll, C.POINTER(d)]
        L.edt_stream_query.argtypes = [vp, ll, C.POINTER(i)]
        L.edt_stream_epoch.argtypes = [vp]
        L.edt_stream_get_stats.argtypes = [vp, C.POINTER(edt_stream_stats)]
        L.edt_stream_set_profiling.argtypes = [vp, i]
        L.edt_stream_set_wait_test.argtypes = [vp, C.c_longlong, i]
        L.edt_stream_read_profile.argtypes = [vp, C.POINTER(d), C.POINTER(C.c_char_p), i, C.POINTER(ll)]
        L.edt_stream_destroy.argtypes = [vp]
        L.edt_stream_destroy.restype = None
        for name in ("edt_stream_plan", "edt_stream_create", "edt_stream_set_workspace",
                     "edt_stream_submit", "edt_stream_wait", "edt_stream_query", "edt_stream_epoch",
                     "edt_stream_get_stats", "edt_stream_set_profiling", "edt_stream_read_profile",
                     "edt_stream_set_wait_test"):
            getattr(L, name).restype = i
        _LIB = L
    return _LIB


def _check(code: int, where: str) -> int:
    if code < 0:
        raise EdtError(code, where)
    return code


# ---- raw C-ABI calls with the same names -------------------------------------------------
def edt_create(cfg: edt_config):
    ctx, ws = C.c_void_p(), C.c_size_t()
    _check(_lib().edt_create(C.byref(ctx), C.byref(cfg), C.byref(ws)), "edt_create")
    return ctx, ws.value


def edt_set_workspace(ctx, ptr: int, nbytes: int):
    _check(_lib().edt_set_workspace(ctx, C.c_void_p(ptr), nbytes), "edt_set_workspace")


def edt_invert(ctx, D_ptr: int, D_dtype: int, V_ptr: int, V_dtype: int, stream: int):
    _check(_lib().edt_invert(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(V_ptr), V_dtype,
                             C.c_void_p(stream)), "edt_invert")


def edt_invert_host(ctx, D_ptr: int, D_dtype: int, V_ptr: int, V_dtype: int, stream: int):
    _check(_lib().edt_invert_host(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(V_ptr), V_dtype,
                                  C.c_void_p(stream)), "edt_invert_host")


def edt_forward(ctx, V_ptr: int, V_dtype: int, D_ptr: int, D_dtype: int, stream: int):
    _check(_lib().edt_forward(ctx, C.c_void_p(V_ptr), V_dtype, C.c_void_p(D_ptr), D_dtype,
                              C.c_void_p(stream)), "edt_forward")


def edt_adjoint(ctx, D_ptr: int, D_dtype: int, V_ptr: int, V_dtype: int, stream: int):
    _check(_lib().edt_adjoint(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(V_ptr), V_dtype,
                              C.c_void_p(stream)), "edt_adjoint")


def edt_green(ctx, g_ptr: int, stream: int):
    _check(_lib().edt_green(ctx, C.c_void_p(g_ptr), C.c_void_p(stream)), "edt_green")


def edt_row_offsets(ctx, nsub: int) -> np.ndarray:
    out = (C.c_longlong * (nsub + 1))()
    _check(_lib().edt_row_offsets(ctx, out), "edt_row_offsets")
    return np.array(out[:], dtype=np.int64)


def edt_export_rhs(ctx, D_ptr: int, D_dtype: int, rhs_ptr: int, stream: int):
    _check(_lib().edt_export_rhs(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(rhs_ptr), C.c_void_p(stream)),
           "edt_export_rhs")


def edt_import_rhs(ctx, block_ptr: int, nrows: int, f_begin: int, f_end: int, stream: int):
    _check(_lib().edt_import_rhs(ctx, C.c_void_p(block_ptr), nrows, f_begin, f_end, C.c_void_p(stream)),
           "edt_import_rhs")


def edt_solve_imported(ctx, vhat_ptr: int, stream: int):
    _check(_lib().edt_solve_imported(ctx, C.c_void_p(vhat_ptr), C.c_void_p(stream)), "edt_solve_imported")


def edt_inverse_vhat(ctx, vhat_ptr: int, V_ptr: int, V_dtype: int, stream: int):
    _check(_lib().edt_inverse_vhat(ctx, C.c_void_p(vhat_ptr), C.c_void_p(V_ptr), V_dtype, C.c_void_p(stream)),
           "edt_inverse_vhat")


def edt_get_factor(ctx, ptr: int, stream: int):
    _check(_lib().edt_get_factor(ctx, C.c_void_p(ptr), C.c_void_p(stream)), "edt_get_factor")


def edt_get_vhat(ctx, ptr: int, stream: int):
    _check(_lib().edt_get_vhat(ctx, C.c_void_p(ptr), C.c_void_p(stream)), "edt_get_vhat")


def edt_gram(ctx, D_ptr: int, D_dtype: int, G_ptr: int, b_ptr: int, tr_ptr: int, stream: int):
    _check(_lib().edt_gram(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(G_ptr), C.c_void_p(b_ptr),
                           C.c_void_p(tr_ptr), C.c_void_p(stream)), "edt_gram")


def edt_green_noalloc(nx, dx, nz, dz, z0, freq_hz, eps, layer_top, layer_vel, g_ptr: int,
                      stream: int):
    """Allocation-free depth march into caller memory (complex128 [nfreq][nx/2+1][nz])."""
    dp = C.POINTER(C.c_double)
    fr = np.ascontiguousarray(freq_hz, dtype=np.float64)
    tp = np.ascontiguousarray(layer_top, dtype=np.float64)
    vl = np.ascontiguousarray(layer_vel, dtype=np.float64)
    _check(_lib().edt_green_noalloc(nx, dx, nz, dz, z0, len(fr), fr.ctypes.data_as(dp), eps,
                                    len(tp), tp.ctypes.data_as(dp), vl.ctypes.data_as(dp),
                                    C.c_void_p(g_ptr), C.c_void_p(stream)), "edt_green_noalloc")


def edt_measure_fma_rates():
    """(FP64, FP32) multiply-add rates of the current device in TFLOP/s."""
    f64, f32 = C.c_double(), C.c_double()
    _check(_lib().edt_measure_fma_rates(C.byref(f64), C.byref(f32)), "edt_measure_fma_rates")
    return f64.value, f32.value


def edt_row_counts(ctx, nsub: int) -> np.ndarray:
    out = (C.c_longlong * nsub)()
    _check(_lib().edt_row_counts(ctx, out), "edt_row_counts")
    return np.array(out[:], dtype=np.int64)


def edt_kz_disk_columns(ctx, nsub: int) -> np.ndarray:
    out = np.zeros(nsub, dtype=np.int32)
    _check(_lib().edt_kz_disk_columns(ctx, out.ctypes.data_as(C.POINTER(C.c_int))), "edt_kz_disk_columns")
    return out


def edt_get_stats(ctx) -> edt_stats:
    st = edt_stats()
    _check(_lib().edt_get_stats(ctx, C.byref(st)), "edt_get_stats")
    return st


def edt_autotune(ctx, D_ptr: int, D_dtype: int, V_ptr: int, V_dtype: int, stream: int, reps: int = 2):
    _check(_lib().edt_autotune(ctx, C.c_void_p(D_ptr), D_dtype, C.c_void_p(V_ptr), V_dtype,
                               C.c_void_p(stream), reps), "edt_autotune")


def edt_get_tuning(ctx) -> edt_tuning:
    t = edt_tuning()
    _check(_lib().edt_get_tuning(ctx, C.byref(t)), "edt_get_tuning")
    return t


def edt_set_tuning(ctx, t: edt_tuning):
    _check(_lib().edt_set_tuning(ctx, C.byref(t)), "edt_set_tuning")


def edt_set_graph(ctx, on: bool):
    _check(_lib().edt_set_graph(ctx, int(bool(on))), "edt_set_graph")


def edt_set_profiling(ctx, on: bool):
    _check(_lib().edt_set_profiling(ctx, int(bool(on))), "edt_set_profiling")


def edt_read_profile(ctx, max_stages: int = 16):
    ms = (C.c_double * max_stages)()
    names = (C.c_char_p * max_stages)()
    ncalls = C.c_int()
    n = _check(_lib().edt_read_profile(ctx, ms, names, max_stages, C.byref(ncalls)),
               "edt_read_profile")
    return {names[i].decode(): ms[i] for i in range(n)}, ncalls.value


def edt_misfit_grad(ctx, V_ptr: int, V_dtype: int, D_ptr: int, D_dtype: int, J_ptr: int,
                    gV_ptr: int, gc_ptr: int, stream: int):
    _check(_lib().edt_misfit_grad(ctx, C.c_void_p(V_ptr), V_dtype, C.c_void_p(D_ptr), D_dtype,
                                  C.c_void_p(J_ptr), C.c_void_p(gV_ptr), C.c_void_p(gc_ptr),
                                  C.c_void_p(stream)), "edt_misfit_grad")


def edt_invert_vjp(ctx, Vbar_ptr: int, Vbar_dtype: int, Dbar_ptr: int, Dbar_dtype: int, gc_ptr: int,
                   stream: int):
    _check(_lib().edt_invert_vjp(ctx, C.c_void_p(Vbar_ptr), Vbar_dtype, C.c_void_p(Dbar_ptr), Dbar_dtype,
                                 C.c_void_p(gc_ptr), C.c_void_p(stream)), "edt_invert_vjp")


def edt_invert_adjoint(ctx, Vbar_ptr: int, Vbar_dtype: int, Dbar_ptr: int, Dbar_dtype: int,
                       stream: int):
    _check(_lib().edt_invert_adjoint(ctx, C.c_void_p(Vbar_ptr), Vbar_dtype, C.c_void_p(Dbar_ptr),
                                     Dbar_dtype, C.c_void_p(stream)), "edt_invert_adjoint")


def edt_set_host_pipeline(ctx, on: bool):
    _check(_lib().edt_set_host_pipeline(ctx, int(bool(on))), "edt_set_host_pipeline")


def edt_set_reference(ctx, vel: np.ndarray, stream: int):
    v = np.ascontiguousarray(vel, dtype=np.float64)
    _check(_lib().edt_set_reference(ctx, v.ctypes.data_as(C.POINTER(C.c_double)),
                                    C.c_void_p(stream)), "edt_set_reference")


def edt_set_wait_test(ctx, wait_cycles: int, stall: bool):
    _check(_lib().edt_set_wait_test(ctx, int(wait_cycles), int(bool(stall))), "edt_set_wait_test")


def edt_destroy(ctx):
    if ctx:
        _lib().edt_destroy(ctx)


# ---- convenience wrapper owning the workspace ---------------------------------------------
@dataclass
class Config:
    nx: int
    dx: float
    nz: int
    dz: float
    z0: float
    freq_hz: Sequence[float]
    eps: float
    layer_top: Sequence[float]
    layer_vel: Sequence[float]
    precision: int = EDT_FP64
    passes: int = 3
    refine: int = 1
    alpha: float = 1e-2
    cutoff: float = 1.0
    fold: int = 1
    chol_df: int = 0
    freq_chunk: int = 0
    geometry: int = EDT_GEOM_LINE
    ny: int = 1
    dy: float = 1.0
    wx: int = 1
    wy: int = 1
    solver: int = 0            # EDT_SOLVE_DAMPED or EDT_SOLVE_TSVD (FP64 line path)
    tsvd_tol: float = 0.0      # truncated SVD: > 0 absolute sigma, < 0 relative to s_max
    kz_disk: float = 0.0       # > 0: |(k_m, k_z)| <= kz_disk omega_max / c_min
    gram_seg_rows: int = 0     # mixed: rows per FP32 Gram accumulation (0 = automatic)
    resid: int = 0             # mixed: refinement residual, 1 FP32, 2 double-float, 0 automatic
    sub_begin: int = 0         # line geometry: solve only subproblems [sub_begin, sub_end)
    sub_end: int = 0           #   (0, 0: all)

    @classmethod
    def from_workload(cls, wl, **kw):
        base = dict(nx=wl.nx, dx=wl.dx, nz=wl.nz, dz=wl.dz, z0=wl.z0, freq_hz=wl.freq_hz,
                    eps=wl.eps, layer_top=wl.layer_top, layer_vel=wl.layer_vel,
                    alpha=wl.alpha, cutoff=wl.cutoff)
        if hasattr(wl, "wx"):          # finite-aperture workload
            base.update(geometry=EDT_GEOM_WINDOW, ny=wl.ny, dy=wl.dy, wx=wl.wx, wy=wl.wy,
                        precision=EDT_MIXED, fold=0)
        base.update(kw)
        return cls(**base)

    def c_config(self):
        """(edt_config, arrays): the C configuration and the FP64 arrays it points into, which
        the caller keeps alive for as long as the context is being created."""
        arrays = tuple(np.ascontiguousarray(a, dtype=np.float64)
                       for a in (self.freq_hz, self.layer_top, self.layer_vel))
        freq, top, vel = arrays
        dp = C.POINTER(C.c_double)
        c = edt_config(
            nx=self.nx, dx=self.dx, nz=self.nz, dz=self.dz, z0=self.z0,
            nfreq=len(freq), freq_hz=freq.ctypes.data_as(dp), eps=self.eps,
            nlayer=len(top), layer_top_m=top.ctypes.data_as(dp),
            layer_vel_mps=vel.ctypes.data_as(dp), precision=self.precision,
            passes=self.passes, refine=self.refine, alpha=self.alpha, cutoff=self.cutoff,
            fold=self.fold, chol_df=self.chol_df, freq_chunk=self.freq_chunk,
            geometry=self.geometry, ny=self.ny, dy=self.dy, wx=self.wx, wy=self.wy,
            solver=self.solver, tsvd_tol=self.tsvd_tol, kz_disk=self.kz_disk,
            gram_seg_rows=self.gram_seg_rows, resid=self.resid, sub_begin=self.sub_begin,
            sub_end=self.sub_end)
        return c, arrays

    @property
    def window(self) -> bool:
        return self.geometry == EDT_GEOM_WINDOW

    def data_shape(self, nfreq):
        if self.window:
            return (nfreq, self.ny, self.nx, self.wy, self.wx)
        return (nfreq, self.nx, self.nx)

    def model_shape(self):
        return (self.ny, self.nx, self.nz) if self.window else (self.nx, self.nz)


class Solver:
    """A context plus a torch-owned workspace on the current CUDA device."""

    def __init__(self, cfg: Config, device=None):
        import torch
        self._torch = torch
        self.cfg = cfg
        c, (self._freq, self._top, self._vel) = cfg.c_config()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.ctx = None
        self.ctx, self.ws_bytes = edt_create(c)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        edt_set_workspace(self.ctx, self.workspace.data_ptr(), self.ws_bytes)
        self.nsub = int(edt_get_stats(self.ctx).n_sub)

    def __del__(self):
        if getattr(self, "ctx", None):
            edt_destroy(self.ctx)
            self.ctx = None

    def _stream(self):
        return self._torch.cuda.current_stream(self.device).cuda_stream

    @staticmethod
    def _cdtype(t):
        import torch
        return {torch.complex64: EDT_C64, torch.complex128: EDT_C128}[t.dtype]

    @staticmethod
    def _rdtype(t):
        import torch
        return {torch.float32: EDT_F32, torch.float64: EDT_F64}[t.dtype]

    def invert(self, D, out=None, out_dtype=None):
        torch = self._torch
        nf = len(self._freq)
        if not (D.is_cuda and D.is_contiguous()) or tuple(D.shape) != self.cfg.data_shape(nf):
            raise ValueError(f"D must be a contiguous CUDA tensor of shape {self.cfg.data_shape(nf)}")
        if out is None:
            out = torch.empty(self.cfg.model_shape(), device=self.device,
                              dtype=out_dtype or torch.float64)
        edt_invert(self.ctx, D.data_ptr(), self._cdtype(D), out.data_ptr(), self._rdtype(out),
                   self._stream())
        return out

    def set_host_pipeline(self, on=True):
        """Overlap invert_host's input copy with the previous call (see edt_set_host_pipeline)."""
        edt_set_host_pipeline(self.ctx, on)

    def invert_host(self, D_host, V_host):
        """Host-buffer entry point: copies in, inverts, copies out on the current stream."""
        edt_invert_host(self.ctx, D_host.data_ptr(), self._cdtype(D_host), V_host.data_ptr(),
                        self._rdtype(V_host), self._stream())
        return V_host

    def forward(self, V, out_dtype=None):
        torch = self._torch
        nf = len(self._freq)
        D = torch.empty((nf, self.cfg.nx, self.cfg.nx), device=self.device,
                        dtype=out_dtype or torch.complex128)
        edt_forward(self.ctx, V.data_ptr(), self._rdtype(V), D.data_ptr(), self._cdtype(D),
                    self._stream())
        return D

    def adjoint(self, D, out_dtype=None):
        """V = F^T D, the adjoint Born operator (see edt_adjoint)."""
        torch = self._torch
        nf = len(self._freq)
        if not (D.is_cuda and D.is_contiguous()) or tuple(D.shape) != self.cfg.data_shape(nf):
            raise ValueError(f"D must be a contiguous CUDA tensor of shape {self.cfg.data_shape(nf)}")
        V = torch.empty(self.cfg.model_shape(), device=self.device, dtype=out_dtype or torch.float64)
        edt_adjoint(self.ctx, D.data_ptr(), self._cdtype(D), V.data_ptr(), self._rdtype(V), self._stream())
        return V

    def misfit_grad(self, V, D):
        """(J, dJ/dV, dJ/dc) of J = ||F V - D||^2 (see edt_misfit_grad): J a 0-d float64
        device tensor, dJ/dV of V's shape and dtype, dJ/dc float64 [nlayer] on the device."""
        torch = self._torch
        nf = len(self._freq)
        if not (D.is_cuda and D.is_contiguous()) or tuple(D.shape) != self.cfg.data_shape(nf):
            raise ValueError(f"D must be a contiguous CUDA tensor of shape {self.cfg.data_shape(nf)}")
        if not (V.is_cuda and V.is_contiguous()) or tuple(V.shape) != self.cfg.model_shape():
            raise ValueError(f"V must be a contiguous CUDA tensor of shape {self.cfg.model_shape()}")
        J = torch.empty((), device=self.device, dtype=torch.float64)
        gV = torch.empty_like(V)
        gc = torch.empty((len(self._top),), device=self.device, dtype=torch.float64)
        edt_misfit_grad(self.ctx, V.data_ptr(), self._rdtype(V), D.data_ptr(), self._cdtype(D),
                        J.data_ptr(), gV.data_ptr(), gc.data_ptr(), self._stream())
        return J, gV, gc

    def invert_adjoint(self, Vbar, out_dtype=None):
        """Dbar = S^T Vbar for the linear map S: D -> V of the last invert (see
        edt_invert_adjoint); Dbar has the data's shape."""
        torch = self._torch
        nf = len(self._freq)
        if not (Vbar.is_cuda and Vbar.is_contiguous()) or tuple(Vbar.shape) != self.cfg.model_shape():
            raise ValueError(f"Vbar must be a contiguous CUDA tensor of shape {self.cfg.model_shape()}")
        Dbar = torch.empty(self.cfg.data_shape(nf), device=self.device,
                           dtype=out_dtype or torch.complex128)
        edt_invert_adjoint(self.ctx, Vbar.data_ptr(), self._rdtype(Vbar), Dbar.data_ptr(),
                           self._cdtype(Dbar), self._stream())
        return Dbar

    def invert_vjp(self, Vbar, want_D=True, want_c=True, out_dtype=None):
        """(Dbar, gc) for Vbar = dL/dV after the last invert (see edt_invert_vjp): Dbar = dL/dD
        with the data's shape, gc[l] = dL/dc_l through the damped solve; either may be None
        when not wanted."""
        torch = self._torch
        nf = len(self._freq)
        if not (Vbar.is_cuda and Vbar.is_contiguous()) or tuple(Vbar.shape) != self.cfg.model_shape():
            raise ValueError(f"Vbar must be a contiguous CUDA tensor of shape {self.cfg.model_shape()}")
        Dbar = torch.empty(self.cfg.data_shape(nf), device=self.device,
                           dtype=out_dtype or torch.complex128) if want_D else None
        gc = torch.empty((len(self._top),), device=self.device, dtype=torch.float64) if want_c else None
        edt_invert_vjp(self.ctx, Vbar.data_ptr(), self._rdtype(Vbar), Dbar.data_ptr() if want_D else 0,
                       self._cdtype(Dbar) if want_D else EDT_C64, gc.data_ptr() if want_c else 0,
                       self._stream())
        return Dbar, gc

    def set_reference(self, layer_vel):
        """Replace the layer velocities of the reference (same layer tops)."""
        vel = np.ascontiguousarray(np.asarray(layer_vel, dtype=np.float64))
        edt_set_reference(self.ctx, vel, self._stream())
        self._vel = vel

    def green(self):
        torch = self._torch
        nf = len(self._freq)
        g = torch.empty((nf, self.cfg.nx // 2 + 1, self.cfg.nz), device=self.device,
                        dtype=torch.complex128)
        edt_green(self.ctx, g.data_ptr(), self._stream())
        return g

    def factor(self):
        """Cholesky factors of the last invert, [nsub][nz][nz] float64, L in the lower triangle
        (the strict upper triangle is unspecified; see edt_get_factor)."""
        torch = self._torch
        L = torch.empty((self.nsub, self.cfg.nz, self.cfg.nz), device=self.device, dtype=torch.float64)
        edt_get_factor(self.ctx, L.data_ptr(), self._stream())
        return L

    def vhat(self):
        torch = self._torch
        v = torch.empty((self.nsub, self.cfg.nz), device=self.device, dtype=torch.complex128)
        edt_get_vhat(self.ctx, v.data_ptr(), self._stream())
        return v

    def gram(self, D):
        """(G [nsub][nz][nz], b [nsub][nz][2], trace [nsub]) of the split systems for data D."""
        torch = self._torch
        nz = self.cfg.nz
        G = torch.empty((self.nsub, nz, nz), device=self.device, dtype=torch.float64)
        b = torch.empty((self.nsub, nz, 2), device=self.device, dtype=torch.float64)
        tr = torch.empty((self.nsub,), device=self.device, dtype=torch.float64)
        edt_gram(self.ctx, D.data_ptr(), self._cdtype(D), G.data_ptr(), b.data_ptr(),
                 tr.data_ptr(), self._stream())
        return G, b, tr

    def row_counts(self):
        return edt_row_counts(self.ctx, self.nsub)

    def stats(self):
        return edt_get_stats(self.ctx)

    def set_graph(self, on=True):
        edt_set_graph(self.ctx, on)

    def autotune(self, D, out=None, reps=2):
        """Pick the fastest launch shapes on data D (see edt_autotune); returns the tuning."""
        torch = self._torch
        if out is None:
            out = torch.empty(self.cfg.model_shape(), device=self.device, dtype=torch.float64)
        edt_autotune(self.ctx, D.data_ptr(), self._cdtype(D), out.data_ptr(), self._rdtype(out),
                     self._stream(), reps)
        return self.tuning()

    def tuning(self):
        t = edt_get_tuning(self.ctx)
        return {k: getattr(t, k) for k, _ in edt_tuning._fields_}

    def set_tuning(self, **kw):
        t = edt_get_tuning(self.ctx)
        for k, v in kw.items():
            setattr(t, k, v)
        edt_set_tuning(self.ctx, t)

    def set_profiling(self, on=True):
        edt_set_profiling(self.ctx, on)

    def set_wait_test(self, wait_cycles=0, stall=False):
        """Test hook: short bounded-wait budget and a Gram stall (see edt_set_wait_test)."""
        edt_set_wait_test(self.ctx, wait_cycles, stall)

    def read_profile(self):
        return edt_read_profile(self.ctx)


# ---- streaming 1D subproblems (edt_stream_*) ---------------------------------------------
def _sub1d_array(subs):
    """ctypes array of edt_sub1d for objects with the fields of synth.stream.Sub1D, plus the
    numpy arrays it points into (kept alive by the caller until the submit returns)."""
    arr = (edt_sub1d * max(len(subs), 1))()
    keep = []
    dp, ip, fp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)
    for i, s in enumerate(subs):
        tops = np.ascontiguousarray(s.layer_top, dtype=np.float64)
        vel = np.ascontiguousarray(s.layer_vel, dtype=np.float64)
        fr = np.ascontiguousarray(s.freq_hz, dtype=np.float64)
        kv = np.ascontiguousarray(s.kval, dtype=np.float64)
        rows = np.ascontiguousarray(s.rows, dtype=np.int32).reshape(-1, 3)
        data = np.ascontiguousarray(s.data, dtype=np.complex64).reshape(-1, 2).view(np.float32)
        keep += [tops, vel, fr, kv, rows, data]
        e = arr[i]
        e.nz, e.dz, e.z0 = int(s.nz), float(s.dz), float(s.z0)
        e.eps, e.alpha, e.dx = float(s.eps), float(s.alpha), float(s.dx)
        e.nlayer = len(tops)
        e.layer_top_m, e.layer_vel_mps = tops.ctypes.data_as(dp), vel.ctypes.data_as(dp)
        e.nfreq, e.freq_hz = len(fr), fr.ctypes.data_as(dp)
        e.nk, e.kval = len(kv), kv.ctypes.data_as(dp)
        e.nrow, e.rows, e.data = rows.shape[0], rows.ctypes.data_as(ip), data.ctypes.data_as(fp)
    return arr, keep


def edt_stream_request_bytes(sub) -> int:
    arr, keep = _sub1d_array([sub])
    return _check(_lib().edt_stream_request_bytes(arr), "edt_stream_request_bytes")


def edt_stream_plan(request_bytes, arena_bytes: int, max_batch: int):
    """(number of batches, batch index of every request) of the admission plan."""
    rb = np.ascontiguousarray(request_bytes, dtype=np.int64)
    out = np.zeros(len(rb), dtype=np.int32)
    nb = _check(_lib().edt_stream_plan(len(rb), rb.ctypes.data_as(C.POINTER(C.c_longlong)),
                                       int(arena_bytes), int(max_batch),
                                       out.ctypes.data_as(C.POINTER(C.c_int))), "edt_stream_plan")
    return nb, out


def edt_stream_create(max_batch: int, stream: int = 0):
    ctx, ws = C.c_void_p(), C.c_size_t()
    _check(_lib().edt_stream_create(C.byref(ctx), int(max_batch), C.c_void_p(stream), C.byref(ws)),
           "edt_stream_create")
    return ctx, ws.value


def edt_stream_set_workspace(ctx, ptr: int, nbytes: int):
    _check(_lib().edt_stream_set_workspace(ctx, C.c_void_p(ptr), nbytes), "edt_stream_set_workspace")


def edt_stream_submit(ctx, subs, vhat: np.ndarray, status: np.ndarray) -> int:
    arr, keep = _sub1d_array(subs)
    t = C.c_longlong()
    _check(_lib().edt_stream_submit(ctx, len(subs), arr, vhat.ctypes.data, status.ctypes.data, C.byref(t)),
           "edt_stream_submit")
    return t.value


def edt_stream_wait(ctx, ticket: int) -> float:
    ms = C.c_double()
    _check(_lib().edt_stream_wait(ctx, int(ticket), C.byref(ms)), "edt_stream_wait")
    return ms.value


def edt_stream_query(ctx, ticket: int) -> bool:
    done = C.c_int()
    _check(_lib().edt_stream_query(ctx, int(ticket), C.byref(done)), "edt_stream_query")
    return bool(done.value)


def edt_stream_epoch(ctx):
    _check(_lib().edt_stream_epoch(ctx), "edt_stream_epoch")


def edt_stream_get_stats(ctx) -> edt_stream_stats:
    st = edt_stream_stats()
    _check(_lib().edt_stream_get_stats(ctx, C.byref(st)), "edt_stream_get_stats")
    return st


def edt_stream_set_profiling(ctx, on: bool):
    _check(_lib().edt_stream_set_profiling(ctx, int(bool(on))), "edt_stream_set_profiling")


def edt_stream_set_wait_test(ctx, wait_cycles: int, stall: bool):
    _check(_lib().edt_stream_set_wait_test(ctx, int(wait_cycles), int(bool(stall))),
           "edt_stream_set_wait_test")


def edt_stream_read_profile(ctx, max_kernels: int = 8):
    """({kernel name: summed ms}, batches covered) since the last read."""
    ms = (C.c_double * max_kernels)()
    names = (C.c_char_p * max_kernels)()
    nb = C.c_longlong()
    n = _check(_lib().edt_stream_read_profile(ctx, ms, names, max_kernels, C.byref(nb)),
               "edt_stream_read_profile")
    return {names[i].decode(): ms[i] for i in range(n)}, nb.value


class Stream:
    """A streaming solver of independent 1D subproblems with a torch-owned device workspace.

    ``submit(subs)`` admits the requests (objects with the fields of ``synth.stream.Sub1D``)
    and returns a ticket; ``wait(ticket)`` returns the list of Vhat arrays (complex128, one per
    request), their status codes and the completion time in ms after the last ``epoch()``.
    """

    def __init__(self, max_batch: int = 512, workspace_bytes: Optional[int] = None, device=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.ctx, self.ws_min = edt_stream_create(max_batch, 0)
        nbytes = max(int(self.ws_min), int(workspace_bytes or 0))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        edt_stream_set_workspace(self.ctx, self.workspace.data_ptr(), nbytes)
        self._pending = {}

    def submit(self, subs) -> int:
        nz = [int(s.nz) for s in subs]
        vhat = np.empty(sum(nz), dtype=np.complex128)
        status = np.empty(len(subs), dtype=np.int32)
        t = edt_stream_submit(self.ctx, subs, vhat, status)
        self._pending[t] = (nz, vhat, status)
        return t

    def wait(self, ticket: int):
        ms = edt_stream_wait(self.ctx, ticket)
        nz, vhat, status = self._pending.pop(ticket)
        cuts = np.cumsum([0] + nz)
        return [vhat[cuts[i]:cuts[i + 1]] for i in range(len(nz))], status, ms

    def query(self, ticket: int) -> bool:
        return edt_stream_query(self.ctx, ticket)

    def solve(self, subs):
        """Submit and wait: (list of Vhat, status)."""
        v, st, _ = self.wait(self.submit(subs))
        return v, st

    def epoch(self):
        edt_stream_epoch(self.ctx)

    def set_profiling(self, on=True):
        edt_stream_set_profiling(self.ctx, on)

    def set_wait_test(self, wait_cycles=0, stall=False):
        """Test hook: short bounded-wait budget and a Gram stall (see edt_stream_set_wait_test)."""
        edt_stream_set_wait_test(self.ctx, wait_cycles, stall)

    def read_profile(self):
        return edt_stream_read_profile(self.ctx)

    def stats(self):
        st = edt_stream_get_stats(self.ctx)
        return {k: getattr(st, k) for k, _ in edt_stream_stats._fields_}

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            _lib().edt_stream_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
