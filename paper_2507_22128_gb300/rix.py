"""Thin Python binding of librix.so (include/rix.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device arrays are torch tensors on the job's CUDA device (PyTorch
provides memory and streams); the default stream argument is torch's current
stream.  Functions carry the names of the C ABI without its ``rix_`` prefix.
Importing this module fails loudly when librix.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librix.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, EBUSY, EINTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
FP32, FP64 = 0, 1
PSF_AUTO, PSF_DOUBLE_GRID, PSF_TILES = 0, 1, 2


class RixError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rix error {code}: {msg}")
        self.code = code


class JobDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("cell_rad", C.c_double), ("n_wplanes", C.c_int32),
                ("nchan", C.c_int32), ("freq_hz", C.POINTER(C.c_double)), ("precision", C.c_int32),
                ("n_part", C.c_int32), ("tile", C.c_int32), ("weighting", C.c_int32), ("exchange", C.c_int32)]


WEIGHT_NATURAL, WEIGHT_UNIFORM = 0, 1
EXCHANGE_IMAGE, EXCHANGE_SPECTRAL = 0, 1


MAX_PART = 8


class JobStats(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("n_samples", C.c_int64), ("n_outside", C.c_int64),
                ("n_entries", C.c_int64), ("part_count", C.c_int64 * MAX_PART),
                ("part_weight", C.c_double * MAX_PART), ("ell_px", C.c_double * (MAX_PART - 1)),
                ("delta_px", C.c_double), ("w_min", C.c_double), ("dw", C.c_double), ("max_dw_nm1", C.c_double),
                ("window_lo", C.c_int32 * MAX_PART), ("window_size", C.c_int32 * MAX_PART),
                ("n_work_items", C.c_int64), ("cycle", C.c_int32 * MAX_PART)]


class MscleanParams(C.Structure):
    _fields_ = [("scales", C.POINTER(C.c_float)), ("n_scales", C.c_int32), ("gain", C.c_double),
                ("niter", C.c_int32), ("threshold", C.c_double)]


class FistaParams(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("lambda_rel", C.c_double), ("iters", C.c_int32),
                ("levels", C.c_int32), ("dictionary", C.c_int32), ("reserved", C.c_int32),
                ("sched_a", C.c_double), ("sched_b", C.c_double)]


DICT_DB4, DICT_DB1_8 = 0, 1


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2507_22128_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "rix_create": (C.c_int, [C.POINTER(vp), C.c_int, sz]),
        "rix_destroy": (C.c_int, [vp]),
        "rix_job_workspace_bytes": (sz, [C.POINTER(JobDesc), i64]),
        "rix_job_create": (C.c_int, [vp, C.POINTER(JobDesc), i64, C.POINTER(vp)]),
        "rix_job_destroy": (C.c_int, [vp]),
        "rix_job_sync": (C.c_int, [vp]),
        "rix_job_get_stats": (C.c_int, [vp, C.POINTER(JobStats)]),
        "rix_set_uv_partition": (C.c_int, [vp, vp, i64, vp, C.POINTER(dbl), dbl, vp, vp]),
        "rix_get_sorted_entries": (C.c_int, [vp, vp, vp, vp]),
        "rix_get_weights": (C.c_int, [vp, vp, vp]),
        "rix_degrid": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "rix_grid": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "rix_grid_noalloc": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "rix_psf": (C.c_int, [vp, C.c_int, vp, C.POINTER(dbl), vp]),
        "rix_major_cycle": (C.c_int, [vp, C.c_int, vp, vp, vp, vp]),
        "rix_minor_cycle_msclean": (C.c_int, [vp, C.c_int, C.POINTER(MscleanParams), vp, vp]),
        "rix_minor_cycle_fista": (C.c_int, [vp, C.c_int, C.POINTER(FistaParams), vp, vp]),
        "rix_minor_cycle_fista_batch": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(FistaParams), vp]),
        "rix_get_components": (C.c_int, [vp, C.c_int, C.POINTER(i32), i32, vp, vp, vp, vp]),
        "rix_get_model": (C.c_int, [vp, C.c_int, vp, vp]),
        "rix_combine": (C.c_int, [vp, vp, vp]),
        "rix_last_error": (C.c_char_p, []),
        "rix_kernel_launches": (C.c_uint64, []),
        "rix_device_allocations": (C.c_uint64, []),
        "rix_timing_enable": (C.c_int, [C.c_int]),
        "rix_timing_read": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "rix_selftest_barrier_timeout": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "rix_daubechies_lowpass": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
        "rix_job_tune": (C.c_int, [vp, i32, i32]),
        "rix_job_set_psf_method": (C.c_int, [vp, i32]),
        "rix_batch_create": (C.c_int, [vp, i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(vp)]),
        "rix_batch_destroy": (C.c_int, [vp]),
        "rix_batch_major_cycle": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), vp]),
        "rix_gridder_probe": (C.c_int, [vp, C.c_int, vp, i32, C.POINTER(dbl)]),
        "rix_major_cycle_probe": (C.c_int, [vp, C.c_int, vp, i32, C.POINTER(dbl)]),
        "rix_phi_support": (C.c_int, [vp, C.c_int, C.POINTER(i64)]),
        "rix_phi_pack": (C.c_int, [vp, C.c_int, vp, vp]),
        "rix_phi_unpack": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "rix_bda_rows": (C.c_int, [vp, vp, i64, i64, C.POINTER(dbl), i32, i32, dbl, dbl, vp, C.POINTER(i64), vp]),
        "rix_bda_average": (C.c_int, [vp, vp, vp, vp, i64, i64, C.POINTER(dbl), i32, i32, i32, dbl, dbl, vp, vp, vp,
                                      i64, C.POINTER(i64), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()

EXPORTED = ("rix_create", "rix_destroy", "rix_job_workspace_bytes", "rix_job_create", "rix_job_destroy",
            "rix_job_sync", "rix_job_get_stats", "rix_set_uv_partition", "rix_get_sorted_entries",
            "rix_degrid", "rix_grid", "rix_psf", "rix_major_cycle", "rix_minor_cycle_msclean",
            "rix_minor_cycle_fista", "rix_get_components", "rix_get_model", "rix_combine", "rix_last_error",
            "rix_kernel_launches", "rix_timing_enable", "rix_timing_read", "rix_grid_noalloc",
            "rix_selftest_barrier_timeout", "rix_daubechies_lowpass", "rix_get_weights",
            "rix_minor_cycle_fista_batch", "rix_device_allocations", "rix_bda_rows", "rix_bda_average",
            "rix_phi_support", "rix_phi_pack", "rix_phi_unpack", "rix_job_tune", "rix_job_set_psf_method",
            "rix_batch_create",
            "rix_batch_destroy", "rix_batch_major_cycle", "rix_gridder_probe",
            "rix_major_cycle_probe")


def _check(rc: int):
    if rc != OK:
        raise RixError(rc, _lib.rix_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t, dtype=None, numel=None, name="tensor", min_numel=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} has {t.numel()} elements, at least {min_numel} needed")
    return C.c_void_p(t.data_ptr())


# The library takes untyped device pointers; the binding checks each buffer
# against the job it is passed with: element type by the job's precision,
# images by their size, visibility arrays by the rows of the current
# partitioning.
_JOBS: dict = {}      # job handle -> [precision, n, nchan, rows partitioned (0 before)]


def _real_t(job):
    j = _JOBS.get(job)
    return _RT if j is None else (torch.float64 if j[0] == FP64 else torch.float32)


def _cplx_t(job):
    j = _JOBS.get(job)
    return _CT if j is None else (torch.complex128 if j[0] == FP64 else torch.complex64)


def _img(job, t, name, side=1):
    j = _JOBS.get(job)
    return _ptr(t, _real_t(job), None if j is None else (side * j[1]) ** 2, name)


def _visp(job, t, name):
    j = _JOBS.get(job)
    return _ptr(t, _cplx_t(job), name=name, min_numel=None if j is None else j[2] * j[3])


# ---------------------------------------------------------------- lifetime --
def create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = C.c_void_p()
    _check(_lib.rix_create(C.byref(h), device, mem_budget_bytes))
    return h.value


def destroy(ctx: int):
    _check(_lib.rix_destroy(ctx))


def _desc(n, cell_rad, n_wplanes, freq_hz, precision, n_part, tile, weighting=WEIGHT_NATURAL,
          exchange=EXCHANGE_IMAGE):
    f = (C.c_double * len(freq_hz))(*[float(x) for x in freq_hz])
    d = JobDesc(n, cell_rad, n_wplanes, len(freq_hz), C.cast(f, C.POINTER(C.c_double)), precision,
                n_part, tile, weighting, exchange)
    return d, f


def job_workspace_bytes(n, cell_rad, n_wplanes, freq_hz, precision, n_part, nrow, tile=0,
                        weighting=WEIGHT_NATURAL, exchange=EXCHANGE_IMAGE) -> int:
    d, _keep = _desc(n, cell_rad, n_wplanes, freq_hz, precision, n_part, tile, weighting, exchange)
    return int(_lib.rix_job_workspace_bytes(C.byref(d), nrow))


def job_create(ctx, n, cell_rad, n_wplanes, freq_hz, precision, n_part, max_rows, tile=0,
               weighting=WEIGHT_NATURAL, exchange=EXCHANGE_IMAGE) -> int:
    d, _keep = _desc(n, cell_rad, n_wplanes, freq_hz, precision, n_part, tile, weighting, exchange)
    h = C.c_void_p()
    _check(_lib.rix_job_create(ctx, C.byref(d), max_rows, C.byref(h)))
    _JOBS[h.value] = [int(precision), int(n), len(freq_hz), 0]
    return h.value


def job_destroy(job: int):
    _check(_lib.rix_job_destroy(job))
    _JOBS.pop(job, None)


def job_sync(job: int):
    _check(_lib.rix_job_sync(job))


def job_get_stats(job: int) -> dict:
    s = JobStats()
    _check(_lib.rix_job_get_stats(job, C.byref(s)))
    out = {}
    for name, _ in JobStats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if not isinstance(v, (int, float)) else v
    return out


# --------------------------------------------------------------- a1 - a3 --
def set_uv_partition(job, uvw, weight=None, ell_px=None, delta_px=1.0, mask_out=None, stream=None):
    nrow = uvw.shape[0]
    ells = None
    if ell_px is not None:
        ells = (C.c_double * len(ell_px))(*[float(x) for x in ell_px])
    _check(_lib.rix_set_uv_partition(job, _ptr(uvw, torch.float64, nrow * 3, "uvw"), nrow,
                                     _ptr(weight, torch.float32, name="weight"),
                                     C.cast(ells, C.POINTER(C.c_double)) if ells is not None else None,
                                     float(delta_px), _ptr(mask_out, torch.uint8, name="mask_out"),
                                     _stream(stream)))
    if job in _JOBS:
        _JOBS[job][3] = int(nrow)


def get_sorted_entries(job, keys_out, samples_out, stream=None):
    _check(_lib.rix_get_sorted_entries(job, _ptr(keys_out, torch.int32, name="keys_out"),
                                       _ptr(samples_out, torch.int32, name="samples_out"), _stream(stream)))


def get_weights(job, weight_out, stream=None):
    """The weights the job images with (after its weighting), float32 [nrow * nchan]."""
    _check(_lib.rix_get_weights(job, _ptr(weight_out, torch.float32, name="weight_out"), _stream(stream)))


# --------------------------------------------------------------- a4 - a7 --
_RT = (torch.float32, torch.float64)
_CT = (torch.complex64, torch.complex128)


def degrid(job, part, image, vis_out, stream=None):
    _check(_lib.rix_degrid(job, part, _img(job, image, "image"), _visp(job, vis_out, "vis_out"),
                           _stream(stream)))


def grid(job, part, vis, image_out, stream=None):
    _check(_lib.rix_grid(job, part, _visp(job, vis, "vis"), _img(job, image_out, "image_out"),
                         _stream(stream)))


# ------------------------------------------ tuning and batched major cycles --
def job_tune(job, chunk_limit=64, ctas_per_sm=0):
    _check(_lib.rix_job_tune(job, int(chunk_limit), int(ctas_per_sm)))


def job_set_psf_method(job, method=0):
    """PSF_AUTO, PSF_DOUBLE_GRID or PSF_TILES (how rix_psf forms the PSF)."""
    _check(_lib.rix_job_set_psf_method(job, int(method)))


def batch_create(ctx, jobs, parts) -> int:
    n = len(jobs)
    ja = (C.c_void_p * n)(*[C.c_void_p(j) for j in jobs])
    pa = (C.c_int32 * n)(*[int(p) for p in parts])
    h = C.c_void_p()
    _check(_lib.rix_batch_create(ctx, n, ja, pa, C.byref(h)))
    _BATCHES[h.value] = list(jobs)
    return h.value


_BATCHES: dict = {}   # batch handle -> the job of each pair


def batch_destroy(batch):
    _check(_lib.rix_batch_destroy(batch))
    _BATCHES.pop(batch, None)


def batch_major_cycle(batch, vis_list, residual_out=None, stream=None):
    """vis_list: one complex64 device tensor per pair; residual_out: None or
    one float32 N x N device tensor (or None) per pair."""
    jobs = _BATCHES.get(batch)
    if jobs is not None and (len(vis_list) != len(jobs) or (residual_out is not None and len(residual_out) != len(jobs))):
        raise ValueError(f"the batch has {len(jobs)} pairs")
    pick = (lambda i: jobs[i]) if jobs is not None else (lambda i: None)
    arr = (C.c_void_p * len(vis_list))(*[_visp(pick(i), v, "vis_obs") if jobs else
                                         _ptr(v, torch.complex64, name="vis_obs") for i, v in enumerate(vis_list)])
    res = None
    if residual_out is not None:
        res = (C.c_void_p * len(residual_out))(*[_img(pick(i), r, "residual_out") if jobs else
                                                 _ptr(r, torch.float32, name="residual_out")
                                                 for i, r in enumerate(residual_out)])
    _check(_lib.rix_batch_major_cycle(batch, arr, res, _stream(stream)))


def major_cycle_probe(job, part, vis, reps=3) -> float:
    """Mean device ms of the partition's fused major-cycle operator."""
    ms = C.c_double()
    _check(_lib.rix_major_cycle_probe(job, part, _visp(job, vis, "vis"), int(reps), C.byref(ms)))
    return ms.value


def gridder_probe(job, part, vis, reps=3) -> float:
    """Mean device ms per launch of the partition's FP32 w-stacked gridder."""
    ms = C.c_double()
    _check(_lib.rix_gridder_probe(job, part, _visp(job, vis, "vis"), int(reps), C.byref(ms)))
    return ms.value


# ------------------------------------------------- band-limited exchange --
def phi_support(job, part) -> int:
    c = C.c_int64()
    _check(_lib.rix_phi_support(job, part, C.byref(c)))
    return int(c.value)


def phi_pack(job, part, packed_out, stream=None):
    cnt = phi_support(job, part)
    _check(_lib.rix_phi_pack(job, part, _ptr(packed_out, _cplx_t(job), name="packed_out", min_numel=cnt),
                             _stream(stream)))


def phi_unpack(job, part, packed, phi_out, stream=None):
    cnt = phi_support(job, part)
    _check(_lib.rix_phi_unpack(job, part, _ptr(packed, _cplx_t(job), name="packed", min_numel=cnt),
                               _img(job, phi_out, "phi_out"), _stream(stream)))


# ------------------------------------------- baseline-dependent averaging --
def bda_rows(ctx, uvw, n_times, n_baselines, freq_hz, n, cell_rad, max_shift_px, stream=None):
    """(number of averaged rows, numpy int32 window per baseline)."""
    import numpy as np
    f = (C.c_double * len(freq_hz))(*[float(x) for x in freq_hz])
    win = np.zeros(n_baselines, np.int32)
    nrow = C.c_int64()
    _check(_lib.rix_bda_rows(ctx, _ptr(uvw, torch.float64, n_times * n_baselines * 3, "uvw"), n_times, n_baselines,
                             f, len(freq_hz), n, cell_rad, max_shift_px, win.ctypes.data_as(C.c_void_p),
                             C.byref(nrow), _stream(stream)))
    return int(nrow.value), win


def bda_average(ctx, uvw, vis, weight, n_times, n_baselines, freq_hz, n, cell_rad, max_shift_px, stream=None):
    """Averaged (uvw, vis, weight) as new device tensors: [rows][3] float64,
    [rows][nchan] of vis's complex type, [rows][nchan] float32."""
    nchan = len(freq_hz)
    prec = FP64 if vis.dtype == torch.complex128 else FP32
    nrow, _ = bda_rows(ctx, uvw, n_times, n_baselines, freq_hz, n, cell_rad, max_shift_px, stream)
    dev = uvw.device
    uvw_o = torch.empty((nrow, 3), dtype=torch.float64, device=dev)
    vis_o = torch.empty((nrow, nchan), dtype=vis.dtype, device=dev)
    w_o = torch.empty((nrow, nchan), dtype=torch.float32, device=dev)
    f = (C.c_double * nchan)(*[float(x) for x in freq_hz])
    got = C.c_int64()
    nv = n_times * n_baselines * nchan
    _check(_lib.rix_bda_average(ctx, _ptr(uvw, torch.float64, n_times * n_baselines * 3, "uvw"),
                                _ptr(vis, (torch.complex64, torch.complex128), nv, "vis"),
                                _ptr(weight, torch.float32, nv, "weight"), n_times, n_baselines, f, nchan, prec, n,
                                cell_rad, max_shift_px, _ptr(uvw_o, name="uvw_out"), _ptr(vis_o, name="vis_out"),
                                _ptr(w_o, name="weight_out"), nrow, C.byref(got), _stream(stream)))
    return uvw_o, vis_o, w_o


def grid_noalloc(job, part, vis, image_out, stream=None):
    """rix_grid with its scratch in the library's fixed device array (no
    device allocation at call time; FP32 jobs; overlapping calls race)."""
    _check(_lib.rix_grid_noalloc(job, part, _ptr(vis, torch.complex64, name="vis"),
                                 _ptr(image_out, torch.float32, name="image_out"), _stream(stream)))


def psf(job, part, psf_out=None, stream=None) -> float:
    w = C.c_double()
    _check(_lib.rix_psf(job, part, _img(job, psf_out, "psf_out", 2), C.byref(w), _stream(stream)))
    return w.value


def major_cycle(job, part, vis_obs, model=None, residual_out=None, stream=None):
    _check(_lib.rix_major_cycle(job, part, _visp(job, vis_obs, "vis_obs"), _img(job, model, "model"),
                                _img(job, residual_out, "residual_out"), _stream(stream)))


# -------------------------------------------------------------- a8 - a11 --
def minor_cycle_msclean(job, part, scales, gain, niter, threshold, delta_out=None, stream=None):
    sc = (C.c_float * len(scales))(*[float(s) for s in scales])
    p = MscleanParams(C.cast(sc, C.POINTER(C.c_float)), len(scales), float(gain), int(niter), float(threshold))
    _check(_lib.rix_minor_cycle_msclean(job, part, C.byref(p), _img(job, delta_out, "delta_out"),
                                        _stream(stream)))


def minor_cycle_fista(job, part, lam=0.0, lam_rel=1e-3, iters=50, levels=4, delta_out=None, stream=None,
                      dictionary=DICT_DB4, schedule=None):
    """schedule: (a, b) for lambda_n = a ||residual_n||_2 b^n, or None."""
    a, b = schedule if schedule is not None else (0.0, 0.0)
    p = FistaParams(float(lam), float(lam_rel), int(iters), int(levels), int(dictionary), 0, float(a), float(b))
    _check(_lib.rix_minor_cycle_fista(job, part, C.byref(p), _img(job, delta_out, "delta_out"),
                                      _stream(stream)))


def minor_cycle_fista_batch(job, parts, lam=0.0, lam_rel=1e-3, iters=50, levels=4, stream=None,
                            dictionary=DICT_DB4, schedule=None):
    """The FISTA minor cycles of `parts` (same cycle, same parameters) as one loop launch."""
    a, b = schedule if schedule is not None else (0.0, 0.0)
    p = FistaParams(float(lam), float(lam_rel), int(iters), int(levels), int(dictionary), 0, float(a), float(b))
    arr = (C.c_int32 * max(len(parts), 1))(*[int(q) for q in parts])
    _check(_lib.rix_minor_cycle_fista_batch(job, len(parts), arr, C.byref(p), _stream(stream)))


def get_components(job, part, capacity=1 << 16, stream=None):
    import numpy as np
    cnt = C.c_int32()
    s = np.zeros(capacity, np.int32)
    px = np.zeros(capacity, np.int32)
    amp = np.zeros(capacity, np.float64)
    _check(_lib.rix_get_components(job, part, C.byref(cnt), capacity, s.ctypes.data_as(C.c_void_p),
                                   px.ctypes.data_as(C.c_void_p), amp.ctypes.data_as(C.c_void_p), _stream(stream)))
    k = min(cnt.value, capacity)
    return s[:k].copy(), px[:k].copy(), amp[:k].copy()


def get_model(job, part, image_out, stream=None):
    _check(_lib.rix_get_model(job, part, _img(job, image_out, "image_out"), _stream(stream)))


def kernel_launches() -> int:
    return int(_lib.rix_kernel_launches())


def device_allocations() -> int:
    """Device allocations the library has made in this process."""
    return int(_lib.rix_device_allocations())


TIME_TILES, TIME_FFT, TIME_PARTITION, TIME_MINOR_LOOP = 0, 1, 2, 3


def timing_enable(on: bool = True):
    _check(_lib.rix_timing_enable(1 if on else 0))


def timing_read(kernel_class: int):
    """(summed launch ms, busy ms = union of launch intervals, launches) of one
    kernel class since the last read."""
    ms = C.c_double()
    busy = C.c_double()
    n = C.c_int64()
    _check(_lib.rix_timing_read(kernel_class, C.byref(ms), C.byref(busy), C.byref(n)))
    return ms.value, busy.value, n.value


def combine(job, image_out, stream=None):
    _check(_lib.rix_combine(job, _img(job, image_out, "image_out"), _stream(stream)))


def selftest_barrier_timeout(ctx):
    """Runs the bounded-barrier self-test; returns (status word, CTAs that gave up)."""
    status, gave_up = C.c_int(), C.c_int()
    _check(_lib.rix_selftest_barrier_timeout(ctx, C.byref(status), C.byref(gave_up)))
    return status.value, gave_up.value


def daubechies_lowpass(p: int):
    """The library's db_p low-pass filter (2p taps) as a list of floats."""
    h = (C.c_double * 16)()
    k = _lib.rix_daubechies_lowpass(int(p), h)
    _check(min(k, 0))
    return [h[i] for i in range(k)]
