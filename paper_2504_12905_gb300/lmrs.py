"""Thin ctypes binding of include/lmrs.h (argument marshalling only).

Every function has the name and argument order of its C entry point.  Vector
arguments may be torch tensors (their ``data_ptr()`` is passed), integers
(raw pointers) or None where the C API accepts NULL.  All arithmetic runs in
liblmrs.so; if the library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

LMRS_OK = 0
STATUS = ["LMRS_OK", "LMRS_ERR_INVALID_ARG", "LMRS_ERR_OOM", "LMRS_ERR_CUDA", "LMRS_ERR_NOT_PREPROCESSED",
          "LMRS_ERR_NUMERIC", "LMRS_ERR_TIMEOUT", "LMRS_ERR_BUDGET"]


class LmrsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}" if msg else name)


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_cam", C.c_float * 12), ("znear", C.c_float)]


class Config(C.Structure):
    _fields_ = [("sh_degree", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("sample_frac", C.c_double), ("samples_per_tile", C.c_int32), ("weight_mode", C.c_int32),
                ("lambda_", C.c_double), ("damping_mode", C.c_int32), ("cg_iters", C.c_int32),
                ("lr_warm", C.c_double), ("lr_cap", C.c_double), ("color_bound", C.c_double),
                ("warm_iters", C.c_int32), ("cache_bf16", C.c_int32), ("seed", C.c_uint64),
                ("sample_dist", C.c_int32), ("ssim_weight", C.c_double)]


class CgStats(C.Structure):
    _fields_ = [("rz0", C.c_double), ("rz_final", C.c_double), ("res_norm", C.c_double),
                ("alpha", C.c_double * 64), ("beta", C.c_double * 64), ("iters", C.c_int32)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("launches", C.c_int64), ("total_ms", C.c_double)]


class Peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("sm_clock_max_mhz", C.c_double), ("fp32_tflops", C.c_double),
                ("fp64_tflops", C.c_double), ("ex2_gops", C.c_double), ("atomic_scattered_gops", C.c_double),
                ("red_v4_scattered_gops", C.c_double), ("atomic_same_address_gops", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("loss", C.c_double), ("eta", C.c_double), ("max_dc", C.c_double), ("rz0", C.c_double),
                ("rz_final", C.c_double), ("n_samples", C.c_int64), ("n_pairs", C.c_int64)]


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("max_active", C.c_int32), ("setup_threads", C.c_int32),
                ("tiles_per_pair", C.c_double), ("policy", C.c_int32), ("stop_full_frame", C.c_int32),
                ("full_frame_gate", C.c_double), ("solo_min_samples", C.c_int64)]


class JobInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("converged", C.c_int32), ("steps", C.c_int32),
                ("loss", C.c_double), ("full_mse", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double),
                ("footprint_est", C.c_int64), ("footprint_peak", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int32), ("active", C.c_int32), ("finished", C.c_int64), ("bytes_in_use", C.c_int64),
                ("bytes_peak", C.c_int64), ("iterations", C.c_int64)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


class FitConfig(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("views_first", C.c_int32), ("views_later", C.c_int32),
                ("cg_first", C.c_int32), ("cg_later", C.c_int32), ("switch_step", C.c_int32),
                ("view_mode", C.c_int32), ("eval_every", C.c_int32), ("seed", C.c_uint64)]


class FitRecord(C.Structure):
    _fields_ = [("step", C.c_int32), ("n_views", C.c_int32), ("cg_iters", C.c_int32), ("loss", C.c_double),
                ("eta", C.c_double), ("mse_full", C.c_double), ("psnr", C.c_double), ("ms", C.c_double)]

_P = C.c_void_p
_S = C.c_int
_SIGS = {
    "lmrs_config_default": (_S, [C.POINTER(Config)]),
    "lmrs_scene_create": (_S, [C.POINTER(Config), C.c_int64, _P, _P, C.c_int32, _P, _P, C.POINTER(_P)]),
    "lmrs_scene_destroy": (_S, [_P]),
    "lmrs_set_params": (_S, [_P, _P]),
    "lmrs_get_params": (_S, [_P, _P]),
    "lmrs_preprocess": (_S, [_P, _P, C.c_int32, C.c_int64]),
    "lmrs_render": (_S, [_P, _P, _P]),
    "lmrs_jvp": (_S, [_P, _P, _P]),
    "lmrs_vjp": (_S, [_P, _P, _P]),
    "lmrs_rhs": (_S, [_P, _P]),
    "lmrs_jtj_diag": (_S, [_P, _P]),
    "lmrs_jtjv": (_S, [_P, _P, _P]),
    "lmrs_cg_solve": (_S, [_P, _P, _P, C.c_int32, C.POINTER(CgStats)]),
    "lmrs_step_size": (_S, [_P, _P, C.c_int64, C.POINTER(C.c_double)]),
    "lmrs_step_size_noalloc": (_S, [_P, C.c_int64, C.c_int32, C.c_int64, C.c_double, C.c_double, C.c_double,
                                    C.c_int32, _P, C.POINTER(C.c_double)]),
    "lmrs_lm_step": (_S, [_P, _P, C.c_int32, C.c_int64, C.POINTER(StepStats)]),
    "lmrs_get_solution": (_S, [_P, _P]),
    "lmrs_num_params": (C.c_int64, [_P]),
    "lmrs_num_samples": (C.c_int64, [_P]),
    "lmrs_num_pairs": (C.c_int64, [_P]),
    "lmrs_num_visible": (C.c_int64, [_P]),
    "lmrs_get_samples": (_S, [_P, _P, _P]),
    "lmrs_get_tile_lists": (_S, [_P, _P, _P]),
    "lmrs_get_sample_weights": (_S, [_P, _P]),
    "lmrs_get_ssim": (_S, [_P, _P, _P]),
    "lmrs_set_timing": (_S, [_P, C.c_int32]),
    "lmrs_get_timing": (_S, [_P, C.POINTER(KernelTime), C.c_int32, C.POINTER(C.c_int32)]),
    "lmrs_batch_create": (_S, [_P, C.c_int32, C.c_int32, _P, C.POINTER(_P)]),
    "lmrs_batch_destroy": (_S, [_P]),
    "lmrs_batch_lm_step": (_S, [_P, _P, _P, _P, _P]),
    "lmrs_batch_last_error": (C.c_char_p, [_P]),
    "lmrs_autotune_tile": (_S, [C.POINTER(Config), C.c_int64, _P, _P, C.c_int32, _P, _P, C.c_int32, _P, C.c_int32,
                                C.c_int32, _P, C.POINTER(C.c_int32), _P]),
    "lmrs_batch_scene_status": (_S, [_P, C.c_int32]),
    "lmrs_batch_set_persistent": (_S, [_P, C.c_int32]),
    "lmrs_grid_barrier_selftest": (_S, [C.c_int32, C.c_double, _P]),
    "lmrs_server_create": (_S, [C.POINTER(ServerConfig), C.POINTER(_P)]),
    "lmrs_server_submit": (_S, [_P, C.POINTER(Config), C.c_int64, _P, _P, C.c_int32, _P, C.c_int32, C.c_double,
                                C.c_int32, C.POINTER(C.c_int64)]),
    "lmrs_server_poll": (_S, [_P, C.c_int64, C.POINTER(JobInfo)]),
    "lmrs_server_wait": (_S, [_P, C.c_int64, C.c_double, C.POINTER(JobInfo)]),
    "lmrs_server_result": (_S, [_P, C.c_int64, _P]),
    "lmrs_server_forget": (_S, [_P, C.c_int64]),
    "lmrs_server_get_stats": (_S, [_P, C.POINTER(ServerStats)]),
    "lmrs_server_destroy": (_S, [_P]),
    "lmrs_footprint_bytes": (C.c_int64, [C.POINTER(Config), C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_double]),
    "lmrs_scene_device_bytes": (C.c_int64, [_P]),
    "lmrs_num_evaluations": (C.c_int64, [_P]),
    "lmrs_num_walked_entries": (C.c_int64, [_P]),
    "lmrs_uniform_views": (_S, [C.c_int32, C.c_int32, C.c_uint64, C.c_int64, _P]),
    "lmrs_view_sampler_create": (_S, [_P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(_P)]),
    "lmrs_view_sampler_destroy": (_S, [_P]),
    "lmrs_view_sampler_labels": (_S, [_P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lmrs_view_sampler_draw": (_S, [_P, C.c_int64, _P, C.POINTER(C.c_int32)]),
    "lmrs_eval_mse": (_S, [_P, C.POINTER(C.c_double)]),
    "lmrs_fit": (_S, [_P, C.POINTER(FitConfig), _P]),
    "lmrs_synchronize": (_S, [_P]),
    "lmrs_status_str": (C.c_char_p, [_S]),
    "lmrs_last_error": (C.c_char_p, [_P]),
    "lmrs_launch_count": (C.c_int64, []),
    "lmrs_measure_peaks": (_S, [_P, C.POINTER(Peaks)]),
    "lmrs_debug_build": (C.c_int32, []),
    "lmrs_debug_status": (_S, [_P, C.POINTER(C.c_uint32)]),
}
EXPORTS = tuple(_SIGS)


def library_path() -> str:
    """The release library, or the bounds-checked LMRS_DEBUG build when the
    environment sets LMRS_DEBUG_LIBRARY=1 (include/lmrs.h)."""
    return _build.library_path(debug=os.environ.get("LMRS_DEBUG_LIBRARY") == "1")


def lib():
    """Load liblmrs.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2504_12905_gb300.build.build() "
                               "(there is no fallback implementation)")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "cuda_stream"):  # a torch.cuda.Stream: its cudaStream_t handle
        return x.cuda_stream
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(status, scene=None):
    if status != LMRS_OK:
        msg = ""
        if scene:
            m = lib().lmrs_last_error(scene)
            msg = m.decode() if m else ""
        raise LmrsError(status, msg)


def cameras(cams):
    """numpy records (synthetic.CAMERA_DTYPE) -> ctypes array."""
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width = int(c["width"])
        arr[i].height = int(c["height"])
        arr[i].fx = float(c["fx"])
        arr[i].fy = float(c["fy"])
        arr[i].cx = float(c["cx"])
        arr[i].cy = float(c["cy"])
        for k in range(12):
            arr[i].world_to_cam[k] = float(c["world_to_cam"][k])
        arr[i].znear = float(c["znear"])
    return arr


def lmrs_config_default(**overrides) -> Config:
    cfg = Config()
    _check(lib().lmrs_config_default(C.byref(cfg)))
    for k, v in overrides.items():
        setattr(cfg, "lambda_" if k == "lambda" else k, v)
    return cfg


def lmrs_scene_create(cfg, n_gauss, params, cams, targets=None, stream=None):
    h = _P()
    cam_arr = cams if isinstance(cams, C.Array) else cameras(cams)
    _check(lib().lmrs_scene_create(C.byref(cfg), int(n_gauss), _ptr(params), C.cast(cam_arr, _P), len(cam_arr),
                                   _ptr(targets), _ptr(stream) if stream is not None else None, C.byref(h)))
    return h.value


def lmrs_scene_destroy(scene):
    _check(lib().lmrs_scene_destroy(scene))


def lmrs_set_params(scene, src):
    _check(lib().lmrs_set_params(scene, _ptr(src)), scene)


def lmrs_get_params(scene, dst):
    _check(lib().lmrs_get_params(scene, _ptr(dst)), scene)


def lmrs_preprocess(scene, view_ids, lm_step=0):
    v = np.ascontiguousarray(view_ids, dtype=np.int32)
    _check(lib().lmrs_preprocess(scene, v.ctypes.data, len(v), int(lm_step)), scene)


def lmrs_render(scene, images=None, residuals=None):
    _check(lib().lmrs_render(scene, _ptr(images), _ptr(residuals)), scene)


def lmrs_jvp(scene, v, u):
    _check(lib().lmrs_jvp(scene, _ptr(v), _ptr(u)), scene)


def lmrs_vjp(scene, u, g):
    _check(lib().lmrs_vjp(scene, _ptr(u), _ptr(g)), scene)


def lmrs_rhs(scene, b):
    _check(lib().lmrs_rhs(scene, _ptr(b)), scene)


def lmrs_jtj_diag(scene, d=None):
    _check(lib().lmrs_jtj_diag(scene, _ptr(d)), scene)


def lmrs_jtjv(scene, v, out):
    _check(lib().lmrs_jtjv(scene, _ptr(v), _ptr(out)), scene)


def lmrs_cg_solve(scene, b, x, iters, stats=True):
    st = CgStats() if stats else None
    _check(lib().lmrs_cg_solve(scene, _ptr(b), _ptr(x), int(iters), C.byref(st) if st is not None else None), scene)
    return st


def lmrs_step_size(scene, x, lm_step):
    eta = C.c_double()
    _check(lib().lmrs_step_size(scene, _ptr(x), int(lm_step), C.byref(eta)), scene)
    return eta.value


def lmrs_step_size_noalloc(x, n_gauss, sh_degree, lm_step, lr_warm, lr_cap, color_bound, warm_iters, stream=None):
    """Step size without a scene and without device allocation (for callers
    that cannot call cudaMalloc); see include/lmrs.h."""
    eta = C.c_double()
    _check(lib().lmrs_step_size_noalloc(_ptr(x), int(n_gauss), int(sh_degree), int(lm_step), float(lr_warm),
                                        float(lr_cap), float(color_bound), int(warm_iters),
                                        _ptr(stream) if stream is not None else None, C.byref(eta)))
    return eta.value


def lmrs_lm_step(scene, view_ids, lm_step, stats=True):
    v = np.ascontiguousarray(view_ids, dtype=np.int32)
    st = StepStats() if stats else None
    _check(lib().lmrs_lm_step(scene, v.ctypes.data, len(v), int(lm_step), C.byref(st) if st is not None else None),
           scene)
    return st


def lmrs_get_solution(scene, dst):
    _check(lib().lmrs_get_solution(scene, _ptr(dst)), scene)


def lmrs_num_params(scene):
    return int(lib().lmrs_num_params(scene))


def lmrs_num_samples(scene):
    return int(lib().lmrs_num_samples(scene))


def lmrs_num_pairs(scene):
    return int(lib().lmrs_num_pairs(scene))


def lmrs_num_visible(scene):
    return int(lib().lmrs_num_visible(scene))


def lmrs_get_samples(scene, n_views, n_tiles):
    S = lmrs_num_samples(scene)
    off = np.empty(S, np.uint8)
    tile_off = np.empty(n_views * n_tiles + 1, np.int32)
    _check(lib().lmrs_get_samples(scene, off.ctypes.data, tile_off.ctypes.data), scene)
    return off, tile_off


def lmrs_get_tile_lists(scene, n_views, n_tiles):
    n = lmrs_num_pairs(scene)
    ranges = np.empty((n_views * n_tiles, 2), np.int32)
    ids = np.empty(max(n, 1), np.int32)
    _check(lib().lmrs_get_tile_lists(scene, ranges.ctypes.data, ids.ctypes.data), scene)
    return ranges, ids[:n]


def lmrs_get_sample_weights(scene, n_samples):
    out = np.empty(int(n_samples), np.float32)
    _check(lib().lmrs_get_sample_weights(scene, out.ctypes.data), scene)
    return out


def lmrs_get_ssim(scene, n_samples):
    """(s, d), each n_samples x 3: the SSIM residual and its own-pixel derivative."""
    s = np.empty((int(n_samples), 3), np.float32)
    d = np.empty((int(n_samples), 3), np.float32)
    _check(lib().lmrs_get_ssim(scene, s.ctypes.data, d.ctypes.data), scene)
    return s, d


def lmrs_set_timing(scene, enable=True):
    _check(lib().lmrs_set_timing(scene, 1 if enable else 0), scene)


def lmrs_get_timing(scene):
    """{kernel name: (launches, total ms)} since the previous call."""
    buf = (KernelTime * 128)()
    n = C.c_int32()
    _check(lib().lmrs_get_timing(scene, buf, 128, C.byref(n)), scene)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, 128))}


def lmrs_batch_create(scenes, n_threads=8, stream=None):
    """scenes: scene handles (ints).  Returns the batch handle."""
    arr = (_P * len(scenes))(*scenes)
    h = _P()
    _check(lib().lmrs_batch_create(arr, len(scenes), int(n_threads), _ptr(stream) if stream is not None else None,
                                   C.byref(h)))
    return h.value


def lmrs_batch_destroy(batch):
    _check(lib().lmrs_batch_destroy(batch))


def lmrs_batch_last_error(batch):
    m = lib().lmrs_batch_last_error(batch)
    return m.decode() if m else ""


def lmrs_batch_lm_step(batch, views, lm_steps, stats=True):
    """views: one sequence of camera indices per scene; lm_steps: one step
    index per scene.  Returns the per-scene StepStats (or None)."""
    n = len(views)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(v, np.int32) for v in views]), np.int32)
    nv = np.ascontiguousarray([len(v) for v in views], np.int32)
    steps = np.ascontiguousarray(lm_steps, np.int64)
    st = (StepStats * n)() if stats else None
    status = lib().lmrs_batch_lm_step(batch, flat.ctypes.data, nv.ctypes.data, steps.ctypes.data,
                                      C.cast(st, _P) if st is not None else None)
    if status != LMRS_OK:
        raise LmrsError(status, lmrs_batch_last_error(batch))
    return list(st) if st is not None else None


def lmrs_autotune_tile(cfg, n_gauss, params, cams, targets, views, shapes, reps=3, stream=None):
    """Times each (tile_w, tile_h) in ``shapes`` on a private copy of the
    scene; returns (index of the fastest, per-shape median ms per LM step)."""
    cam_arr = cams if isinstance(cams, C.Array) else cameras(cams)
    v = np.ascontiguousarray(views, dtype=np.int32)
    sh = np.ascontiguousarray(shapes, dtype=np.int32).reshape(-1, 2)
    ms = np.zeros(len(sh), np.float32)
    best = C.c_int32(-1)
    _check(lib().lmrs_autotune_tile(C.byref(cfg), int(n_gauss), _ptr(params), C.cast(cam_arr, _P), len(cam_arr),
                                    _ptr(targets), v.ctypes.data, len(v), sh.ctypes.data, len(sh), int(reps),
                                    _ptr(stream) if stream is not None else None, C.byref(best), ms.ctypes.data))
    return best.value, ms


def lmrs_batch_scene_status(batch, i):
    return int(lib().lmrs_batch_scene_status(batch, int(i)))


def lmrs_batch_set_persistent(batch, on):
    _check(lib().lmrs_batch_set_persistent(batch, int(on)))


def lmrs_grid_barrier_selftest(missing, timeout_s=0.25, stream=None):
    """Status of a grid-barrier launch missing `missing` blocks (see include/lmrs.h)."""
    return int(lib().lmrs_grid_barrier_selftest(int(missing), float(timeout_s), _ptr(stream)))


def lmrs_server_create(budget_bytes, max_active=64, setup_threads=8, tiles_per_pair=0.0, policy=0,
                       stop_full_frame=0, full_frame_gate=0.0, solo_min_samples=0):
    cfg = ServerConfig(int(budget_bytes), int(max_active), int(setup_threads), float(tiles_per_pair), int(policy),
                       int(stop_full_frame), float(full_frame_gate), int(solo_min_samples))
    h = _P()
    _check(lib().lmrs_server_create(C.byref(cfg), C.byref(h)))
    return h.value


def lmrs_server_submit(server, cfg, n_gauss, params_host, cams, targets_host, views_per_step=0, target_loss=0.0,
                       max_steps=20):
    """params_host [P] and targets_host [n_cams, H, W, 3]: float32 host arrays
    (copied).  Returns the job id."""
    p = np.ascontiguousarray(params_host, np.float32)
    t = np.ascontiguousarray(targets_host, np.float32)
    cam_arr = cams if isinstance(cams, C.Array) else cameras(cams)
    jid = C.c_int64(0)
    status = lib().lmrs_server_submit(server, C.byref(cfg), int(n_gauss), p.ctypes.data, C.cast(cam_arr, _P),
                                      len(cam_arr), t.ctypes.data, int(views_per_step), float(target_loss),
                                      int(max_steps), C.byref(jid))
    if status != LMRS_OK:
        raise LmrsError(status, "server submit")
    return jid.value


def lmrs_server_poll(server, job):
    info = JobInfo()
    _check(lib().lmrs_server_poll(server, int(job), C.byref(info)))
    return info


def lmrs_server_wait(server, job, timeout_s=60.0):
    """Returns (status, JobInfo); status LMRS_ERR_TIMEOUT if not finished in time."""
    info = JobInfo()
    status = lib().lmrs_server_wait(server, int(job), float(timeout_s), C.byref(info))
    if status not in (LMRS_OK, 6):
        raise LmrsError(status, "server wait")
    return status, info


def lmrs_server_result(server, job, n_params):
    out = np.empty(int(n_params), np.float32)
    _check(lib().lmrs_server_result(server, int(job), out.ctypes.data))
    return out


def lmrs_server_forget(server, job):
    _check(lib().lmrs_server_forget(server, int(job)))


def lmrs_server_get_stats(server):
    st = ServerStats()
    _check(lib().lmrs_server_get_stats(server, C.byref(st)))
    return st


def lmrs_server_destroy(server):
    _check(lib().lmrs_server_destroy(server))


def lmrs_footprint_bytes(cfg, n_gauss, n_cams, width, height, views_per_step=0, tiles_per_pair=0.0):
    return int(lib().lmrs_footprint_bytes(C.byref(cfg), int(n_gauss), int(n_cams), int(width), int(height),
                                          int(views_per_step), float(tiles_per_pair)))


def lmrs_num_evaluations(scene):
    return int(lib().lmrs_num_evaluations(scene))


def lmrs_num_walked_entries(scene):
    return int(lib().lmrs_num_walked_entries(scene))


def lmrs_scene_device_bytes(scene):
    return int(lib().lmrs_scene_device_bytes(scene))


def lmrs_uniform_views(n_cams, n_views, seed, step):
    out = np.empty(int(n_cams), np.int32)
    _check(lib().lmrs_uniform_views(int(n_cams), int(n_views), C.c_uint64(seed), int(step), out.ctypes.data))
    k = n_cams if (n_views <= 0 or n_views >= n_cams) else n_views
    return out[:k].copy()


class ViewSampler:
    """K-means view sampler (Sec. 4.3)."""

    def __init__(self, cams, n_clusters, seed=0):
        self._arr = cams if isinstance(cams, C.Array) else cameras(cams)
        h = _P()
        _check(lib().lmrs_view_sampler_create(C.cast(self._arr, _P), len(self._arr), int(n_clusters),
                                              C.c_uint64(seed), C.byref(h)))
        self.h = h.value
        self.n_cams = len(self._arr)

    def labels(self):
        out = np.empty(self.n_cams, np.int32)
        k, it = C.c_int32(0), C.c_int32(0)
        _check(lib().lmrs_view_sampler_labels(self.h, out.ctypes.data, C.byref(k), C.byref(it)))
        return out, k.value, it.value

    def draw(self, step):
        out = np.empty(self.n_cams, np.int32)
        n = C.c_int32(0)
        _check(lib().lmrs_view_sampler_draw(self.h, int(step), out.ctypes.data, C.byref(n)))
        return out[:n.value].copy()

    def close(self):
        if getattr(self, "h", None):
            lib().lmrs_view_sampler_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lmrs_eval_mse(scene):
    m = C.c_double(0.0)
    _check(lib().lmrs_eval_mse(scene, C.byref(m)), scene)
    return m.value


def lmrs_fit(scene, n_steps, views_first, views_later=None, cg_first=8, cg_later=None, switch_step=0,
             view_mode=0, eval_every=0, seed=0):
    cfg = FitConfig(int(n_steps), int(views_first), int(views_later or views_first), int(cg_first),
                    int(cg_first if cg_later is None else cg_later), int(switch_step), int(view_mode),
                    int(eval_every), int(seed))
    recs = (FitRecord * int(n_steps))()
    _check(lib().lmrs_fit(scene, C.byref(cfg), C.cast(recs, _P)), scene)
    return list(recs)


def lmrs_synchronize(scene):
    _check(lib().lmrs_synchronize(scene), scene)


def lmrs_status_str(status):
    return lib().lmrs_status_str(status).decode()


def lmrs_last_error(scene):
    m = lib().lmrs_last_error(scene)
    return m.decode() if m else ""


def lmrs_launch_count():
    return int(lib().lmrs_launch_count())


def lmrs_debug_build():
    return int(lib().lmrs_debug_build())


def lmrs_debug_status(scene):
    """The scene's debug word (0: every check passed), then cleared."""
    bits = C.c_uint32()
    _check(lib().lmrs_debug_status(scene, C.byref(bits)), scene)
    return int(bits.value)


def lmrs_measure_peaks(stream=None):
    """Measured peak rates of the current device as a dict (see include/lmrs.h)."""
    pk = Peaks()
    _check(lib().lmrs_measure_peaks(_ptr(stream), C.byref(pk)))
    return {name: getattr(pk, name) for name, _ in Peaks._fields_}


class Scene:
    """Owner of one lmrs_scene plus the torch tensors it borrows."""

    def __init__(self, params, cams, n_gauss, sh_degree=0, targets=None, stream=None, **cfg):
        import torch
        c = lmrs_config_default(sh_degree=sh_degree, **cfg)
        self.cfg = c
        self.n_gauss = int(n_gauss)
        self.sh_degree = sh_degree
        self.cams = cams
        self.width = int(cams[0]["width"])
        self.height = int(cams[0]["height"])
        self.tiles_x = (self.width + c.tile_w - 1) // c.tile_w
        self.tiles_y = (self.height + c.tile_h - 1) // c.tile_h
        self.n_tiles = self.tiles_x * self.tiles_y
        self.targets = targets  # kept alive: the scene borrows it
        p = params if hasattr(params, "data_ptr") else torch.as_tensor(np.ascontiguousarray(params, np.float32))
        self.h = lmrs_scene_create(c, n_gauss, p.contiguous() if p.is_cuda else p.contiguous(), cams, targets, stream)
        self.n_params = lmrs_num_params(self.h)
        self.n_views = 0

    def close(self):
        if getattr(self, "h", None):
            lmrs_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def preprocess(self, views, step=0):
        lmrs_preprocess(self.h, views, step)
        self.n_views = len(views)

    @property
    def n_samples(self):
        return lmrs_num_samples(self.h)

    @property
    def n_pairs(self):
        return lmrs_num_pairs(self.h)
