"""FP64 CPU oracle of the LM-RS hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA library.

The library is compiled from ``oracle/lmrs_oracle.cpp`` by
``oracle.build.build()`` (plain g++ with OpenMP and FP contraction disabled).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None


class _Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_cam", C.c_float * 12), ("znear", C.c_float)]


class _Config(C.Structure):
    _fields_ = [("sh_degree", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("sample_frac", C.c_double), ("samples_per_tile", C.c_int32), ("weight_mode", C.c_int32),
                ("lambda_", C.c_double), ("damping_mode", C.c_int32), ("cg_iters", C.c_int32),
                ("lr_warm", C.c_double), ("lr_cap", C.c_double), ("color_bound", C.c_double),
                ("warm_iters", C.c_int32), ("seed", C.c_uint64),
                ("margin_alpha", C.c_double), ("margin_T", C.c_double), ("sample_dist", C.c_int32),
                ("ssim_weight", C.c_double), ("list_mode", C.c_int32)]


DEFAULTS = dict(sh_degree=0, tile_w=16, tile_h=16, sample_frac=1.0, samples_per_tile=0, weight_mode=0,
                lambda_=1e-2, damping_mode=1, cg_iters=10, lr_warm=0.05, lr_cap=0.2, color_bound=1.0,
                warm_iters=10, seed=0x1A5E0000, margin_alpha=1e-4, margin_T=1e-3, sample_dist=0,
                ssim_weight=0.0, list_mode=0)

_P = C.c_void_p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.library_path()
        if not os.path.exists(path):
            _build.build()
        L = C.CDLL(path)
        sig = {
            "orc_create": (_P, [C.POINTER(_Config), C.c_int32, _P, _P, C.c_int32, _P]),
            "orc_destroy": (None, [_P]),
            "orc_set_params": (C.c_int32, [_P, _P]),
            "orc_get_params": (C.c_int32, [_P, _P]),
            "orc_num_params": (C.c_int64, [_P]),
            "orc_begin_step": (C.c_int32, [_P, _P, C.c_int32, C.c_int64]),
            "orc_num_samples": (C.c_int64, [_P]),
            "orc_get_samples": (C.c_int32, [_P, _P, _P, _P, _P, _P, _P]),
            "orc_get_sample_flags": (C.c_int32, [_P, _P]),
            "orc_get_ssim": (C.c_int32, [_P, _P, _P, _P]),
            "orc_num_pairs": (C.c_int64, [_P]),
            "orc_get_lists": (C.c_int32, [_P, _P, _P]),
            "orc_get_geom": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
            "orc_get_features": (C.c_int32, [_P, C.c_int32, _P]),
            "orc_render_samples": (C.c_int32, [_P, _P, _P, _P]),
            "orc_render_samples_subset": (C.c_int32, [_P, _P, C.c_int64, _P, _P]),
            "orc_render_full": (C.c_int32, [_P, C.c_int32, _P, _P]),
            "orc_pixel_counts": (C.c_int32, [_P, C.c_int32, _P]),
            "orc_render_full_f32": (C.c_int32, [_P, C.c_int32, _P]),
            "orc_jvp": (C.c_int32, [_P, _P, _P]),
            "orc_jvp_subset": (C.c_int32, [_P, _P, _P, C.c_int64, _P]),
            "orc_vjp": (C.c_int32, [_P, _P, _P]),
            "orc_vjp_gauss": (C.c_int32, [_P, _P, _P, C.c_int32, _P]),
            "orc_diag": (C.c_int32, [_P, _P]),
            "orc_diag_magnitude": (C.c_int32, [_P, _P]),
            "orc_set_flips": (C.c_int32, [_P, _P, _P, C.c_int64]),
            "orc_clear_flips": (C.c_int32, [_P]),
            "orc_near_counts": (C.c_int32, [_P, _P, C.c_int64, _P]),
            "orc_sample_outcomes": (C.c_int32, [_P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P]),
            "orc_diag_gauss": (C.c_int32, [_P, _P, C.c_int32, _P]),
            "orc_apply": (C.c_int32, [_P, _P, _P, _P]),
            "orc_apply_gauss": (C.c_int32, [_P, _P, _P, _P, C.c_int32, _P]),
            "orc_rhs": (C.c_int32, [_P, _P]),
            "orc_precond": (C.c_int32, [_P, _P, _P]),
            "orc_cg": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P]),
            "orc_step_size": (C.c_double, [_P, _P, C.c_int64]),
            "orc_lm_step": (C.c_int32, [_P, _P, C.c_int32, C.c_int64, _P, _P]),
            "orc_sh_basis": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, _P]),
            "orc_splitmix64": (None, [C.c_uint64, C.c_int32, _P]),
            "orc_tile_seed": (C.c_uint64, [C.c_uint64, C.c_int64, C.c_int32, C.c_int32]),
            "orc_sample_tile": (None, [C.c_uint64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P]),
            "orc_num_threads": (C.c_int32, []),
            "orc_ssim_pixel": (None, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def cams_to_struct(cams):
    arr = (_Camera * len(cams))()
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


class OracleScene:
    """One scene held by the oracle.  ``params`` are the FP32 inputs (the
    same values the CUDA path receives); the oracle works on their FP64
    widening."""

    def __init__(self, params, cams, n_gauss, sh_degree=0, targets=None, **cfg):
        c = dict(DEFAULTS)
        c["sh_degree"] = sh_degree
        c.update(cfg)
        self.cfg = c
        self._cfg = _Config(**c)
        self.n_gauss = int(n_gauss)
        self.sh_degree = sh_degree
        self.Pg = 11 + 3 * (sh_degree + 1) ** 2
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._cams = cams_to_struct(cams)
        self.width = int(cams[0]["width"])
        self.height = int(cams[0]["height"])
        self._targets = None if targets is None else np.ascontiguousarray(targets, dtype=np.float32)
        self._h = lib().orc_create(C.byref(self._cfg), self.n_gauss, _ptr(p), C.cast(self._cams, C.c_void_p),
                                   len(cams), None if self._targets is None else _ptr(self._targets))
        if not self._h:
            raise ValueError("orc_create rejected its arguments")
        self.n_views = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.orc_destroy(h)
            self._h = None

    # -- parameters -----------------------------------------------------------
    @property
    def n_params(self):
        return int(lib().orc_num_params(self._h))

    def get_params(self):
        out = np.empty(self.n_params)
        lib().orc_get_params(self._h, _ptr(out))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        lib().orc_set_params(self._h, _ptr(p))

    # -- one LM step's setup --------------------------------------------------
    def begin_step(self, views, step=0):
        v = np.ascontiguousarray(views, dtype=np.int32)
        if lib().orc_begin_step(self._h, _ptr(v), len(v), int(step)):
            raise ValueError("orc_begin_step failed")
        self.n_views = len(v)
        self.views = v

    @property
    def n_samples(self):
        return int(lib().orc_num_samples(self._h))

    def samples(self):
        S = self.n_samples
        tiles = self.n_tiles
        off = np.empty(S, np.uint8)
        tile_off = np.empty(self.n_views * tiles + 1, np.int32)
        w = np.empty(S)
        px = np.empty(S, np.int32)
        py = np.empty(S, np.int32)
        slot = np.empty(S, np.int32)
        lib().orc_get_samples(self._h, _ptr(off), _ptr(tile_off), _ptr(w), _ptr(px), _ptr(py), _ptr(slot))
        return dict(off=off, tile_off=tile_off, w=w, px=px, py=py, slot=slot)

    def render_full_f32(self, slot):
        """The view's frame with the preprocessing and compositing in
        binary32 over the same lists (FP32 rounding against the FP64 frame)."""
        img = np.empty((self.height, self.width, 3))
        lib().orc_render_full_f32(self._h, slot, _ptr(img))
        return img

    def pixel_counts(self, slot):
        out = np.empty((self.height, self.width), np.int32)
        lib().orc_pixel_counts(self._h, int(slot), _ptr(out))
        return out

    def sample_flags(self):
        out = np.empty(self.n_samples, np.uint8)
        lib().orc_get_sample_flags(self._h, _ptr(out))
        return out

    def ssim(self):
        """Per sample and channel the SSIM residual s = 1 - SSIM and its
        own-pixel derivative d (S x 3 each), and per sample the window flag."""
        S = self.n_samples
        sv = np.empty((S, 3))
        dv = np.empty((S, 3))
        fl = np.empty(S, np.uint8)
        lib().orc_get_ssim(self._h, _ptr(sv), _ptr(dv), _ptr(fl))
        return sv, dv, fl

    @property
    def tiles_x(self):
        return (self.width + self.cfg["tile_w"] - 1) // self.cfg["tile_w"]

    @property
    def tiles_y(self):
        return (self.height + self.cfg["tile_h"] - 1) // self.cfg["tile_h"]

    @property
    def n_tiles(self):
        return self.tiles_x * self.tiles_y

    def lists(self):
        n = int(lib().orc_num_pairs(self._h))
        ranges = np.empty((self.n_views * self.n_tiles, 2), np.int32)
        ids = np.empty(n, np.int32)
        lib().orc_get_lists(self._h, _ptr(ranges), _ptr(ids))
        return ranges, ids

    def geom(self, slot):
        G = self.n_gauss
        vis = np.empty(G, np.int32)
        depth = np.empty(G, np.float32)
        rect = np.empty((G, 4), np.int32)
        lib().orc_get_geom(self._h, slot, _ptr(vis), _ptr(depth), _ptr(rect))
        return vis, depth, rect

    def features(self, slot):
        out = np.empty((self.n_gauss, 9))
        lib().orc_get_features(self._h, slot, _ptr(out))
        return out

    # -- forward ----------------------------------------------------------------
    def render_samples(self):
        S = self.n_samples
        rgb = np.empty((S, 3))
        res = np.empty((S, 3))
        flags = np.empty(S, np.uint8)
        lib().orc_render_samples(self._h, _ptr(rgb), _ptr(res), _ptr(flags))
        return rgb, res, flags

    def render_samples_subset(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        rgb = np.empty((len(idx), 3))
        flags = np.empty(len(idx), np.uint8)
        lib().orc_render_samples_subset(self._h, _ptr(idx), len(idx), _ptr(rgb), _ptr(flags))
        return rgb, flags

    def render_full(self, slot):
        img = np.empty((self.height, self.width, 3))
        flags = np.empty((self.height, self.width), np.uint8)
        lib().orc_render_full(self._h, slot, _ptr(img), _ptr(flags))
        return img, flags

    # -- derivatives --------------------------------------------------------------
    def jvp(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        u = np.empty((self.n_samples, 3))
        lib().orc_jvp(self._h, _ptr(v), _ptr(u))
        return u

    def jvp_subset(self, v, idx):
        v = np.ascontiguousarray(v, dtype=np.float64)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        u = np.empty((len(idx), 3))
        lib().orc_jvp_subset(self._h, _ptr(v), _ptr(idx), len(idx), _ptr(u))
        return u

    def vjp(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        g = np.empty(self.n_params)
        lib().orc_vjp(self._h, _ptr(u), _ptr(g))
        return g

    def vjp_gauss(self, u, gids):
        u = np.ascontiguousarray(u, dtype=np.float64)
        gids = np.ascontiguousarray(gids, dtype=np.int32)
        out = np.empty((len(gids), self.Pg))
        lib().orc_vjp_gauss(self._h, _ptr(u), _ptr(gids), len(gids), _ptr(out))
        return out

    def diag(self):
        D = np.empty(self.n_params)
        lib().orc_diag(self._h, _ptr(D))
        return D

    def set_flips(self, idx, masks):
        """Bit k of masks[j] inverts the k-th near decision of sample idx[j]
        (clamp, skip, termination per entry, in list order)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        masks = np.ascontiguousarray(masks, dtype=np.uint32)
        assert idx.shape == masks.shape
        if lib().orc_set_flips(self._h, _ptr(idx), _ptr(masks), len(idx)) != 0:
            raise ValueError("sample index out of range")

    def clear_flips(self):
        lib().orc_clear_flips(self._h)

    def near_counts(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.zeros(len(idx), np.int32)
        lib().orc_near_counts(self._h, _ptr(idx), len(idx), _ptr(out))
        return out

    def sample_outcomes(self, v, idx, max_bits=4):
        """(n_near [n], rgb [n, 2^max_bits, 3], u [n, 2^max_bits, 3]): the
        colour and J v of each sample under every mask of its near decisions
        (NaN beyond 2^min(n_near, max_bits))."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        M = 1 << max_bits
        nn = np.zeros(len(idx), np.int32)
        rgb = np.empty((len(idx), M, 3))
        u = np.empty((len(idx), M, 3))
        lib().orc_sample_outcomes(self._h, _ptr(v), _ptr(idx), len(idx), int(max_bits), _ptr(nn), _ptr(rgb), _ptr(u))
        return nn, rgb, u

    def diag_magnitude(self):
        """Per entry of diag(J^T W J): the sum over rows of w (sum_f |dC/df
        a_fj|)^2, against which an FP32 evaluation of the entry rounds."""
        M = np.empty(self.n_params)
        lib().orc_diag_magnitude(self._h, _ptr(M))
        return M

    def diag_gauss(self, gids):
        gids = np.ascontiguousarray(gids, dtype=np.int32)
        out = np.empty((len(gids), self.Pg))
        lib().orc_diag_gauss(self._h, _ptr(gids), len(gids), _ptr(out))
        return out

    def apply(self, v, D):
        v = np.ascontiguousarray(v, dtype=np.float64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        out = np.empty(self.n_params)
        lib().orc_apply(self._h, _ptr(v), _ptr(D), _ptr(out))
        return out

    def apply_gauss(self, v, D, gids):
        v = np.ascontiguousarray(v, dtype=np.float64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        gids = np.ascontiguousarray(gids, dtype=np.int32)
        out = np.empty((len(gids), self.Pg))
        lib().orc_apply_gauss(self._h, _ptr(v), _ptr(D), _ptr(gids), len(gids), _ptr(out))
        return out

    def rhs(self):
        b = np.empty(self.n_params)
        lib().orc_rhs(self._h, _ptr(b))
        return b

    def precond(self, D):
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = np.empty(self.n_params)
        lib().orc_precond(self._h, _ptr(D), _ptr(m))
        return m

    def cg(self, b, D, iters):
        b = np.ascontiguousarray(b, dtype=np.float64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        x = np.empty(self.n_params)
        st = np.zeros(2 + 2 * max(iters, 1))
        lib().orc_cg(self._h, _ptr(b), _ptr(D), iters, _ptr(x), _ptr(st))
        return x, st

    def step_size(self, x, step):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(lib().orc_step_size(self._h, _ptr(x), int(step)))

    def lm_step(self, views, step):
        v = np.ascontiguousarray(views, dtype=np.int32)
        x = np.empty(self.n_params)
        st = np.zeros(3)
        if lib().orc_lm_step(self._h, _ptr(v), len(v), int(step), _ptr(x), _ptr(st)):
            raise ValueError("orc_lm_step failed")
        self.n_views = len(v)
        self.views = v
        return x, st


def sh_basis(deg, x, y, z):
    Y = np.zeros(16)
    lib().orc_sh_basis(deg, float(x), float(y), float(z), _ptr(Y))
    return Y[: (deg + 1) ** 2]


def splitmix64(state, n):
    out = np.empty(n, np.uint64)
    lib().orc_splitmix64(C.c_uint64(state), n, _ptr(out))
    return out


def tile_seed(seed, step, view, tile):
    return int(lib().orc_tile_seed(C.c_uint64(seed), step, view, tile))


def sample_tile(seed, step, view, tile, n_valid, k):
    out = np.empty(k, np.uint8)
    lib().orc_sample_tile(C.c_uint64(seed), step, view, tile, n_valid, k, _ptr(out))
    return out


def num_threads():
    return int(lib().orc_num_threads())


def ssim_pixel(X, Y, px, py):
    """(s, d) of the three channels at pixel (px, py) of H x W x 3 images."""
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    H, W = X.shape[:2]
    sv = np.empty(3)
    dv = np.empty(3)
    lib().orc_ssim_pixel(_ptr(X), _ptr(Y), H, W, int(px), int(py), _ptr(sv), _ptr(dv))
    return sv, dv
