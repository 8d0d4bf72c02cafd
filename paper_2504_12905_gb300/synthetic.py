"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameters, pinhole cameras and noise
images.  It holds none of the method's arithmetic (no projection, no
rendering, no derivatives), so both the CUDA path and the FP64 oracle can be
fed from it.  Targets that must be renders of perturbed parameters are made by
whichever side consumes them.

Parameter layout (one float per entry, group-major structure of arrays, the
same for every P-vector of the method):

    [ means G x 3 | log_scales G x 3 | quats G x 4 (w, x, y, z) |
      opacity_logits G | sh G x (d+1)^2 x 3 ]

so a Gaussian has P_g = 11 + 3 (d+1)^2 entries (14 for SH degree 0, the
parameter set of Sec. 4.1: opacity, colour, mean, scale, quaternion).

Camera record (little-endian, 76 bytes, matches ``lmrs_camera``):
    int32 width, height; float fx, fy, cx, cy; float world_to_cam[12]
    (row-major 3x4 [R | t], OpenCV axes: x right, y down, z forward);
    float znear.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CAMERA_DTYPE = np.dtype([
    ("width", "<i4"), ("height", "<i4"),
    ("fx", "<f4"), ("fy", "<f4"), ("cx", "<f4"), ("cy", "<f4"),
    ("world_to_cam", "<f4", (12,)),
    ("znear", "<f4"),
])
assert CAMERA_DTYPE.itemsize == 76

# Half-range of the SH degree-0 coefficient that maps to colours in [0, 1]:
# 1/(2 C0) with C0 = 1/(2 sqrt(pi)), i.e. sqrt(pi) ~ 1.77 (the colour-parameter
# range quoted in Sec. 4.5).
SH_DC_HALF_RANGE = math.sqrt(math.pi)


def n_coeffs(sh_degree: int) -> int:
    return (sh_degree + 1) ** 2


def params_per_gaussian(sh_degree: int) -> int:
    return 11 + 3 * n_coeffs(sh_degree)


def group_offsets(n_gauss: int, sh_degree: int) -> dict:
    """Start index of each parameter group inside a P-vector."""
    G = n_gauss
    return {"means": 0, "log_scales": 3 * G, "quats": 6 * G, "opacity": 10 * G,
            "sh": 11 * G, "end": G * params_per_gaussian(sh_degree)}


@dataclasses.dataclass
class Scene:
    n_gauss: int
    sh_degree: int
    params: np.ndarray          # float32 [P]
    cams: np.ndarray            # CAMERA_DTYPE [n_cams]
    seed: int

    @property
    def width(self) -> int:
        return int(self.cams["width"][0])

    @property
    def height(self) -> int:
        return int(self.cams["height"][0])

    @property
    def n_params(self) -> int:
        return self.params.size


def look_at_camera(eye, width, height, hfov_deg=60.0, znear=0.2):
    """Pinhole camera at ``eye`` looking at the origin with +z as world up."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = -eye / np.linalg.norm(eye)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    cam = np.zeros((), dtype=CAMERA_DTYPE)
    cam["width"] = width
    cam["height"] = height
    f = (0.5 * width) / math.tan(math.radians(hfov_deg) * 0.5)
    cam["fx"] = f
    cam["fy"] = f
    cam["cx"] = 0.5 * width
    cam["cy"] = 0.5 * height
    w2c = np.zeros((3, 4))
    w2c[:, :3] = R
    w2c[:, 3] = t
    cam["world_to_cam"] = w2c.reshape(-1)
    cam["znear"] = znear
    return cam


def ring_cameras(n, radius, width, height, elev_deg=0.0, hfov_deg=60.0):
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        az = 2.0 * math.pi * i / n
        el = math.radians(elev_deg)
        eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams[i] = look_at_camera(eye, width, height, hfov_deg)
    return cams


def hemisphere_cameras(n, radius, width, height, min_elev_deg=10.0, hfov_deg=60.0):
    """Fibonacci points on the upper hemisphere above ``min_elev_deg``."""
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    z0 = math.sin(math.radians(min_elev_deg))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n):
        z = z0 + (1.0 - z0) * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        az = golden * i
        eye = radius * np.array([r * math.cos(az), r * math.sin(az), z])
        cams[i] = look_at_camera(eye, width, height, hfov_deg)
    return cams


def orbit_cameras(rng, n, radius, width, height, elev_jitter_deg=15.0, hfov_deg=60.0):
    """``n`` views evenly spaced in azimuth, elevation uniform in +-jitter."""
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        az = 2.0 * math.pi * i / n
        el = math.radians(rng.uniform(-elev_jitter_deg, elev_jitter_deg))
        eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams[i] = look_at_camera(eye, width, height, hfov_deg)
    return cams


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _random_rotation(rng):
    """Haar-random rotation from the QR factorisation of a Gaussian matrix."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def pack_params(means, log_scales, quats, opacity_logits, sh):
    G = means.shape[0]
    return np.concatenate([
        means.reshape(-1), log_scales.reshape(-1), quats.reshape(-1),
        opacity_logits.reshape(-1), sh.reshape(G, -1).reshape(-1),
    ]).astype(np.float32)


def draw_gaussians(rng, n_gauss, sh_degree, means=None, sh_sigma=None):
    """Gaussian parameters with the laws of the tiny configuration:
    means U[-1,1]^3, log-scales N(-3.5, 0.3), unit quaternions (normalised
    N(0,1)^4), opacity logits N(0,1); SH degree 0 draws the DC coefficient
    uniformly in +-sqrt(pi) (colours uniform in [0,1]); higher bands, or all
    bands when ``sh_sigma`` is given, are N(0, sh_sigma)."""
    if means is None:
        means = rng.uniform(-1.0, 1.0, (n_gauss, 3))
    log_scales = rng.normal(-3.5, 0.3, (n_gauss, 3))
    quats = _unit_quats(rng, n_gauss)
    opac = rng.normal(0.0, 1.0, n_gauss)
    K = n_coeffs(sh_degree)
    sh = np.zeros((n_gauss, K, 3))
    if sh_sigma is None:
        sh[:, 0, :] = rng.uniform(-SH_DC_HALF_RANGE, SH_DC_HALF_RANGE, (n_gauss, 3))
        if K > 1:
            sh[:, 1:, :] = rng.normal(0.0, 0.2, (n_gauss, K - 1, 3))
    else:
        sh[:] = rng.normal(0.0, sh_sigma, (n_gauss, K, 3))
    return pack_params(means, log_scales, quats, opac, sh)


def blob_means(rng, n_gauss, n_blobs=32):
    """Means from an equal-weight mixture of anisotropic Gaussian blobs:
    centres U[-1,1]^3, per-axis sigma U[0.05, 0.3], random orientation."""
    centres = rng.uniform(-1.0, 1.0, (n_blobs, 3))
    sig = rng.uniform(0.05, 0.3, (n_blobs, 3))
    rots = [_random_rotation(rng) for _ in range(n_blobs)]
    which = rng.integers(0, n_blobs, n_gauss)
    z = rng.standard_normal((n_gauss, 3))
    out = np.empty((n_gauss, 3))
    for b in range(n_blobs):
        m = which == b
        out[m] = centres[b] + (z[m] * sig[b]) @ rots[b].T
    return out


def perturb(rng, params, sigma=0.05):
    """Every raw parameter plus N(0, sigma); the fit target of a scene."""
    return (params.astype(np.float64) + rng.normal(0.0, sigma, params.shape)).astype(np.float32)


def noise_targets(rng, n_cams, height, width):
    return rng.uniform(0.0, 1.0, (n_cams, height, width, 3)).astype(np.float32)


# ----------------------------------------------------------------------------
# Named workloads.
# ----------------------------------------------------------------------------

def tiny_scene(seed=0x1A5E0000, n_gauss=1000, width=64, height=64, sh_degree=0):
    """1,000 Gaussians, 4 cameras of 64x64 at radius 3 (azimuth 0/90/180/270,
    elevation 0), 60 degree FOV."""
    rng = np.random.default_rng(seed)
    params = draw_gaussians(rng, n_gauss, sh_degree)
    cams = ring_cameras(4, 3.0, width, height)
    return Scene(n_gauss, sh_degree, params, cams, seed)


def moderate_scene(seed=0x1A5E0001, n_gauss=200_000, n_views=24, width=1024, height=672, sh_degree=3):
    """200k Gaussians from 32 anisotropic blobs, SH degree 3 with N(0, 0.2)
    coefficients, 24 views of 1024x672 on a Fibonacci hemisphere."""
    rng = np.random.default_rng(seed)
    means = blob_means(rng, n_gauss)
    params = draw_gaussians(rng, n_gauss, sh_degree, means=means, sh_sigma=0.2)
    cams = hemisphere_cameras(n_views, 3.0, width, height)
    return Scene(n_gauss, sh_degree, params, cams, seed)


def large_scene(seed=0x1A5E0002, n_gauss=1_500_000, n_views=100, width=1297, height=840, sh_degree=3):
    """1.5M Gaussians, SH degree 3, 100 views of 1297x840 on a 360 degree
    orbit with +-15 degree elevation jitter."""
    rng = np.random.default_rng(seed)
    means = blob_means(rng, n_gauss)
    params = draw_gaussians(rng, n_gauss, sh_degree, means=means, sh_sigma=0.2)
    cams = orbit_cameras(rng, n_views, 3.0, width, height)
    return Scene(n_gauss, sh_degree, params, cams, seed)


def small_fit_scenes(seed=0x1A5E0003, n_scenes=64, g_lo=5_000, g_hi=50_000, v_lo=4, v_hi=16,
                     width=256, height=256, sh_degree=0):
    """Independent small scenes: Gaussian counts log-uniform in [g_lo, g_hi],
    v_lo..v_hi views each at width x height."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        G = int(round(math.exp(rng.uniform(math.log(g_lo), math.log(g_hi)))))
        nv = int(rng.integers(v_lo, v_hi + 1))
        sub = np.random.default_rng([seed, i])
        means = blob_means(sub, G, n_blobs=8)
        params = draw_gaussians(sub, G, sh_degree, means=means)
        cams = hemisphere_cameras(nv, 3.0, width, height)
        out.append(Scene(G, sh_degree, params, cams, int(seed) * 1000 + i))
    return out


def serving_requests(seed=0x1A5E0004, n_requests=100, rate=20.0, g_lo=2_000, g_hi=300_000, v_lo=8, v_hi=32,
                     width=512, height=512, sh_degree=1):
    """A stream of fit requests: Poisson arrivals (exponential gaps of mean
    1/rate seconds), Gaussian counts log-uniform in [g_lo, g_hi], v_lo..v_hi
    views of width x height on a Fibonacci hemisphere, means from 16 blobs.
    Returns [(arrival time in seconds, Scene)]; the Scene holds the ground
    truth of the fit."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        G = int(round(math.exp(rng.uniform(math.log(g_lo), math.log(g_hi)))))
        nv = int(rng.integers(v_lo, v_hi + 1))
        sub = np.random.default_rng([seed, i])
        params = draw_gaussians(sub, G, sh_degree, means=blob_means(sub, G, n_blobs=16))
        cams = hemisphere_cameras(nv, 3.0, width, height)
        out.append((t, Scene(G, sh_degree, params, cams, int(seed) * 1000 + i)))
    return out


def perturb_appearance(rng, params, n_gauss, sh_degree, sh_sigma=0.1, opacity_sigma=0.3):
    """Start of a serving fit: SH coefficients + N(0, sh_sigma) and opacity
    logits + N(0, opacity_sigma); geometry unchanged."""
    off = group_offsets(n_gauss, sh_degree)
    p = params.astype(np.float64).copy()
    p[off["opacity"]:off["sh"]] += rng.normal(0.0, opacity_sigma, n_gauss)
    p[off["sh"]:off["end"]] += rng.normal(0.0, sh_sigma, off["end"] - off["sh"])
    return p.astype(np.float32)


def view_subset(rng, n_cams, n_views):
    """Views of one LM step: uniform without replacement."""
    return np.sort(rng.choice(n_cams, size=n_views, replace=False)).astype(np.int32)
