"""Seeded synthetic stereo pairs (stand-ins for the Middlebury pairs of the paper's
experiments, which are not available here).

This module holds no part of the matching method: it only draws inputs.  Both the
CUDA path and the CPU oracle consume the arrays it returns, so every random number is
produced here once.

Determinism: every random draw comes from a counter-based SplitMix64 stream
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
``z = seed + (i + 1) * 0x9E3779B97F4A7C15`` followed by the published finaliser.
Blurs, stretches, warps and noise are integer arithmetic (plus IEEE float64
add/multiply for the plane equations), so x86-64 and aarch64 produce identical bytes.

Recipe for one pair (W x H, D labels, K planes, noise sigma):
  * texture: uniform bytes blurred twice with the binomial kernel C(8, k)/256
    (sigma = sqrt(2) px per pass), replicate borders, stretched to [0, 255];
  * disparity: K Voronoi cells around uniform seed points; cell k carries the plane
    d = a_k + b_k (x - sx_k) + c_k (y - sy_k) with a_k ~ U[0.1 D, 0.9 D] and
    |b_k|, |c_k| <= 0.3 D / W, clamped to [0, D - 1] and rounded to integers;
  * right view: the left texture forward-warped to x - d(x, y) with a z-buffer that
    keeps the largest disparity (the nearest surface); right pixels nobody hits are
    filled from a second, independent texture (occlusion holes);
  * noise: approximately Gaussian, sigma * (sum of 12 uniforms - 6) rounded to an
    integer, added to the right view and clamped to [0, 255];
  * occlusion mask: left pixels whose warp target falls outside the image or was taken
    by a nearer surface.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers: one independent SplitMix64 stream per purpose
_S_TEX, _S_FILL, _S_SEEDS, _S_PLANES, _S_NOISE = 1, 2, 3, 4, 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n uint64 draws of the counter-based SplitMix64 stream (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 1_000_003 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64)
        return _mix(key + ctr * _GAMMA)


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n float64 uniforms in [0, 1): the top 53 bits of each draw times 2**-53."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


_BINOM8 = np.array([1, 8, 28, 56, 70, 56, 28, 8, 1], dtype=np.int64)


def _blur_binomial(img: np.ndarray) -> np.ndarray:
    """Separable binomial blur, sum of weights 256 per axis, replicate borders, floor division."""
    r = 4
    out = img.astype(np.int64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="edge")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for k, w in enumerate(_BINOM8):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(k, k + n)
            acc += w * p[tuple(sl)]
        out = acc // 256
    return out


def texture(seed: int, stream: int, W: int, H: int) -> np.ndarray:
    """Smoothed-noise texture, uint8 [H][W], stretched to the full [0, 255] range."""
    raw = (splitmix64(seed, stream, W * H) >> np.uint64(56)).astype(np.int64).reshape(H, W)
    t = _blur_binomial(_blur_binomial(raw))
    lo, hi = int(t.min()), int(t.max())
    if hi == lo:
        return np.full((H, W), 128, dtype=np.uint8)
    return ((t - lo) * 255 // (hi - lo)).astype(np.uint8)


@dataclass
class StereoPair:
    left: np.ndarray       # uint8 [H][W]
    right: np.ndarray      # uint8 [H][W]
    disparity: np.ndarray  # int32 [H][W], ground-truth disparity of the left view
    occluded: np.ndarray   # bool [H][W], left pixels with no visible match
    D: int
    seed: int


def disparity_planes(seed: int, W: int, H: int, D: int, planes: int) -> np.ndarray:
    """Piecewise-planar integer disparity map, int32 [H][W], values in [0, D - 1]."""
    u = uniform01(seed, _S_SEEDS, 2 * planes)
    sx = np.floor(u[0::2] * W).astype(np.int64)
    sy = np.floor(u[1::2] * H).astype(np.int64)
    v = uniform01(seed, _S_PLANES, 3 * planes)
    a = 0.1 * D + 0.8 * D * v[0::3]
    slope = 0.3 * D / max(W, 1)
    b = (2.0 * v[1::3] - 1.0) * slope
    c = (2.0 * v[2::3] - 1.0) * slope
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs[None] - sx[:, None, None]) ** 2 + (ys[None] - sy[:, None, None]) ** 2
    cell = np.argmin(d2, axis=0)  # ties go to the lowest cell index
    d = a[cell] + b[cell] * (xs - sx[cell]) + c[cell] * (ys - sy[cell])
    d = np.clip(np.floor(d + 0.5), 0, D - 1)
    return d.astype(np.int32)


def make_pair(seed: int, W: int, H: int, D: int, planes: int = 3, sigma: float = 2.0) -> StereoPair:
    """One synthetic rectified pair; the left view is the reference (d >= 0 shifts left in R)."""
    if W < 1 or H < 1 or D < 1:
        raise ValueError("W, H and D must be >= 1")
    L = texture(seed, _S_TEX, W, H)
    fill = texture(seed, _S_FILL, W, H)
    disp = disparity_planes(seed, W, H, D, max(planes, 1))
    R = fill.astype(np.int64).copy()
    zbuf = np.full((H, W), -1, dtype=np.int64)
    occluded = np.zeros((H, W), dtype=bool)
    ys, xs = np.mgrid[0:H, 0:W]
    tx = xs - disp
    inside = tx >= 0
    occluded[~inside] = True
    # z-buffer: the largest disparity wins each target; among equals the largest source x
    yy, xx, tt, dd = ys[inside], xs[inside], tx[inside], disp[inside].astype(np.int64)
    key = dd * (W + 1) + xx
    order = np.lexsort((key, yy * W + tt))
    flat = (yy * W + tt)[order]
    last = np.ones(flat.shape[0], dtype=bool)
    last[:-1] = flat[1:] != flat[:-1]
    win = order[last]
    R.reshape(-1)[flat[last]] = L[yy[win], xx[win]]
    zbuf.reshape(-1)[flat[last]] = key[win]
    lost = zbuf[yy, tt] != key
    occluded[yy[lost], xx[lost]] = True
    if sigma > 0:
        u = uniform01(seed, _S_NOISE, 12 * W * H).reshape(12, H, W)
        g = u.sum(axis=0) - 6.0
        R = R + np.floor(sigma * g + 0.5).astype(np.int64)
    R = np.clip(R, 0, 255).astype(np.uint8)
    return StereoPair(L, R, disp, occluded, D, seed)


# Workloads with the shapes of the paper's test pairs (section "Experimental Results"):
# name -> (W, H, D, window, planes, sigma, seed)
WORKLOADS = {
    "tiny_96x72_d16": (96, 72, 16, 5, 3, 2.0, 1),
    "tsukuba_384x288_d16": (384, 288, 16, 7, 8, 3.0, 2),
    "teddy_450x375_d64": (450, 375, 64, 7, 8, 3.0, 3),
    "hd_1920x1080_d256": (1920, 1080, 256, 9, 8, 3.0, 5),
    "qhd_960x540_d256": (960, 540, 256, 9, 8, 3.0, 6),  # a quarter of the HD pair, for profiling
    "c3_1280x720_d64": (1280, 720, 64, 7, 8, 3.0, 7),  # the largest pair size of the mixed batches
}


def workload_pair(name: str, seed_offset: int = 0) -> tuple[StereoPair, int]:
    W, H, D, window, planes, sigma, seed = WORKLOADS[name]
    return make_pair(seed + seed_offset, W, H, D, planes, sigma), window


def batch_specs(n: int, seed0: int = 1000) -> list[tuple[int, int, int, int]]:
    """(seed, W, H, D) of a mixed batch: W ~ U[320, 1280], H ~ U[240, 720], D ~ U{32, 64, 96, 128}."""
    out = []
    for k in range(n):
        u = uniform01(seed0 + k, 9, 3)
        W = 320 + int(u[0] * 961)
        H = 240 + int(u[1] * 481)
        D = (32, 64, 96, 128)[int(u[2] * 4)]
        out.append((seed0 + k, W, H, D))
    return out
