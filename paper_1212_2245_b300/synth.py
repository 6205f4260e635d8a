"""Seeded synthetic inputs shaped like the paper's deblurring workloads.

This module is the only code shared between the CUDA path's tests/benchmark and
the FP64 oracle.  It holds none of the deblurring method's arithmetic: it paints
sharp test scenes, builds point-spread functions and degrades the scenes with
the blur model of Sec. 2, Eq. (1) (f = g*h + n), using a library FFT
convolution on an edge-replicated image.  The blur uses constant continuation at
the boundary, as the paper does for its synthetic test images to avoid the
"inverse crime" (Sec. 3.1).

Scenes: a smooth linear gradient around grey 128 plus piecewise-constant
rectangles and discs with grey values in [20, 235], about 20 shapes per 256x256
area; noise is Gaussian plus optional salt-and-pepper outliers; values are
clipped to the grey range [0, 255] of the paper's 8-bit images.  The sharp
image, the observation and the PSF are returned as float32 arrays, so both
sides of a parity test consume bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.signal

from .params import Params

SEED_BASE = 12122245


def rng_for(config: int, index: int = 0) -> np.random.Generator:
    """Deterministic generator for image `index` of workload `config`."""
    return np.random.default_rng(SEED_BASE + 1000 * config + index)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
def scene(H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """Sharp grey image: linear gradient (+-20 around 128) plus shapes."""
    yy = (np.arange(H, dtype=np.float64)[:, None] / max(H - 1, 1)) * 2.0 - 1.0
    xx = (np.arange(W, dtype=np.float64)[None, :] / max(W - 1, 1)) * 2.0 - 1.0
    cx, cy = rng.uniform(-0.5, 0.5, size=2)
    g = 128.0 + 20.0 * (cx * xx + cy * yy)
    g = np.broadcast_to(g, (H, W)).copy()
    n_shapes = max(1, int(round(20.0 * H * W / 65536.0)))
    short = min(H, W)
    for s in range(n_shapes):
        size = rng.uniform(0.05, 0.30) * short
        ci, cj = rng.uniform(0, H), rng.uniform(0, W)
        grey = rng.uniform(20.0, 235.0)
        if s % 2 == 0:
            hh = 0.5 * size
            hw = 0.5 * size * rng.uniform(0.5, 1.5)
            i0, i1 = int(max(0, math.floor(ci - hh))), int(min(H, math.ceil(ci + hh)))
            j0, j1 = int(max(0, math.floor(cj - hw))), int(min(W, math.ceil(cj + hw)))
            g[i0:i1, j0:j1] = grey
        else:
            r = 0.5 * size
            i0, i1 = int(max(0, math.floor(ci - r))), int(min(H, math.ceil(ci + r) + 1))
            j0, j1 = int(max(0, math.floor(cj - r))), int(min(W, math.ceil(cj + r) + 1))
            if i0 >= i1 or j0 >= j1:
                continue
            ii = np.arange(i0, i1, dtype=np.float64)[:, None] + 0.5
            jj = np.arange(j0, j1, dtype=np.float64)[None, :] + 0.5
            inside = (ii - ci) ** 2 + (jj - cj) ** 2 <= r * r
            sub = g[i0:i1, j0:j1]
            sub[inside] = grey
    return g


# --------------------------------------------------------------------------
# point-spread functions (odd extents, centre tap at index (kh//2, kw//2),
# except even-length boxes whose centre is at index L//2)
# --------------------------------------------------------------------------
def _normalise(h: np.ndarray) -> np.ndarray:
    h = np.asarray(h, dtype=np.float64)
    return (h / h.sum()).astype(np.float32)


def box_psf(L: int, axis: str = "row") -> np.ndarray:
    """Uniform linear motion of integer length L along a coordinate axis."""
    h = np.full((1, L), 1.0 / L)
    return _normalise(h if axis == "row" else h.T)


def box_psf_frac(L: float, axis: str = "row") -> np.ndarray:
    """Uniform linear motion of non-integer length L, centred on the middle
    tap: each pixel's weight is the length of [-L/2, L/2] that falls inside
    it, so the two end pixels carry the fractional remainder."""
    half = 0.5 * float(L)
    K = int(np.ceil(half - 0.5))
    k = np.arange(-K, K + 1, dtype=np.float64)
    w = np.clip(np.minimum(k + 0.5, half) - np.maximum(k - 0.5, -half), 0.0, None)[None, :]
    return _normalise(w if axis == "row" else w.T)


def raised_cosine_1d(L: int, axis: str = "row", period: float | None = None) -> np.ndarray:
    """Non-uniform linear motion: taps 0.5*(1+cos(2*pi*t/P)), t centred."""
    P = float(L + 1) if period is None else float(period)
    t = np.arange(L, dtype=np.float64) - (L - 1) / 2.0
    h = (0.5 * (1.0 + np.cos(2.0 * np.pi * t / P)))[None, :]
    return _normalise(h if axis == "row" else h.T)


def random_motion_1d(L: int, rng: np.random.Generator, axis: str = "row", zeros: float = 0.15) -> np.ndarray:
    """Non-uniform linear motion along a coordinate axis with an irregular
    speed profile: L positive dwell weights U(0.05, 1), about `zeros` of the
    interior ones set to zero (the camera skipping pixels)."""
    w = rng.uniform(0.05, 1.0, L)
    if L > 2:
        w[1:-1][rng.random(L - 2) < zeros] = 0.0
    h = w[None, :]
    return _normalise(h if axis == "row" else h.T)


def line_psf(L: int = 31, angle_deg: float = 30.0, period: float = 32.0) -> np.ndarray:
    """Motion along a line at `angle_deg` (counter-clockwise from the +x axis,
    rows pointing down).  Samples t_j = j-(L-1)/2 of a raised-cosine profile
    are splatted bilinearly at (x, y) = (t cos a, -t sin a); the support is
    cropped symmetrically so the origin is the centre tap."""
    a = math.radians(angle_deg)
    t = np.arange(L, dtype=np.float64) - (L - 1) / 2.0
    w = 0.5 * (1.0 + np.cos(2.0 * np.pi * t / period))
    xs, ys = t * math.cos(a), -t * math.sin(a)
    R = int(math.ceil(max(np.abs(xs).max(), np.abs(ys).max()))) + 2
    grid = np.zeros((2 * R + 1, 2 * R + 1))
    for x, y, wt in zip(xs, ys, w):
        x0, y0 = math.floor(x), math.floor(y)
        fx, fy = x - x0, y - y0
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                grid[R + y0 + dy, R + x0 + dx] += wt * wy * wx
    nz_r = np.nonzero(np.abs(grid).sum(axis=1) > 0)[0]
    nz_c = np.nonzero(np.abs(grid).sum(axis=0) > 0)[0]
    ry = max(R - nz_r.min(), nz_r.max() - R)
    rx = max(R - nz_c.min(), nz_c.max() - R)
    return _normalise(grid[R - ry:R + ry + 1, R - rx:R + rx + 1])


def gaussian_mixture_psf(S: int, rng: np.random.Generator, n_comp: int = 3,
                         scale: float | None = None) -> np.ndarray:
    """S x S (S odd) sum of anisotropic Gaussians sampled at pixel centres.
    For S = 31: sigma_major in [1.5, 5], sigma_minor in [0.7, sigma_major],
    orientation in [0, pi), mean offset in [-4, 4]^2, weight in [0.5, 1];
    smaller windows scale sigmas and offsets by S/31."""
    assert S % 2 == 1
    sc = (S / 31.0) if scale is None else scale
    r = S // 2
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1].astype(np.float64)
    h = np.zeros((S, S))
    for _ in range(n_comp):
        smaj = rng.uniform(1.5, 5.0) * sc
        smin = rng.uniform(0.7 * sc, smaj)
        th = rng.uniform(0.0, math.pi)
        my, mx = rng.uniform(-4.0, 4.0, size=2) * sc
        wt = rng.uniform(0.5, 1.0)
        c, s = math.cos(th), math.sin(th)
        dx, dy = xx - mx, yy - my
        p = c * dx + s * dy
        q = -s * dx + c * dy
        h += wt * np.exp(-0.5 * ((p / smaj) ** 2 + (q / smin) ** 2))
    return _normalise(h)


# --------------------------------------------------------------------------
# degradation (Eq. 1): f = clip(g*h + n), constant continuation at borders
# --------------------------------------------------------------------------
def blur_replicate(g: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Spatial blur of g by h with edge replication, via a library FFT
    convolution of the padded image ('valid' part)."""
    kh, kw = h.shape
    cy, cx = kh // 2, kw // 2
    gp = np.pad(g.astype(np.float64), ((kh - 1 - cy, cy), (kw - 1 - cx, cx)), mode="edge")
    return scipy.signal.fftconvolve(gp, h.astype(np.float64), mode="valid")


def degrade(g: np.ndarray, h: np.ndarray, sigma: float, rng: np.random.Generator,
            salt_pepper: float = 0.0) -> np.ndarray:
    f = blur_replicate(g, h)
    if sigma > 0:
        f = f + rng.normal(0.0, sigma, size=f.shape)
    if salt_pepper > 0:
        hit = rng.random(f.shape) < salt_pepper
        salt = rng.random(f.shape) < 0.5
        f = np.where(hit, np.where(salt, 255.0, 0.0), f)
    return np.clip(f, 0.0, 255.0).astype(np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass
class Case:
    name: str
    g: np.ndarray             # sharp image, float32 (H, W)
    f: np.ndarray             # observed image, float32 (H, W)
    h: np.ndarray             # PSF taps, float32 (kh, kw)
    iters: int
    params: Params
    psf_kind: str = "general"  # "box_row", "box_col" or "general"
    extra: dict = field(default_factory=dict)


def case_box256(H: int = 256, W: int = 256, iters: int = 10) -> Case:
    """256x256, uniform horizontal motion L=15, sigma=2, Wiener K=0.006,
    10 RRRL iterations, TV, alpha=0.003."""
    rng = rng_for(0)
    g = scene(H, W, rng).astype(np.float32)
    h = box_psf(15, "row")
    f = degrade(g, h, 2.0, rng)
    return Case("box256", g, f, h, iters, Params(K=0.006), psf_kind="box_row")


def case_line1024(H: int = 1024, W: int = 1024, iters: int = 20) -> Case:
    """1024x1024, 30-degree line PSF L=31 with raised-cosine taps, sigma=2
    plus 1% salt-and-pepper, Wiener K=0.01, 20 RRRL iterations."""
    rng = rng_for(1)
    g = scene(H, W, rng).astype(np.float32)
    h = line_psf(31, 30.0)
    f = degrade(g, h, 2.0, rng, salt_pepper=0.01)
    return Case("line1024", g, f, h, iters, Params(K=0.01))


def case_gauss2048(H: int = 2048, W: int = 2048, iters: int = 30) -> Case:
    """2048x2048, 31x31 mixture of 3 Gaussians, sigma=1, FFT Wiener K=0.006,
    30 RRRL iterations with periodic (Fourier) blur and correlation."""
    rng = rng_for(2)
    g = scene(H, W, rng).astype(np.float32)
    h = gaussian_mixture_psf(31, rng)
    f = degrade(g, h, 1.0, rng)
    return Case("gauss2048", g, f, h, iters, Params(K=0.006, conv="periodic"))


def case_gauss3072(H: int = 3072, W: int = 3072, iters: int = 10) -> Case:
    """3072x3072, 25x25 mixture of 3 Gaussians (the largest PSF of the
    batch), sigma=2, Wiener K=0.006, 10 RRRL iterations with constant
    continuation (spatial: the FFT tiles' workload)."""
    rng = rng_for(5)
    g = scene(H, W, rng).astype(np.float32)
    h = gaussian_mixture_psf(25, rng)
    f = degrade(g, h, 2.0, rng)
    return Case("gauss3072", g, f, h, iters, Params(K=0.006))


def batch_case(index: int, size_cap: int = 1024) -> Case:
    """Image `index` (0..511) of the uneven batch: sides U{128..1024};
    images 0-255 carry axis-aligned 1D motion of length U{5..41} (even
    index: box, odd: raised cosine; direction random), images 256-511 an
    S x S Gaussian mixture, S odd in 7..25.  sigma=2, K=0.006, 10 iters."""
    rng = rng_for(3, index)
    H = int(rng.integers(128, size_cap + 1))
    W = int(rng.integers(128, size_cap + 1))
    g = scene(H, W, rng).astype(np.float32)
    if index < 256:
        L = int(rng.integers(5, 42))
        axis = "row" if rng.random() < 0.5 else "col"
        if index % 2 == 0:
            h, kind = box_psf(L, axis), "box_" + axis
        else:
            h, kind = raised_cosine_1d(L, axis), "general"
    else:
        S = int(rng.choice(np.arange(7, 26, 2)))
        h, kind = gaussian_mixture_psf(S, rng), "general"
    f = degrade(g, h, 2.0, rng)
    return Case(f"batch{index}", g, f, h, 10, Params(K=0.006), psf_kind=kind)


def case_learn512(n_images: int = 64, H: int = 512, W: int = 512, iters: int = 15) -> Case:
    """Batch of 512x512 images blurred horizontally (true PSF: 15-tap box in a
    21-tap window); the learnable PSF starts as a 21-tap raised cosine,
    alpha=0.003, K=0.006; 15 RRRL iterations; loss = MSE to the sharp image."""
    gs, fs = [], []
    true_h = np.zeros((1, 21), dtype=np.float64)
    true_h[0, 3:18] = 1.0 / 15.0
    true_h = _normalise(true_h)
    for n in range(n_images):
        rng = rng_for(4, n)
        g = scene(H, W, rng).astype(np.float32)
        gs.append(g)
        fs.append(degrade(g, true_h, 2.0, rng))
    h0 = raised_cosine_1d(21, "row")
    return Case("learn512", np.stack(gs), np.stack(fs), h0, iters, Params(K=0.006),
                extra={"true_h": true_h})
