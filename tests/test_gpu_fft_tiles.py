"""FFT tiles: the spatial iteration's blur and correlations of 2D PSFs as
64 x 64 circular convolutions of constant-continuation windows (Sec. 4.2
"Fourier transform"; the general 2D variant of Sec. 4.3).  Against the FP64
oracle's direct sums on ragged shapes, odd and even PSF sides up to 48,
images smaller than one window, dense and sparse PSFs; and the batched
kernel and the N-image launches give the single-image bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu

MAX_ABS, RMS = 1e-3, 1e-4


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


@pytest.fixture
def fft_all(lib):
    """FFT tiles for every PSF of their shape range (sides 2..48)."""
    lib.set_fft_tiles(1)
    yield
    lib.set_fft_tiles(0)


def _case(H, W, h, seed, salt_pepper=0.01):
    rng = np.random.default_rng(seed)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng, salt_pepper=salt_pepper)
    u0 = np.maximum(f, 0.1).astype(np.float32)
    return f, u0


def _psf(kh, kw, rng, sparse=False):
    h = rng.uniform(0.05, 1.0, size=(kh, kw))
    if sparse:
        h *= rng.random((kh, kw)) < 0.2
    h[kh // 2, kw // 2] += 1.0
    return (h / h.sum()).astype(np.float32)


def _check(u, ref, what):
    d = (u.double().cpu() - torch.as_tensor(ref)).abs()
    m, r = float(d.max()), float(d.pow(2).mean().sqrt())
    assert m <= MAX_ABS and r <= RMS, f"{what}: max-abs {m:.3e} rms {r:.3e}"
    return m, r


@pytest.mark.parametrize("H,W,kh,kw", [
    (77, 131, 9, 9),      # several tiles and pairs, ragged in both directions
    (64, 64, 25, 25),     # image = one window; 40 x 40 outputs per tile
    (33, 40, 15, 15),     # image smaller than a window
    (130, 300, 31, 17),   # not dense-eligible (side 31)
    (200, 150, 4, 6),     # even sides: the window offsets differ for blur and correlation
    (97, 201, 48, 2),     # the largest height: 17-row tiles
    (65, 129, 2, 48),     # the largest width: 17-column tiles, odd pair count
    (129, 67, 21, 23),
])
def test_fft_tiles_match_oracle(lib, fft_all, H, W, kh, kw):
    rng = np.random.default_rng(kh * 100 + kw)
    h = _psf(kh, kw, rng)
    p = Params()
    f, u0 = _case(H, W, h, H + W)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
    _check(u, ref, f"{kh}x{kw} on {H}x{W}")


def test_fft_tiles_sparse_and_line_psfs(lib, fft_all):
    """A 30-degree line PSF (17 x 27, 71 taps) and a random sparse 19 x 13
    PSF: the transform does not care about zero taps."""
    rng = np.random.default_rng(5)
    for h in (synth.line_psf(31, 30.0, 32.0), _psf(19, 13, rng, sparse=True)):
        H, W = 150, 170
        p = Params()
        f, u0 = _case(H, W, h, 17)
        ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 5)
        u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 5)
        _check(u, ref, f"sparse {h.shape}")


def test_fft_tiles_parameter_variants(lib, fft_all):
    """Phi' = 1 (plain data term), linear diffusion, and no regulariser."""
    rng = np.random.default_rng(8)
    h = _psf(11, 11, rng)
    H, W = 90, 110
    f, u0 = _case(H, W, h, 3)
    for kw in (dict(phi_robust=0), dict(psi_tv=0, alpha=0.001), dict(alpha=0.0)):
        p = Params(**kw)
        ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
        u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
        _check(u, ref, str(kw))


def test_fft_tiles_full_pipeline_and_plan(lib, fft_all):
    """Wiener + 6 RRRL iterations on a 2D Gaussian mixture, through
    db_deblur and through a plan (bit for bit)."""
    rng = np.random.default_rng(21)
    h = synth.gaussian_mixture_psf(17, rng).astype(np.float32)
    H, W = 160, 224
    p = Params(K=0.006)
    f, _ = _case(H, W, h, 4, salt_pepper=0.0)
    _, ref = oracle.wr3l(f, h, p, 6)
    fd, hd = cuda(f), cuda(h)
    u = lib.deblur(fd, hd, p, 6)
    _check(u, ref, "wr3l 17x17")
    plan = lib.Plan(H, W, hd, p, 6)
    assert torch.equal(plan.run(fd), u)


def test_fft_tiles_batch_equals_single_images(lib, fft_all):
    """A batch mixing FFT-tile images (2D PSFs of several sizes, odd pair
    counts), a one-axis image and a small 2D PSF equals the single-image
    pipeline bit for bit; one FFT image also against the oracle."""
    rng = np.random.default_rng(12)
    shapes = [(150, 200, 25, 25), (97, 131, 7, 9), (64, 64, 13, 13), (128, 300, 19, 4), (201, 77, 3, 3),
              (90, 70, 1, 15)]
    fs, hs, ps, cases = [], [], [], []
    for H, W, kh, kw in shapes:
        h = _psf(kh, kw, rng)
        f, _ = _case(H, W, h, H * W)
        fs.append(cuda(f)); hs.append(cuda(h)); ps.append(Params(K=0.006)); cases.append((f, h))
    outs = lib.deblur_batch(fs, hs, ps, 5)
    for (f, h), fd, hd, u in zip(cases, fs, hs, outs):
        assert torch.equal(u, lib.deblur(fd, hd, Params(K=0.006), 5)), h.shape
    f, h = cases[0]
    _, ref = oracle.wr3l(f, h, Params(K=0.006), 5)
    _check(outs[0], ref, "batched 25x25")


def test_fft_tiles_n_images_equal_single(lib, fft_all):
    """db_deblur_n: the FFT-tile launches over all images (gridDim.z) give
    each image's single-call bits."""
    rng = np.random.default_rng(13)
    h = _psf(15, 15, rng)
    H, W, n = 100, 140, 3
    fs = np.stack([_case(H, W, h, 40 + k)[0] for k in range(n)])
    p = Params(K=0.006)
    out = lib.deblur_n(cuda(fs), cuda(h), p, 4)
    for k in range(n):
        assert torch.equal(out[k], lib.deblur(cuda(fs[k]), cuda(h), p, 4)), k


def test_fft_tiles_checkpoints(lib, fft_all):
    """Checkpointed iterations (the split schedule writes the iterates) give
    the same final iterate as an uncheckpointed run."""
    rng = np.random.default_rng(14)
    h = _psf(9, 11, rng)
    H, W = 80, 96
    f, u0 = _case(H, W, h, 6)
    p = Params()
    a = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6)
    ck = torch.empty((3, H, W), device="cuda")
    b = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6, ckpt=ck, ckpt_every=2)
    assert torch.equal(a, b)
    assert torch.equal(ck[0], cuda(u0))


@pytest.mark.parametrize("H,W,kh,kw", [
    (77, 132, 9, 9),      # ragged rows, TMA windows over every edge
    (36, 40, 15, 15),     # image smaller than a window: clamped on all four sides
    (97, 200, 48, 2),     # the largest height
    (68, 128, 2, 48),     # the largest width: the box's widest reach (130 of 136 columns)
    (300, 516, 25, 24),   # many interior tiles, even width of the PSF
    (77, 131, 9, 9),      # row stride not a multiple of 4: element-wise loads on the caller's buffer
])
def test_fft_tiles_tma_equals_elementwise(lib, fft_all, H, W, kh, kw):
    """The q phase's windows staged by one TMA tensor copy (with the
    constant continuation applied in shared memory) give the bits of the
    element-wise clamped loads."""
    rng = np.random.default_rng(kh * 7 + kw)
    h = _psf(kh, kw, rng)
    p = Params()
    f, u0 = _case(H, W, h, H + 3 * W)
    outs = []
    try:
        for on in (True, False):
            lib.set_tma(on)
            outs.append(lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 3))
    finally:
        lib.set_tma(True)
    assert torch.equal(outs[0], outs[1])


def test_fft_tiles_tma_n_images(lib, fft_all):
    """db_deblur_n over three images: one 3D tensor map (image index as the
    third coordinate) gives each image's element-wise bits."""
    rng = np.random.default_rng(14)
    h = _psf(13, 17, rng)
    H, W, n = 90, 116, 3
    fs = np.stack([_case(H, W, h, 60 + k)[0] for k in range(n)])
    p = Params(K=0.006)
    outs = []
    try:
        for on in (True, False):
            lib.set_tma(on)
            outs.append(lib.deblur_n(cuda(fs), cuda(h), p, 4))
    finally:
        lib.set_tma(True)
    assert torch.equal(outs[0], outs[1])
