"""Dense 2D PSFs (odd sides 3..25, at least half the taps non-zero): the
register-blocked dense tile bodies against the FP64 oracle on ragged shapes,
for every tap-table width they are compiled for; PSFs of the same shapes
with mostly zero taps keep the tap-group bodies; and the batched kernel
gives the single-image bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu

MAX_ABS, RMS = 1e-3, 1e-4


@pytest.fixture(autouse=True)
def _no_fft_tiles(lib):
    """These tests cover the direct-sum bodies: FFT tiles off."""
    lib.set_fft_tiles(2305)
    yield
    lib.set_fft_tiles(0)


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def _case(H, W, h, seed):
    rng = np.random.default_rng(seed)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng, salt_pepper=0.01)
    u0 = np.maximum(f, 0.1).astype(np.float32)
    return f, u0


def _dense_psf(kh, kw, rng):
    h = rng.uniform(0.05, 1.0, size=(kh, kw))
    h[kh // 2, kw // 2] += 1.0
    return (h / h.sum()).astype(np.float32)


def _check(u, ref, what):
    d = (u.double().cpu() - torch.as_tensor(ref)).abs()
    m, r = float(d.max()), float(d.pow(2).mean().sqrt())
    assert m <= MAX_ABS and r <= RMS, f"{what}: max-abs {m:.3e} rms {r:.3e}"


@pytest.mark.parametrize("kh,kw", [(3, 3), (5, 7), (7, 5), (9, 9), (11, 13), (13, 11), (15, 15), (17, 19),
                                   (19, 17), (21, 23), (23, 21), (25, 25), (25, 3), (3, 25)])
@pytest.mark.parametrize("H,W", [(77, 131), (64, 96), (33, 40)])
def test_dense_bodies_match_oracle(lib, kh, kw, H, W):
    if kh > H or kw > W:
        pytest.skip("PSF larger than image")
    rng = np.random.default_rng(kh * 100 + kw)
    h = _dense_psf(kh, kw, rng)
    p = Params()
    f, u0 = _case(H, W, h, H + W)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
    _check(u, ref, f"{kh}x{kw} on {H}x{W}")


def test_mostly_zero_taps_of_an_eligible_shape_keep_tap_groups(lib):
    """A 15x15 diagonal line PSF (few non-zero taps) and a 9x9 PSF with 40 of
    81 taps non-zero: both against the oracle."""
    rng = np.random.default_rng(3)
    line = np.zeros((15, 15))
    for t in range(15):           # a diagonal line: 15 of 225 taps
        line[t, t] = 1.0 + t % 3
    line /= line.sum()
    sparse = _dense_psf(9, 9, rng)
    sparse.flat[:42] = 0.0        # with the centre below: 40 of 81 non-zero
    sparse[4, 4] = 0.5
    for h in (line.astype(np.float32), (sparse / sparse.sum()).astype(np.float32)):
        H, W = 90, 120
        p = Params()
        f, u0 = _case(H, W, h, 9)
        ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
        u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
        _check(u, ref, f"sparse {h.shape}")


def test_dense_batch_equals_single_images_and_oracle(lib):
    """Batched images with dense PSFs of several widths (tiles of 32 x 64)
    equal the single-image split schedule (tiles of 32 x 32) bit for bit."""
    rng = np.random.default_rng(11)
    shapes = [(150, 200, 25), (97, 131, 7), (64, 64, 13), (128, 300, 19), (201, 77, 3)]
    fs, hs, ps, cases = [], [], [], []
    for H, W, k in shapes:
        h = _dense_psf(k, k, rng)
        f, _ = _case(H, W, h, H * W)
        fs.append(cuda(f)); hs.append(cuda(h)); ps.append(Params(K=0.006)); cases.append((f, h))
    outs = lib.deblur_batch(fs, hs, ps, 5)
    for (f, h), fd, hd, u in zip(cases, fs, hs, outs):
        assert torch.equal(u, lib.deblur(fd, hd, Params(K=0.006), 5)), h.shape
    f, h = cases[0]
    _, ref = oracle.wr3l(f, h, Params(K=0.006), 5)
    _check(outs[0], ref, "batched 25x25")
