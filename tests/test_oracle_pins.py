"""Pins for the FP64 oracle: each test ties one oracle function to something
other than the oracle itself (brute force on tiny inputs, a library routine
for a special case, a closed form, or an invariant the paper's method has)."""
import cmath
import math

import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import oracle
from paper_1212_2245_b300 import synth
from oracle import ops

RNG = np.random.default_rng(7)


class P:
    def __init__(self, **kw):
        self.K = 0.006
        self.alpha = 0.003
        self.eps_phi = 1.0
        self.eps_psi = 1.0
        self.pos_floor = 0.1
        self.phi_robust = 1
        self.psi_tv = 1
        self.conv = "clamp"
        self.__dict__.update(kw)


def rand_img(H, W, lo=20.0, hi=235.0):
    return RNG.uniform(lo, hi, size=(H, W))


def rand_psf(kh, kw):
    h = RNG.uniform(0.05, 1.0, size=(kh, kw))
    return h / h.sum()


# --------------------------------------------------------------------------
# convolution conventions (Sec. 2, Eq. 1; h*(x) = h(-x))
# --------------------------------------------------------------------------
def test_delta_blurs_to_psf_and_correlation_flips():
    h = rand_psf(3, 5)  # asymmetric
    u = np.zeros((15, 15))
    u[7, 7] = 1.0
    b = oracle.conv_clamp(u, h).numpy()
    c = oracle.corr_clamp(u, h).numpy()
    np.testing.assert_allclose(b[6:9, 5:10], h, atol=0)
    np.testing.assert_allclose(c[6:9, 5:10], h[::-1, ::-1], atol=0)
    assert abs(b.sum() - 1) < 1e-14


def _brute_conv(u, h, sign, wrap):
    H, W = u.shape
    kh, kw = h.shape
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            s = 0.0
            for a in range(kh):
                for b in range(kw):
                    y = i - sign * (a - kh // 2)
                    x = j - sign * (b - kw // 2)
                    if wrap:
                        y, x = y % H, x % W
                    else:
                        y, x = min(max(y, 0), H - 1), min(max(x, 0), W - 1)
                    s += h[a, b] * u[y, x]
            out[i, j] = s
    return out


@pytest.mark.parametrize("shape,k", [((5, 7), (3, 5)), ((6, 4), (5, 3)), ((1, 9), (1, 7)), ((9, 1), (5, 1))])
def test_conv_corr_brute_force(shape, k):
    u, h = rand_img(*shape), rand_psf(*k)
    np.testing.assert_allclose(oracle.conv_clamp(u, h), _brute_conv(u, h, +1, False), rtol=1e-13)
    np.testing.assert_allclose(oracle.corr_clamp(u, h), _brute_conv(u, h, -1, False), rtol=1e-13)
    np.testing.assert_allclose(oracle.conv_periodic(u, h), _brute_conv(u, h, +1, True), rtol=1e-13)
    np.testing.assert_allclose(oracle.corr_periodic(u, h), _brute_conv(u, h, -1, True), rtol=1e-13)


def test_conv_matches_library_nearest_and_wrap():
    u, h = rand_img(40, 33), rand_psf(7, 9)
    np.testing.assert_allclose(oracle.conv_clamp(u, h), ndi.convolve(u, h, mode="nearest"), rtol=1e-12)
    np.testing.assert_allclose(oracle.corr_clamp(u, h), ndi.correlate(u, h, mode="nearest"), rtol=1e-12)
    np.testing.assert_allclose(oracle.conv_periodic(u, h), ndi.convolve(u, h, mode="wrap"), rtol=1e-12)
    np.testing.assert_allclose(ops.conv_fourier(u, h), ndi.convolve(u, h, mode="wrap"), rtol=1e-11)
    np.testing.assert_allclose(ops.corr_fourier(u, h), ndi.correlate(u, h, mode="wrap"), rtol=1e-11)


# --------------------------------------------------------------------------
# running-sum box filter (Sec. 4.3, uniform linear motion)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [1, 2, 3, 4, 7, 15, 16, 27, 41])
@pytest.mark.parametrize("W", [1, 2, 5, 17, 64])
def test_running_sum_equals_direct(L, W):
    u = rand_img(3, W)
    h = np.full((1, L), 1.0 / L)
    np.testing.assert_allclose(oracle.box_running_sum_rows(u, L), oracle.conv_clamp(u, h), rtol=1e-12)
    np.testing.assert_allclose(oracle.box_running_sum_rows(u, L, adjoint=True), oracle.corr_clamp(u, h), rtol=1e-12)
    uc = rand_img(W, 2)
    np.testing.assert_allclose(oracle.box_running_sum_cols(uc, L), oracle.conv_clamp(uc, h.T), rtol=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 9, 17, 41])
@pytest.mark.parametrize("W", [1, 5, 64])
def test_running_sum_with_light_ends_equals_direct(L, W):
    """Box with lighter end taps (non-integer blur length, Sec. 4.3): the
    sliding-window form equals the direct clamped sums with those taps, for
    convolution and correlation, along rows and columns."""
    rng = np.random.default_rng(L * 100 + W)
    u = rng.uniform(0, 255, (3, W))
    taps = np.full(L, 1.0)
    taps[0], taps[-1] = rng.uniform(0.05, 1.0, 2) if L > 1 else (0.7, 0.7)
    h = taps[None, :]
    np.testing.assert_allclose(oracle.box_ends_running_sum_rows(u, taps), oracle.conv_clamp(u, h), rtol=1e-12)
    np.testing.assert_allclose(oracle.box_ends_running_sum_rows(u, taps, adjoint=True), oracle.corr_clamp(u, h),
                               rtol=1e-12)
    uc = u.T.copy()
    np.testing.assert_allclose(oracle.box_ends_running_sum_cols(uc, taps), oracle.conv_clamp(uc, h.T), rtol=1e-12)


@pytest.mark.parametrize("L", [3.0, 4.5, 15.4, 26.9])
def test_fractional_box_taps(L):
    """The fractional box integrates a centred segment of length L over the
    pixels: weights sum to L before normalisation, interior pixels get 1, the
    two end pixels the same remainder, and an odd integer length gives a
    plain box."""
    h = synth.box_psf_frac(L)[0].astype(np.float64)
    raw = h * L
    assert abs(raw.sum() - L) < 1e-5
    assert np.allclose(raw[1:-1], 1.0, atol=1e-5)
    assert abs(raw[0] - raw[-1]) < 1e-6
    n_int = len(raw) - 2
    assert abs(2 * raw[0] - (L - n_int)) < 1e-5
    if float(L).is_integer() and int(L) % 2 == 1:
        assert np.allclose(raw, 1.0, atol=1e-6)



# --------------------------------------------------------------------------
# Wiener filter (Sec. 2.1, Eq. 2)
# --------------------------------------------------------------------------
def test_wiener_inverts_invertible_psf_without_noise():
    g = rand_img(16, 32)
    k1 = np.array([[0.2, 0.6, 0.2]])          # |h-hat| >= 0.2
    for h in (k1, k1.T, k1.T @ k1):
        f = oracle.conv_periodic(g, h)
        np.testing.assert_allclose(oracle.wiener(f, h, 1e-12), g, atol=1e-8)
    f = oracle.conv_periodic(g, k1)
    np.testing.assert_allclose(oracle.wiener_rows(f, k1, 1e-12), g, atol=1e-8)


@pytest.mark.parametrize("ky,kx", [(0, 0), (1, 3), (5, 2), (8, 16)])
def test_wiener_attenuation_closed_form(ky, kx):
    H, W, K = 16, 32, 0.05
    a, b = 0.25, 0.5
    h = np.outer([a, b, a], [a, b, a])
    yy, xx = np.mgrid[0:H, 0:W]
    g = np.cos(2 * np.pi * (ky * yy / H + kx * xx / W))
    hh = (b + 2 * a * math.cos(2 * math.pi * ky / H)) * (b + 2 * a * math.cos(2 * math.pi * kx / W))
    np.testing.assert_allclose(oracle.wiener(g, h, K), g * hh / (hh * hh + K), atol=1e-12)


def test_wiener_rows_equals_2d_for_one_row_psf():
    f = rand_img(12, 20)
    h = rand_psf(1, 7)
    np.testing.assert_allclose(oracle.wiener_rows(f, h, 0.01), oracle.wiener(f, h, 0.01), atol=1e-10)
    np.testing.assert_allclose(oracle.wiener_cols(f, h.T, 0.01), oracle.wiener(f, h.T, 0.01), atol=1e-10)


def _naive_dft2(x, sign):
    H, W = x.shape
    out = np.zeros((H, W), dtype=complex)
    for p in range(H):
        for q in range(W):
            s = 0j
            for i in range(H):
                for j in range(W):
                    s += x[i, j] * cmath.exp(sign * 2j * math.pi * (p * i / H + q * j / W))
            out[p, q] = s
    return out


def test_wiener_brute_force_dft():
    H, W, K = 5, 6, 0.02
    f = rand_img(H, W)
    h = rand_psf(3, 3)
    hp = np.zeros((H, W))
    for a in range(3):
        for b in range(3):
            hp[(a - 1) % H, (b - 1) % W] += h[a, b]
    F, Hh = _naive_dft2(f, -1), _naive_dft2(hp, -1)
    U = F * np.conj(Hh) / (np.abs(Hh) ** 2 + K)
    u = (_naive_dft2(U, +1) / (H * W)).real
    np.testing.assert_allclose(oracle.wiener(f, h, K), u, atol=1e-10)


# --------------------------------------------------------------------------
# information divergence (Eq. 7)
# --------------------------------------------------------------------------
def test_information_divergence_properties():
    f = RNG.uniform(0.1, 255, size=1000)
    s = RNG.uniform(0.1, 255, size=1000)
    r = oracle.info_divergence(s, f).numpy()
    assert np.all(r >= -1e-12)
    assert np.all(np.abs(oracle.info_divergence(f, f).numpy()) < 1e-12)
    # second-order behaviour near s = f: r ~ (s-f)^2 / (2 f)
    d = 1e-3 * f
    r2 = oracle.info_divergence(f + d, f).numpy()
    np.testing.assert_allclose(r2, d * d / (2 * f), rtol=2e-3)
    # scaling r_f(s) = f r_1(s/f)
    np.testing.assert_allclose(r, f * oracle.info_divergence(s / f, np.ones_like(f)).numpy(), rtol=1e-9, atol=1e-9)


def test_penaliser_derivatives():
    z = np.array([0.0, 1.0, 3.0, 99.0])
    np.testing.assert_allclose(oracle.phi_prime(z, 1.0), 1 / np.sqrt(z + 1), rtol=1e-15)
    assert float(oracle.phi_prime(0.0, 2.0)) == 1.0
    np.testing.assert_allclose(oracle.psi_prime(z, 0.5), 1 / np.sqrt(z + 0.25), rtol=1e-15)
    # d/dz sqrt(z + e^2) = 1 / (2 sqrt(z + e^2)): phi' is that derivative times 2e
    e = 1.7
    zz = 3.3
    num = (math.sqrt(zz + 1e-6 + e * e) - math.sqrt(zz - 1e-6 + e * e)) / 2e-6
    assert abs(float(oracle.phi_prime(zz, e)) - 2 * e * num) < 1e-8


# --------------------------------------------------------------------------
# diffusion term (Eq. 11, Sec. 4.1)
# --------------------------------------------------------------------------
def test_diffusion_invariants():
    u = rand_img(13, 17)
    D = oracle.diffusion(u, 1.0).numpy()
    assert abs(D.sum()) < 1e-10                      # zero flux: telescoping
    assert np.abs(oracle.diffusion(np.full((9, 8), 42.0), 1.0).numpy()).max() == 0.0
    # psi' == 1: 5-point Laplacian with reflecting (Neumann) boundary
    np.testing.assert_allclose(oracle.diffusion(u, 1.0, tv=False), ndi.laplace(u, mode="nearest"), atol=1e-11)


def _brute_diffusion(u, eps):
    H, W = u.shape
    U = lambda i, j: u[min(max(i, 0), H - 1), min(max(j, 0), W - 1)]  # noqa: E731

    def g(i, j):
        gx = (U(i, j + 1) - U(i, j - 1)) / 2
        gy = (U(i + 1, j) - U(i - 1, j)) / 2
        return 1 / math.sqrt(gx * gx + gy * gy + eps * eps)

    D = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            s = 0.0
            for (di, dj) in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                ii, jj = i + di, j + dj
                if 0 <= ii < H and 0 <= jj < W:
                    s += 0.5 * (g(ii, jj) + g(i, j)) * (u[ii, jj] - u[i, j])
            D[i, j] = s
    return D


def test_diffusion_brute_force_tv():
    u = rand_img(6, 9)
    np.testing.assert_allclose(oracle.diffusion(u, 0.7), _brute_diffusion(u, 0.7), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# RRRL iteration (Eq. 9-12)
# --------------------------------------------------------------------------
def test_rrrl_reduces_to_richardson_lucy():
    u, f, h = rand_img(20, 24), rand_img(20, 24), rand_psf(3, 5)
    p = P(alpha=0.0, phi_robust=0)
    rl = u * ndi.correlate(f / ndi.convolve(u, h, mode="nearest"), h, mode="nearest")
    np.testing.assert_allclose(oracle.rrrl_step(u, f, h, p), rl, rtol=1e-12)


def test_identity_psf_alpha0_fixed_point_is_f():
    u, f = rand_img(10, 11), rand_img(10, 11)
    for robust in (0, 1):
        out = oracle.rrrl_step(u, f, np.ones((1, 1)), P(alpha=0.0, phi_robust=robust))
        np.testing.assert_allclose(out, f, rtol=1e-13)
        np.testing.assert_allclose(oracle.rrrl_step(f, f, np.ones((1, 1)), P(alpha=0.0)), f, rtol=1e-13)


def test_constant_image_is_fixed_point():
    c = np.full((12, 10), 77.0)
    h = rand_psf(5, 3)
    for conv in ("clamp", "periodic"):
        out = oracle.rrrl_step(c, c, h, P(alpha=0.003, conv=conv))
        np.testing.assert_allclose(out, c, rtol=1e-13)


def test_rl_flux_conservation_and_positivity_periodic():
    f = rand_img(16, 16, 0.5, 255)
    u = rand_img(16, 16, 0.5, 255)
    h = rand_psf(3, 5)
    p = P(alpha=0.0, phi_robust=0, conv="periodic")
    for _ in range(4):
        u = oracle.rrrl_step(u, f, h, p)
        assert float(u.min()) > 0
        assert abs(float(u.sum()) - f.sum()) < 1e-9 * f.sum()


# --------------------------------------------------------------------------
# whole pipeline on a tiny case, against an independent naive implementation
# --------------------------------------------------------------------------
def _naive_pipeline(f, h, K, alpha, eps_phi, eps_psi, delta, iters):
    H, W = f.shape
    kh, kw = h.shape
    f = np.maximum(f, delta)
    hp = np.zeros((H, W))
    for a in range(kh):
        for b in range(kw):
            hp[(a - kh // 2) % H, (b - kw // 2) % W] += h[a, b]
    F, Hh = _naive_dft2(f, -1), _naive_dft2(hp, -1)
    u = (_naive_dft2(F * np.conj(Hh) / (np.abs(Hh) ** 2 + K), +1) / (H * W)).real
    u = np.maximum(u, delta)
    for _ in range(iters):
        b = _brute_conv(u, h, +1, False)
        Wt = np.zeros((H, W))
        for i in range(H):
            for j in range(W):
                r = b[i, j] - f[i, j] - f[i, j] * math.log(b[i, j] / f[i, j])
                Wt[i, j] = eps_phi / math.sqrt(r + eps_phi ** 2)
        A = _brute_conv(Wt * f / b, h, -1, False)
        B = _brute_conv(Wt, h, -1, False)
        D = _brute_diffusion(u, eps_psi)
        new = np.zeros((H, W))
        for i in range(H):
            for j in range(W):
                d = D[i, j]
                new[i, j] = u[i, j] * (A[i, j] + alpha * max(d, 0.0)) / (B[i, j] - alpha * min(d, 0.0))
        u = new
    return u


@pytest.mark.parametrize("kshape", [(3, 3), (1, 5), (3, 1)])
def test_tiny_pipeline_brute_force(kshape):
    H, W = 8, 8
    f = rand_img(H, W, 0.0, 255.0)
    f[2, 3] = 0.0                                  # a pepper pixel: positivity floor
    h = rand_psf(*kshape)
    p = P(K=0.01, alpha=0.05)                      # large alpha: regulariser matters
    u0, u = oracle.wr3l(f, h, p, 3)
    ref = _naive_pipeline(f, h, p.K, p.alpha, p.eps_phi, p.eps_psi, p.pos_floor, 3)
    np.testing.assert_allclose(u, ref, rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("kshape", [(1, 5), (3, 3), (3, 1)])
@pytest.mark.parametrize("grad", [False, True])
def test_loss_forward_equals_naive_pipeline(kshape, grad):
    """The loss of the tuning workload (mean square error of WR3L against the
    sharp image) equals the same mean taken over the independent naive
    pipeline's outputs, with and without gradients on the taps, alpha and K
    (the gradient path keeps zero taps and goes through the same Wiener
    functions)."""
    N, H, W, iters = 2, 8, 8, 3
    fs = np.stack([rand_img(H, W, 0.0, 255.0) for _ in range(N)])
    fs[1, 5, 2] = 0.0
    gs = np.stack([rand_img(H, W) for _ in range(N)])
    h = rand_psf(*kshape)
    h.flat[0] = 0.0                                 # a zero tap
    p = P(K=0.01, alpha=0.05)
    ref = np.mean([(_naive_pipeline(fs[n], h, p.K, p.alpha, p.eps_phi, p.eps_psi, p.pos_floor, iters) - gs[n]) ** 2
                   for n in range(N)])
    hT = torch.tensor(h, dtype=torch.float64, requires_grad=grad)
    aT = torch.tensor(p.alpha, dtype=torch.float64, requires_grad=grad)
    kT = torch.tensor(p.K, dtype=torch.float64, requires_grad=grad)
    loss = oracle.wr3l_loss(torch.tensor(fs, dtype=torch.float64), gs, hT, aT, kT, p, iters)
    assert abs(float(loss) - ref) <= 1e-11 * ref


# --------------------------------------------------------------------------
# FP64 reverse mode (autograd through the oracle) against central differences
# --------------------------------------------------------------------------
def test_reverse_mode_matches_central_differences():
    N, H, W, iters = 2, 8, 12, 3
    g = rand_img(H, W)
    fs = np.stack([oracle.conv_clamp(rand_img(H, W), rand_psf(1, 5)).numpy() for _ in range(N)])
    gs = np.stack([g, g[::-1].copy()])
    h0 = torch.tensor(rand_psf(1, 5), dtype=torch.float64, requires_grad=True)
    al = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
    K = torch.tensor(0.01, dtype=torch.float64, requires_grad=True)
    fT = torch.tensor(fs, dtype=torch.float64, requires_grad=True)
    p = P()
    loss = oracle.wr3l_loss(fT, gs, h0, al, K, p, iters)
    loss.backward()

    def L(hv, av, kv, fv):
        with torch.no_grad():
            return float(oracle.wr3l_loss(fv, gs, hv, av, kv, p, iters))

    e = 1e-6
    for t in range(5):
        hp_, hm_ = h0.detach().clone(), h0.detach().clone()
        hp_[0, t] += e
        hm_[0, t] -= e
        fd = (L(hp_, al.detach(), K.detach(), fT.detach()) - L(hm_, al.detach(), K.detach(), fT.detach())) / (2 * e)
        assert abs(fd - float(h0.grad[0, t])) <= 1e-5 * max(1.0, abs(fd))
    fd = (L(h0.detach(), al.detach() + e, K.detach(), fT.detach()) - L(h0.detach(), al.detach() - e, K.detach(), fT.detach())) / (2 * e)
    assert abs(fd - float(al.grad)) <= 1e-5 * max(1.0, abs(fd))
    fd = (L(h0.detach(), al.detach(), K.detach() + e, fT.detach()) - L(h0.detach(), al.detach(), K.detach() - e, fT.detach())) / (2 * e)
    assert abs(fd - float(K.grad)) <= 1e-5 * max(1.0, abs(fd))
    for (n, i, j) in ((0, 0, 0), (1, 4, 7), (0, 7, 11)):
        fp_, fm_ = fT.detach().clone(), fT.detach().clone()
        fp_[n, i, j] += 1e-4
        fm_[n, i, j] -= 1e-4
        fd = (L(h0.detach(), al.detach(), K.detach(), fp_) - L(h0.detach(), al.detach(), K.detach(), fm_)) / 2e-4
        assert abs(fd - float(fT.grad[n, i, j])) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_snr_closed_forms():
    """SNR(u, u0) = 10 log10(var u / var(u - u0)) (Sec. 3.1) on patterns with
    known variances: u = 2x with x = +-1 checkerboard gives 10 log10 4; u = x +
    0.1 y with y = +-1 in stripes (orthogonal, zero mean) gives 10 log10 101."""
    i, j = np.indices((8, 8))
    x = np.where((i + j) % 2 == 0, 1.0, -1.0)
    y = np.where(i % 2 == 0, 1.0, -1.0)
    assert abs(oracle.snr_db(2 * x, x) - 10 * math.log10(4.0)) < 1e-12
    assert abs(oracle.snr_db(x + 0.1 * y, x) - 10 * math.log10(101.0)) < 1e-9
    # the library's helper computes the same quantity
    from paper_1212_2245_b300 import quality
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(20, 30)), rng.normal(size=(20, 30))
    assert abs(quality.snr_db(a + b, a) - oracle.snr_db(a + b, a)) < 1e-12



def test_r1_lookup_table_pins():
    """Table evaluation of r_1 (Sec. 4.1): exact at the grid points, within
    the linear-interpolation bound h^2/8 max r_1'' = h^2/(8 s_j^2) between
    them, the closed form below the first entry, and beyond 65 the tangent
    line (value and slope r_1'(65) = 1 - 1/65 continuous at 65)."""
    h = oracle.RF_LUT_SMAX / oracle.RF_LUT_N
    grid = torch.tensor([h, 2 * h, 0.5, 1.0, 7.3125, 64.0, 65.0], dtype=torch.float64)
    grid = torch.round(grid / h) * h
    assert torch.allclose(oracle.r1_lut(grid), oracle.r1(grid), rtol=1e-12, atol=1e-15)
    x = torch.rand(20000, dtype=torch.float64, generator=torch.Generator().manual_seed(1)) * (65 - h) + h
    sj = torch.floor(x / h) * h
    bound = h * h / (8 * sj * sj)
    assert torch.all((oracle.r1_lut(x) - oracle.r1(x)).abs() <= bound * (1 + 1e-9) + 1e-15)
    # interpolation overestimates a convex function
    assert torch.all(oracle.r1_lut(x) >= oracle.r1(x) - 1e-15)
    small = torch.tensor([1e-6, 0.3 * h, 0.99 * h], dtype=torch.float64)
    assert torch.allclose(oracle.r1_lut(small), oracle.r1(small), rtol=1e-14)
    big = torch.tensor([65.0 + 1e-9, 70.0, 200.0], dtype=torch.float64)
    expect = oracle.r1(torch.tensor(65.0, dtype=torch.float64)) + (1 - 1 / 65) * (big - 65)
    assert torch.allclose(oracle.r1_lut(big), expect, rtol=1e-12)
    # r_f(s) = f r_1(s/f)
    s, f = torch.tensor([30.0, 80.0]), torch.tensor([40.0, 20.0])
    assert torch.allclose(oracle.info_divergence_lut(s, f), f.double() * oracle.r1_lut(s.double() / f.double()))



@pytest.mark.parametrize("H,W,shape", [(7, 9, (1, 5)), (6, 11, (3, 4)), (1, 8, (1, 3)), (9, 2, (5, 1)), (5, 5, (5, 5))])
def test_clamped_transposes_dot_product(H, W, shape):
    """<C x, y> = <x, C^T y> and <C' x, y> = <x, C'^T y> for the clamped
    (constant-continuation) convolution and correlation, whose transposes
    differ from each other at the borders; and the transposes equal the
    preimage form the reverse mode uses on rows: at an end pixel j of a row,
    the sum over i with clip(i - d) = j."""
    rng = np.random.default_rng(H * 31 + W)
    h = rng.uniform(0.1, 1.0, shape)
    x, y = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    lhs = float((oracle.conv_clamp(x, h) * torch.as_tensor(y)).sum())
    rhs = float((torch.as_tensor(x) * oracle.conv_clamp_T(y, h)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    lhs = float((oracle.corr_clamp(x, h) * torch.as_tensor(y)).sum())
    rhs = float((torch.as_tensor(x) * oracle.corr_clamp_T(y, h)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    if shape[0] == 1:  # row PSF: preimage sums along the row
        cx = shape[1] // 2
        ref = np.zeros((H, W))
        for j in range(W):
            for c in range(shape[1]):
                d = c - cx
                pre = [i for i in range(W) if min(max(i - d, 0), W - 1) == j]
                ref[:, j] += h[0, c] * y[:, pre].sum(axis=1)
        np.testing.assert_allclose(oracle.conv_clamp_T(y, h), ref, rtol=1e-12, atol=1e-12)
