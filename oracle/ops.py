"""FP64 reference of every step of the WR3L pipeline (test infrastructure).

Conventions (Sec. 2, Eq. 1 and the adjoint h*(x) = h(-x)):
  * images are (H, W) float64 tensors, index (i, j) = (row, column);
  * a PSF is a (kh, kw) tensor; tap (a, b) sits at offset
    (dy, dx) = (a - kh//2, b - kw//2) from the origin;
  * convolution  (u*h)(i,j)  = sum_ab h[a,b] u(i-dy, j-dx);
  * correlation  (v*h*)(i,j) = sum_ab h[a,b] v(i+dy, j+dx);
  * spatial operations continue the image constantly along the normal of
    the boundary (index clamping), Fourier operations periodically
    (Sec. 4.2).

Readings taken where the paper is silent or garbled (each also listed in the
design notes of the repository):
  R1 Eq. (9) as printed lacks the factor u^k and Eq. (3) lacks the correlation
     with h*; the multiplicative RL-style scheme the text derives is
       u <- u * ((W f/(u*h))*h* + alpha [D]+) / (W*h* - alpha [D]-).
  R2 phi'(z) = eps_phi / sqrt(z + eps_phi^2) (the regularised L1 penaliser of
     Sec. 2.3, scaled so phi'(0) = 1); psi'(z) = 1/sqrt(z + eps_psi^2) (TV).
  R3 The diffusion term D = div(psi'(|grad u|^2) grad u) uses central
     differences for |grad u|^2, arithmetic means of psi' at half-pixels and
     zero flux across the image boundary (Sec. 4.1, "standard central
     differences"), in both convolution modes.
  R4 The Wiener filter (Eq. 2) is applied literally at the native image size
     with periodic continuation; no DC correction.
  R5 "Zero or negative grey-values are replaced by a small positive value"
     (Sec. 3.2) is read as u <- max(u, delta); the same floor is applied to
     the observed image f, whose information divergence needs f > 0.
"""
from __future__ import annotations

import math

import torch

F64 = torch.float64


def _t(x) -> torch.Tensor:
    if torch.is_tensor(x) and x.dtype == F64:
        return x
    return torch.as_tensor(x, dtype=F64)


def _offsets(h: torch.Tensor):
    """Yield (dy, dx, weight) for every tap of h (zero taps are skipped unless
    h carries gradients, whose tap derivatives need every tap)."""
    kh, kw = h.shape
    cy, cx = kh // 2, kw // 2
    keep_all = h.requires_grad
    for a in range(kh):
        for b in range(kw):
            if keep_all:
                yield a - cy, b - cx, h[a, b]
            elif float(h[a, b]) != 0.0:
                yield a - cy, b - cx, float(h[a, b])


# ---------------------------------------------------------------------------
# convolution and correlation (Sec. 2 Eq. 1; Sec. 4.1 "Convolution"; Sec. 4.2)
# ---------------------------------------------------------------------------
def conv_clamp(u, h):
    """(u*h)(i,j) = sum h[a,b] u(clip(i-dy), clip(j-dx)); constant continuation."""
    u, h = _t(u), _t(h)
    H, W = u.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(u)
    for dy, dx, w in _offsets(h):
        rows = (ri - dy).clamp(0, H - 1)
        cols = (cj - dx).clamp(0, W - 1)
        out += w * u[rows][:, cols]
    return out


def corr_clamp(v, h):
    """(v*h*)(i,j) = sum h[a,b] v(clip(i+dy), clip(j+dx)); h*(x) = h(-x)."""
    v, h = _t(v), _t(h)
    H, W = v.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(v)
    for dy, dx, w in _offsets(h):
        rows = (ri + dy).clamp(0, H - 1)
        cols = (cj + dx).clamp(0, W - 1)
        out += w * v[rows][:, cols]
    return out


def conv_clamp_T(y, h):
    """Exact transpose of conv_clamp: (C^T y)(j) = sum_d h(d) sum_{i: clip(i-d) = j} y(i),
    by scatter-adding every term of the forward sum to the pixel it read."""
    y, h = _t(y), _t(h)
    H, W = y.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(y)
    for dy, dx, w in _offsets(h):
        rows = (ri - dy).clamp(0, H - 1)
        cols = (cj - dx).clamp(0, W - 1)
        out.index_put_((rows[:, None].expand(H, W), cols[None, :].expand(H, W)), w * y, accumulate=True)
    return out


def corr_clamp_T(z, h):
    """Exact transpose of corr_clamp: (C'^T z)(j) = sum_d h(d) sum_{i: clip(i+d) = j} z(i)."""
    z, h = _t(z), _t(h)
    H, W = z.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(z)
    for dy, dx, w in _offsets(h):
        rows = (ri + dy).clamp(0, H - 1)
        cols = (cj + dx).clamp(0, W - 1)
        out.index_put_((rows[:, None].expand(H, W), cols[None, :].expand(H, W)), w * z, accumulate=True)
    return out


def conv_periodic(u, h):
    """(u*h)(i,j) = sum h[a,b] u((i-dy) mod H, (j-dx) mod W)."""
    u, h = _t(u), _t(h)
    H, W = u.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(u)
    for dy, dx, w in _offsets(h):
        out += w * u[(ri - dy) % H][:, (cj - dx) % W]
    return out


def corr_periodic(v, h):
    """(v*h*)(i,j) = sum h[a,b] v((i+dy) mod H, (j+dx) mod W)."""
    v, h = _t(v), _t(h)
    H, W = v.shape
    ri, cj = torch.arange(H), torch.arange(W)
    out = torch.zeros_like(v)
    for dy, dx, w in _offsets(h):
        out += w * v[(ri + dy) % H][:, (cj + dx) % W]
    return out


def psf_transfer(h, H, W):
    """h-hat: DFT of the PSF wrapped periodically onto an H x W grid with its
    origin (centre tap) at index (0, 0) (Sec. 2.1)."""
    h = _t(h)
    hp = torch.zeros(H, W, dtype=F64)
    for dy, dx, w in _offsets(h):
        hp[dy % H, dx % W] += w
    return torch.fft.fft2(hp)


def conv_fourier(u, h):
    """Periodic convolution through the Fourier domain (Sec. 4.3, 2D case)."""
    u = _t(u)
    H, W = u.shape
    return torch.fft.ifft2(torch.fft.fft2(u) * psf_transfer(h, H, W)).real


def corr_fourier(v, h):
    """Periodic correlation with h* through the Fourier domain: the transfer
    function of h* is the complex conjugate of h-hat (Sec. 2.1)."""
    v = _t(v)
    H, W = v.shape
    return torch.fft.ifft2(torch.fft.fft2(v) * psf_transfer(h, H, W).conj()).real


def conv(u, h, mode="clamp"):
    return conv_clamp(u, h) if mode == "clamp" else conv_fourier(u, h)


def corr(v, h, mode="clamp"):
    return corr_clamp(v, h) if mode == "clamp" else corr_fourier(v, h)


# ---------------------------------------------------------------------------
# uniform linear motion: running-sum box filter (Sec. 4.3, "Uniform linear
# motion").  Per row: the first window sum is formed directly, then the
# window slides, adding the entering and subtracting the leaving grey value.
# ---------------------------------------------------------------------------
def box_running_sum_rows(u, L, weight=None, adjoint=False):
    """Convolution (or, with adjoint=True, correlation) of every row with a
    uniform box of length L (centre index L//2), constant continuation."""
    u = _t(u)
    H, W = u.shape
    c = L // 2
    w = 1.0 / L if weight is None else float(weight)
    # window for output j covers columns j - dx, dx in [-c, L-1-c] (conv),
    # i.e. [j-(L-1-c), j+c]; correlation covers [j-c, j+(L-1-c)].
    lo_off, hi_off = (-(L - 1 - c), c) if not adjoint else (-c, L - 1 - c)
    out = torch.empty_like(u)
    col = lambda j: u[:, min(max(j, 0), W - 1)]  # noqa: E731  constant continuation
    s = torch.zeros(H, dtype=F64)
    for k in range(lo_off, hi_off + 1):
        s = s + col(k)
    out[:, 0] = w * s
    for j in range(1, W):
        s = s + col(j + hi_off) - col(j - 1 + lo_off)
        out[:, j] = w * s
    return out


def box_running_sum_cols(u, L, weight=None, adjoint=False):
    return box_running_sum_rows(_t(u).T.contiguous(), L, weight, adjoint).T.contiguous()


def box_ends_running_sum_rows(u, taps, adjoint=False):
    """Row convolution (correlation with adjoint=True), constant continuation,
    with a box whose end taps may be lighter: taps = [e0, w, ..., w, e1] in
    tap order (centre index L//2).  This is the non-integer blur length of
    Sec. 4.3 ("Uniform linear motion"): single pixels of smaller weight at
    one or both ends.  The window of interior pixels slides by one pixel per
    output (one pixel enters, one leaves); the two end pixels are added with
    their own weights, so each step costs at most two additions and two
    subtractions beyond the products."""
    u = _t(u)
    taps = [float(t) for t in _t(taps).reshape(-1)]
    H, W = u.shape
    L = len(taps)
    c = L // 2
    col = lambda j: u[:, min(max(j, 0), W - 1)]  # noqa: E731  constant continuation
    # output j reads positions p = j + c - k (conv) or p = j + k - c (corr) for
    # tap k; `pos(j, k)` gives that position
    pos = (lambda j, k: j + k - c) if adjoint else (lambda j, k: j + c - k)  # noqa: E731
    out = torch.empty_like(u)
    if L == 1:
        for j in range(W):
            out[:, j] = taps[0] * col(j)
        return out
    w = taps[1] if L > 2 else 0.0
    inner = torch.zeros(H, dtype=F64)  # sum over taps 1..L-2 for output 0
    for k in range(1, L - 1):
        inner = inner + col(pos(0, k))
    for j in range(W):
        if j > 0 and L > 2:
            # the interior window moves by one pixel: the pixel of tap 1 (or
            # L-2) at j enters, the one that tap L-2 (or 1) read at j-1 leaves
            enter, leave = (pos(j, 1), pos(j - 1, L - 2)) if not adjoint else (pos(j, L - 2), pos(j - 1, 1))
            inner = inner + col(enter) - col(leave)
        out[:, j] = w * inner + taps[0] * col(pos(j, 0)) + taps[L - 1] * col(pos(j, L - 1))
    return out


def box_ends_running_sum_cols(u, taps, adjoint=False):
    return box_ends_running_sum_rows(_t(u).T.contiguous(), taps, adjoint).T.contiguous()


# ---------------------------------------------------------------------------
# Wiener filter (Sec. 2.1, Eq. 2), periodic, native size, literal (R4)
# ---------------------------------------------------------------------------
def wiener(f, h, K):
    """u = Re IDFT( f-hat * conj(h-hat) / (|h-hat|^2 + K) )."""
    f = _t(f)
    H, W = f.shape
    hh = psf_transfer(h, H, W)
    uh = torch.fft.fft2(f) * hh.conj() / (hh.abs() ** 2 + K)
    return torch.fft.ifft2(uh).real


def wiener_rows(f, h_row, K):
    """Wiener filter for a PSF supported on one row: one 1D DFT per image row
    (Sec. 4.3, "Non-uniform linear motion")."""
    f = _t(f)
    H, W = f.shape
    h_row = _t(h_row).reshape(1, -1)
    hh = psf_transfer(h_row, 1, W)[0]
    uh = torch.fft.fft(f, dim=1) * hh.conj() / (hh.abs() ** 2 + K)
    return torch.fft.ifft(uh, dim=1).real


def wiener_cols(f, h_col, K):
    return wiener_rows(_t(f).T, _t(h_col).reshape(1, -1), K).T.contiguous()


# ---------------------------------------------------------------------------
# positivity (Sec. 3.2, R5)
# ---------------------------------------------------------------------------
def positivity_floor(u, delta):
    return torch.clamp(_t(u), min=delta)


def condition_input(f, delta):
    """Observed image with the positivity floor the divergence r_f needs."""
    return positivity_floor(f, delta)


# ---------------------------------------------------------------------------
# robust data term (Sec. 2.3, Eq. 6-7, Eq. 10) and regulariser (Eq. 11)
# ---------------------------------------------------------------------------
def info_divergence(s, f):
    """r_f(s) = s - f - f ln(s/f) (Eq. 7)."""
    s, f = _t(s), _t(f)
    return s - f - f * torch.log(s / f)


# Lookup-table evaluation of r_1 (Sec. 4.1, "Function evaluations"): r_1 is
# tabulated on (0, 65], r_f(s) = f r_1(s/f), with a linear continuation of r_1
# beyond 65.  The paper gives no table resolution or interpolation rule; the
# reading taken: RF_LUT_N entries at s_j = j h, h = 65 / RF_LUT_N, linear
# interpolation between them, the closed form below the first entry.
RF_LUT_N = 8192
RF_LUT_SMAX = 65.0


def r1(x):
    """r_1(x) = x - 1 - ln x (Eq. 7 with f = 1)."""
    x = _t(x)
    return x - 1.0 - torch.log(x)


def r1_lut_table():
    h = RF_LUT_SMAX / RF_LUT_N
    s = torch.arange(1, RF_LUT_N + 1, dtype=F64) * h
    return r1(s)


def r1_lut(x):
    """r_1 from the table: linear interpolation between s_j = j h on
    [h, 65], the closed form on (0, h), and beyond 65 the tangent line at 65
    (r_1'(s) = 1 - 1/s)."""
    x = _t(x)
    T = r1_lut_table()
    h = RF_LUT_SMAX / RF_LUT_N
    k = x / h
    j = torch.clamp(torch.floor(k), 1, RF_LUT_N - 1).long()
    fr = k - j.to(F64)
    inside = T[j - 1] + fr * (T[j] - T[j - 1])
    beyond = T[-1] + (1.0 - 1.0 / RF_LUT_SMAX) * (x - RF_LUT_SMAX)
    below = r1(torch.clamp(x, min=1e-300))
    return torch.where(x < h, below, torch.where(x > RF_LUT_SMAX, beyond, inside))


def info_divergence_lut(s, f):
    """r_f(s) = f r_1(s/f) with r_1 from the table (Sec. 4.1)."""
    s, f = _t(s), _t(f)
    return f * r1_lut(s / f)


def phi_prime(z, eps, robust=True):
    """Derivative of the data penaliser, normalised to phi'(0) = 1 (R2)."""
    z = _t(z)
    if not robust:
        return torch.ones_like(z)
    return eps / torch.sqrt(z + eps * eps)


def psi_prime(z, eps, tv=True):
    """TV diffusivity psi'(|grad u|^2) = 1/sqrt(|grad u|^2 + eps^2) (R2)."""
    z = _t(z)
    if not tv:
        return torch.ones_like(z)
    return 1.0 / torch.sqrt(z + eps * eps)


def diffusion(u, eps, tv=True):
    """D(u) = div(psi'(|grad u|^2) grad u) with central differences and zero
    flux across the boundary (Eq. 11, Sec. 4.1; reading R3)."""
    u = _t(u)
    H, W = u.shape
    # ghost cells replicate the boundary values
    up = torch.nn.functional.pad(u[None, None], (1, 1, 1, 1), mode="replicate")[0, 0]
    ux = 0.5 * (up[1:-1, 2:] - up[1:-1, :-2])
    uy = 0.5 * (up[2:, 1:-1] - up[:-2, 1:-1])
    g = psi_prime(ux * ux + uy * uy, eps, tv)
    D = torch.zeros_like(u)
    # flux between (i, j) and (i, j+1), j = 0..W-2
    fx = 0.5 * (g[:, 1:] + g[:, :-1]) * (u[:, 1:] - u[:, :-1])
    D[:, :-1] += fx
    D[:, 1:] -= fx
    # flux between (i, j) and (i+1, j), i = 0..H-2
    fy = 0.5 * (g[1:, :] + g[:-1, :]) * (u[1:, :] - u[:-1, :])
    D[:-1, :] += fy
    D[1:, :] -= fy
    return D


# ---------------------------------------------------------------------------
# RRRL iteration (Sec. 2.3, Eq. 9-12; reading R1)
# ---------------------------------------------------------------------------
def rrrl_step(u, f, h, p):
    """One robust regularised Richardson-Lucy step.  `p` carries alpha,
    eps_phi, eps_psi, phi_robust, psi_tv and conv ("clamp"/"periodic")."""
    u, f = _t(u), _t(f)
    mode = p.conv
    b = conv(u, h, mode)                                   # u^k * h
    rf = info_divergence_lut(b, f) if getattr(p, "rf_eval", "log1p") == "lut" else info_divergence(b, f)
    Wk = phi_prime(rf, p.eps_phi, bool(p.phi_robust))      # Eq. 10
    A = corr(Wk * f / b, h, mode)                          # (W f/(u*h)) * h*
    B = corr(Wk, h, mode)                                  # W * h*
    D = diffusion(u, p.eps_psi, bool(p.psi_tv))            # Eq. 11
    Dp = 0.5 * (D + D.abs())                               # [D]+ (Eq. 12)
    Dm = 0.5 * (D - D.abs())                               # [D]-
    return u * (A + p.alpha * Dp) / (B - p.alpha * Dm)


def rrrl(u0, f, h, p, iters):
    u = _t(u0)
    for _ in range(iters):
        u = rrrl_step(u, f, h, p)
    return u


def _wiener_any(f, h, K):
    kh, kw = h.shape
    if kh == 1:
        return wiener_rows(f, h, K)
    if kw == 1:
        return wiener_cols(f, h, K)
    return wiener(f, h, K)


def wr3l(f, h, p, iters):
    """Wiener initialisation, positivity floor, `iters` RRRL steps (Sec. 3.2).
    Returns (u0, u_iters)."""
    h = _t(h)
    f0 = condition_input(f, p.pos_floor)
    u0 = positivity_floor(_wiener_any(f0, h, p.K), p.pos_floor)
    return u0, rrrl(u0, f0, h, p, iters)


# ---------------------------------------------------------------------------
# differentiable form (mean-square loss against the sharp image)
# ---------------------------------------------------------------------------
def wr3l_loss(f, g, h, alpha, K, p, iters):
    """Mean over a batch (N, H, W) and its pixels of (WR3L(f; h, alpha, K) - g)^2:
    the same steps as `wr3l` (conditioning, Wiener of Eq. 2, floor, `iters`
    steps of Eq. 9), with alpha and K taken from the arguments.  Every
    argument may require grad; torch autograd then gives the FP64 reverse
    mode (taps with gradients keep their zero entries, see `_offsets`)."""
    class _P:
        pass
    q = _P()
    for k in ("eps_phi", "eps_psi", "pos_floor", "phi_robust", "psi_tv", "conv"):
        setattr(q, k, getattr(p, k))
    q.alpha = alpha
    h = _t(h)
    f = _t(f)
    total = 0.0
    for n in range(f.shape[0]):
        f0 = condition_input(f[n], p.pos_floor)
        u = positivity_floor(_wiener_any(f0, h, K), p.pos_floor)
        for _ in range(iters):
            u = rrrl_step(u, f0, h, q)
        total = total + ((u - _t(g[n])) ** 2).sum()
    return total / (f.shape[0] * f.shape[1] * f.shape[2])


# ---------------------------------------------------------------------------
# quality measure (Sec. 3.1)
# ---------------------------------------------------------------------------
def snr_db(u, u0):
    """SNR(u, u0) = 10 log10(var(u) / var(u - u0)) dB."""
    u, u0 = _t(u), _t(u0)
    return 10.0 * math.log10(float(u.var(unbiased=False) / (u - u0).var(unbiased=False)))
