"""Reverse mode of the WR3L chain (db_rrl_backward behind DeblurFn) against
the FP64 oracle: its autograd reverse mode on small cases, and central finite
differences of the FP64 forward at full size."""
import numpy as np
import pytest
import torch

import oracle
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu

REL = 1e-3


def _setup(N, H, W, kw, seed):
    rng = np.random.default_rng(seed)
    gs = np.stack([synth.scene(H, W, rng) for _ in range(N)]).astype(np.float32)
    true_h = synth.raised_cosine_1d(kw)
    fs = np.stack([synth.degrade(g, true_h, 2.0, rng) for g in gs])
    h0 = rng.uniform(0.2, 1.0, size=(1, kw))
    h0 = (h0 / h0.sum()).astype(np.float32)
    return gs, fs, h0


def _gpu_grads(lib, fs, gs, h0, alpha, K, p, iters, every):
    f = torch.tensor(fs, device="cuda", requires_grad=True)
    taps = torch.tensor(h0, device="cuda", requires_grad=True)
    al = torch.tensor(alpha, device="cuda", requires_grad=True)
    kk = torch.tensor(K, device="cuda", requires_grad=True)
    u = lib.DeblurFn.apply(f, taps, al, kk, p, iters, every)
    loss = ((u - torch.tensor(gs, device="cuda")) ** 2).mean()
    loss.backward()
    return (float(loss.detach()), f.grad.double().cpu(), taps.grad.double().cpu(), float(al.grad),
            float(kk.grad))


def _oracle_grads(fs, gs, h0, alpha, K, p, iters):
    fT = torch.tensor(fs, dtype=torch.float64, requires_grad=True)
    hT = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    aT = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    kT = torch.tensor(K, dtype=torch.float64, requires_grad=True)
    loss = oracle.wr3l_loss(fT, gs, hT, aT, kT, p, iters)
    loss.backward()
    ga = float(aT.grad) if aT.grad is not None else 0.0  # alpha does not enter with 0 iterations
    return float(loss.detach()), fT.grad, hT.grad, ga, float(kT.grad)


@pytest.mark.parametrize("iters,every", [(0, 1), (1, 1), (3, 2), (6, 4), (6, 1), (5, 5)])
def test_backward_matches_fp64_reverse_mode(lib, iters, every):
    gs, fs, h0 = _setup(2, 40, 56, 7, 11 + iters)
    p = Params(alpha=0.02, K=0.01)
    lg, gf, gt, ga, gk = _gpu_grads(lib, fs, gs, h0, 0.02, 0.01, p, iters, every)
    lo, of, ot, oa, ok = _oracle_grads(fs, gs, h0, 0.02, 0.01, p, iters)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert float((gf - of).abs().max()) <= REL * float(of.abs().max()), "grad f"
    assert float((gt - ot).abs().max()) <= REL * float(ot.abs().max()), f"grad taps {gt} vs {ot}"
    assert abs(ga - oa) <= REL * abs(oa) + 1e-9, f"grad alpha {ga} vs {oa}"
    assert abs(gk - ok) <= REL * abs(ok) + 1e-9, f"grad K {gk} vs {ok}"


def test_backward_full_size_against_reverse_mode_and_fd(lib):
    """Two 512x512 images, 21 learnable taps, 15 iterations, checkpoints every
    5.  (1) Every gradient equals the FP64 oracle's reverse mode within 1e-3.
    (2) Central differences of the FP64 forward with a step of 1e-3 relative
    to each parameter (1e-3 absolute along a pixel direction) agree with the
    GPU gradient within 1e-3.  (An absolute step of 1e-3 would be a third of
    alpha = 0.003; the loss also has kinks at [D]+- = 0 and at the floors.)"""
    case = synth.case_learn512(n_images=2)
    gs, fs, h0 = case.g, case.f, case.h
    p = case.params
    alpha, K = p.alpha, p.K
    _, gf, gt, ga, gk = _gpu_grads(lib, fs, gs, h0, alpha, K, p, 15, 5)
    _, of, ot, oa, ok = _oracle_grads(fs, gs, h0, alpha, K, p, 15)
    print(f"learn512 (2 images) gradient rel. errors: f {float((gf - of).abs().max() / of.abs().max()):.2e} "
          f"taps {float((gt - ot).abs().max() / ot.abs().max()):.2e} alpha {abs(ga - oa) / abs(oa):.2e} "
          f"K {abs(gk - ok) / abs(ok):.2e}")
    assert float((gf - of).abs().max()) <= REL * float(of.abs().max()), "grad f"
    assert float((gt - ot).abs().max()) <= REL * float(ot.abs().max()), "grad taps"
    assert abs(ga - oa) <= REL * abs(oa) and abs(gk - ok) <= REL * abs(ok)

    def L(h, a, k, f):
        with torch.no_grad():
            return float(oracle.wr3l_loss(torch.tensor(f, dtype=torch.float64), gs,
                                          torch.tensor(h, dtype=torch.float64), a, k, p, 15))

    rel = 1e-3
    e = rel * alpha
    fd = (L(h0, alpha + e, K, fs) - L(h0, alpha - e, K, fs)) / (2 * e)
    assert abs(ga - fd) <= REL * abs(fd), f"alpha: {ga} vs {fd}"
    e = rel * K
    fd = (L(h0, alpha, K + e, fs) - L(h0, alpha, K - e, fs)) / (2 * e)
    assert abs(gk - fd) <= REL * abs(fd), f"K: {gk} vs {fd}"
    for t in (0, 10, 20):
        d = np.zeros_like(h0, dtype=np.float64)
        d[0, t] = rel * abs(float(h0[0, t]))
        fd = (L(h0 + d, alpha, K, fs) - L(h0 - d, alpha, K, fs)) / (2 * d[0, t])
        assert abs(float(gt[0, t]) - fd) <= REL * abs(fd) + 1e-6 * float(gt.abs().max()), f"tap {t}: {float(gt[0, t])} vs {fd}"
    vf = np.random.default_rng(5).standard_normal(fs.shape)
    fd = (L(h0, alpha, K, fs + 1e-3 * vf) - L(h0, alpha, K, fs - 1e-3 * vf)) / 2e-3
    an = float((gf * torch.tensor(vf)).sum())
    assert abs(an - fd) <= REL * abs(fd), f"f: {an} vs {fd}"


def test_backward_rejects_2d_psf(lib):
    f = torch.full((32, 32), 50.0, device="cuda")
    taps = torch.ones(3, 3, device="cuda") / 9
    gt = torch.zeros(9, dtype=torch.float64, device="cuda")
    ga = torch.zeros(1, dtype=torch.float64, device="cuda")
    gk = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.DeblurError):
        lib.rrl_backward(f, f.clone(), f.clone(), taps, Params(), 2, 1, gt, ga, gk)


@pytest.mark.parametrize("H,W,kw", [(12, 53, 7), (10, 37, 15), (9, 61, 21), (8, 45, 31), (6, 27, 25), (5, 7, 7),
                                    (4, 1, 1), (7, 16, 3)])
def test_backward_row_runs_ragged_rows(lib, H, W, kw):
    """The row kernels of the reverse pass take runs of 8 outputs per thread:
    rows whose length is not a multiple of 8, a run longer than the row, a
    row as long as the PSF, a single column, and every tap bucket (8, 16,
    24, 32) against the FP64 reverse mode."""
    gs, fs, h0 = _setup(2, H, W, kw, 100 + W + kw)
    p = Params(alpha=0.02, K=0.01)
    lg, gf, gt, ga, gk = _gpu_grads(lib, fs, gs, h0, 0.02, 0.01, p, 3, 2)
    lo, of, ot, oa, ok = _oracle_grads(fs, gs, h0, 0.02, 0.01, p, 3)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert float((gf - of).abs().max()) <= REL * float(of.abs().max()), "grad f"
    assert float((gt - ot).abs().max()) <= REL * float(ot.abs().max()), f"grad taps {gt} vs {ot}"
    assert abs(ga - oa) <= REL * abs(oa) + 1e-9, f"grad alpha {ga} vs {oa}"
    assert abs(gk - ok) <= REL * abs(ok) + 1e-9, f"grad K {gk} vs {ok}"
