"""Lookup-table evaluation of r_1 (Sec. 4.1): the GPU table path against the
oracle's table path, and its distance from the log1p path."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_1212_2245_b300 as db
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


@pytest.fixture
def lut_mode(lib):
    db.set_rf_eval("lut")
    yield
    db.set_rf_eval("log1p")


@pytest.mark.parametrize("psf,H,W", [("line", 160, 224), ("box", 128, 200), ("gauss", 77, 131)])
def test_lut_iterations_match_oracle_lut(lib, lut_mode, psf, H, W):
    rng = np.random.default_rng(H + W)
    h = {"line": synth.line_psf(15, 30.0, 16.0), "box": synth.box_psf(9),
         "gauss": synth.gaussian_mixture_psf(9, rng)}[psf]
    kind = "box" if psf == "box" else "general"
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng, salt_pepper=0.01)
    p = Params()
    p_lut = dataclasses.replace(p, rf_eval="lut")
    u0_ref, u_ref = oracle.wr3l(f, h, p_lut, 8)
    u = lib.deblur(cuda(f), cuda(h), p, 8, kind=kind)
    d = (u.double().cpu() - u_ref).abs()
    assert float(d.max()) <= 1e-3 and float(d.pow(2).mean().sqrt()) <= 1e-4, (float(d.max()), psf)
    # the table changes the result by far more than rounding: the two
    # oracles differ, and the GPU follows the table one
    _, u_log = oracle.wr3l(f, h, p, 8)
    assert float((u_ref - u_log).abs().max()) > 10 * float(d.max())


def test_lut_mode_in_plans_batches_and_backward(lib, lut_mode):
    H, W = 64, 96
    h = synth.raised_cosine_1d(7)
    rng = np.random.default_rng(5)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = cuda(synth.degrade(g, h, 2.0, rng))
    p = Params()
    plan = db.Plan(H, W, cuda(h), p, 5)
    u_plan = plan.run(f)
    assert torch.equal(u_plan, lib.deblur(f, cuda(h), p, 5))
    b = db.Batch([f], [cuda(h)], p, 5)
    b.run()
    assert torch.equal(b.us[0], u_plan)
    plan.close(); b.close()
    with pytest.raises(db.DeblurError, match="unsupported"):
        taps = cuda(h)
        ck = torch.empty(1, 1, H, W, device="cuda")
        gt = torch.zeros(taps.numel(), dtype=torch.float64, device="cuda")
        ga = torch.zeros(1, dtype=torch.float64, device="cuda")
        gk = torch.zeros(1, dtype=torch.float64, device="cuda")
        db.rrl_backward(f[None], ck, torch.zeros_like(f)[None], taps, p, 1, 5, gt, ga, gk)
