"""N equally sized images in one call (db_deblur_n): every image equals the
single-image pipeline, checkpoints land in the layout the reverse mode reads."""
import numpy as np
import pytest
import torch

import paper_1212_2245_b300 as db
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu


def _stack(n, H, W, h, seed, ld=None):
    rng = np.random.default_rng(seed)
    fs = [synth.degrade(synth.scene(H, W, rng).astype(np.float32), h, 2.0, rng) for _ in range(n)]
    ld = W if ld is None else ld
    f = torch.zeros(n, H, ld, device="cuda")
    f[:, :, :W] = torch.as_tensor(np.stack(fs)).cuda()
    return f[:, :, :W]


@pytest.mark.parametrize("psf,kind,H,W", [("line", "general", 96, 128), ("rc", "general", 65, 100),
                                          ("rc", "general", 64, 100), ("box", "box", 50, 77),
                                          ("gauss", "general", 40, 33)])
def test_deblur_n_equals_single(lib, psf, kind, H, W):
    rng = np.random.default_rng(7)
    h = {"line": synth.line_psf(15, 30.0, 16.0), "rc": synth.raised_cosine_1d(9), "box": synth.box_psf(7),
         "gauss": synth.gaussian_mixture_psf(7, rng)}[psf]
    taps = torch.as_tensor(h).cuda()
    p = Params()
    f = _stack(3, H, W, h, H + W, ld=W + 12)
    iters, every = 5, 2
    ck = torch.empty(3, 3, H, W, device="cuda")
    u = db.deblur_n(f, taps, p, iters, kind=kind, ckpt=ck, ckpt_every=every)
    db.set_schedule("split")
    try:
        for z in range(3):
            fz = f[z].contiguous()
            ref = lib.deblur(fz, taps, p, iters, kind=kind)
            assert torch.equal(u[z], ref), (psf, z)
            u0 = lib.wiener(fz, taps, p, kind=kind)
            for c, k in enumerate((0, 2, 4)):
                uk = lib.rrl_iterate(fz, u0.clone(), taps, p, k, kind=kind)
                assert torch.equal(ck[z, c], uk), (psf, z, k)
    finally:
        db.set_schedule("auto")
