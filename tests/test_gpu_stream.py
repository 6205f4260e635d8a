"""Streaming form: transfers overlapped with computation give the same frames
as running the plan on each frame alone."""
import numpy as np
import pytest
import torch

import paper_1212_2245_b300 as db
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [2, 3])
def test_stream_equals_plan(lib, depth):
    H, W, iters = 96, 160, 6
    h = synth.line_psf(15, 30.0, 16.0)
    p = Params()
    rng = np.random.default_rng(depth)
    frames = []
    for _ in range(7):
        g = synth.scene(H, W, rng).astype(np.float32)
        frames.append(torch.as_tensor(synth.degrade(g, h, 2.0, rng)).pin_memory())
    taps = torch.as_tensor(h).cuda()
    fs = db.FrameStream(H, W, taps, p, iters, depth=depth)
    outs = fs.run(frames)
    plan = db.Plan(H, W, taps, p, iters)
    for fr, out in zip(frames, outs):
        ref = plan.run(fr.cuda())
        assert torch.equal(out, ref.cpu())
    fs.close()
    plan.close()
