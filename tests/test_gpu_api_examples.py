"""The usage shown in the README runs as written (smaller sizes)."""
import numpy as np
import pytest
import torch

import paper_1212_2245_b300 as db
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu


def test_readme_usage(lib):
    case = synth.case_line1024(256, 256, 5)
    f, h = torch.as_tensor(case.f).cuda(), torch.as_tensor(case.h).cuda()
    u = db.deblur(f, h, case.params, iters=5)
    plan = db.Plan(256, 256, h, case.params, 5)
    assert torch.equal(plan.run(f), u)
    plan.close()
    fs = [torch.rand(300, 420, device="cuda") * 255 for _ in range(3)]
    hs = [torch.as_tensor(synth.box_psf(15)).cuda()] * 3
    outs = db.deblur_batch(fs, hs, Params(), 4, kinds=["box"] * 3)
    for fi, oi in zip(fs, outs):
        assert torch.equal(oi, db.deblur(fi, hs[0], Params(), 4, kind="box"))


def test_plan_run_host_equals_device_run(lib):
    """db_plan_run_host (copy in, pipeline, copy out on one stream) gives the
    device run's result bit for bit, from page-locked HostBuffers and from
    ordinary CPU tensors; bad host buffers are rejected before any copy."""
    case = synth.case_line1024(192, 160, 4)
    f, h = torch.as_tensor(case.f).cuda(), torch.as_tensor(case.h).cuda()
    plan = db.Plan(192, 160, h, case.params, 4)
    ref = plan.run(f).cpu()
    fh, uh = db.HostBuffer((192, 160)), db.HostBuffer((192, 160))
    fh.copy_from(case.f)
    plan.run_host(fh, uh)
    assert torch.equal(uh.tensor, ref)
    out = torch.empty(192, 160)
    plan.run_host(torch.as_tensor(case.f).contiguous(), out)
    assert torch.equal(out, ref)
    with pytest.raises(ValueError):
        plan.run_host(torch.empty(10, 10), out)
    with pytest.raises(ValueError):
        plan.run_host(fh, torch.empty(192, 160, dtype=torch.float64))
    fh.close()
    uh.close()
    plan.close()


@pytest.mark.parametrize("form", ["line", "gauss", "row", "col-box"])
def test_plan_autotune_keeps_a_form_equal_to_the_global_setting(lib, form):
    """db_plan_autotune times every schedule (and one-axis or FFT-tile form) and keeps the
    fastest for the plan: the tuned plan's result equals, bit for bit, a run
    with that choice set process-wide, and stays within FP32 rounding of the
    untuned plan's."""
    rng = np.random.default_rng(11)
    H, W, kind = 384, 352, "general"
    if form == "line":
        h = synth.line_psf(15, 30.0)
    elif form == "gauss":
        h = synth.gaussian_mixture_psf(21, rng)
    elif form == "row":
        h = synth.random_motion_1d(31, rng, "row")
    else:
        h, kind = synth.box_psf(13, "col"), "box"
    f = torch.as_tensor(rng.uniform(0.0, 255.0, (H, W)).astype(np.float32)).cuda()
    taps = torch.as_tensor(np.ascontiguousarray(h, dtype=np.float32)).cuda()
    p = Params()
    plan = db.Plan(H, W, taps, p, 6, kind=kind)
    base = plan.run(f).clone()
    sched, axis = plan.autotune(f, reps=2)
    assert sched in ("split", "flow", "fused", "cluster")
    if form == "row" and sched != "cluster":
        assert axis == "groups" if sched == "fused" else axis in ("groups", "windows")
    elif form in ("line", "gauss"):  # 2D PSFs: direct sums, or FFT tiles (split schedule)
        assert axis == "groups" or (axis == "fft" and sched == "split")
    else:
        assert axis is None
    tuned = plan.run(f).clone()
    try:
        db.set_schedule(sched)
        if form in ("line", "gauss"):
            db.set_fft_tiles(1 if axis == "fft" else 2305)
        elif axis is not None:
            db.set_one_axis_min(1 if axis == "windows" else 256)
        assert torch.equal(tuned, db.deblur(f, taps, p, 6, kind=kind))
    finally:
        db.set_schedule("auto")
        db.set_one_axis_min(0)
        db.set_fft_tiles(0)
    err = (tuned - base).abs().max().item()
    assert err <= 1e-3 * max(1.0, base.abs().max().item()), err
    plan.close()
