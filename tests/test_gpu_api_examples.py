"""The usage shown in the README runs as written (smaller sizes)."""
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
