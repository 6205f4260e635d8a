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


def test_batch_stream_equals_batch(lib):
    """Sub-batches with overlapped transfers give the single batch's results
    bit for bit, over repeated calls, for any split."""
    from paper_1212_2245_b300 import synth
    cases = [synth.batch_case(i, size_cap=192) for i in (0, 1, 2, 3, 256, 257, 300)]
    taps = [torch.as_tensor(c.h).cuda().contiguous() for c in cases]
    ps = [c.params for c in cases]
    kinds = [c.psf_kind for c in cases]
    fs = [torch.as_tensor(c.f).cuda() for c in cases]
    ref = [u.cpu() for u in lib.deblur_batch(fs, taps, ps, 4, kinds=kinds)]
    for parts in (1, 3, 5):
        bs = lib.BatchStream([c.f.shape for c in cases], taps, ps, 4, kinds=kinds, parts=parts)
        f_host = [torch.as_tensor(c.f).contiguous().pin_memory() for c in cases]
        u_host = [torch.empty(c.f.shape, dtype=torch.float32).pin_memory() for c in cases]
        for _ in range(2):
            for u in u_host:
                u.zero_()
            bs.run(f_host, u_host)
            for a, b in zip(u_host, ref):
                assert torch.equal(a, b)
        bs.close()


def test_batch_stream_pitched_staging(lib):
    """Staging buffers with a row stride above the width (copies by rows)
    give the single batch's results bit for bit."""
    import ctypes
    from paper_1212_2245_b300 import Workspace, _check, _db_params, _db_psf, _lib, _stream
    cases = [synth.batch_case(i, size_cap=160) for i in (4, 5, 260, 261)]
    taps = [torch.as_tensor(c.h).cuda().contiguous() for c in cases]
    ps = [c.params for c in cases]
    kinds = [c.psf_kind for c in cases]
    ref = [u.cpu() for u in lib.deblur_batch([torch.as_tensor(c.f).cuda() for c in cases], taps, ps, 3,
                                            kinds=kinds)]
    n = len(cases)
    pad = [torch.zeros(c.f.shape[0], c.f.shape[1] + 5, device="cuda") for c in cases]
    padu = [torch.zeros_like(t) for t in pad]
    descs = (_lib.DbImageDesc * n)()
    for k, c in enumerate(cases):
        H, W = c.f.shape
        descs[k] = _lib.DbImageDesc(pad[k].data_ptr(), padu[k].data_ptr(), H, W, W + 5,
                                    _db_psf(taps[k], kinds[k]), _db_params(ps[k]))
    L = _lib.load()
    nbytes = L.db_batch_stream_workspace_bytes(descs, n, 3, 2)
    assert nbytes > 0
    ws = Workspace(nbytes)
    ws.reset_status()
    h = ctypes.c_void_p()
    _check(L.db_batch_stream_create(descs, n, 3, 2, ws.ptr, ws.nbytes, ws.status.data_ptr(), _stream(),
                                    ctypes.byref(h)), "db_batch_stream_create")
    f_host = [torch.as_tensor(c.f).contiguous().pin_memory() for c in cases]
    u_host = [torch.full(c.f.shape, -1.0).pin_memory() for c in cases]
    fp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in f_host])
    up = (ctypes.c_void_p * n)(*[t.data_ptr() for t in u_host])
    _check(L.db_batch_stream_run_host(h, fp, up, ws.status.data_ptr(), _stream()), "db_batch_stream_run_host")
    torch.cuda.current_stream().synchronize()
    ws.raise_on_flags("pitched streamed batch")
    L.db_batch_stream_destroy(h)
    for a, b in zip(u_host, ref):
        assert torch.equal(a, b)
