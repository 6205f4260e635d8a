"""The allocation-free entry point, called through the C ABI.

db_rrl_iterate_noalloc is for callers that cannot allocate device memory at
run time: a deblurring step inside a fixed-latency frame loop cannot risk a
cudaMalloc (it may synchronise the device and take unbounded time), and a
plugin inside a framework that owns all GPU memory may have no allocator at
all.  It takes its scratch from a fixed array inside the library instead of
a caller workspace, so it must give what db_rrl_iterate gives, call after
call, even though consecutive calls reuse the same array.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1212_2245_b300 import _db_params, _lib, synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu


def _inputs(H, W, h, seed):
    rng = np.random.default_rng(seed)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng, salt_pepper=0.01)
    u0 = np.maximum(f, 0.1).astype(np.float32)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()  # noqa: E731
    return dev(f), dev(u0), dev(h)


def _with_workspace(lib, f, u, h, p, iters):
    """The existing entry point, with a caller workspace."""
    H, W = f.shape
    psf = _lib.DbPsf(h.shape[0], h.shape[1], 0, h.data_ptr())
    par = _db_params(p)
    nbytes = lib.db_workspace_bytes(H, W, ctypes.byref(psf), ctypes.byref(par))
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = ws.data_ptr() + (-ws.data_ptr()) % 256
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.db_rrl_iterate(f.data_ptr(), u.data_ptr(), H, W, W, ctypes.byref(psf), ctypes.byref(par),
                            iters, None, 0, ptr, nbytes, status.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return u


def _without_allocation(lib, f, u, h, p, iters):
    H, W = f.shape
    psf = _lib.DbPsf(h.shape[0], h.shape[1], 0, h.data_ptr())
    par = _db_params(p)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.db_rrl_iterate_noalloc(f.data_ptr(), u.data_ptr(), H, W, W, ctypes.byref(psf),
                                    ctypes.byref(par), iters, status.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.db_status_string(rc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return u


def test_no_alloc_matches_workspace_entry_point_on_consecutive_calls():
    """Both entry points launch the same kernels on the same inputs, so their
    results must agree bit for bit, whichever call ran before on the shared
    scratch.  The shapes cover the split schedule (below 512K pixels), the
    flow schedule (512K to 2M pixels, whose dependency counters live in the
    scratch and are cleared by each call), tap groups (2D PSFs) and one-axis
    register windows (row PSFs)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib.load()
    p = Params()
    cases = [(_inputs(200, 300, synth.line_psf(15, 30.0, 16.0), 1), 6),
             (_inputs(97, 131, synth.raised_cosine_1d(9), 2), 5),
             (_inputs(1024, 1024, synth.raised_cosine_1d(31), 3), 4),
             (_inputs(1024, 1024, synth.line_psf(31, 30.0, 32.0), 4), 3)]
    refs = [_with_workspace(lib, f, u0.clone(), h, p, it) for (f, u0, h), it in cases]
    # every case twice in a row after a call of another shape, then the first
    # again after the largest
    for k in [0, 1, 2, 2, 1, 3, 3, 0]:
        (f, u0, h), it = cases[k]
        out = _without_allocation(lib, f, u0.clone(), h, p, it)
        assert torch.equal(out, refs[k]), f"call on {tuple(f.shape)} differs from db_rrl_iterate"


def test_no_alloc_rejects_images_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib.load()
    p = Params()
    h = torch.ones(3, 3, device="cuda") / 9
    psf = _lib.DbPsf(3, 3, 0, h.data_ptr())
    par = _db_params(p)
    H = W = 2048  # needs far more than the fixed scratch
    assert lib.db_workspace_bytes(H, W, ctypes.byref(psf), ctypes.byref(par)) > _lib.NOALLOC_SCRATCH_BYTES
    f = torch.full((H, W), 100.0, device="cuda")
    u = f.clone()
    rc = lib.db_rrl_iterate_noalloc(f.data_ptr(), u.data_ptr(), H, W, W, ctypes.byref(psf),
                                    ctypes.byref(par), 2, None, torch.cuda.current_stream().cuda_stream)
    assert rc == 4  # DB_ERR_WORKSPACE, nothing enqueued
    torch.cuda.synchronize()
    assert torch.equal(u, f)
