"""Batched form: many uneven images with their own PSFs in one planned run
(five batched Wiener launches + one persistent RRRL launch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1212_2245_b300 import synth

pytestmark = pytest.mark.gpu

MAX_ABS, RMS = 1e-3, 1e-4


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def small_batch(idx, cap=300):
    return [synth.batch_case(i, size_cap=cap) for i in idx]


def test_batch_equals_single_image_pipeline(lib):
    cases = small_batch(list(range(0, 8)) + list(range(256, 264)))
    fs = [cuda(c.f) for c in cases]
    hs = [cuda(c.h) for c in cases]
    outs = lib.deblur_batch(fs, hs, [c.params for c in cases], 10, kinds=[c.psf_kind for c in cases])
    for c, f, h, u in zip(cases, fs, hs, outs):
        ref = lib.deblur(f, h, c.params, 10, kind=c.psf_kind)
        d = float((u - ref).abs().max())
        assert d == 0.0, f"{c.name} {c.f.shape} psf {c.h.shape}: batch differs from single image by {d}"


@pytest.mark.parametrize("iters", [0, 1, 4, 10])
def test_batch_against_oracle(lib, iters):
    cases = small_batch([4, 5, 258, 300], cap=200)
    fs = [cuda(c.f) for c in cases]
    outs = lib.deblur_batch(fs, [cuda(c.h) for c in cases], [c.params for c in cases], iters,
                            kinds=[c.psf_kind for c in cases])
    for c, u in zip(cases, outs):
        _, ref = oracle.wr3l(c.f, c.h, c.params, iters)
        d = (u.double().cpu() - ref).abs()
        assert float(d.max()) <= MAX_ABS and float(d.pow(2).mean().sqrt()) <= RMS, c.name


def test_batch_graph_capture_and_replay(lib):
    cases = small_batch([10, 11, 270, 271], cap=256)
    fs = [cuda(c.f) for c in cases]
    hs = [cuda(c.h) for c in cases]
    b = lib.Batch(fs, hs, [c.params for c in cases], 6, kinds=[c.psf_kind for c in cases])
    first = [u.clone() for u in b.run()]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(check=False)
    g.replay()
    torch.cuda.synchronize()
    for u, v in zip(b.us, first):
        assert torch.equal(u, v)
    # new pixel values, same shapes: the replayed plan deblurs them
    for f in fs:
        f.mul_(0.9).add_(5.0)
    b.ws.reset_status()
    g.replay()
    torch.cuda.synchronize()
    b.ws.raise_on_flags("replay")
    for c, f, h, u in zip(cases, fs, hs, b.us):
        assert torch.equal(u, lib.deblur(f, h, c.params, 6, kind=c.psf_kind))
    b.close()


@pytest.mark.parametrize("order", ["dependency", "barrier"])
def test_batch_bounded_barrier_reports_timeout(lib, order):
    """With a zero wait budget the persistent kernel's waits (per-image
    dependency waits, or grid barriers) give up at once: the run returns,
    the status word carries the time-out flag and the context stays usable."""
    cases = small_batch([20, 280], cap=200)
    fs = [cuda(c.f) for c in cases]
    hs = [cuda(c.h) for c in cases]
    lib.set_spin_limit(0)
    lib.set_batch_order(order)
    try:
        b = lib.Batch(fs, hs, [c.params for c in cases], 5, kinds=[c.psf_kind for c in cases])
        b.ws.reset_status()
        b.run(check=False)
        torch.cuda.synchronize()
        flags = int(b.ws.status.item())
        b.close()
    finally:
        lib.set_spin_limit(4_000_000_000)
        lib.set_batch_order("barrier")
    if flags == 0:
        pytest.skip("every CTA reached each barrier before checking its budget")
    assert flags & 0x4, f"flags 0x{flags:x}"
    u = lib.deblur(fs[0], hs[0], cases[0].params, 3, kind=cases[0].psf_kind)
    assert torch.isfinite(u).all()


def test_batch_rejects_bad_descriptors(lib):
    f = cuda(np.full((64, 64), 50.0))
    with pytest.raises(lib.DeblurError):
        lib.deblur_batch([f], [cuda(np.ones((1, 80)) / 80)], [synth.Params()], 2)
    with pytest.raises(lib.DeblurError):
        lib.deblur_batch([f], [cuda(np.ones((3, 3)) / 9)], [synth.Params(conv="periodic")], 2)


def test_uneven_batch_512_subset_against_oracle(lib):
    """The full 512-image batch (sides 128..1024, half 1D motion, half 2D
    Gaussian mixtures), compared with the oracle on 16 + 16 images."""
    cases = [synth.batch_case(i) for i in range(512)]
    fs = [cuda(c.f) for c in cases]
    outs = lib.deblur_batch(fs, [cuda(c.h) for c in cases], [c.params for c in cases], 10,
                            kinds=[c.psf_kind for c in cases])
    worst = (0.0, 0.0)
    for i in list(range(0, 256, 16)) + list(range(256, 512, 16)):
        _, ref = oracle.wr3l(cases[i].f, cases[i].h, cases[i].params, 10)
        d = (outs[i].double().cpu() - ref).abs()
        m, r = float(d.max()), float(d.pow(2).mean().sqrt())
        worst = (max(worst[0], m), max(worst[1], r))
        assert m <= MAX_ABS and r <= RMS, f"{cases[i].name} {cases[i].f.shape}: {m:.3e} {r:.3e}"
    print(f"batch512 subset worst max-abs {worst[0]:.3e} rms {worst[1]:.3e}")


def test_uneven_batch_512_all_fft_tiles_against_oracle(lib):
    """The full batch with FFT tiles for every 2D PSF (the lowest threshold
    db_batch_autotune can choose: 7x7 up), in one run; 12 of its 2D images,
    one of each size class and the smallest and largest images, against the
    oracle."""
    cases = [synth.batch_case(i) for i in range(512)]
    fs = [cuda(c.f) for c in cases]
    lib.set_fft_tiles(1)
    try:
        outs = lib.deblur_batch(fs, [cuda(c.h) for c in cases], [c.params for c in cases], 10,
                                kinds=[c.psf_kind for c in cases])
    finally:
        lib.set_fft_tiles(0)
    by_size = {}
    for i in range(256, 512):
        by_size.setdefault(cases[i].h.shape[0], i)
    px = sorted(range(256, 512), key=lambda i: cases[i].f.size)
    pick = sorted(set(by_size.values()) | {px[0], px[-1]})
    for i in pick:
        _, ref = oracle.wr3l(cases[i].f, cases[i].h, cases[i].params, 10)
        d = (outs[i].double().cpu() - ref).abs()
        m, r = float(d.max()), float(d.pow(2).mean().sqrt())
        assert m <= MAX_ABS and r <= RMS, f"{cases[i].name} {cases[i].f.shape} {cases[i].h.shape}: {m:.3e} {r:.3e}"


def test_batch_plans_with_different_shared_memory_coexist(lib):
    """A plan made after another one with smaller tiles (less shared memory
    per CTA) must not stop the earlier plan from launching."""
    big = small_batch([259], cap=160)     # 25x25 Gaussian mixture: large halo
    small = small_batch([0], cap=160)     # 1D box: small tiles
    fb, fs_ = [cuda(c.f) for c in big], [cuda(c.f) for c in small]
    bb = lib.Batch(fb, [cuda(c.h) for c in big], [c.params for c in big], 3, kinds=[c.psf_kind for c in big])
    bs = lib.Batch(fs_, [cuda(c.h) for c in small], [c.params for c in small], 3,
                   kinds=[c.psf_kind for c in small])
    for b, cases, fs in ((bb, big, fb), (bs, small, fs_)):
        for c, f, u in zip(cases, fs, b.run()):
            assert torch.equal(u, lib.deblur(f, cuda(c.h), c.params, 3, kind=c.psf_kind))
    bb.close()
    bs.close()


def test_batch_autotune_keeps_the_results_of_the_chosen_forms(lib):
    """The batch's autotuner times the dense-sum and one-axis forms and keeps
    the fastest; every image then equals the single-image pipeline under the
    matching process-wide settings, bit for bit, and the oracle."""
    cases = small_batch([0, 1, 3, 5, 256, 257, 259, 300], cap=200)
    fs = [cuda(c.f) for c in cases]
    hs = [cuda(c.h) for c in cases]
    b = lib.Batch(fs, hs, [c.params for c in cases], 4, kinds=[c.psf_kind for c in cases])
    choice = b.autotune(reps=2)
    assert set(choice) == {"fft", "dense", "windows"} and choice["windows"] in ("rule", "all", "none")
    outs = [u.clone() for u in b.run()]
    lib.set_fft_tiles(choice["fft"] or 2305)
    lib.set_dense_min(50 if choice["dense"] else 101)
    lib.set_one_axis_min({"rule": 0, "all": 1, "none": 256}[choice["windows"]])
    try:
        for c, f, h, u in zip(cases, fs, hs, outs):
            assert torch.equal(u, lib.deblur(f, h, c.params, 4, kind=c.psf_kind)), c.name
    finally:
        lib.set_fft_tiles(0)
        lib.set_dense_min(0)
        lib.set_one_axis_min(0)
    for c, u in zip(cases[:2] + cases[4:6], outs[:2] + outs[4:6]):
        _, ref = oracle.wr3l(c.f, c.h, c.params, 4)
        d = (u.double().cpu() - ref).abs()
        assert float(d.max()) <= MAX_ABS and float(d.pow(2).mean().sqrt()) <= RMS, c.name
    b.close()


def test_batch_dependency_order_equals_barrier_order(lib):
    """The dependency-ordered run (each tile waits for its own image's
    previous phase) and the run with grid barriers between phases give the
    same bits on a mix of 1D, dense 2D and FFT-tile images."""
    cases = small_batch([0, 1, 2, 3, 256, 257, 258, 300, 301, 400], cap=320)
    fs = [cuda(c.f) for c in cases]
    hs = [cuda(c.h) for c in cases]
    outs = {}
    try:
        for order in ("barrier", "dependency"):
            lib.set_batch_order(order)
            b = lib.Batch(fs, hs, [c.params for c in cases], 6, kinds=[c.psf_kind for c in cases])
            outs[order] = [u.clone() for u in b.run()]
            b.close()
    finally:
        lib.set_batch_order("barrier")
    for c, a, d in zip(cases, outs["barrier"], outs["dependency"]):
        assert torch.equal(a, d), c.name
