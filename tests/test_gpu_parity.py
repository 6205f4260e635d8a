"""GPU parity: the CUDA path against the FP64 oracle on the same seeded
inputs.  Bar: max-abs <= 1e-3 and RMS <= 1e-4 grey levels (0-255 scale)
after the stated iteration count."""
import numpy as np
import pytest
import torch

import oracle
from paper_1212_2245_b300 import synth
from paper_1212_2245_b300.params import Params

pytestmark = pytest.mark.gpu

MAX_ABS, RMS = 1e-3, 1e-4


def err(gpu, ref):
    d = (gpu.double().cpu() - torch.as_tensor(ref, dtype=torch.float64)).abs()
    return float(d.max()), float(d.pow(2).mean().sqrt())


def assert_close(gpu, ref, what, max_abs=MAX_ABS, rms=RMS):
    m, r = err(gpu, ref)
    assert m <= max_abs and r <= rms, f"{what}: max-abs {m:.3e} rms {r:.3e}"
    return m, r


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


@pytest.fixture(params=["fused", "split", "flow", "cluster"])
def sched(request, lib):
    lib.set_schedule(request.param)
    yield request.param
    lib.set_schedule("auto")


def oracle_pipeline(case):
    return oracle.ops.wr3l(case.f, case.h, case.params, case.iters)


@pytest.mark.parametrize("maker", [synth.case_box256, synth.case_line1024])
def test_full_pipeline_configs(lib, maker, sched):
    case = maker()
    f, h = cuda(case.f), cuda(case.h)
    u0_ref, u_ref = oracle_pipeline(case)
    u0 = lib.wiener(f, h, case.params, kind=case.psf_kind)
    m0, r0 = assert_close(u0, u0_ref, f"{case.name} Wiener")
    print(f"{case.name} Wiener max-abs {m0:.3e} rms {r0:.3e}")
    u = lib.rrl_iterate(f, u0.clone(), h, case.params, case.iters, kind=case.psf_kind)
    m, r = assert_close(u, u_ref, f"{case.name} WR3L")
    print(f"{case.name} [{sched}] WR3L max-abs {m:.3e} rms {r:.3e}")
    ud = lib.deblur(f, h, case.params, case.iters, kind=case.psf_kind)
    assert torch.equal(ud, u)
    # the same schedule with direct sums only (line1024's 17 x 27 PSF takes the
    # FFT tiles by the size rule, so the flow kernel and the tap groups run here)
    lib.set_fft_tiles(2305)
    try:
        u2 = lib.rrl_iterate(f, u0.clone(), h, case.params, case.iters, kind=case.psf_kind)
    finally:
        lib.set_fft_tiles(0)
    m, r = assert_close(u2, u_ref, f"{case.name} WR3L direct sums")
    print(f"{case.name} [{sched}, direct sums] WR3L max-abs {m:.3e} rms {r:.3e}")


@pytest.mark.parametrize("maker", [synth.case_box256, synth.case_line1024])
def test_full_pipeline_tuned_plan(lib, maker):
    """The configuration the bench times: a plan whose schedule and tile
    form db_plan_autotune chose, at full size, against the oracle."""
    case = maker()
    f, h = cuda(case.f), cuda(case.h)
    _, u_ref = oracle_pipeline(case)
    plan = lib.Plan(*case.f.shape, h, case.params, case.iters, kind=case.psf_kind)
    sched, form = plan.autotune(f, reps=2)
    u = plan.run(f)
    m, r = assert_close(u, u_ref, f"{case.name} tuned plan ({sched}, {form})")
    print(f"{case.name} tuned plan [{sched}, {form}] WR3L max-abs {m:.3e} rms {r:.3e}")
    plan.close()


def test_full_pipeline_fourier_gauss2048(lib):
    """2048x2048, 31x31 Gaussian mixture, Wiener + 30 RRRL with Fourier-domain
    (periodic) blur and correlation."""
    case = synth.case_gauss2048()
    f, h = cuda(case.f), cuda(case.h)
    u0_ref, u_ref = oracle_pipeline(case)
    u0 = lib.wiener(f, h, case.params)
    m0, r0 = assert_close(u0, u0_ref, "gauss2048 Wiener")
    u = lib.rrl_iterate(f, u0.clone(), h, case.params, case.iters)
    m, r = assert_close(u, u_ref, "gauss2048 WR3L")
    print(f"gauss2048 Wiener max-abs {m0:.3e} rms {r0:.3e}; WR3L max-abs {m:.3e} rms {r:.3e}")


@pytest.mark.parametrize("H,W,psf", [(64, 64, "line"), (128, 32, "gauss"), (32, 256, "row"), (256, 512, "gauss"),
                                     (16, 16, "identity"), (8, 1024, "row"), (1024, 8, "col")])
def test_fourier_iterations_shapes(lib, H, W, psf):
    rng = np.random.default_rng(H * 7 + W)
    h = {"line": synth.line_psf(9, 30.0, 10.0), "row": synth.raised_cosine_1d(7), "col": synth.box_psf(5, "col"),
         "gauss": synth.gaussian_mixture_psf(7, rng), "identity": np.ones((1, 1), np.float32)}[psf]
    p = Params(conv="periodic")
    f, u0 = _iterate_case(H, W, h, 4, p, seed=5)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
    assert_close(u, ref, f"fourier {psf} {H}x{W}")


@pytest.mark.parametrize("H,W", [(16, 4096), (4096, 16)])
def test_fourier_iterations_at_the_largest_side(lib, H, W):
    """Periodic iterations on images whose long side is the largest the
    library takes (4096): row transforms of 4096 points, column passes of
    4096 points."""
    rng = np.random.default_rng(H + 3 * W)
    h = synth.gaussian_mixture_psf(7, rng)
    p = Params(conv="periodic")
    f, u0 = _iterate_case(H, W, h, 3, p, seed=9)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 3)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 3)
    assert_close(u, ref, f"fourier {H}x{W}")


def test_fourier_checkpoints_and_pitch(lib):
    H, W, ld = 64, 128, 160
    h = synth.gaussian_mixture_psf(5, np.random.default_rng(3))
    p = Params(conv="periodic")
    f, u0 = _iterate_case(H, W, h, 5, p)
    fp = torch.zeros(H, ld, device="cuda"); fp[:, :W] = cuda(f)
    up = torch.full((H, ld), -3.0, device="cuda"); up[:, :W] = cuda(u0)
    ck = torch.empty(3, H, W, device="cuda")
    lib.rrl_iterate(fp[:, :W], up[:, :W], cuda(h), p, 5, ckpt=ck, ckpt_every=2)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 5)
    assert_close(up[:, :W], ref, "fourier pitched")
    assert torch.all(up[:, W:] == -3.0)
    u2 = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 2)
    u4 = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
    assert torch.equal(ck[0], cuda(u0)) and torch.equal(ck[1], u2) and torch.equal(ck[2], u4)


def _iterate_case(H, W, h, iters, params, kind="general", seed=0, ld=None):
    rng = np.random.default_rng(seed)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng, salt_pepper=0.01)
    u0 = np.maximum(synth.blur_replicate(f, np.ones((1, 1))), 0.1).astype(np.float32)  # any positive start
    return f, u0


@pytest.mark.parametrize("H,W", [(77, 131), (1, 1), (3, 200), (200, 3), (65, 64), (33, 97)])
@pytest.mark.parametrize("psf", ["line", "box", "gauss", "col", "identity"])
def test_iterations_ragged_shapes(lib, H, W, psf, sched):
    rng = np.random.default_rng(H * 1000 + W)
    h = {"line": synth.line_psf(9, 30.0, 10.0), "box": synth.box_psf(7), "col": synth.raised_cosine_1d(5, "col"),
         "gauss": synth.gaussian_mixture_psf(7, rng), "identity": np.ones((1, 1), np.float32)}[psf]
    if h.shape[0] > H or h.shape[1] > W:
        pytest.skip("PSF larger than image")
    kind = "box" if psf == "box" else "general"
    p = Params()
    iters = 5
    f, u0 = _iterate_case(H, W, h, iters, p)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, iters)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, iters, kind=kind)
    assert_close(u, ref, f"{psf} {H}x{W}")


def test_pitched_rows_and_odd_iteration_count(lib, sched):
    H, W, ld = 70, 90, 128
    h = synth.line_psf(11, 30.0, 12.0)
    p = Params(alpha=0.01)
    f, u0 = _iterate_case(H, W, h, 3, p)
    fp = torch.zeros(H, ld, device="cuda"); fp[:, :W] = cuda(f)
    up = torch.full((H, ld), -7.0, device="cuda"); up[:, :W] = cuda(u0)
    lib.rrl_iterate(fp[:, :W], up[:, :W], cuda(h), p, 3)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 3)
    assert_close(up[:, :W], ref, "pitched")
    assert torch.all(up[:, W:] == -7.0), "wrote outside the image"


@pytest.mark.parametrize("variant", [dict(phi_robust=0), dict(psi_tv=0, alpha=1e-4), dict(alpha=0.0),
                                     dict(eps_phi=0.5, eps_psi=3.0, alpha=0.002)])
def test_parameter_variants(lib, variant):
    H, W = 96, 128
    h = synth.line_psf(13, 45.0, 14.0)
    p = Params(**variant)
    f, u0 = _iterate_case(H, W, h, 6, p, seed=3)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 6)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6)
    assert_close(u, ref, str(variant))


@pytest.mark.parametrize("psf", ["line", "gauss"])
def test_small_tv_epsilon_few_iterations(lib, psf):
    """eps_psi = 1 (the survey's suggested TV epsilon, not the default): the
    explicit diffusion step then exceeds the stable range and amplifies
    rounding differences over many iterations, but after 3 iterations the
    FP32 path still matches the FP64 oracle at the usual bar."""
    rng = np.random.default_rng(17)
    h = synth.line_psf(13, 45.0, 14.0) if psf == "line" else synth.gaussian_mixture_psf(11, rng)
    p = Params(eps_psi=1.0)
    f, u0 = _iterate_case(96, 128, h, 3, p, seed=21)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 3)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 3)
    assert_close(u, ref, f"eps_psi=1 {psf}")


@pytest.mark.parametrize("H,W", [(16, 4096), (4096, 16), (40, 4095)])
def test_iterations_at_the_largest_side(lib, H, W, sched):
    """Spatial iterations and the whole pipeline on images whose long side is
    the largest the library takes, in every schedule."""
    h = synth.line_psf(9, 30.0, 10.0)
    p = Params()
    f, u0 = _iterate_case(H, W, h, 3, p, seed=13)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 3)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 3)
    assert_close(u, ref, f"{H}x{W}")
    _, u_ref = oracle.wr3l(f, h, p, 3)
    assert_close(lib.deblur(cuda(f), cuda(h), p, 3), u_ref, f"WR3L {H}x{W}")


@pytest.mark.parametrize("H,W,shape", [(128, 256, (1, 15)), (256, 128, (9, 1)), (64, 512, (5, 7)),
                                       (512, 64, (17, 27)), (1, 256, (1, 31)), (256, 1, (7, 1)),
                                       (2, 2, (1, 1)), (4096, 16, (3, 5)),
                                       (100, 150, (1, 15)), (77, 64, (9, 1)), (129, 127, (5, 7)),
                                       (1021, 48, (1, 41)), (40, 1021, (25, 25)), (3, 5, (1, 3)),
                                       (1000, 1000, (25, 25)), (4095, 33, (9, 1)), (1, 1, (1, 1))])
def test_wiener_shapes(lib, H, W, shape):
    rng = np.random.default_rng(H + W)
    h = rng.uniform(0.1, 1.0, size=shape)
    h = (h / h.sum()).astype(np.float32)
    g = synth.scene(H, W, rng).astype(np.float32)
    f = synth.degrade(g, h, 2.0, rng)
    p = Params(K=0.01)
    ref = oracle.positivity_floor(oracle.ops._wiener_any(oracle.condition_input(f, p.pos_floor),
                                                         torch.tensor(h, dtype=torch.float64), p.K), p.pos_floor)
    u0 = lib.wiener(cuda(f), cuda(h), p)
    assert_close(u0, ref, f"wiener {H}x{W} psf {shape}")


@pytest.mark.parametrize("index", [0, 1, 2, 3, 256, 257, 300, 511])
def test_uneven_batch_images_single_calls(lib, index):
    """Images of the uneven batch (non-power-of-two sides, 1D box / raised
    cosine or 2D Gaussian-mixture PSFs) through the single-image pipeline."""
    case = synth.batch_case(index)
    f, h = cuda(case.f), cuda(case.h)
    u0_ref, u_ref = oracle_pipeline(case)
    u0 = lib.wiener(f, h, case.params, kind=case.psf_kind)
    m0, r0 = assert_close(u0, u0_ref, f"{case.name} {case.f.shape} Wiener")
    u = lib.rrl_iterate(f, u0.clone(), h, case.params, case.iters, kind=case.psf_kind)
    m, r = assert_close(u, u_ref, f"{case.name} {case.f.shape} psf {case.h.shape} WR3L")
    print(f"{case.name} {case.f.shape} psf {case.h.shape}: Wiener {m0:.2e}/{r0:.2e} WR3L {m:.2e}/{r:.2e}")


def test_checkpoints_hold_intermediate_iterates(lib, sched):
    H, W = 64, 96
    h = synth.raised_cosine_1d(9)
    p = Params()
    f, u0 = _iterate_case(H, W, h, 7, p)
    ck = torch.empty(3, H, W, device="cuda")
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 7, ckpt=ck, ckpt_every=3)
    u3 = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 3)
    u6 = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6)
    assert torch.equal(ck[0], cuda(u0)) and torch.equal(ck[1], u3) and torch.equal(ck[2], u6)
    assert torch.equal(lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 7), u)


def test_device_flags_for_bad_taps(lib):
    f = cuda(np.full((32, 32), 100.0))
    p = Params()
    with pytest.raises(lib.DeblurError, match="taps"):
        lib.rrl_iterate(f, f.clone(), cuda(np.array([[0.5, -0.1, 0.6]])), p, 1)
    with pytest.raises(lib.DeblurError, match="taps"):
        lib.rrl_iterate(f, f.clone(), cuda(np.array([[0.2, 0.3, 0.1, 0.4]])), p, 1, kind="box")
    # lighter end taps are a valid box (non-integer blur length)
    lib.rrl_iterate(f, f.clone(), cuda(np.array([[0.3, 0.4, 0.3]])), p, 1, kind="box")
    with pytest.raises(lib.DeblurError):
        lib.wiener(f, cuda(np.zeros((1, 3))), p)


def test_unsupported_is_reported(lib):
    f = cuda(np.full((32, 48), 100.0))
    with pytest.raises(lib.DeblurError, match="unsupported"):
        lib.rrl_iterate(f, f.clone(), cuda(np.ones((3, 3)) / 9), Params(conv="periodic"), 1)


@pytest.mark.parametrize("maker,kind", [(lambda: synth.case_line1024(256, 320, 5), "general"),
                                        (lambda: synth.case_box256(200, 256, 4), "box_row"),
                                        (lambda: synth.batch_case(2, size_cap=300), None),
                                        (lambda: synth.case_gauss2048(256, 256, 4), "general")])
def test_plan_equals_deblur(lib, maker, kind):
    case = maker()
    kind = kind or case.psf_kind
    f, h = cuda(case.f), cuda(case.h)
    H, W = case.f.shape
    plan = lib.Plan(H, W, h, case.params, case.iters, kind=kind)
    u1 = plan.run(f)
    u2 = plan.run(f)
    ref = lib.deblur(f, h, case.params, case.iters, kind=kind)
    assert torch.equal(u1, ref) and torch.equal(u2, ref)
    plan.close()


@pytest.mark.parametrize("H,W,psf,kind", [(256, 320, "line", "general"), (77, 131, "gauss", "general"),
                                          (40, 300, "row", "general"), (300, 40, "col", "general"),
                                          (130, 300, "row", "box"), (97, 200, "rowrnd", "general")])
def test_flow_equals_split_bitwise(lib, H, W, psf, kind):
    """The persistent dependency-ordered launch runs the split schedule's tile
    bodies (tap groups, box sums or register windows), so it must reproduce
    the split result exactly."""
    rng = np.random.default_rng(H + W)
    h = {"line": synth.line_psf(31, 30.0, 32.0), "row": synth.box_psf(15), "rowrnd": synth.random_motion_1d(23, rng),
         "col": synth.raised_cosine_1d(9, "col"), "gauss": synth.gaussian_mixture_psf(9, rng)}[psf]
    p = Params()
    f, u0 = _iterate_case(H, W, h, 7, p, seed=11)
    out = {}
    lib.set_fft_tiles(2305)  # direct sums: the flow kernel runs them (FFT tiles run split)
    try:
        for knob in (1, 256):  # one-axis PSFs: register windows, then tap groups
            lib.set_one_axis_min(knob)
            for name in ("split", "flow"):
                lib.set_schedule(name)
                out[name, knob] = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 7, kind=kind)
    finally:
        lib.set_schedule("auto")
        lib.set_one_axis_min(0)
        lib.set_fft_tiles(0)
    for knob in (1, 256):
        assert torch.equal(out["split", knob], out["flow", knob])


@pytest.mark.parametrize("H,W,psf,kind,iters", [(256, 256, "box15", "box", 10), (128, 64, "rowrnd31", "general", 7),
                                                (64, 8, "box7", "box", 3), (64, 512, "rowrnd41", "general", 5),
                                                (192, 200, "box1", "box", 4), (512, 128, "row5", "general", 6),
                                                (128, 96, "box16", "box", 1), (100, 96, "box15", "box", 3)])
def test_cluster_equals_split_bitwise(lib, H, W, psf, kind, iters):
    """The cluster-resident schedule (whole image in one cluster's shared
    memory, TV halo rows through distributed shared memory) computes every
    pixel with the split schedule's one-axis device functions, so it must
    reproduce the split result exactly -- at every row split across the 8
    CTAs, for box and register-window sums, even box lengths, a box of
    length 1, one iteration, and (100 rows: not a multiple of 64) the
    fallback to the split schedule."""
    rng = np.random.default_rng(H * 7 + W)
    h = {"box15": synth.box_psf(15), "box7": synth.box_psf(7), "box1": synth.box_psf(1), "box16": synth.box_psf(16),
         "rowrnd31": synth.random_motion_1d(31, rng), "rowrnd41": synth.random_motion_1d(41, rng),
         "row5": synth.raised_cosine_1d(5)}[psf]
    p = Params()
    f, u0 = _iterate_case(H, W, h, iters, p, seed=5)
    out = {}
    try:
        lib.set_one_axis_min(1)  # the split schedule sums non-box rows with register windows too
        for name in ("split", "cluster"):
            lib.set_schedule(name)
            out[name] = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, iters, kind=kind)
    finally:
        lib.set_schedule("auto")
        lib.set_one_axis_min(0)
    assert torch.equal(out["split"], out["cluster"])
    if psf == "box15" and H == 256:  # and the oracle, at the box256 workload's PSF
        ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, iters)
        d = (out["cluster"].double().cpu() - torch.as_tensor(ref)).abs()
        assert float(d.max()) <= 1e-3 and float(d.pow(2).mean().sqrt()) <= 1e-4


def test_flow_bounded_waits_report_timeout(lib):
    """With a zero wait budget every dependency wait of the persistent launch
    gives up at once: the call returns, the status word carries the time-out
    flag (unless no wait ever found a dependency pending) and the context
    stays usable."""
    h = synth.line_psf(31, 30.0, 32.0)
    p = Params()
    f, u0 = _iterate_case(256, 256, h, 6, p, seed=2)
    ws = lib.Workspace.for_image(256, 256, h.shape[0], h.shape[1], p)
    lib.set_schedule("flow")
    lib.set_spin_limit(0)
    try:
        ws.reset_status()
        lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6, ws=ws, check=False)
        torch.cuda.synchronize()
        flags = int(ws.status.item())
    finally:
        lib.set_spin_limit(4_000_000_000)
        lib.set_schedule("auto")
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 2)
    assert torch.isfinite(u).all()
    if flags == 0:
        pytest.skip("no wait found a dependency pending")
    assert flags & 0x4, f"flags 0x{flags:x}"


@pytest.mark.parametrize("L,axis", [(15.4, "row"), (4.5, "col"), (26.9, "row"), (3.0, "row"), (1.0, "col"),
                                    (41.0, "col"), (2.5, "row")])
@pytest.mark.parametrize("H,W", [(77, 131), (64, 64), (200, 45)])
def test_box_sliding_window_matches_oracle(lib, L, axis, H, W):
    """Box PSFs, plain and of non-integer length (lighter end pixels, Sec.
    4.3): the sliding-window iterations against the oracle's direct sums."""
    h = synth.box_psf_frac(L, axis)
    if h.shape[0] > H or h.shape[1] > W:
        pytest.skip("PSF larger than image")
    p = Params()
    f, u0 = _iterate_case(H, W, h, 6, p, seed=int(L * 10))
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 6)
    u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6, kind="box")
    assert_close(u, ref, f"box L={L} {axis} {H}x{W}")
    ug = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 6)  # tap groups
    assert_close(u, ug.double().cpu().numpy(), "box vs tap groups")


def _sparse_psf(kind, rng):
    if kind == "random":      # irregular zero gaps: clusters of every length
        h = rng.uniform(0.1, 1.0, (15, 11)) * (rng.random((15, 11)) < 0.45)
    elif kind == "tall":      # columns longer than a group: split into parts
        h = rng.uniform(0.1, 1.0, (41, 3))
    elif kind == "dotted":    # taps one and two zero rows apart
        h = np.zeros((13, 5))
        h[[0, 2, 4, 7, 10, 12], :] = rng.uniform(0.1, 1.0, (6, 5))
    else:                     # checkerboard
        h = ((np.add.outer(np.arange(9), np.arange(9)) % 2) == 0) * rng.uniform(0.1, 1.0, (9, 9))
    h[h.shape[0] // 2, h.shape[1] // 2] += 0.5
    return (h / h.sum()).astype(np.float32)


@pytest.mark.parametrize("kind", ["random", "tall", "dotted", "checker"])
def test_tap_groups_of_every_height_match_oracle(lib, kind, sched):
    """PSFs whose columns cut into tap groups of every height 1..7 (zero gaps
    of one and two rows, columns longer than a group): the grouped sums
    against the oracle's direct sums, in every schedule."""
    rng = np.random.default_rng({"random": 1, "tall": 2, "dotted": 3, "checker": 4}[kind])
    h = _sparse_psf(kind, rng)
    H, W = 77, 131
    p = Params()
    f, u0 = _iterate_case(H, W, h, 4, p, seed=5)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
    lib.set_fft_tiles(2305)  # the tap groups themselves, not FFT tiles
    try:
        u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
    finally:
        lib.set_fft_tiles(0)
    assert_close(u, ref, f"{kind} {h.shape}")


@pytest.mark.parametrize("L", [1, 2, 7, 8, 9, 16, 33, 100, 255])
@pytest.mark.parametrize("axis", ["row", "col"])
def test_one_axis_register_windows_match_oracle(lib, L, axis):
    """Non-uniform one-axis PSFs with irregular weights (zeros included): the
    register-window tap sums of the split schedule against the oracle, and
    against the tap-group form of the fused schedule, on ragged shapes."""
    rng = np.random.default_rng(1000 + L)
    h = synth.random_motion_1d(L, rng, axis)
    H, W = 61, max(L, 37) + 13
    if axis == "col":
        H, W = W, H
    p = Params()
    f, u0 = _iterate_case(H, W, h, 4, p, seed=L)
    ref = oracle.rrrl(u0, oracle.condition_input(f, p.pos_floor), h, p, 4)
    lib.set_schedule("split")
    lib.set_one_axis_min(1)  # register windows at every length
    ug = None
    try:
        u = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
        lib.set_schedule("fused")
        try:  # the fused tiles hold a halo of kw columns: not every width fits
            ug = lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 4)
        except lib.DeblurError as e:
            assert "unsupported" in str(e) and L > 128
    finally:
        lib.set_schedule("auto")
        lib.set_one_axis_min(0)
    assert_close(u, ref, f"1D L={L} {axis} {H}x{W}")
    if ug is not None:
        assert_close(u, ug.double().cpu().numpy(), "register windows vs tap groups")


def test_box_full_pipeline_fractional(lib):
    """Wiener + 10 RRRL on a 256x256 image blurred by a box of length 15.4."""
    rng = np.random.default_rng(1540)
    g = synth.scene(256, 256, rng).astype(np.float32)
    h = synth.box_psf_frac(15.4)
    f = synth.degrade(g, h, 2.0, rng)
    p = Params()
    u0_ref, u_ref = oracle.wr3l(f, h, p, 10)
    u = lib.deblur(cuda(f), cuda(h), p, 10, kind="box")
    assert_close(u, u_ref, "fractional box WR3L")


@pytest.mark.parametrize("sched", ["split", "flow", "fused"])
def test_nonfinite_values_raise_the_device_flag(lib, sched):
    """A NaN in the iterate or an infinite grey value does not trap: it is
    reported through the device status word (DB_FLAG_NONFINITE) and the call
    raises on the host afterwards."""
    h = synth.line_psf(9, 30.0, 10.0)
    p = Params()
    f, u0 = _iterate_case(64, 96, h, 2, p, seed=3)
    lib.set_schedule(sched)
    try:
        u = cuda(u0)
        u[10, 20] = float("nan")
        with pytest.raises(lib.DeblurError, match="non-finite|nonfinite|NaN"):
            lib.rrl_iterate(cuda(f), u, cuda(h), p, 2)
        fi = cuda(f)
        fi[5, 5] = float("inf")
        with pytest.raises(lib.DeblurError, match="non-finite|nonfinite|NaN"):
            lib.rrl_iterate(fi, cuda(u0), cuda(h), p, 2)
    finally:
        lib.set_schedule("auto")
    assert torch.isfinite(lib.rrl_iterate(cuda(f), cuda(u0), cuda(h), p, 2)).all()
