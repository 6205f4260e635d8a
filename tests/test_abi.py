"""CPU checks of the C ABI: the library builds, loads and exports every
function include/libdeblur.h declares; argument errors are reported
synchronously without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1212_2245_b300 import _lib, build
from paper_1212_2245_b300.params import Params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(db_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("db_wiener", "db_rrl_iterate", "db_deblur", "db_workspace_bytes", "db_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(_lib.SIGNATURES), "binding misses a declared function"


def test_status_strings_and_version(lib):
    assert lib.db_status_string(0) == b"ok"
    assert b"sm_103a" in lib.db_version()
    assert lib.db_status_from_flags(0) == 0
    assert lib.db_status_from_flags(_lib.FLAG_TIMEOUT) == 7
    assert lib.db_status_from_flags(_lib.FLAG_TAPS) == 9
    assert lib.db_status_from_flags(_lib.FLAG_NONFINITE) == 8


def _args(H=64, W=64, kh=1, kw=15, **pk):
    p = Params(**pk)
    from paper_1212_2245_b300 import _db_params
    return _lib.DbPsf(kh, kw, 0, 0x1000), _db_params(p)


def test_workspace_query(lib):
    psf, p = _args()
    n = lib.db_workspace_bytes(256, 256, ctypes.byref(psf), ctypes.byref(p))
    assert n >= 256 * 256 * 4
    assert lib.db_workspace_bytes(0, 256, ctypes.byref(psf), ctypes.byref(p)) == 0
    big = _lib.DbPsf(1, 300, 0, 0x1000)
    assert lib.db_workspace_bytes(256, 512, ctypes.byref(big), ctypes.byref(p)) == 0


def test_argument_errors_are_synchronous(lib):
    """Invalid arguments return a status before anything is enqueued (fake,
    never-dereferenced device addresses are fine: nothing is launched)."""
    psf, p = _args()
    fake_f, fake_u, ws = 0x10000, 0x20000, 0x40000
    call = lambda **kw: lib.db_rrl_iterate(kw.get("f", fake_f), kw.get("u", fake_u), kw.get("H", 64),  # noqa: E731
                                           kw.get("W", 64), kw.get("ld", 64), ctypes.byref(kw.get("psf", psf)),
                                           ctypes.byref(kw.get("p", p)), kw.get("iters", 3), None, 0,
                                           kw.get("ws", ws), kw.get("wsb", 1 << 30), None, None)
    assert call(f=0) == 1                       # NULL pointer
    assert call(H=0) == 2 and call(ld=10) == 2  # shape
    assert call(psf=_lib.DbPsf(1, 65, 0, 0x1000)) == 3  # PSF wider than image
    assert call(psf=_lib.DbPsf(3, 3, 1, 0x1000)) == 3   # box PSF not on one axis
    assert call(ws=0x40001) == 4 and call(wsb=16) == 4  # workspace
    assert call(iters=-1) == 1
    bad = _args(K=0.0)[1]
    assert call(p=bad) == 1
    assert call(f=fake_u) == 1                  # f aliases u


def test_process_wide_knobs_validate_their_arguments(lib):
    for bad in (-1, 5, 99):
        assert lib.db_set_schedule(bad) == 1
    for good in (4, 0):  # the cluster schedule, then back to auto
        assert lib.db_set_schedule(good) == 0
    for bad in (-1, 257, 1000):
        assert lib.db_set_one_axis_min(bad) == 1
    for good in (1, 16, 256, 0):
        assert lib.db_set_one_axis_min(good) == 0
    for bad in (-1, 102):
        assert lib.db_set_dense_min(bad) == 1
    assert lib.db_set_dense_min(0) == 0
    assert lib.db_set_fft_tiles(-1) == 1
    assert lib.db_set_fft_tiles(0) == 0
    for bad in (-1, 2):
        assert lib.db_set_batch_order(bad) == 1
        assert lib.db_set_tma(bad) == 1
    assert lib.db_set_batch_order(1) == 0
    assert lib.db_set_tma(1) == 0


def test_host_path_arguments_are_checked_before_any_cuda_call(lib):
    """db_plan_run_host and db_host_alloc reject null or empty arguments
    synchronously (no plan, no allocation, nothing enqueued)."""
    fake = 0x10000
    assert lib.db_plan_run_host(None, fake, fake, fake, fake + 64, None, None) == 1
    out = ctypes.c_void_p(123)
    assert lib.db_host_alloc(0, ctypes.byref(out)) == 1 and out.value is None
    assert lib.db_host_alloc(16, None) == 1
    lib.db_host_free(None)  # a null pointer is ignored
