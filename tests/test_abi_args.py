"""Argument checks of the C ABI that return before any device work, so they run without a GPU:
every entry point answers a bad argument with a status (never a crash), creation leaves *out NULL
and explains itself through hz_last_error(NULL), and non-finite or non-positive medium values are
rejected while the medium is read on the host."""
import ctypes as ct

import numpy as np
import pytest

from paper_1801_08655_gb300 import build, hz


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hz.load()


def _create(lib, n=12, npml=2, L=2, omega=1.0, prec=1, m=None, b=None, grid=True, pml=True):
    m = np.ones((n, n, n)) if m is None else m
    g = hz.Grid(n, n, n, 1.0)
    p = hz.Pml(npml, 10.0, -1)
    out = ct.c_void_p(1234)
    st = lib.hz_create_ex(ct.byref(g) if grid else None, m.ctypes.data,
                          b.ctypes.data if b is not None else None, omega, ct.byref(p) if pml else None, L, prec,
                          None, ct.byref(out))
    return st, out.value, lib.hz_last_error(None).decode()


@pytest.mark.parametrize("kw,word", [
    (dict(grid=False), "null"), (dict(pml=False), "null"), (dict(n=2), "grid"),
    (dict(omega=0.0), "omega"), (dict(omega=-1.0), "omega"), (dict(omega=float("inf")), "omega"),
    (dict(npml=-1), "pml"), (dict(prec=7), "precision"), (dict(L=0), "n_layers"), (dict(L=9), "n_layers"),
])
def test_create_rejects_bad_arguments(lib, kw, word):
    st, out, msg = _create(lib, **kw)
    assert st == hz.HZ_ERR_ARG and out is None and word in msg


def test_create_rejects_bad_medium(lib):
    m = np.ones((12, 12, 12))
    m[3, 4, 5] = np.nan
    st, out, msg = _create(lib, m=m)
    assert st == hz.HZ_ERR_NONFINITE and out is None and "m" in msg
    b = np.ones((12, 12, 12))
    b[1, 2, 3] = 0.0
    st, out, msg = _create(lib, b=b)
    assert st == hz.HZ_ERR_ARG and out is None and "positive" in msg
    b[1, 2, 3] = np.inf
    st, out, msg = _create(lib, b=b)
    assert st == hz.HZ_ERR_NONFINITE and out is None


def test_null_handles_are_statuses(lib):
    ARG = hz.HZ_ERR_ARG
    i64, d, f = ct.c_int64(), ct.c_double(), ct.c_float()
    assert lib.hz_factor(None) == ARG
    assert lib.hz_solve(None, None, 1, None, None, None) == ARG
    assert lib.hz_solve_host(None, None, 1, None, None, None) == ARG
    assert lib.hz_trace_blocks(None, 4, ct.byref(i64)) == ARG and i64.value == 0
    assert lib.hz_layer_solve(None, 0, None, 1, None) == ARG
    assert lib.hz_apply_mpol(None, None, 1, None) == ARG
    assert lib.hz_apply_precond(None, None, 1, None) == ARG
    assert lib.hz_volume_residual(None, None, None, 1, None, None) == ARG
    assert lib.hz_volume_residual_noalloc(None, None, None, 1, None, None) == ARG
    assert lib.hz_layer_info(None, 0, None, None, None, None) == ARG
    assert lib.hz_factor_stats(None, None, None, None, None, None) == ARG
    assert lib.hz_profile_kernel(None, 0, None, None, None, None) == ARG
    assert lib.hz_profile_end(None, None, None, None, None) == ARG
    out = ct.c_void_p(99)
    assert lib.hz_create_shared(None, None, ct.byref(out)) == ARG and out.value is None
    assert lib.hz_destroy(None) == hz.HZ_OK


def test_group_solve_rejects_missing_handles(lib):
    hs = (ct.c_void_p * 2)(None, None)
    rp = (ct.c_void_p * 2)(None, None)
    Rs = (ct.c_int32 * 2)(1, 1)
    sts = (ct.c_int * 2)()
    assert lib.hz_solve_group(hs, 1, rp, Rs, rp, None, None, sts) == hz.HZ_ERR_ARG
    assert lib.hz_solve_group(hs, 2, rp, Rs, rp, None, None, sts) == hz.HZ_ERR_ARG
    assert lib.hz_solve_group(None, 1, rp, Rs, rp, None, None, sts) == hz.HZ_ERR_ARG
    assert lib.hz_solve_group(hs, 0, rp, Rs, rp, None, None, sts) == hz.HZ_ERR_ARG


def test_create_without_a_device_is_a_cuda_status(lib):
    """With valid arguments but no usable GPU the first device allocation fails: a status
    (HZ_ERR_CUDA, not HZ_ERR_OOM: nothing ran out of memory) with the runtime's reason."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, out, msg = _create(lib)
    assert st == hz.HZ_ERR_CUDA and out is None and "allocation" in msg
