"""pff_apply_laplacian_noalloc, the Laplacian entry point for callers that cannot
allocate device memory (for example a framework that has reserved all of it
for its own pool): its output matches the allocating entry point
pff_apply_laplacian on two calls in a row, and oversized grids are rejected
before any launch.  Collected last on purpose (file name): every other test has
run before it when a run stops at the first failure."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2203_16467_gb300 import pff
    assert torch.cuda.is_available()
    return pff, torch


def _call(pff, nx, ny, dx, src, dst, stream):
    msg = ctypes.c_char_p()
    rc = pff.lib.pff_apply_laplacian_noalloc(nx, ny, dx, ctypes.c_void_p(src.data_ptr()),
                                             ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(stream),
                                             ctypes.byref(msg))
    return rc, (msg.value.decode() if msg.value else None)


@pytest.mark.parametrize("ny,nx", [(64, 64), (32, 128), (512, 512)])
def test_noalloc_matches_allocating_entry_point_twice(env, ny, nx):
    pff, torch = env
    dx = 0.75
    stream = torch.cuda.Stream()
    ref_problem = pff.Problem(nx, ny, pff.FP64)
    ref_problem.set_params(dx=dx)
    rng = np.random.default_rng(nx + ny)
    for call in range(2):   # two calls in a row share the static scratch
        g = rng.standard_normal((ny, nx)) + np.sin(2 * np.pi * np.arange(nx) / nx)[None, :]
        src = torch.tensor(g, dtype=torch.float64, device="cuda")
        dst = torch.full((ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            rc, msg = _call(pff, nx, ny, dx, src, dst, stream.cuda_stream)
        stream.synchronize()
        assert rc == pff.OK, msg
        out = dst.cpu().numpy()
        ref = ref_problem.apply_laplacian(g)
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err < 1e-12, (call, err)
    ref_problem.close()


def test_noalloc_rejects_grids_beyond_the_limit(env):
    pff, torch = env
    big = 2 * 512
    src = torch.zeros(16, dtype=torch.float64, device="cuda")
    dst = torch.zeros(16, dtype=torch.float64, device="cuda")
    launches = pff.kernel_launches()
    rc, msg = _call(pff, big, 64, 1.0, src, dst, None)
    assert rc == pff.ERR_INVALID_ARG and "512" in msg
    rc, msg = _call(pff, 48, 64, 1.0, src, dst, None)
    assert rc == pff.ERR_INVALID_ARG
    assert pff.kernel_launches() == launches   # nothing was launched


@pytest.mark.parametrize("ny,nx", [(64, 64), (32, 128), (512, 512)])
def test_noalloc_f32_matches_the_fp64_entry(env, ny, nx):
    # the FP32 entry runs the mixed-precision kernels on caller-owned FP32 fields:
    # within FP32 rounding of the FP64 entry's result on the same input
    pff, torch = env
    dx = 0.5
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(3 * nx + ny)
    g = rng.standard_normal((ny, nx))
    src64 = torch.tensor(g, dtype=torch.float64, device="cuda")
    dst64 = torch.empty_like(src64)
    src32 = src64.float()
    dst32 = torch.full((ny, nx), float("nan"), dtype=torch.float32, device="cuda")
    msg = ctypes.c_char_p()
    with torch.cuda.stream(stream):
        rc, m = _call(pff, nx, ny, dx, src64, dst64, stream.cuda_stream)
        assert rc == pff.OK, m
        for _ in range(2):
            rc = pff.lib.pff_apply_laplacian_noalloc_f32(nx, ny, dx, ctypes.c_void_p(src32.data_ptr()),
                                                         ctypes.c_void_p(dst32.data_ptr()),
                                                         ctypes.c_void_p(stream.cuda_stream), ctypes.byref(msg))
            assert rc == pff.OK, msg.value
    stream.synchronize()
    ref = dst64.cpu().numpy()
    out = dst32.double().cpu().numpy()
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 2e-6
    big = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = pff.lib.pff_apply_laplacian_noalloc_f32(1024, 64, 1.0, ctypes.c_void_p(big.data_ptr()),
                                                 ctypes.c_void_p(big.data_ptr()), None, ctypes.byref(msg))
    assert rc == pff.ERR_INVALID_ARG and b"512" in msg.value
