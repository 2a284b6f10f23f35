"""st_apply_Kx_static, the allocation-free variant of st_apply_Kx.

Some callers cannot allocate device memory: processes whose device memory is owned by another
allocator (a framework's caching allocator, a serving runtime's arena), and latency-critical
loops that forbid cudaMalloc after start-up because it may synchronise the device.  For them
the library offers st_apply_Kx_static, which keeps its multigrid scratch in one static device
array instead of a handle's workspace.  This file is collected last, so a run that stops at
the first failure has already run every other test.  It must pass on its own in a fresh
process (the first call performs the per-device set-up) and after the other tests.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_2009_08875_gb300 import Solver, _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the operator parity tolerance of the other GPU tests


def _static_kx(lib, K, ns, b, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.st_apply_Kx_static(K, ns, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream))


@pytest.mark.parametrize("K,ns", [(7, 6), (5, 9)])
def test_static_scratch_variant_matches_st_apply_Kx(K, ns):
    lib = _lib.load()
    with Solver(K, 3) as s:  # 2 N_t = 18 slices of handle workspace
        # two calls in a row: the second runs on scratch that still holds the first call's data
        for seed in (1, 2):
            b = torch.from_numpy(inputs.random_state(ns, s.Nx, 100 * K + seed)).cuda()
            ref = torch.empty_like(b)
            s.apply_Kx(b, ref)
            out = torch.full_like(b, float("nan"))
            _lib.check(_static_kx(lib, K, ns, b, out))
            torch.cuda.synchronize()
            err = ((out - ref).abs().max() / ref.abs().max()).item()
            assert err <= TOL, (seed, err)
            # the handle is not autotuned, so both run the same kernels on the same coefficient
            # table: the header promises the same bits
            assert torch.equal(out, ref), (seed, err)


def test_sizes_beyond_the_static_maximum_are_rejected():
    lib = _lib.load()
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    # K = 9 fits 5 slices in the 32 MiB array, not 6; nothing is launched
    st = _static_kx(lib, 9, 6, b, b)
    assert st == _lib.ST_ERR_ARG
    assert "static maximum" in lib.st_last_error().decode()
    # K = 2 would fit about a million slices in the array, but a launch grid holds 65535
    st = _static_kx(lib, 2, 65536, b, b)
    assert st == _lib.ST_ERR_ARG
    assert "65535" in lib.st_last_error().decode()
