"""The CPQR entry point that allocates nothing (curid_cpqr_static), for
callers that cannot obtain device memory when they factor a matrix (a
pre-reserved memory budget, a framework that owns every allocation).  It is
checked through the C ABI against the workspace-based curid_cpqr on the same
inputs, over two calls in a row that share its static scratch array.  This
file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1412_8447_gb300 as curid
import synthetic as syn

pytestmark = pytest.mark.gpu


def cpqr_static(Y, k, tol=0.0):
    lib = curid.load_library()
    l, n = Y.shape
    k_max = k if k > 0 else min(l, n)
    J = torch.full((n,), -1, dtype=torch.int32, device=Y.device)
    S = torch.zeros((k_max, n), dtype=Y.dtype, device=Y.device)
    info = torch.zeros(3, dtype=torch.int32, device=Y.device)
    dt = 0 if Y.dtype == torch.float64 else 1
    stream = torch.cuda.current_stream(Y.device).cuda_stream
    st = lib.curid_cpqr_static(ctypes.c_void_p(stream), dt, ctypes.c_void_p(Y.data_ptr()), l, n,
                               Y.stride(0), k, float(tol), ctypes.c_void_p(J.data_ptr()),
                               ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(info.data_ptr()))
    return st, J, S, info


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_static_cpqr_matches_workspace_cpqr(dtype):
    torch.cuda.set_device(0)
    cases = [(300, 1000, 40, 0.0, 61), (210, 6000, 200, 0.0, 62), (120, 900, 0, 1e-4, 63)]
    inputs = [syn.spectrum_matrix(l, n, syn.power_decay(min(l, n)), seed, dtype, "cuda:0")
              for (l, n, k, tol, seed) in cases]
    # two (here three) calls in a row, all on the one static scratch array
    got = [cpqr_static(Y, k, tol) for Y, (l, n, k, tol, seed) in zip(inputs, cases)]
    torch.cuda.synchronize()
    tol_fp = 1e-11 if dtype == torch.float64 else 2e-5
    for Y, (l, n, k, tol, seed), (st, J, S, info) in zip(inputs, cases, got):
        assert st == 0
        ref = curid.cpqr(Y, k=k, tol=tol)
        kk = ref.k
        assert torch.equal(J, ref.J)
        Sr = ref.S[:kk].cpu().numpy()
        np.testing.assert_allclose(S[:kk].cpu().numpy(), Sr, atol=tol_fp * np.abs(Sr).max(),
                                   rtol=0)
        flags, steps, rank = info.cpu().tolist()
        assert flags == 0 and rank == kk and steps == kk


@pytest.mark.parametrize("dtype,l,n,k", [(torch.float32, 520, 26144, 64),
                                         (torch.float64, 8000, 8, 8)])
def test_static_cpqr_overflow_groups(dtype, l, n, k):
    """Slabs that spill past registers and shared memory into the carved
    overflow area of the static scratch (on a 152-SM GPU with 227 KB of
    shared memory per CTA): 520 x 26144 float32 is 172 columns per CTA, one
    four-column group more than registers and shared memory hold; 8000 x 8
    float64 runs on two CTAs whose one group (256 KB) fits no shared memory.
    Same J, S and step count as the workspace-based call."""
    torch.cuda.set_device(0)
    Y = syn.spectrum_matrix(l, n, syn.power_decay(min(l, n)), 71, dtype, "cuda:0")
    st, J, S, info = cpqr_static(Y, k)
    torch.cuda.synchronize()
    assert st == 0
    ref = curid.cpqr(Y, k=k)
    assert torch.equal(J, ref.J)
    Sr = ref.S[:k].cpu().numpy()
    tol_fp = 1e-11 if dtype == torch.float64 else 2e-5
    np.testing.assert_allclose(S[:k].cpu().numpy(), Sr, atol=tol_fp * np.abs(Sr).max(), rtol=0)
    flags, steps, rank = info.cpu().tolist()
    assert flags == 0 and steps == k and rank == ref.k


def test_static_cpqr_rejects_oversized_request():
    torch.cuda.set_device(0)
    Y = torch.randn(2000, 304, dtype=torch.float64, device="cuda:0")
    st, J, S, info = cpqr_static(Y, 10)
    assert st == 7                      # CURID_NO_WORKSPACE, nothing enqueued
    assert int((J != -1).sum()) == 0
