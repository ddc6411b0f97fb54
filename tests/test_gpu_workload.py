"""Parity at the benchmarked size and launch configuration: randomized CUR-ID
of the dense float32 8000 x 6000 matrix (sigma_j = j^-2), k = 200, p = 10,
q = 1, Omega drawn on the device from a seed exactly as bench.py does.
The FP64 oracle runs the same decomposition with the same Omega."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from oracle.philox import gaussian as philox_gaussian
from parity import fro, id_residual, np64, npi

pytestmark = pytest.mark.gpu

M, N, K, P, Q = 8000, 6000, 200, 10, 1
SEED = 1413


@pytest.fixture(scope="module")
def workload():
    A = syn.spectrum_matrix(M, N, syn.power_decay(N), SEED, torch.float32, "cuda:0")
    Ah = A.cpu().numpy().astype(np.float64)
    seed = SEED * 1000
    Om = philox_gaussian(K + P, M, seed).astype(np.float32)
    o, _ = O.randomized_cur(Ah, Om, K, q=Q)
    return A, Ah, seed, o


@pytest.mark.parametrize("tf32", [False, True])
def test_full_size_cur(workload, tf32):
    A, Ah, seed, o = workload
    r = curid.cur(A, K, p=P, q=Q, seed=seed, tf32=tf32, want_c=True, want_r=True, want_t=True)
    assert r.status == 0 and r.k == K
    J, I = npi(r.J), npi(r.I)
    assert sorted(J) == list(range(N)) and sorted(I) == list(range(M))
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:K]]) and np.array_equal(R, Ah[I[:K], :])
    # skeleton quality against the oracle's (pivot gaps here are far below
    # FP32 rounding, so the index sets are compared through their residuals)
    assert id_residual(Ah, J, T, K) <= 1.05 * id_residual(Ah, o.J, o.T, K)
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    # the FP32 criterion on the CUR error itself: within 1e-5 of the oracle's
    assert abs(eg - eo) <= 1e-5, (eg, eo)
    # U precision on the GPU's own skeleton: FP64 least squares on the same J, T, I
    Uo = O.cur_middle(R, O.vstar(J, T, N))
    assert abs(eg - O.rel_err_fro(Ah, C, Uo, R)) <= 1e-5


def test_full_size_sampled_sketch(workload):
    """Sampled rows of Y = Omega A against the oracle computed one by one."""
    A, Ah, seed, o = workload
    l = K + P
    Om = curid.gaussian(l, M, seed, dtype=torch.float32, device=0)
    Y = curid.sketch_matrix(A, Om, q=0)
    Omh = np64(Om)
    rows = [0, 1, 77, 150, l - 1]
    for r in rows:
        ref = Omh[r] @ Ah
        np.testing.assert_allclose(np64(Y[r]), ref, atol=2e-5 * np.abs(ref).max() * 10, rtol=0)
