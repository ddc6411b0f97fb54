"""Truncated-SVD interpolation matrix (Section 4.1) through
curid_interp_tsvd (one-sided Jacobi SVD on the GPU), against the FP64
oracle on the same host-built S: S11 with planted singular values, a clear
gap around the cut, odd and even orders up to the 256 limit."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
from parity import U32, U64

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def planted_s(k, n, kept_lo, dropped_hi, ndrop, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((k, k)))
    Q2, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.concatenate([np.logspace(0, np.log10(kept_lo), k - ndrop),
                        np.logspace(np.log10(dropped_hi), np.log10(dropped_hi) - 2, ndrop)])
    S1 = np.hstack([Q1 @ np.diag(s) @ Q2.T, rng.standard_normal((k, n - k))])
    J = rng.permutation(n)
    S = np.zeros((k, n))
    S[:, J] = S1
    return S, J, S1


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,n", [(12, 40), (101, 700), (200, 1500), (256, 900)])
def test_tsvd_matches_oracle(dtype, k, n):
    if dtype == torch.float64:
        kept_lo, dropped_hi, rtol, u = 1e-4, 1e-8, 1e-6, U64
    else:
        kept_lo, dropped_hi, rtol, u = 1e-2, 1e-5, 1e-3, U32
    S, J, S1 = planted_s(k, n, kept_lo, dropped_hi, max(1, k // 10), k + n)
    Sd = torch.tensor(S, dtype=dtype, device=DEV)
    Jd = torch.tensor(J, dtype=torch.int32, device=DEV)
    T = curid.interp_tsvd(Sd, Jd, k, rtol)
    torch.cuda.synchronize()
    S1r = torch.tensor(S1, dtype=dtype).double().numpy()  # the values the GPU received
    To = O.interpolation_matrix_tsvd(S1r, k, rtol)
    kappa = 1.0 / kept_lo
    err = np.abs(T.double().cpu().numpy() - To).max()
    tol = 1e3 * u * kappa * np.abs(To).max()
    assert err <= tol, (err, tol)


def test_tsvd_well_conditioned_is_back_substitution():
    k, n = 64, 300
    rng = np.random.default_rng(5)
    S11 = np.triu(rng.standard_normal((k, k)) * 0.1) + np.diag(np.linspace(1.0, 0.5, k))
    S1 = np.hstack([S11, rng.standard_normal((k, n - k))])
    J = rng.permutation(n)
    S = np.zeros((k, n))
    S[:, J] = S1
    T = curid.interp_tsvd(torch.tensor(S, device=DEV), torch.tensor(J, dtype=torch.int32,
                                                                    device=DEV), k, 0.0)
    Tb = O.interpolation_matrix(S1, k)
    assert np.abs(T.cpu().numpy() - Tb).max() <= 1e-11 * np.abs(Tb).max()


def test_tsvd_rejects_bad_arguments():
    S = torch.zeros((4, 10), dtype=torch.float64, device=DEV)
    J = torch.arange(10, dtype=torch.int32, device=DEV)
    with pytest.raises(curid.CuridError):
        curid.interp_tsvd(S, J, 4, 1.0)
    S = torch.zeros((300, 400), dtype=torch.float64, device=DEV)
    J = torch.arange(400, dtype=torch.int32, device=DEV)
    with pytest.raises(curid.CuridError):
        curid.interp_tsvd(S, J, 300, 1e-6)
