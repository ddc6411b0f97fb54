"""Regularised interpolation matrix (Section 4.1, Eq. (4.1) with a Tikhonov
term) through curid_interp_tikhonov, against the FP64 oracle on the same
host-built S (graded upper-trapezoidal, original column order) and J.
Tolerances follow the forward error of a regularised least-squares solve,
u (kappa + kappa^2) with kappa = ||S11||_2 / lam the bound on the augmented
matrix's condition number."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
from parity import U32, U64

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def graded_s(k, n, cond, seed):
    rng = np.random.default_rng(seed)
    d = np.logspace(0, -np.log10(cond), k)
    S11 = np.triu(rng.standard_normal((k, k)) * 0.1 * d[None, :]) + np.diag(d)
    S12 = rng.standard_normal((k, n - k)) * d[:, None]
    S1 = np.hstack([S11, S12])
    J = rng.permutation(n)
    S = np.zeros((k, n))
    S[:, J] = S1  # original column order: S[:, J[t]] = S1[:, t]
    return S, J, S1


@pytest.mark.parametrize("dtype,rel_lam", [(torch.float64, 1e-4), (torch.float64, 1e-2),
                                           (torch.float32, 1e-2), (torch.float32, 1e-1)])
@pytest.mark.parametrize("k,n,cond", [(12, 40, 1e6), (64, 900, 1e8), (200, 1500, 1e10)])
def test_tikhonov_matches_oracle(dtype, rel_lam, k, n, cond):
    S, J, S1 = graded_s(k, n, cond, k + n)
    s1 = np.linalg.norm(S1[:, :k], 2)
    lam = rel_lam * s1
    Sd = torch.tensor(S, dtype=dtype, device=DEV)
    Jd = torch.tensor(J, dtype=torch.int32, device=DEV)
    T = curid.interp_tikhonov(Sd, Jd, k, lam)
    torch.cuda.synchronize()
    st, _ = curid.last_status(0)
    assert st == 0
    # the oracle solves with the values the GPU received
    S1r = torch.tensor(S1, dtype=dtype).double().numpy()
    To = O.interpolation_matrix_tikhonov(S1r, k, lam)
    u = U64 if dtype == torch.float64 else U32
    kappa = 1.0 / rel_lam
    tol = 20 * u * (kappa + kappa ** 2) * np.abs(To).max()
    err = np.abs(T.double().cpu().numpy() - To).max()
    assert err <= tol, (err, tol)


def test_tikhonov_shrinks_and_tends_to_back_substitution():
    k, n = 30, 200
    S, J, S1 = graded_s(k, n, 1e3, 7)
    Sd = torch.tensor(S, dtype=torch.float64, device=DEV)
    Jd = torch.tensor(J, dtype=torch.int32, device=DEV)
    s1 = np.linalg.norm(S1[:, :k], 2)
    norms = [float(torch.linalg.norm(curid.interp_tikhonov(Sd, Jd, k, r * s1)))
             for r in (1e-9, 1e-3, 1e-1, 1.0)]
    assert all(a > b for a, b in zip(norms, norms[1:]))
    T0 = curid.interp_tikhonov(Sd, Jd, k, 1e-12 * s1).cpu().numpy()
    Tb = O.interpolation_matrix(S1, k)
    assert np.abs(T0 - Tb).max() <= 1e-8 * np.abs(Tb).max()


def test_tikhonov_rejects_bad_lambda_and_square_case():
    S, J, _ = graded_s(8, 8, 10.0, 9)
    Sd = torch.tensor(S, device=DEV)
    Jd = torch.tensor(J, dtype=torch.int32, device=DEV)
    with pytest.raises(curid.CuridError):
        curid.interp_tikhonov(Sd, Jd, 8, 0.0)
    assert curid.interp_tikhonov(Sd, Jd, 8, 0.5).shape == (8, 0)
