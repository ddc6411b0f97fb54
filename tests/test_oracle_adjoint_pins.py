"""CPU pins of the adjoint oracle (oracle/adjoint.py): the reverse-mode
derivative of the CUR-ID with frozen skeletons (T = C^+ B, Eq. (2.8);
U = V* R^+, Eq. (3.5)) against central finite differences and against float64
torch autograd through an independent forward written with normal-equation
solves."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as syn
from oracle.adjoint import cur_adjoint, cur_frozen, cur_loss_grad


def skeletons(A, k):
    r = O.cur(A, k=k)
    return np.asarray(r.J), np.asarray(r.I)


def pairing(A, J, I, k, Cb, Ub, Rb):
    C, U, R, _ = cur_frozen(A, J, I, k)
    return float(np.sum(Cb * C) + np.sum(Ub * U) + np.sum(Rb * R))


@pytest.mark.parametrize("m,n,k,seed", [(14, 10, 4, 1), (9, 12, 5, 2), (11, 7, 7, 3)])
def test_adjoint_matches_central_differences(m, n, k, seed):
    """Every entry of Abar against a central difference of the pairing
    <Cbar, C> + <Ubar, U> + <Rbar, R> (k = n = 7 in the last case: no
    residual columns, R square)."""
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 3.0), seed).numpy()
    J, I = skeletons(A, k)
    g = np.random.default_rng(seed + 100)
    Cb, Ub, Rb = g.standard_normal((m, k)), g.standard_normal((k, k)), g.standard_normal((k, n))
    Ab = cur_adjoint(A, J, I, k, Cb, Ub, Rb)
    h = 1e-6
    fd = np.zeros_like(A)
    for i in range(m):
        for j in range(n):
            E = np.zeros_like(A)
            E[i, j] = h
            fd[i, j] = (pairing(A + E, J, I, k, Cb, Ub, Rb)
                        - pairing(A - E, J, I, k, Cb, Ub, Rb)) / (2 * h)
    assert np.max(np.abs(fd - Ab)) <= 1e-6 * np.max(np.abs(Ab)), np.max(np.abs(fd - Ab))


@pytest.mark.parametrize("m,n,k,seed", [(30, 20, 6, 4), (25, 40, 8, 5)])
def test_adjoint_matches_torch_autograd(m, n, k, seed):
    """Abar against torch autograd of T = (C^T C)^{-1} C^T B and
    U = V* R^T (R R^T)^{-1} (an independent derivation of the same maps)."""
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 5.0), seed).numpy()
    J, I = skeletons(A, k)
    g = np.random.default_rng(seed + 200)
    Cb, Ub, Rb = g.standard_normal((m, k)), g.standard_normal((k, k)), g.standard_normal((k, n))
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    Jt, It = torch.tensor(J), torch.tensor(I)
    C = At[:, Jt[:k]]
    B = At[:, Jt[k:]]
    R = At[It[:k], :]
    T = torch.linalg.solve(C.T @ C, C.T @ B)
    Vs = torch.zeros((k, n), dtype=torch.float64)
    Vs = Vs.index_put((torch.arange(k), Jt[:k]), torch.ones(k, dtype=torch.float64))
    Vs = Vs.index_put((torch.arange(k)[:, None], Jt[k:][None, :]), T)
    U = Vs @ R.T @ torch.linalg.inv(R @ R.T)
    f = (torch.tensor(Cb) * C).sum() + (torch.tensor(Ub) * U).sum() + (torch.tensor(Rb) * R).sum()
    f.backward()
    Ab = cur_adjoint(A, J, I, k, Cb, Ub, Rb)
    ref = At.grad.numpy()
    assert np.linalg.norm(Ab - ref) <= 1e-10 * np.linalg.norm(ref)


def test_loss_gradient_matches_central_differences():
    """Gradient of 1/2 ||A - C U R||_F^2 (frozen skeletons) on 64 seeded
    entries and two random directions."""
    m, n, k = 24, 18, 5
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 4.0), 7).numpy()
    J, I = skeletons(A, k)
    grad, _ = cur_loss_grad(A, J, I, k)

    def loss(X):
        C, U, R, _ = cur_frozen(X, J, I, k)
        D = X - C @ U @ R
        return 0.5 * float(np.sum(D * D))

    g = np.random.default_rng(8)
    h = 1e-6
    idx = g.choice(m * n, 64, replace=False)
    for e in idx:
        i, j = divmod(int(e), n)
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E) - loss(A - E)) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-6 * np.max(np.abs(grad)) + 1e-12
    for _ in range(2):
        D = g.standard_normal(A.shape)
        D /= np.linalg.norm(D)
        fd = (loss(A + h * D) - loss(A - h * D)) / (2 * h)
        assert abs(fd - np.sum(grad * D)) <= 1e-6 * np.linalg.norm(grad)


def test_frozen_forward_reproduces_cur():
    """cur_frozen on the oracle's own skeletons gives the oracle's T and U
    (T = C^+ B equals S11^{-1} S12 of the deterministic column ID)."""
    A = syn.spectrum_matrix(40, 30, syn.exp_decay(30, 6.0), 9).numpy()
    k = 8
    r = O.cur(A, k=k)
    C, U, R, T = cur_frozen(A, r.J, r.I, k)
    assert np.array_equal(C, r.C) and np.array_equal(R, r.R)
    assert np.linalg.norm(T - r.T) <= 1e-10 * np.linalg.norm(r.T)
    assert np.linalg.norm(U - r.U) <= 1e-10 * np.linalg.norm(r.U)
