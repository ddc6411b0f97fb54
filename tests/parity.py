"""Comparison helpers shared by the GPU parity tests (no GPU needed to
import).  Every expected value comes from ``oracle``."""
import numpy as np
import torch

import oracle as O

U64 = np.finfo(np.float64).eps / 2
U32 = float(np.finfo(np.float32).eps) / 2


def np64(t):
    if isinstance(t, torch.Tensor):
        return t.detach().cpu().to(torch.float64).numpy()
    return np.asarray(t, dtype=np.float64)


def npi(t):
    return t.detach().cpu().numpy().astype(np.int64)


def fro(X):
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def gap_allows_exact(qr, k, u):
    """Pivot order is fixed to working precision when every step's relative
    gap between the two largest candidate norms exceeds 1e3 * u * kappa,
    kappa = nu_1 / nu_k."""
    nu = qr.nu[:k]
    if k == 0 or nu[-1] <= 0:
        return False
    kappa = nu[0] / nu[-1]
    return float(np.min(qr.gaps[:k])) > 1e3 * u * kappa


def id_residual(A, J, T, k):
    """||A - A(:, J[:k]) V*||_F / ||A||_F in float64."""
    A = np64(A)
    V = O.vstar(np.asarray(J), np64(T), A.shape[1])
    return fro(A - A[:, np.asarray(J)[:k]] @ V) / fro(A)


def s_by_column(S1, J, n):
    """Oracle S1 (columns in pivot order) -> original column order."""
    out = np.zeros((S1.shape[0], n))
    out[:, np.asarray(J)] = S1
    return out


def assert_s_rows_match(S_gpu, S_orc_by_col, k, rtol):
    """Rows of S agree up to a sign per row (the Householder sign is free)."""
    Sg = np64(S_gpu)[:k]
    So = S_orc_by_col[:k]
    scale = np.abs(So).max()
    for i in range(k):
        j = np.argmax(np.abs(So[i]))
        sgn = np.sign(So[i, j]) * np.sign(Sg[i, j])
        np.testing.assert_allclose(sgn * Sg[i], So[i], atol=rtol * scale, rtol=0)
