"""FP64 CPU oracle for the adjoint (reverse-mode derivative) of the CUR-ID
with the skeletons frozen.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The decomposition of Algorithm 3 is differentiable once the index sets J
(columns) and I (rows) are held fixed: with C = A(:, J[:k]), B = A(:, J[k:])
and R = A(I[:k], :),

  * T = S11^{-1} S12 of the deterministic column ID equals C^+ B
    (A P = Q [S11 S12; 0 S22] gives C = Q1 S11 and Q1^* B = S12), i.e. the
    least-squares solution of C T = B (Section 2.3, Eq. (2.8));
  * U = V* R^+ with V* = [I T] P^* (Eq. (3.5)), R of full row rank.

Given cotangents (Cbar, Ubar, Rbar) of the outputs (C, U, R), this module
returns Abar, the gradient with respect to A of <Cbar, C> + <Ubar, U> +
<Rbar, R>.  The steps follow the chain rule through those two definitions:

  1. U = V* R^+:  Vsbar = Ubar R^{+T};  with M = V Ubar (V = (V*)^T),
     Rbar += -R^{+T} M R^{+T} + (R R^T)^{-1} M^T (I - R^+ R)
     (the derivative of R^+ for full row rank R);
  2. Tbar = Vsbar(:, J[k:]);
  3. T = (C^T C)^{-1} C^T B:  K = (C^T C)^{-1} Tbar,
     Cbar += (B - C T) K^T - C K T^T,  Bbar = C K;
  4. Abar = Cbar scattered to columns J[:k] + Bbar scattered to columns
     J[k:] + Rbar scattered to rows I[:k] (overlapping entries add).

Pinned in ``tests/test_oracle_pins.py`` by central finite differences of the
frozen-skeleton map and by float64 torch autograd through an independent
forward written with ``torch.linalg`` solves.
"""
import numpy as np
import scipy.linalg

__all__ = ["cur_frozen", "cur_adjoint", "cur_loss_grad"]


def cur_frozen(A, J, I, k):
    """Forward map with frozen skeletons: C = A(:, J[:k]), R = A(I[:k], :),
    T the least-squares solution of C T = A(:, J[k:]) (Householder QR of C),
    U = V* R^+ (least squares through the QR of R^T, as ``cur_middle``).
    Returns (C, U, R, T)."""
    A = np.asarray(A, dtype=np.float64)
    J = np.asarray(J)
    I = np.asarray(I)
    n = A.shape[1]
    C = A[:, J[:k]]
    B = A[:, J[k:]]
    R = A[I[:k], :]
    Qc, Sc = np.linalg.qr(C)
    T = scipy.linalg.solve_triangular(Sc, Qc.T @ B, lower=False)
    Vs = np.zeros((k, n))
    Vs[np.arange(k), J[:k]] = 1.0
    Vs[:, J[k:]] = T
    Qr, Sr = np.linalg.qr(R.T)
    U = scipy.linalg.solve_triangular(Sr, Qr.T @ Vs.T, lower=False).T
    return C, U, R, T


def cur_adjoint(A, J, I, k, Cbar, Ubar, Rbar):
    """Abar for cotangents (Cbar m x k, Ubar k x k, Rbar k x n) of the
    frozen-skeleton outputs (C, U, R); steps 1-4 of the module docstring."""
    A = np.asarray(A, dtype=np.float64)
    J = np.asarray(J)
    I = np.asarray(I)
    m, n = A.shape
    Cbar = np.asarray(Cbar, dtype=np.float64)
    Ubar = np.asarray(Ubar, dtype=np.float64)
    Rbar = np.asarray(Rbar, dtype=np.float64)
    C, U, R, T = cur_frozen(A, J, I, k)
    B = A[:, J[k:]]
    # R^+ = R^T (R R^T)^{-1} through the QR of R^T = Qr Sr: R^+ = Qr Sr^{-T}
    Qr, Sr = np.linalg.qr(R.T)
    Rp = scipy.linalg.solve_triangular(Sr, Qr.T, lower=False).T        # n x k
    RRt_inv = scipy.linalg.cho_solve((Sr, False), np.eye(k))            # (R R^T)^{-1}
    V = np.zeros((n, k))
    V[J[:k], np.arange(k)] = 1.0
    V[J[k:], :] = T.T
    # 1. through U = V* R^+
    M = V @ Ubar                                                        # n x k
    Vsbar = Ubar @ Rp.T                                                 # k x n
    Rbar_t = Rbar - Rp.T @ M @ Rp.T + RRt_inv @ M.T @ (np.eye(n) - Rp @ R)
    # 2. cotangent of T
    Tbar = Vsbar[:, J[k:]]
    # 3. through T = (C^T C)^{-1} C^T B, with C^T C = Sc^T Sc
    Qc, Sc = np.linalg.qr(C)
    K = scipy.linalg.cho_solve((Sc, False), Tbar)                       # k x (n-k)
    E = B - C @ T
    Cbar_t = Cbar + E @ K.T - C @ K @ T.T
    Bbar = C @ K
    # 4. scatter
    Abar = np.zeros((m, n))
    Abar[:, J[:k]] += Cbar_t
    Abar[:, J[k:]] += Bbar
    Abar[I[:k], :] += Rbar_t
    return Abar


def cur_loss_grad(A, J, I, k):
    """Gradient of the loss 1/2 ||A - C U R||_F^2 with frozen skeletons: the
    direct term (A - CUR) plus the adjoint of the outputs' cotangents
    Cbar = G R^T U^T, Ubar = C^T G R^T, Rbar = U^T C^T G, with
    G = -(A - C U R) the cotangent of the product C U R."""
    A = np.asarray(A, dtype=np.float64)
    C, U, R, _ = cur_frozen(A, J, I, k)
    Res = A - C @ U @ R
    G = -Res
    Cbar = G @ R.T @ U.T
    Ubar = C.T @ G @ R.T
    Rbar = U.T @ C.T @ G
    return Res + cur_adjoint(A, J, I, k, Cbar, Ubar, Rbar), 0.5 * float(np.sum(Res * Res))
