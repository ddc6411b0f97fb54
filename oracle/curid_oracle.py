"""Plain FP64 CPU oracle: truncated CPQR, column/row/two-sided ID, CUR-ID and
the randomized sketch of Voronin & Martinsson (arXiv:1412.8447).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Everything is float64
numpy, one step at a time, in the order the paper states the method.  Library
primitives (matrix product, Householder QR of a tall matrix, triangular
solve) serve as single steps; nothing is blocked, fused or reordered.

Conventions fixed here (the paper leaves them open):
  * indices are 0-based; ``J[:k]`` are the pivots in selection order and
    ``J[k:]`` are the unselected columns in ascending index order;
  * among exactly equal pivot norms the smallest column index wins;
  * ``T`` is k x (n-k), its columns follow ``J[k:]``;
  * ``orth`` returns the row-orthonormal Q with Y = L Q, L lower triangular
    with a positive diagonal (unique for full row rank);
  * the adaptive rank is the smallest j with ||A - C V*||_F <= tol ||A||_F.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

__all__ = [
    "as_f64", "CPQR", "cpqr", "interpolation_matrix", "interpolation_matrix_tikhonov",
    "interpolation_matrix_tsvd",
    "vstar", "wmat",
    "IDResult", "id_col", "id_row", "TSIDResult", "tsid", "CURResult",
    "cur_middle", "cur", "cur_middle_corrected", "cur_corrected", "randomized_cur_corrected",
    "orth_rows", "sketch", "randomized_id_col", "randomized_rank_adaptive",
    "randomized_cur", "srft_sketch", "srft_omega_rows", "rel_err_fro", "OK", "RANK_DEFICIENT",
    "rank_threshold", "cpqr_complex", "cur_complex", "sketch_complex",
]

OK = 0
RANK_DEFICIENT = 2


def as_f64(A):
    """Exact upcast of a stored matrix (float32, float64, or bfloat16 values
    already held as float32) to a float64 numpy array."""
    if hasattr(A, "detach"):  # torch tensor
        A = A.detach().to("cpu")
        if str(A.dtype) == "torch.bfloat16":
            A = A.float()
        A = A.numpy()
    return np.array(A, dtype=np.float64, copy=True)


def rank_threshold(shape, nu_first, eps=np.finfo(np.float64).eps):
    """Pivot norm at or below which the factorization is declared rank
    deficient (the case of Section 2.3 where S11 is singular; the paper gives
    no numerical threshold): 2 sqrt(l) eps times the first pivot norm, l the
    column length.  After an exact rank-r part is removed, rounding leaves
    residual columns of relative norm about sqrt(l) eps / 4 or less, while a
    genuine trailing singular value above this level keeps its pivot."""
    return 2.0 * np.sqrt(shape[0]) * eps * nu_first


@dataclass
class CPQR:
    """Result of k steps of column-pivoted QR, Eq. (2.4)-(2.5):
    Y(:, J) = Q1 S1 + Q2 S2 with S1 = [S11 S12] upper trapezoidal.

    J       : full permutation (int64, length n); J[:k] pivots in order.
    S1      : k x n, columns in the order J (S1[:, :k] = S11 upper triangular).
    Q1      : l x k with orthonormal columns.
    k       : number of steps taken.
    k_eff   : numerical rank found (== k unless rank deficient).
    nu      : pivot norms, nu[j] = |S(j, j)|.
    gaps    : relative gap (nu_(1) - nu_(2)) / nu_(1) between the two largest
              candidate norms at every step (inf when only one candidate).
    resid   : ||Y - Q1 Q1^T Y||_F after 0, 1, ..., k steps.
    """
    J: np.ndarray
    S1: np.ndarray
    Q1: np.ndarray
    k: int
    k_eff: int
    nu: np.ndarray
    gaps: np.ndarray
    resid: np.ndarray
    status: int = OK


def cpqr(Y, k=None, tol=None, eps=np.finfo(np.float64).eps):
    """Truncated column-pivoted QR by pivoted Gram-Schmidt (Section 2.2,
    Eq. (2.4)-(2.5); the first step of Algorithm 1; the Gram-Schmidt reading
    of Remark 2.1 and Section 2.4).

    Each step j: (1) recompute the norm of every unselected residual column
    from the vector itself; (2) pick the largest (smallest index on exact
    ties); (3) normalise it to q_j and re-orthogonalise once against
    q_1..q_{j-1}; (4) project q_j out of every unselected residual column.
    Stops after ``k`` steps, or (``tol`` given) at the first j with
    ||residual||_F <= tol * ||Y||_F, or at min(l, n).
    Finally S1 = Q1^T Y(:, J), whose strictly lower part in the first k columns
    is zero in exact arithmetic and is set to zero.
    """
    Y = as_f64(Y)
    l, n = Y.shape
    kmax = min(l, n)
    if k is not None:
        kmax = min(kmax, int(k))
    Rres = Y.copy()
    active = np.ones(n, dtype=bool)
    Q = np.zeros((l, kmax))
    J, nus, gaps = [], [], []
    normY = np.sqrt(np.sum(Y * Y))
    resid = [normY]
    k_eff = None
    nu_first = None
    for j in range(kmax):
        if tol is not None and resid[-1] <= tol * normY:
            break
        nu = np.sqrt(np.sum(Rres * Rres, axis=0))            # (1)
        cand = np.where(active, nu, -1.0)
        p = int(np.argmax(cand))                               # (2) first max
        srt = np.sort(cand[active])[::-1]
        if srt.size > 1 and srt[0] > 0:
            gaps.append((srt[0] - srt[1]) / srt[0])
        else:
            gaps.append(np.inf)
        if nu_first is None:
            nu_first = nu[p]
        if k_eff is None and (nu[p] == 0.0 or
                              nu[p] <= rank_threshold((l, n), nu_first, eps)):
            k_eff = j
        if nu[p] > 0.0:
            q = Rres[:, p] / nu[p]                              # (3)
            q = q - Q[:, :j] @ (Q[:, :j].T @ q)
            nq = np.linalg.norm(q)
            q = q / nq if nq > 0 else q
        else:
            q = np.zeros(l)
        Q[:, j] = q
        nus.append(nu[p])
        J.append(p)
        active[p] = False
        Rres[:, p] = 0.0
        Rres[:, active] -= np.outer(q, q @ Rres[:, active])     # (4)
        resid.append(np.sqrt(np.sum(Rres[:, active] ** 2)))
    kk = len(J)
    Jfull = np.array(J + [i for i in range(n) if active[i]], dtype=np.int64)
    Q1 = Q[:, :kk]
    S1 = Q1.T @ Y[:, Jfull]
    S1[:, :kk] = np.triu(S1[:, :kk])
    status = OK
    if k_eff is None:
        k_eff = kk
    else:
        status = RANK_DEFICIENT
    return CPQR(J=Jfull, S1=S1, Q1=Q1, k=kk, k_eff=k_eff,
                nu=np.array(nus), gaps=np.array(gaps), resid=np.array(resid),
                status=status)


def interpolation_matrix(S1, k, k_eff=None):
    """T solving S11 T = S12 by back substitution (Eq. (2.8), Section 4.1).
    S1 is k x n in pivot order.  When S11 is singular (numerical rank
    k_eff < k) the bottom k - k_eff rows of T are zero and the top rows solve
    the leading k_eff x k_eff system, as Section 2.3 allows."""
    S1 = np.asarray(S1, dtype=np.float64)
    n = S1.shape[1]
    if k_eff is None:
        k_eff = k
    T = np.zeros((k, n - k))
    if k_eff > 0:
        T[:k_eff] = scipy.linalg.solve_triangular(
            S1[:k_eff, :k_eff], S1[:k_eff, k:], lower=False)
    return T


def interpolation_matrix_tikhonov(S1, k, lam):
    """T of the regularised least-squares problem of Section 4.1 (Eq. (4.1)
    amended by a Tikhonov term): T = argmin ||S11 T - S12||_F^2 +
    lam^2 ||T||_F^2, as the plain least-squares solution of the augmented
    system [S11; lam I] T = [S12; 0] (library lstsq as the single step).
    S1 is k x n in pivot order; lam >= 0 (lam = 0 is Eq. (2.8) when S11 is
    nonsingular)."""
    S1 = np.asarray(S1, dtype=np.float64)
    n = S1.shape[1]
    W = np.vstack([S1[:k, :k], lam * np.eye(k)])
    B = np.vstack([S1[:k, k:], np.zeros((k, n - k))])
    return np.linalg.lstsq(W, B, rcond=None)[0]


def interpolation_matrix_tsvd(S1, k, rtol):
    """T from the truncated SVD of S11 (Section 4.1): S11 = U diag(s) V^T
    (library SVD as the single step), singular values s_i <= rtol * s_1
    dropped, T = V diag(1 / s_i) U^T S12 over the kept ones.  S1 is k x n in
    pivot order."""
    S1 = np.asarray(S1, dtype=np.float64)
    U, sv, Vt = np.linalg.svd(S1[:k, :k])
    keep = sv > rtol * sv[0] if sv.size and sv[0] > 0 else np.zeros(sv.size, dtype=bool)
    return Vt[keep].T @ np.diag(1.0 / sv[keep]) @ U[:, keep].T @ S1[:k, k:]


def vstar(J, T, n):
    """V* = [I_k T] P^* as an explicit k x n matrix (Eq. (2.9)):
    V*(:, J[:k]) = I and V*(:, J[k:]) = T."""
    k = T.shape[0]
    V = np.zeros((k, n))
    V[np.arange(k), J[:k]] = 1.0
    V[:, J[k:]] = T
    return V


def wmat(I, TW, m):
    """W = P [I; T_W^*] as an explicit m x k matrix (Eq. (3.11)):
    W(I[:k], :) = I and W(I[k:], :) = T_W^T."""
    k = TW.shape[0]
    W = np.zeros((m, k))
    W[I[:k], np.arange(k)] = 1.0
    W[I[k:], :] = TW.T
    return W


@dataclass
class IDResult:
    """Column ID A ~ A(:, J[:k]) V*, V* = [I T] P^* (Algorithm 1)."""
    J: np.ndarray
    T: np.ndarray
    k: int
    qr: CPQR
    status: int = OK


def id_col(A, k=None, tol=None, eps=np.finfo(np.float64).eps):
    """Rank-k column ID (Algorithm 1, Section 2.3): CPQR of A, then
    T = S11^{-1} S12."""
    res = cpqr(A, k=k, tol=tol, eps=eps)
    T = interpolation_matrix(res.S1, res.k, res.k_eff)
    return IDResult(J=res.J, T=T, k=res.k, qr=res, status=res.status)


def id_row(A, k=None, tol=None, eps=np.finfo(np.float64).eps):
    """Row ID A ~ W A(I[:k], :) by the column ID of A^* (Remark 2.1)."""
    return id_col(as_f64(A).T, k=k, tol=tol, eps=eps)


@dataclass
class TSIDResult:
    """Two-sided ID A ~ W A(I[:k], J[:k]) V* (Algorithm 2, Eq. (2.12))."""
    J: np.ndarray
    T: np.ndarray
    I: np.ndarray
    TW: np.ndarray
    k: int
    col: IDResult
    row: IDResult
    status: int = OK


def tsid(A, k=None, tol=None, Y=None, eps=np.finfo(np.float64).eps):
    """Algorithm 2: a column ID (of A, or of a sketch Y of A when given, as in
    Algorithm 4), then a full rank-k ID of C^* with C = A(:, J[:k])
    (Eq. (2.11)), which is exact."""
    A = as_f64(A)
    col = id_col(A if Y is None else Y, k=k, tol=tol, eps=eps)
    kk = col.k
    C = A[:, col.J[:kk]]
    row = id_col(C.T, k=kk, eps=eps)
    status = col.status if col.status != OK else row.status
    return TSIDResult(J=col.J, T=col.T, I=row.J, TW=row.T, k=kk, col=col,
                      row=row, status=status)


def cur_middle(R, Vs):
    """U = V* R^+ (Eq. (3.5)) as the least-squares solution of U R = V*
    (Eq. (4.2)) through the Householder QR of R^T: R^T = Q_R S_R, then
    U^T = S_R^{-1} Q_R^T V with V = (V*)^T."""
    Qr, Sr = np.linalg.qr(np.asarray(R, dtype=np.float64).T)
    Ut = scipy.linalg.solve_triangular(Sr, Qr.T @ np.asarray(Vs).T,
                                       lower=False)
    return Ut.T


@dataclass
class CURResult:
    """CUR-ID A ~ C U R (Algorithm 3)."""
    J: np.ndarray
    I: np.ndarray
    T: np.ndarray
    TW: np.ndarray
    U: np.ndarray
    C: np.ndarray
    R: np.ndarray
    k: int
    ts: TSIDResult
    status: int = OK


def cur(A, k=None, tol=None, Y=None, eps=np.finfo(np.float64).eps):
    """Algorithm 3: two-sided ID, C = A(:, J[:k]), R = A(I[:k], :),
    U = V* R^+ (Eq. (3.1), (3.5))."""
    A = as_f64(A)
    ts = tsid(A, k=k, tol=tol, Y=Y, eps=eps)
    kk = ts.k
    n = A.shape[1]
    C = A[:, ts.J[:kk]]
    R = A[ts.I[:kk], :]
    U = cur_middle(R, vstar(ts.J, ts.T, n))
    return CURResult(J=ts.J, I=ts.I, T=ts.T, TW=ts.TW, U=U, C=C, R=R, k=kk,
                     ts=ts, status=ts.status)


def cur_middle_corrected(A, C, R, Vs):
    """U from the error-corrected system of Section 4.3, Eq. (4.3): with
    E = A - C V* (the column ID's error), solve U R = V* + C^+ E in the
    least-squares sense.  C^+ E is the least-squares solution of C X = E
    (Householder QR of C), and the system for U is solved like Eq. (4.2)
    (``cur_middle``)."""
    A, C = as_f64(A), as_f64(C)
    Vs = np.asarray(Vs, dtype=np.float64)
    E = A - C @ Vs
    Qc, Sc = np.linalg.qr(C)
    CpE = scipy.linalg.solve_triangular(Sc, Qc.T @ E, lower=False)
    return cur_middle(R, Vs + CpE)


def cur_corrected(A, k=None, tol=None, Y=None, eps=np.finfo(np.float64).eps):
    """Algorithm 3 with U from Eq. (4.3) instead of Eq. (4.2)."""
    A = as_f64(A)
    r = cur(A, k=k, tol=tol, Y=Y, eps=eps)
    U = cur_middle_corrected(A, r.C, r.R, vstar(r.J, r.T, A.shape[1]))
    return CURResult(J=r.J, I=r.I, T=r.T, TW=r.TW, U=U, C=r.C, R=r.R, k=r.k, ts=r.ts,
                     status=r.status)


def randomized_cur_corrected(A, Omega, k, q=0, orth=True, eps=np.finfo(np.float64).eps):
    """CUR-ID with its column ID from Algorithm 4 and U from Eq. (4.3)."""
    Y = sketch(A, Omega, q=q, orth=orth)
    return cur_corrected(A, k=k, Y=Y, eps=eps), Y


def orth_rows(Y):
    """Row orthonormalisation without pivoting (Section 5.3): the unique
    row-orthonormal Q with Y = L Q, L lower triangular with positive
    diagonal, from the Householder QR of Y^T with the signs fixed."""
    Qt, Rt = np.linalg.qr(as_f64(Y).T)
    s = np.sign(np.diag(Rt))
    s[s == 0] = 1.0
    return (Qt * s).T


def sketch(A, Omega, q=0, orth=True):
    """Sample matrix of Algorithm 4 with the power scheme of Section 5.3:
    (2a) Y = Omega A; (2b) for i = 1..q: (2c) Y <- orth(Y) A^*,
    (2d) Y <- orth(Y) A.  ``orth=False`` gives the un-orthonormalised
    variant, Eq. (5.3)."""
    A = as_f64(A)
    Y = as_f64(Omega) @ A
    for _ in range(q):
        Y = (orth_rows(Y) if orth else Y) @ A.T
        Y = (orth_rows(Y) if orth else Y) @ A
    return Y


def randomized_id_col(A, Omega, k, q=0, orth=True,
                      eps=np.finfo(np.float64).eps):
    """Algorithm 4: Y from ``sketch``, k steps of CPQR on Y (the first k
    pivots of the full pivoted QR the algorithm states), T from S of Y."""
    Y = sketch(A, Omega, q=q, orth=orth)
    return id_col(Y, k=k, eps=eps), Y


def randomized_rank_adaptive(A, Omega, tol, p, q=0, orth=True, l0=64, l_cap=4096,
                             eps=np.finfo(np.float64).eps):
    """Rank for a tolerance with a sketch (Algorithm 4 with the tolerance stop
    of Section 3; the sample size l = k + p needs the rank, so l is searched):
    l starts at max(l0, p + 1), capped by min(m, n, l_cap); the sample is the
    first l rows of ``Omega`` applied as in ``sketch``; CPQR of the sample
    runs at most l - p steps with the stop ||Y - Q_j Q_j^T Y||_F <= tol ||Y||_F.
    A stop before l - p steps gives the rank; otherwise l doubles (at the cap
    the rank is l - p).  Returns (k, l, Y)."""
    A = as_f64(A)
    m, n = A.shape
    cap = min(m, n, l_cap)
    l = min(cap, max(l0, p + 1))
    while True:
        Y = sketch(A, np.asarray(Omega)[:l], q=q, orth=orth)
        r = cpqr(Y, k=l - p, tol=tol, eps=eps)
        if r.k < l - p or l >= cap:
            return r.k, l, Y
        l = min(cap, 2 * l)


def randomized_cur(A, Omega, k, q=0, orth=True,
                   eps=np.finfo(np.float64).eps):
    """CUR-ID (Algorithm 3) with its column ID taken from Algorithm 4."""
    Y = sketch(A, Omega, q=q, orth=orth)
    return cur(A, k=k, Y=Y, eps=eps), Y


def srft_sketch(A, rows, signs):
    """Structured sample matrix of Section 5.2, Eq. (5.2), applied to A:
    Y = sqrt(m / l) R F D A with D = diag(signs), F the m x m orthonormal
    transform and R the l sampled rows ``rows`` (0-based, drawn without
    replacement).  Real reading of the paper's complex construction: the
    unit-circle entries of D become random signs +-1 and the unitary DFT
    becomes the orthonormal DCT-II, F(f, t) = c_f cos(pi f (2t + 1) / (2m)),
    c_0 = sqrt(1/m), c_f = sqrt(2/m) -- real, orthogonal, any m.  The
    transform is scipy's DCT along the columns (a library primitive used as
    one step), then row selection and scaling, in the order of Eq. (5.2)."""
    import scipy.fft
    A = as_f64(A)
    m = A.shape[0]
    rows = np.asarray(rows, dtype=np.int64)
    d = np.asarray(signs, dtype=np.float64)
    FDA = scipy.fft.dct(d[:, None] * A, type=2, norm="ortho", axis=0)
    return np.sqrt(m / len(rows)) * FDA[rows, :]


def srft_omega_rows(m, rows, signs, which=None):
    """Rows ``which`` (default all) of the l x m matrix Omega of Eq. (5.2)
    under the reading of ``srft_sketch``: row i is sqrt(m/l) times row
    rows[i] of F, times the signs.  Row f of an orthogonal F equals F^T
    applied to e_f, i.e. the inverse transform (orthonormal DCT-III) of e_f."""
    import scipy.fft
    rows = np.asarray(rows, dtype=np.int64)
    d = np.asarray(signs, dtype=np.float64)
    idx = range(len(rows)) if which is None else which
    out = []
    for i in idx:
        e = np.zeros(m)
        e[rows[i]] = 1.0
        out.append(np.sqrt(m / len(rows)) * scipy.fft.idct(e, type=2, norm="ortho") * d)
    return np.array(out)


def rel_err_fro(A, C, U, R):
    """||A - C U R||_F / ||A||_F in float64."""
    A = as_f64(A)
    E = A - as_f64(C) @ as_f64(U) @ as_f64(R)
    return float(np.sqrt(np.sum(E * E)) / np.sqrt(np.sum(A * A)))


# --- complex A (the paper works over C throughout) ---------------------------

def cpqr_complex(Y, k):
    """k steps of column-pivoted QR of a complex Y by pivoted Gram-Schmidt,
    the complex form of ``cpqr`` (Section 2.2 over C): norms |y|_2 recomputed
    each step, the largest taken (smallest index on exact ties), q_j
    re-orthogonalised once, q_j q_j^* projected out of every unselected
    column.  Returns (J, S1) with J the full permutation (unselected columns
    ascending) and S1 = Q1^* Y(:, J) (k x n, upper triangular in its first k
    columns)."""
    Y = np.asarray(Y, dtype=np.complex128)
    l, n = Y.shape
    R = Y.copy()
    active = np.ones(n, dtype=bool)
    Q = np.zeros((l, k), dtype=np.complex128)
    J = []
    for j in range(k):
        nu = np.sqrt(np.sum(np.abs(R) ** 2, axis=0))
        p = int(np.argmax(np.where(active, nu, -1.0)))
        q = R[:, p] / nu[p]
        q = q - Q[:, :j] @ (Q[:, :j].conj().T @ q)
        q = q / np.linalg.norm(q)
        Q[:, j] = q
        J.append(p)
        active[p] = False
        R[:, p] = 0.0
        R[:, active] -= np.outer(q, q.conj() @ R[:, active])
    Jf = np.array(J + [i for i in range(n) if active[i]], dtype=np.int64)
    S1 = Q.conj().T @ Y[:, Jf]
    S1[:, :k] = np.triu(S1[:, :k])
    return Jf, S1


def cur_complex(A, k, Y=None):
    """CUR-ID of a complex A (Algorithm 3 over C): column ID from the CPQR of
    A (or of a sketch Y), T = S11^{-1} S12, row ID from the full k-step CPQR of
    C^* (conjugate transpose), U = V* R^+ by least squares (Eq. (4.2)).
    Returns a dict with J, I, T, TW, U, C, R."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    J, S1 = cpqr_complex(A if Y is None else Y, k)
    T = scipy.linalg.solve_triangular(S1[:, :k], S1[:, k:], lower=False)
    C = A[:, J[:k]]
    I, SW = cpqr_complex(C.conj().T, k)
    TW = scipy.linalg.solve_triangular(SW[:, :k], SW[:, k:], lower=False)
    R = A[I[:k], :]
    Vs = np.zeros((k, n), dtype=np.complex128)
    Vs[np.arange(k), J[:k]] = 1.0
    Vs[:, J[k:]] = T
    U = np.linalg.lstsq(R.T, Vs.T, rcond=None)[0].T
    return {"J": J, "I": I, "T": T, "TW": TW, "U": U, "C": C, "R": R}


def sketch_complex(A, Omega, q=0):
    """Sample matrix of Algorithm 4 over C with the power scheme of Section
    5.3: Y = Omega A, then q times Y <- orth(Y) A^*, Y <- orth(Y) A, orth the
    row orthonormalisation (Householder QR of Y^*, diagonal made positive)."""
    A = np.asarray(A, dtype=np.complex128)

    def orth(Y):
        Qt, Rt = np.linalg.qr(Y.conj().T)
        d = np.diag(Rt)
        ph = np.where(d == 0, 1.0, d / np.abs(np.where(d == 0, 1.0, d)))
        return (Qt * ph).conj().T

    Y = np.asarray(Omega, dtype=np.complex128) @ A
    for _ in range(q):
        Y = orth(Y) @ A.conj().T
        Y = orth(Y) @ A
    return Y
