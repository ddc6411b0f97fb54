"""Pins for the FP64 oracle: checks against values fixed by the paper's
identities, by library routines (LAPACK dgeqp3 via scipy, lstsq, pinv, SVD,
Cholesky), by closed forms, by a hand-derived example and by brute force.
No check re-types the oracle's own formula."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg
import torch

import oracle as O
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def f64(t):
    return t.numpy().astype(np.float64) if hasattr(t, "numpy") else np.asarray(t, np.float64)


def fro(X):
    return float(np.sqrt(np.sum(np.asarray(X) ** 2)))


# --- hand-derived example ---------------------------------------------------

def test_handworked_example():
    g = json.load(open(os.path.join(GOLDEN, "handworked_2x3.json")))
    A = np.array(g["A"])
    for key, k in (("k1", 1), ("k2", 2)):
        r = O.id_col(A, k=k)
        assert list(r.J) == g[key]["J"]
        np.testing.assert_allclose(r.T, np.array(g[key]["T"]), rtol=0, atol=1e-15)
        np.testing.assert_allclose(r.qr.nu, g[key]["nu"], rtol=1e-15)
        assert abs(r.qr.resid[-1] - g[key]["resid_fro"]) <= 1e-15
    r = O.id_col(A, k=2)
    np.testing.assert_allclose(np.abs(r.qr.S1[:, :2]), np.array(g["k2"]["S11_abs"]), atol=1e-15)


# --- CPQR against LAPACK and against the planted order ---------------------

@pytest.mark.parametrize("m,n,k,seed", [(60, 40, 12, 1), (40, 70, 20, 2),
                                        (128, 96, 33, 3), (33, 257, 30, 4)])
def test_cpqr_planted_and_lapack(m, n, k, seed):
    A, perm = syn.planted_pivots(m, n, k, seed)
    A = f64(A)
    r = O.cpqr(A, k=k)
    assert list(r.J[:k]) == list(perm[:k])
    # LAPACK dgeqp3 (Householder with norm downdating): a different algorithm
    R, P = scipy.linalg.qr(A, mode="r", pivoting=True)
    assert list(P[:k]) == list(r.J[:k])
    # rows of S agree with LAPACK's R up to sign, column by column
    S_by_col = np.zeros((k, n))
    S_by_col[:, r.J] = r.S1
    R_by_col = np.zeros((k, n))
    R_by_col[:, P] = R[:k]
    sgn = np.sign(np.diag(R[:k, :k])) * np.sign(np.diag(r.S1[:, :k]))
    np.testing.assert_allclose(S_by_col, sgn[:, None] * R_by_col,
                               atol=1e-12 * np.abs(R).max())
    # residual columns are ascending
    assert list(r.J[k:]) == sorted(r.J[k:])
    assert sorted(r.J) == list(range(n))


def _brute_force_greedy(A, k):
    """Independent greedy: at each step pick the column with the largest
    least-squares residual against the columns already picked."""
    m, n = A.shape
    sel = []
    for _ in range(k):
        best, bi = -1.0, None
        for c in range(n):
            if c in sel:
                continue
            if sel:
                x, *_ = np.linalg.lstsq(A[:, sel], A[:, c], rcond=None)
                res = np.linalg.norm(A[:, c] - A[:, sel] @ x)
            else:
                res = np.linalg.norm(A[:, c])
            if res > best * (1 + 1e-12):
                best, bi = res, c
        sel.append(bi)
    return sel


@pytest.mark.parametrize("seed", range(6))
def test_cpqr_brute_force_tiny(seed):
    g = np.random.default_rng(100 + seed)
    m, n = g.integers(3, 9), g.integers(3, 10)
    A = g.standard_normal((m, n)) * g.uniform(0.1, 3, n)
    k = min(m, n) - 1
    r = O.cpqr(A, k=k)
    assert list(r.J[:k]) == _brute_force_greedy(A, k)


def test_cpqr_ties_take_smallest_index():
    g = np.random.default_rng(7)
    A = g.standard_normal((8, 6))
    A[:, 4] = A[:, 1] = 10 * g.standard_normal(8)  # exact tie, largest norm
    r = O.cpqr(A, k=3)
    assert r.J[0] == 1


def test_cpqr_decay_property():
    """|S(j,j)| >= ||S(j:k, l)|| for l after j (Section 2.2)."""
    A = f64(syn.spectrum_matrix(80, 60, syn.exp_decay(60, 5.0), 11))
    r = O.cpqr(A, k=30)
    S = r.S1
    for j in range(30):
        col_norms = np.sqrt(np.sum(S[j:, j + 1:] ** 2, axis=0))
        assert np.all(abs(S[j, j]) >= col_norms * (1 - 1e-12))


def test_cpqr_residual_matches_projection():
    """resid[j] = ||A - Q_j Q_j^T A||_F with Q_j from numpy's QR of the
    selected columns (Eq. (2.5), (2.10))."""
    A = f64(syn.spectrum_matrix(50, 70, syn.exp_decay(50, 8.0), 12))
    r = O.cpqr(A, k=20)
    for j in (1, 5, 20):
        Qj, _ = np.linalg.qr(A[:, r.J[:j]])
        assert abs(fro(A - Qj @ (Qj.T @ A)) - r.resid[j]) <= 1e-12 * fro(A)


# --- column ID ---------------------------------------------------------------

def test_id_identities():
    A = f64(syn.spectrum_matrix(90, 70, syn.exp_decay(70), 21))
    k = 25
    r = O.id_col(A, k=k)
    V = O.vstar(r.J, r.T, A.shape[1])
    # V*(:, J[:k]) is exactly the identity (Eq. (2.9))
    assert np.array_equal(V[:, r.J[:k]], np.eye(k))
    C = A[:, r.J[:k]]
    # A - C V* = Q2 S22: its Frobenius norm is the CPQR residual (Eq. (2.10))
    assert abs(fro(A - C @ V) - r.qr.resid[k]) <= 1e-12 * fro(A)
    # T closed form: least-squares coefficients of the residual columns
    Tls, *_ = np.linalg.lstsq(C, A[:, r.J[k:]], rcond=None)
    np.testing.assert_allclose(r.T, Tls, atol=1e-9 * np.abs(Tls).max())
    # Eckart-Young: the ID error is at least sigma_{k+1} (Section 2.2)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.linalg.norm(A - C @ V, 2) >= s[k] * (1 - 1e-12)


def test_exact_rank_reconstruction():
    A = f64(syn.exact_rank(120, 90, 15, 31))
    res = O.cur(A, k=15)
    assert O.rel_err_fro(A, res.C, res.U, res.R) <= 1e-13
    V = O.vstar(res.J, res.T, 90)
    assert fro(A - res.C @ V) <= 1e-13 * fro(A)


def test_rank_deficient_status_and_zero_rows():
    A = f64(syn.exact_rank(40, 30, 6, 32))
    r = O.id_col(A, k=10)
    assert r.status == O.RANK_DEFICIENT and r.qr.k_eff == 6
    assert np.all(r.T[6:] == 0)
    C = A[:, r.J[:10]]
    assert fro(A - C @ O.vstar(r.J, r.T, 30)) <= 1e-12 * fro(A)


def test_adaptive_rank():
    A = f64(syn.spectrum_matrix(100, 80, syn.exp_decay(80, 6.0), 41))
    tol = 1e-6
    r = O.id_col(A, tol=tol)
    k = r.k
    nA = fro(A)
    # residual at k meets the tolerance; at k - 1 (recomputed independently) it does not
    assert r.qr.resid[k] <= tol * nA
    rk1 = O.id_col(A, k=k - 1)
    C = A[:, rk1.J[:k - 1]]
    assert fro(A - C @ O.vstar(rk1.J, rk1.T, 80)) > tol * nA


# --- row ID, two-sided ID, CUR -------------------------------------------------

def test_row_id_and_tsid():
    A = f64(syn.spectrum_matrix(70, 110, syn.exp_decay(70), 51))
    k = 20
    ts = O.tsid(A, k=k)
    C = A[:, ts.J[:k]]
    W = O.wmat(ts.I, ts.TW, 70)
    V = O.vstar(ts.J, ts.T, 110)
    # C = W C(I, :) exactly up to rounding (Eq. (2.11), full-rank ID)
    assert fro(C - W @ C[ts.I[:k]]) <= 1e-12 * fro(C)
    # W(I[:k], :) is the identity
    assert np.array_equal(W[ts.I[:k]], np.eye(k))
    # the two-sided ID adds no error to the column ID (Section 2.4)
    E1 = fro(A - C @ V)
    E2 = fro(A - W @ A[np.ix_(ts.I[:k], ts.J[:k])] @ V)
    assert abs(E1 - E2) <= 1e-12 * fro(A)
    # row ID via the transpose: id_row(A) is id_col(A^T)
    rr = O.id_row(A, k=k)
    Rl, P = scipy.linalg.qr(A.T, mode="r", pivoting=True)
    assert list(rr.J[:k]) == list(P[:k]) or min(rr.qr.gaps) < 1e-8


def test_cur_middle_closed_form_and_bounds():
    A = f64(syn.spectrum_matrix(90, 120, syn.exp_decay(90, 7.0), 61))
    k = 18
    res = O.cur(A, k=k)
    V = O.vstar(res.J, res.T, 120)
    # U = V* R^+ (Eq. (3.5)) against numpy's pinv (SVD based)
    Up = V @ np.linalg.pinv(res.R)
    np.testing.assert_allclose(res.U, Up, atol=1e-8 * np.abs(Up).max())
    # Lemma 3.1, Lemma 3.2 and Corollary 3.3 in the spectral norm
    E = A - res.C @ V
    W = O.wmat(res.I, res.TW, 90)
    Et = A - W @ res.R
    nE, nEt = np.linalg.norm(E, 2), np.linalg.norm(Et, 2)
    ncur = np.linalg.norm(A - res.C @ res.U @ res.R, 2)
    assert ncur <= (nE + nEt) * (1 + 1e-10)
    assert nEt <= (1 + np.linalg.norm(res.TW, 2)) * nE * (1 + 1e-10)
    assert ncur <= (2 + np.linalg.norm(res.TW, 2)) * nE * (1 + 1e-10)
    # Eq. (3.14): E~ = P [0; F E], with F = [-T_W^* I] P^* (Eq. (3.13))
    Ires, Isk = res.I[k:], res.I[:k]
    FE = E[Ires] - res.TW.T @ E[Isk]
    np.testing.assert_allclose(Et[Ires], FE, atol=1e-11 * fro(A))
    assert fro(Et[Isk]) <= 1e-12 * fro(A)
    # F W = 0
    FW = W[Ires] - res.TW.T @ W[Isk]
    assert fro(FW) <= 1e-13


# --- randomized front end ------------------------------------------------------

def test_orth_rows_against_cholesky():
    g = np.random.default_rng(71)
    Y = g.standard_normal((12, 50)) * np.logspace(0, -3, 12)[:, None]
    Q = O.orth_rows(Y)
    np.testing.assert_allclose(Q @ Q.T, np.eye(12), atol=1e-13)
    L = np.linalg.cholesky(Y @ Y.T)          # Y Y^T = L L^T, L with positive diagonal
    np.testing.assert_allclose(Q, np.linalg.solve(L, Y), atol=1e-9)


def _proj(M):
    Qm, _ = np.linalg.qr(M.T)
    return Qm @ Qm.T


def test_sketch_power_spans_closed_form():
    """The orthonormalised scheme (Section 5.3) spans the same row space as
    Omega A (A^* A)^q evaluated directly (Eq. (5.3))."""
    A = f64(syn.spectrum_matrix(60, 45, np.linspace(1, 0.3, 45), 81))
    Om = f64(syn.gaussian(10, 60, 82))
    for q in (0, 1, 2):
        Y = O.sketch(A, Om, q=q, orth=True)
        Yd = Om @ A @ np.linalg.matrix_power(A.T @ A, q)
        assert fro(_proj(Y) - _proj(Yd)) <= 1e-10
        Yn = O.sketch(A, Om, q=q, orth=False)
        np.testing.assert_allclose(Yn, Yd, rtol=1e-10, atol=1e-12 * np.abs(Yd).max())


def test_randomized_exact_rank():
    A = f64(syn.exact_rank(200, 150, 12, 91))
    Om = f64(syn.gaussian(17, 200, 92))
    res, Y = O.randomized_cur(A, Om, k=12, q=1)
    assert O.rel_err_fro(A, res.C, res.U, res.R) <= 1e-12


def test_randomized_close_to_deterministic():
    """With p = 10 and q = 1 the randomized CUR error is within a small
    factor of the optimal rank-k error (Section 5)."""
    A = f64(syn.spectrum_matrix(300, 200, syn.power_decay(200), 93))
    Om = f64(syn.gaussian(30, 300, 94))
    res, _ = O.randomized_cur(A, Om, k=20, q=1)
    s = np.linalg.svd(A, compute_uv=False)
    opt = np.sqrt(np.sum(s[20:] ** 2)) / np.sqrt(np.sum(s ** 2))
    e = O.rel_err_fro(A, res.C, res.U, res.R)
    assert opt <= e <= 10 * opt


def test_exhaustive_best_subset():
    """The greedy skeleton is never better than the best k-subset and is
    within a small factor of it on a tiny input."""
    g = np.random.default_rng(95)
    A = g.standard_normal((7, 9)) @ np.diag(np.logspace(0, -2, 9))
    k = 3
    best = np.inf
    for sub in itertools.combinations(range(9), k):
        C = A[:, sub]
        Qc, _ = np.linalg.qr(C)
        best = min(best, fro(A - Qc @ (Qc.T @ A)))
    r = O.id_col(A, k=k)
    e = fro(A - A[:, r.J[:k]] @ O.vstar(r.J, r.T, 9))
    assert best <= e * (1 + 1e-12)
    assert e <= 3 * best


# --- structured sampling matrix (Section 5.2, Eq. (5.2)) ----------------------

def _srft_draw(m, l, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(m, l, replace=False), rng.choice([-1.0, 1.0], m)


@pytest.mark.parametrize("m,l", [(37, 9), (64, 64), (1000, 80), (997, 250)])
def test_srft_rows_orthogonal(m, l):
    """R F D has orthonormal rows (F orthogonal, D a sign matrix, R a row
    selection without replacement), so Omega Omega^T = (m / l) I."""
    rows, signs = _srft_draw(m, l, m + l)
    Om = O.srft_omega_rows(m, rows, signs)
    np.testing.assert_allclose(Om @ Om.T, (m / l) * np.eye(l), atol=1e-12 * m / l, rtol=0)


@pytest.mark.parametrize("m", [7, 12, 501])
def test_srft_cosine_closed_form(m):
    """Discrete orthogonality of cosines: for g_t = cos(pi f0 (2t+1) / (2m)),
    sum_t g_t cos(pi f (2t+1) / (2m)) = (m/2) delta_{f f0} for f0 > 0 and
    m delta_{f 0} for f0 = 0.  Fed x = D g (so D x = g), the sketch is
    sqrt(m/l) c_{f0} (m/2 or m) at the row that samples f0 and zero
    elsewhere: sqrt(m/l) sqrt(m/2) or sqrt(m/l) sqrt(m)."""
    l = min(m, 5)
    rng = np.random.default_rng(m)
    signs = rng.choice([-1.0, 1.0], m)
    t = np.arange(m)
    for f0 in (0, 1, m // 2, m - 1):
        rows = np.array([f0] + [f for f in rng.permutation(m) if f != f0][: l - 1])
        g = np.cos(np.pi * f0 * (2 * t + 1) / (2 * m))
        Y = O.srft_sketch((signs * g)[:, None], rows, signs)[:, 0]
        expect = np.zeros(l)
        expect[0] = np.sqrt(m / l) * (np.sqrt(m) if f0 == 0 else np.sqrt(m / 2))
        np.testing.assert_allclose(Y, expect, atol=1e-12 * np.sqrt(m), rtol=0)


def test_srft_library_convention_matches_definition():
    """scipy's orthonormal DCT-II (the library step the oracle uses) against
    the transform as defined, F(f, t) = c_f cos(pi f (2t+1) / (2m)), built
    entry by entry on a small m."""
    import scipy.fft
    m = 11
    f, t = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    F = np.where(f == 0, np.sqrt(1 / m), np.sqrt(2 / m)) * np.cos(np.pi * f * (2 * t + 1) / (2 * m))
    X = np.random.default_rng(3).standard_normal((m, 4))
    np.testing.assert_allclose(scipy.fft.dct(X, type=2, norm="ortho", axis=0), F @ X,
                               atol=1e-13, rtol=0)


def test_srft_sketch_equals_omega_times_a():
    m, n, l = 300, 40, 24
    rows, signs = _srft_draw(m, l, 11)
    A = np.random.default_rng(12).standard_normal((m, n))
    np.testing.assert_allclose(O.srft_sketch(A, rows, signs),
                               O.srft_omega_rows(m, rows, signs) @ A, atol=1e-12, rtol=0)


def test_srft_randomized_exact_rank():
    """Algorithm 4 with the structured Omega (l = 2k) recovers an exact
    rank-k matrix to rounding (any sketch whose rows span A's row space)."""
    m, n, k = 400, 300, 20
    rng = np.random.default_rng(21)
    A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    rows, signs = _srft_draw(m, 2 * k, 22)
    Om = O.srft_omega_rows(m, rows, signs)
    o, Y = O.randomized_cur(A, Om, k)
    np.testing.assert_allclose(Y, O.srft_sketch(A, rows, signs), atol=1e-10, rtol=0)
    assert O.rel_err_fro(A, o.C, o.U, o.R) <= 1e-12


# --- error-corrected U (Section 4.3, Eq. (4.3)) --------------------------------

def _randomized_skeleton(seed=61, q=0):
    m, n, k = 300, 220, 25
    A = f64(syn.spectrum_matrix(m, n, syn.power_decay(n), seed, torch.float64))
    Om = np.random.default_rng(seed + 1).standard_normal((k + 5, m))
    return A, Om, k, q


def test_corrected_u_closed_form():
    """U R = V* + C^+ E with E = A - C V* has the least-squares solution
    C^+ (C V* + E) R^+ = C^+ A R^+; checked against library pseudo-inverses
    on a randomized skeleton (where C^+ E is not zero)."""
    A, Om, k, q = _randomized_skeleton()
    o, _ = O.randomized_cur_corrected(A, Om, k, q=q)
    U = np.linalg.pinv(o.C) @ A @ np.linalg.pinv(o.R)
    np.testing.assert_allclose(o.U, U, atol=1e-9 * np.abs(U).max(), rtol=0)
    base, _ = O.randomized_cur(A, Om, k, q=q)
    assert np.abs(base.U - o.U).max() > 1e-6 * np.abs(U).max()  # the correction is not void


def test_corrected_u_is_optimal():
    """For fixed C and R the corrected U minimises ||A - C U R||_F: no
    perturbation and not the uncorrected U of Eq. (4.2) does better."""
    A, Om, k, q = _randomized_skeleton(seed=71)
    o, _ = O.randomized_cur_corrected(A, Om, k, q=q)
    e = O.rel_err_fro(A, o.C, o.U, o.R)
    base, _ = O.randomized_cur(A, Om, k, q=q)
    assert e < O.rel_err_fro(A, base.C, base.U, base.R)
    rng = np.random.default_rng(72)
    for _ in range(5):
        D = rng.standard_normal(o.U.shape) * 1e-3 * np.abs(o.U).max()
        assert e <= O.rel_err_fro(A, o.C, o.U + D, o.R) * (1 + 1e-12)


def test_corrected_u_vanishes_for_deterministic_id():
    """With the column ID from the CPQR of A itself, E = Q2 S22 (Eq. (2.5))
    is orthogonal to range(C) = range(Q1), so C^+ E = 0 and Eq. (4.3)
    reduces to Eq. (4.2)."""
    A = f64(syn.spectrum_matrix(200, 150, syn.exp_decay(150), 81, torch.float64))
    k = 20
    a = O.cur(A, k)
    b = O.cur_corrected(A, k)
    assert list(a.J) == list(b.J) and list(a.I) == list(b.I)
    np.testing.assert_allclose(b.U, a.U, atol=1e-8 * np.abs(a.U).max(), rtol=0)


def test_corrected_u_exact_rank():
    m, n, k = 250, 180, 15
    rng = np.random.default_rng(91)
    A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    Om = rng.standard_normal((k + 5, m))
    o, _ = O.randomized_cur_corrected(A, Om, k)
    assert O.rel_err_fro(A, o.C, o.U, o.R) <= 1e-12


# --- regularised T (Section 4.1, Tikhonov term) --------------------------------

def _graded_s1(k, n, cond, seed):
    """Upper-trapezoidal S1 = [S11 S12] with S11 of condition about cond."""
    rng = np.random.default_rng(seed)
    d = np.logspace(0, -np.log10(cond), k)
    S11 = np.triu(rng.standard_normal((k, k)) * 0.1 * d[None, :]) + np.diag(d)
    S12 = rng.standard_normal((k, n - k)) * d[:, None]
    return np.hstack([S11, S12])


def test_tikhonov_t_zero_lambda_is_back_substitution():
    S1 = _graded_s1(12, 40, 1e3, 1)
    np.testing.assert_allclose(O.interpolation_matrix_tikhonov(S1, 12, 0.0),
                               O.interpolation_matrix(S1, 12), rtol=0, atol=1e-10)


def test_tikhonov_t_filter_factors():
    """Closed form through the SVD S11 = U diag(s) V^T (library SVD): the
    regularised solution is V diag(s / (s^2 + lam^2)) U^T S12."""
    k, n = 15, 50
    S1 = _graded_s1(k, n, 1e6, 2)
    Us, sv, Vt = np.linalg.svd(S1[:, :k])
    for lam in (1e-6, 1e-3, 0.1):
        T = O.interpolation_matrix_tikhonov(S1, k, lam)
        ref = Vt.T @ np.diag(sv / (sv ** 2 + lam ** 2)) @ Us.T @ S1[:, k:]
        np.testing.assert_allclose(T, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_tikhonov_t_normal_equations_and_shrinkage():
    """(S11^T S11 + lam^2 I) T = S11^T S12 holds, and ||T_lam||_F decreases
    as lam grows."""
    k, n = 10, 30
    S1 = _graded_s1(k, n, 1e4, 3)
    S11, S12 = S1[:, :k], S1[:, k:]
    norms = []
    for lam in (1e-5, 1e-3, 1e-1, 1.0):
        T = O.interpolation_matrix_tikhonov(S1, k, lam)
        lhs = (S11.T @ S11 + lam ** 2 * np.eye(k)) @ T
        np.testing.assert_allclose(lhs, S11.T @ S12, rtol=0, atol=1e-10 * np.abs(S11.T @ S12).max())
        norms.append(np.linalg.norm(T))
    assert all(a > b for a, b in zip(norms, norms[1:]))


# --- adaptive rank with a sketch -------------------------------------------------

def test_randomized_adaptive_exact_rank():
    """An exact rank-r matrix: every sample with more than r rows has rank r,
    its residual after r steps is rounding, so the search stops at k = r (in
    the first sample that leaves l - p > r)."""
    m, n, r, p = 500, 400, 70, 10
    rng = np.random.default_rng(101)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    Om = rng.standard_normal((512, m))
    k, l, Y = O.randomized_rank_adaptive(A, Om, 1e-10, p)
    assert k == r and l == 128  # 64 - 10 < 70 <= 128 - 10


def test_randomized_adaptive_stop_is_minimal():
    """The rank returned is the smallest j whose sample residual meets the
    tolerance: the residual of the first k - 1 pivots does not, that of k
    does, both measured by an independent projection of the sample onto the
    span of the chosen columns."""
    m, n, p = 600, 450, 10
    A = f64(syn.spectrum_matrix(m, n, syn.exp_decay(n, 6.0), 102, torch.float64))
    Om = np.random.default_rng(103).standard_normal((600, m))
    tol = 1e-5
    k, l, Y = O.randomized_rank_adaptive(A, Om, tol, p)
    assert 0 < k < l - p
    J = O.cpqr(Y, k=k).J

    def resid(j):
        if j == 0:
            return fro(Y)
        Q, _ = np.linalg.qr(Y[:, J[:j]])
        return fro(Y - Q @ (Q.T @ Y))
    assert resid(k) <= tol * fro(Y) < resid(k - 1)


# --- truncated-SVD T (Section 4.1) ------------------------------------------------

def test_tsvd_t_full_rank_is_back_substitution():
    S1 = _graded_s1(14, 50, 1e4, 11)
    np.testing.assert_allclose(O.interpolation_matrix_tsvd(S1, 14, 1e-12),
                               O.interpolation_matrix(S1, 14), rtol=0, atol=1e-9)


def test_tsvd_t_drops_planted_singular_values():
    """S11 = Q1 diag(s) Q2^T with planted s (five of them below the cut):
    the result equals the least-squares solution restricted to the kept
    right singular directions, computed by library lstsq on S11 Q2_keep,
    and it is orthogonal to the dropped directions."""
    k, n = 16, 45
    rng = np.random.default_rng(12)
    Q1, _ = np.linalg.qr(rng.standard_normal((k, k)))
    Q2, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.concatenate([np.logspace(0, -2, k - 5), np.logspace(-7, -9, 5)])
    S11 = Q1 @ np.diag(s) @ Q2.T
    S12 = rng.standard_normal((k, n - k))
    S1 = np.hstack([S11, S12])
    T = O.interpolation_matrix_tsvd(S1, k, 1e-5)
    Vk = Q2[:, : k - 5]
    Y = np.linalg.lstsq(S11 @ Vk, S12, rcond=None)[0]
    np.testing.assert_allclose(T, Vk @ Y, rtol=0, atol=1e-9 * np.abs(T).max())
    assert np.abs(Q2[:, k - 5:].T @ T).max() <= 1e-9 * np.abs(T).max()


def test_tsvd_t_rank_deficient_is_minimum_norm():
    """Exactly singular S11 (rank 9 of 12): with the zero singular values
    dropped, T is the minimum-norm least-squares solution (library pinv)."""
    k, n = 12, 30
    rng = np.random.default_rng(13)
    S11 = rng.standard_normal((k, 9)) @ rng.standard_normal((9, k))
    S1 = np.hstack([S11, rng.standard_normal((k, n - k))])
    T = O.interpolation_matrix_tsvd(S1, k, 1e-10)
    np.testing.assert_allclose(T, np.linalg.pinv(S11, rcond=1e-10) @ S1[:, k:], rtol=0,
                               atol=1e-9 * np.abs(T).max())


# --- complex A ----------------------------------------------------------------

def _complex_spectrum(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return U @ np.diag(np.exp(-np.arange(n) / decay)) @ V.conj().T


def test_complex_oracle_on_real_input_is_the_real_oracle():
    A = f64(syn.spectrum_matrix(120, 90, syn.exp_decay(90), 301, torch.float64))
    r = O.cur(A, 15)
    c = O.cur_complex(A.astype(np.complex128), 15)
    assert list(c["J"]) == list(r.J) and list(c["I"]) == list(r.I)
    np.testing.assert_allclose(c["T"].real, r.T, atol=1e-10, rtol=0)
    np.testing.assert_allclose(c["U"].real, r.U, atol=1e-8 * np.abs(r.U).max(), rtol=0)
    assert np.abs(c["U"].imag).max() <= 1e-10 * np.abs(r.U).max()


def test_complex_pivots_invariant_under_unitary_rows():
    """Norms and projections of columns are unchanged by a unitary factor on
    the left, so the pivots are too (against LAPACK-free brute force: the
    same routine on W Y)."""
    A = _complex_spectrum(80, 60, 6.0, 302)
    W, _ = np.linalg.qr(np.random.default_rng(303).standard_normal((80, 80))
                        + 1j * np.random.default_rng(304).standard_normal((80, 80)))
    J1, _ = O.cpqr_complex(A, 12)
    J2, _ = O.cpqr_complex(W @ A, 12)
    assert list(J1[:12]) == list(J2[:12])


def test_complex_closed_forms_and_exact_rank():
    A = _complex_spectrum(100, 70, 5.0, 305)
    k = 14
    c = O.cur_complex(A, k)
    # T = C^+ A(:, J[k:]) and U = V* R^+ (library complex lstsq / pinv)
    Tls = np.linalg.lstsq(c["C"], A[:, c["J"][k:]], rcond=None)[0]
    np.testing.assert_allclose(c["T"], Tls, atol=1e-9 * np.abs(Tls).max(), rtol=0)
    Vs = np.zeros((k, 70), dtype=complex)
    Vs[np.arange(k), c["J"][:k]] = 1.0
    Vs[:, c["J"][k:]] = c["T"]
    np.testing.assert_allclose(c["U"], Vs @ np.linalg.pinv(c["R"]), atol=1e-8 * np.abs(c["U"]).max(),
                               rtol=0)
    rng = np.random.default_rng(306)
    B = (rng.standard_normal((90, 9)) + 1j * rng.standard_normal((90, 9))) @ \
        (rng.standard_normal((9, 60)) + 1j * rng.standard_normal((9, 60)))
    e = O.cur_complex(B, 9)
    E = B - e["C"] @ e["U"] @ e["R"]
    assert np.linalg.norm(E) <= 1e-12 * np.linalg.norm(B)


def test_complex_power_scheme_spans_closed_form():
    """With q = 1 the sample's row space is that of Omega (A A^*) A (the
    orthonormalisations change only a left factor): compare the orthogonal
    projectors onto the two row spaces."""
    rng = np.random.default_rng(307)
    A = _complex_spectrum(90, 70, 4.0, 308)
    Om = rng.standard_normal((12, 90)) + 1j * rng.standard_normal((12, 90))
    Y = O.sketch_complex(A, Om, q=1)
    Z = Om @ (A @ A.conj().T) @ A

    def proj(X):
        Q, _ = np.linalg.qr(X.conj().T)
        return Q @ Q.conj().T
    assert np.abs(proj(Y) - proj(Z)).max() <= 1e-9


def test_complex_row_id_reconstructs_c():
    """The row ID of C (CPQR of the conjugate transpose, Eq. (2.11) over C)
    is exact: C(I[k:], :) = T_W^* C(I[:k], :)."""
    A = _complex_spectrum(90, 60, 5.0, 309)
    k = 12
    c = O.cur_complex(A, k)
    C, I, TW = c["C"], c["I"], c["TW"]
    np.testing.assert_allclose(C[I[k:], :], TW.conj().T @ C[I[:k], :],
                               atol=1e-10 * np.abs(C).max(), rtol=0)
