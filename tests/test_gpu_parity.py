"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on
seeded synthetic inputs: sizes the oracle finishes in seconds, spanning
several column slabs per CTA, ragged tails and the degenerate cases."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from oracle.philox import gaussian as philox_gaussian
from parity import (U32, U64, assert_s_rows_match, fro, gap_allows_exact, id_residual, np64,
                    npi, s_by_column)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cuda(t):
    return t.to(DEV)


# --- Omega generator -----------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gaussian_matches_philox_reference(dtype):
    rows, cols, seed = 37, 1001, 0x1234567890AB
    g = np64(curid.gaussian(rows, cols, seed, dtype=dtype, device=0))
    ref = philox_gaussian(rows, cols, seed)
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    np.testing.assert_allclose(g, ref, atol=tol * 10, rtol=tol)


# --- sketch products -------------------------------------------------------------

@pytest.mark.parametrize("dtype,q", [(torch.float64, 0), (torch.float64, 1), (torch.float32, 0),
                                     (torch.float32, 1), (torch.float64, 2)])
def test_sketch_matrix(dtype, q):
    m, n, l = 700, 515, 37
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 30.0), 501, dtype)
    Om = syn.gaussian(l, m, 502, dtype)
    Y = np64(curid.sketch_matrix(cuda(A), cuda(Om), q=q))
    Yo = O.sketch(np64(A), np64(Om), q=q)
    if q == 0:
        tol = 1e-12 if dtype == torch.float64 else 2e-5
        np.testing.assert_allclose(Y, Yo, atol=tol * np.abs(Yo).max(), rtol=0)
    else:
        # orth is unique up to the rounding of each side; compare row spaces
        def proj(M):
            Qm, _ = np.linalg.qr(M.T)
            return Qm @ Qm.T
        d = fro(proj(Y) - proj(Yo))
        assert d <= (1e-8 if dtype == torch.float64 else 2e-3), d


# --- CPQR ----------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,k,seed", [(60, 40, 12, 1), (40, 70, 20, 2), (128, 1000, 33, 3),
                                        (33, 4099, 30, 4), (300, 157, 60, 5)])
def test_cpqr_planted(dtype, m, n, k, seed):
    # FP32 keeps every planted diagonal far above its rounding level
    decay = 2.0 ** -0.5 if dtype == torch.float64 else 0.85
    A, perm = syn.planted_pivots(m, n, k, seed, decay=decay, dtype=dtype)
    r = curid.cpqr(cuda(A), k=k)
    J = npi(r.J)
    assert list(J[:k]) == list(perm[:k])
    assert sorted(J) == list(range(n))
    assert list(J[k:]) == sorted(J[k:])
    o = O.cpqr(np64(A), k=k)
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    assert_s_rows_match(r.S, s_by_column(o.S1, o.J, n), k, tol)


@pytest.mark.parametrize("m,n,k,seed", [(400, 300, 40, 11), (64, 2000, 50, 12),
                                        (1000, 1999, 80, 13)])
def test_cpqr_random_f64(m, n, k, seed):
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 10.0), seed)
    r = curid.cpqr(cuda(A), k=k)
    o = O.cpqr(np64(A), k=k)
    J = npi(r.J)
    if gap_allows_exact(o, k, U64):
        assert list(J[:k]) == list(o.J[:k])
        assert_s_rows_match(r.S, s_by_column(o.S1, o.J, n), k, 1e-10)
    else:
        T = O.interpolation_matrix(np64(r.S)[:, J], k)
        assert id_residual(A, J, T, k) <= 1.05 * id_residual(A, o.J, O.id_col(np64(A), k).T, k)


def test_cpqr_adaptive_tolerance():
    A = syn.spectrum_matrix(500, 400, syn.exp_decay(400, 8.0), 21)
    tol = 1e-6
    r = curid.cpqr(cuda(A), k=0, tol=tol)
    o = O.cpqr(np64(A), tol=tol)
    assert r.k == o.k
    assert list(npi(r.J)[:o.k]) == list(o.J[:o.k])


@pytest.mark.parametrize("dtype,l,n,k", [(torch.float32, 250, 9728, 60),
                                         (torch.float32, 200, 5000, 60),
                                         (torch.float32, 161, 2437, 40),
                                         (torch.float64, 100, 7600, 40),
                                         (torch.float64, 128, 9700, 48)])
def test_cpqr_register_slabs(dtype, l, n, k):
    """Orders that keep the slab in registers (l <= 256 in float32, <= 128 in
    float64; up to 64 columns per CTA: 9728 = 64 x 152): 4, 7 and 8 rows per
    lane, full and ragged slabs.  Planted pivot order exact, S rows as the
    oracle's."""
    decay = 0.85 if dtype == torch.float32 else 2 ** -0.5
    A, perm = syn.planted_pivots(l, n, k, 45 + l, decay=decay, dtype=dtype)
    r = curid.cpqr(cuda(A), k=k)
    J = npi(r.J)
    assert list(J[:k]) == list(perm[:k])
    assert sorted(J.tolist()) == list(range(n)) and list(J[k:]) == sorted(J[k:].tolist())
    o = O.cpqr(np64(A), k=k)
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    assert_s_rows_match(r.S, s_by_column(o.S1, o.J, n), k, tol)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cpqr_adaptive_register_slabs(dtype):
    """Tolerance stop on a register-resident slab (120 x 3000): the rank and
    pivots of the oracle's stop."""
    A = syn.spectrum_matrix(120, 3000, syn.exp_decay(120, 6.0), 46, dtype)
    tol = 1e-6 if dtype == torch.float64 else 1e-3
    r = curid.cpqr(cuda(A), k=0, tol=tol)
    o = O.cpqr(np64(A), tol=tol)
    u = U64 if dtype == torch.float64 else U32
    if gap_allows_exact(o, o.k, u):
        assert r.k == o.k
        assert list(npi(r.J)[:o.k]) == list(o.J[:o.k])
    else:
        assert abs(r.k - o.k) <= 1


def test_cpqr_ties_smallest_index():
    g = np.random.default_rng(7)
    A = g.standard_normal((64, 300))
    A[:, 250] = A[:, 17] = 10 * g.standard_normal(64)
    r = curid.cpqr(cuda(torch.from_numpy(A)), k=3)
    assert int(r.J[0]) == 17


def test_cpqr_full_rank_steps_and_k1():
    A = syn.spectrum_matrix(50, 30, syn.exp_decay(30, 5.0), 22)
    for k in (1, 30):
        r = curid.cpqr(cuda(A), k=k)
        o = O.cpqr(np64(A), k=k)
        assert list(npi(r.J)[:k]) == list(o.J[:k])


# --- deterministic ID / tsID / CUR in FP64 (400 x 300, sigma_j = exp(-j/10), k = 40) ---

def small_f64():
    w = syn.workload_small_f64()
    return w["A"], w["k"]


def test_id_col_f64():
    A, k = small_f64()
    r = curid.id_col(cuda(A), k)
    o = O.id_col(np64(A), k)
    assert gap_allows_exact(o.qr, k, U64)
    assert list(npi(r.J)) == list(o.J)
    np.testing.assert_allclose(np64(r.T), o.T, atol=1e-11 * np.abs(o.T).max(), rtol=0)


def test_id_row_f64():
    A, k = small_f64()
    r = curid.id_row(cuda(A), k)
    o = O.id_row(np64(A), k)
    assert list(npi(r.I)) == list(o.J)
    np.testing.assert_allclose(np64(r.TW), o.T, atol=1e-11 * np.abs(o.T).max(), rtol=0)


def test_tsid_f64():
    A, k = small_f64()
    r = curid.tsid(cuda(A), k)
    o = O.tsid(np64(A), k)
    assert list(npi(r.J)) == list(o.J)
    assert list(npi(r.I)) == list(o.I)
    np.testing.assert_allclose(np64(r.T), o.T, atol=1e-11 * np.abs(o.T).max(), rtol=0)
    np.testing.assert_allclose(np64(r.TW), o.TW, atol=1e-11 * np.abs(o.TW).max(), rtol=0)


def test_cur_f64():
    A, k = small_f64()
    r = curid.cur(cuda(A), k, want_c=True, want_r=True, want_t=True, want_tw=True)
    o = O.cur(np64(A), k)
    J, I = npi(r.J), npi(r.I)
    assert list(J) == list(o.J) and list(I) == list(o.I)
    Ah = np64(A)
    # C and R are exact copies
    assert np.array_equal(np64(r.C), Ah[:, J[:k]])
    assert np.array_equal(np64(r.R), Ah[I[:k], :])
    U = np64(r.U)
    np.testing.assert_allclose(U, o.U, rtol=0, atol=1e-8 * np.abs(o.U).max())
    eg = O.rel_err_fro(Ah, np64(r.C), U, np64(r.R))
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert abs(eg - eo) <= 1e-12, (eg, eo)


def test_cur_exact_rank_f64():
    A = syn.exact_rank(333, 257, 17, 23)
    r = curid.cur(cuda(A), 17, want_c=True, want_r=True)
    assert O.rel_err_fro(np64(A), np64(r.C), np64(r.U), np64(r.R)) <= 1e-12


# --- randomized CUR ------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_randomized_cur_moderate(dtype):
    m, n, k, p, q = 1500, 1100, 50, 10, 1
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), 31, dtype)
    Om = syn.gaussian(k + p, m, 32, dtype)
    r = curid.cur(cuda(A), k, p=p, q=q, omega=cuda(Om), want_c=True, want_r=True, want_t=True)
    o, _ = O.randomized_cur(np64(A), np64(Om), k, q=q)
    Ah = np64(A)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    # same skeleton: U against the FP64 least-squares U on the GPU's J, T, I
    Uo = O.cur_middle(R, O.vstar(J, T, n))
    e_same = O.rel_err_fro(Ah, C, Uo, R)
    if dtype == torch.float64:
        assert list(J) == list(o.J) and list(I) == list(o.I)
        assert abs(eg - eo) <= 1e-12
    else:
        assert abs(eg - e_same) <= 1e-5, (eg, e_same)
        assert eg <= 1.05 * eo, (eg, eo)
        assert abs(eg - eo) <= 1e-5, (eg, eo)


@pytest.mark.parametrize("dtype,k,p", [(torch.float32, 246, 10), (torch.float64, 182, 10),
                                       (torch.float32, 300, 20), (torch.float64, 240, 10)])
def test_randomized_cur_large_order(dtype, k, p):
    """l = k + p at the largest one-CTA orders of the Gram factorisation (256
    float32, 192 float64) and beyond them (blocked Cholesky and triangular
    solves; the T and U solves of order k blocked as well), with a power
    step."""
    m, n, q = 1200, 900, 1
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 60.0), 41, dtype)
    Om = syn.gaussian(k + p, m, 42, dtype)
    r = curid.cur(cuda(A), k, p=p, q=q, omega=cuda(Om), want_c=True, want_r=True, want_t=True)
    o, _ = O.randomized_cur(np64(A), np64(Om), k, q=q)
    Ah = np64(A)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)
    if dtype == torch.float64:
        assert list(J) == list(o.J) and list(I) == list(o.I)
        assert abs(eg - eo) <= 1e-12


def test_order_beyond_limit_is_unsupported():
    m = n = 4200
    A = torch.zeros((m, n), dtype=torch.float32, device="cuda:0")
    with pytest.raises(curid.CuridError) as e:
        curid.cur(A, 4090, p=10, q=1, seed=5)
    assert e.value.status == 8


@pytest.mark.parametrize("dtype,l,n,k", [(torch.float32, 520, 20000, 64),
                                         (torch.float32, 520, 30000, 64),
                                         (torch.float32, 600, 20000, 64),
                                         (torch.float64, 300, 40000, 48)])
def test_cpqr_overflow_columns(dtype, l, n, k):
    """Large slabs of the grouped shared-memory kernel.  520 x 20000 float32
    (132 columns of a CTA): 15 register groups and 18 groups in shared
    memory.  520 x 30000 (200 columns): register groups, shared memory and 8
    overflow groups in global memory.  600 x 20000 (rows beyond the register
    groups) and 300 x 40000 float64: shared memory and overflow only.  The
    planted pivot order must come out exactly, and S must match the oracle's
    rows up to sign."""
    Y, perm = syn.planted_pivots(l, n, k, 44, decay=0.85 if dtype == torch.float32 else 2 ** -0.5,
                                 dtype=dtype)
    r = curid.cpqr(cuda(Y), k=k)
    J = npi(r.J)
    assert list(J[:k]) == list(perm[:k])
    assert sorted(J.tolist()) == list(range(n)) and list(J[k:]) == sorted(J[k:].tolist())
    o = O.cpqr(np64(Y), k=k)
    S = np64(r.S)
    So = np.zeros((k, n))
    So[:, o.J] = o.S1
    for i in range(k):
        sgn = np.sign(S[i, J[i]]) * np.sign(So[i, J[i]])
        tol = 1e-4 if dtype == torch.float32 else 1e-10
        assert np.max(np.abs(sgn * S[i] - So[i])) <= tol * np.max(np.abs(So[i]))


@pytest.mark.parametrize("l,n,k,ctas", [(210, 6000, 120, None), (200, 3000, 80, "3")])
def test_cpqr_grouped_throughput_layout(monkeypatch, l, n, k, ctas):
    """The layout the library picks with eight or more decompositions in
    flight: the grouped kernel with 7-row register groups on the fewest CTAs
    that hold the sample (210 x 6000 float32: 19 CTAs).  With the grid forced
    down to three CTAs (200 x 3000: 1000 columns per CTA) most groups live in
    the global overflow area.  The planted pivot order must come out exactly,
    S must match the oracle's rows up to sign, and the concurrency is put
    back afterwards."""
    Y, perm = syn.planted_pivots(l, n, k, 45, decay=0.9, dtype=torch.float32)
    if ctas:
        monkeypatch.setenv("CURID_CPQR_KERNEL", "grouped")
        monkeypatch.setenv("CURID_CPQR_CTAS", ctas)
    curid.set_concurrency(8)
    try:
        r = curid.cpqr(cuda(Y), k=k)
    finally:
        curid.set_concurrency(1)
    J = npi(r.J)
    assert list(J[:k]) == list(perm[:k])
    assert sorted(J.tolist()) == list(range(n)) and list(J[k:]) == sorted(J[k:].tolist())
    o = O.cpqr(np64(Y), k=k)
    S = np64(r.S)
    So = np.zeros((k, n))
    So[:, o.J] = o.S1
    for i in range(k):
        sgn = np.sign(S[i, J[i]]) * np.sign(So[i, J[i]])
        assert np.max(np.abs(sgn * S[i] - So[i])) <= 1e-4 * np.max(np.abs(So[i]))


def test_random_omega_generated_on_device():
    m, n, k, p = 900, 700, 30, 10
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 6.0), 33)
    r = curid.cur(cuda(A), k, p=p, q=1, seed=99, want_c=True, want_r=True)
    Om = philox_gaussian(k + p, m, 99)
    o, _ = O.randomized_cur(np64(A), Om, k, q=1)
    assert list(npi(r.J)[:k]) == list(o.J[:k])
    eg = O.rel_err_fro(np64(A), np64(r.C), np64(r.U), np64(r.R))
    eo = O.rel_err_fro(np64(A), o.C, o.U, o.R)
    assert abs(eg - eo) <= 1e-11


# --- degenerate and invalid inputs -------------------------------------------------

def test_rank_deficient_status():
    A = syn.exact_rank(200, 150, 8, 41)
    r = curid.id_col(cuda(A), 12)
    assert r.status == 2 and r.k == 8
    T = np64(r.T)
    assert np.all(T[8:] == 0)
    assert id_residual(A, npi(r.J), T, 12) <= 1e-12


def test_nonfinite_input():
    A = syn.spectrum_matrix(100, 80, syn.exp_decay(80), 42)
    A[17, 33] = float("nan")
    with pytest.raises(curid.CuridError) as e:
        curid.id_col(cuda(A), 10)
    assert e.value.status == 4


def test_invalid_arguments():
    A = cuda(syn.spectrum_matrix(50, 40, syn.exp_decay(40), 43))
    with pytest.raises(curid.CuridError) as e:
        curid.id_col(A, 41)
    assert e.value.status == 1
    with pytest.raises(curid.CuridError):
        curid.cur(A, 10, p=40, q=0)          # k + p > min(m, n)
    with pytest.raises(curid.CuridError):
        curid.cur(A.double(), 5, p=5, tf32=True)  # TF32 needs float32


def test_handworked_example_gpu():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked_2x3.json")))
    A = torch.tensor(g["A"], dtype=torch.float64)
    for key, k in (("k1", 1), ("k2", 2)):
        r = curid.id_col(cuda(A), k)
        assert list(npi(r.J)) == g[key]["J"]
        np.testing.assert_allclose(np64(r.T), np.array(g[key]["T"]).reshape(k, -1)[:, :3 - k],
                                   atol=1e-15)


# --- tensor-core (tcgen05) products: X A_hi + X A_lo with X read as TF32 ---------

def tf32_exact(x):
    """Round-free TF32 values: float32 with the 13 low mantissa bits cleared."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


@pytest.mark.parametrize("m,n,lda,l", [(700, 516, 516, 37), (1000, 1024, 1024, 128),
                                       (333, 4000, 4000, 210), (8000, 6000, 6000, 210),
                                       (64, 132, 132, 16), (260, 257, 260, 256),
                                       (97, 1001, 1004, 33)])
def test_tensor_core_sketch_product(m, n, lda, l):
    """Y = Omega A on the tensor cores against tf32(Omega) A in float64: the
    differences are the truncation of A's low part (2^-22 |A|) and the
    tensor core's float32 accumulation over K (measured up to 6e-5 of |Y|
    at K = 8000; a tile-layout error would be O(1)).  Ragged shapes: n not a multiple of the 128-column
    tile, m (the K extent) not a multiple of 32, l not a multiple of 16, A
    with a padded leading dimension, Omega rows not 16-byte aligned."""
    g = np.random.default_rng(m + n + l)
    Afull = torch.from_numpy(g.standard_normal((m, lda)).astype(np.float32))
    A = cuda(Afull)[:, :n]
    Om = torch.from_numpy(tf32_exact(g.standard_normal((l, m))))
    Y = np64(curid.sketch_matrix(A, cuda(Om), q=0, tf32=True))
    ref = np64(Om) @ np64(Afull[:, :n])
    err = np.abs(Y - ref).max() / np.abs(ref).max()
    assert err <= 1e-4, err


def test_tensor_core_rejects_misaligned_rows():
    A = cuda(torch.randn(100, 130))
    Om = cuda(torch.randn(10, 100))
    with pytest.raises(curid.CuridError) as e:
        curid.sketch_matrix(A, Om, q=0, tf32=True)
    assert e.value.status == 8


@pytest.mark.parametrize("q", [1, 2])
def test_tensor_core_sketch_power(q):
    """Power steps use both product kinds (Q A^T and Q A); compare row spaces."""
    m, n, l = 1500, 1100, 60
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 40.0), 503, torch.float32)
    Om = syn.gaussian(l, m, 504, torch.float32)
    Y = np64(curid.sketch_matrix(cuda(A), cuda(Om), q=q, tf32=True))
    Yo = O.sketch(np64(A), np64(Om), q=q)

    def proj(M):
        Qm, _ = np.linalg.qr(M.T)
        return Qm @ Qm.T
    assert fro(proj(Y) - proj(Yo)) <= 5e-3


def test_tensor_core_randomized_cur():
    m, n, k, p, q = 1500, 1100, 50, 10, 1
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), 31, torch.float32)
    Om = syn.gaussian(k + p, m, 32, torch.float32)
    r = curid.cur(cuda(A), k, p=p, q=q, omega=cuda(Om), tf32=True, want_c=True, want_r=True,
                  want_t=True)
    o, _ = O.randomized_cur(np64(A), np64(Om), k, q=q)
    Ah = np64(A)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    assert abs(eg - eo) <= 1e-5, (eg, eo)
    assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)
    Uo = O.cur_middle(R, O.vstar(J, T, n))
    assert abs(eg - O.rel_err_fro(Ah, C, Uo, R)) <= 1e-5


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_adaptive_rank_decompositions(tol):
    """k = 0, tol > 0 (deterministic): the rank, skeletons and factors of the
    oracle's tolerance stop, through id_col, tsid and cur."""
    A = syn.spectrum_matrix(500, 400, syn.exp_decay(400, 8.0), 23)
    o = O.cur(np64(A), tol=tol)
    ko = o.k
    r1 = curid.id_col(cuda(A), 0, tol=tol)
    assert r1.k == ko and list(npi(r1.J)) == list(o.J)
    # both T are backward-stable solves of S11 T = S12: kappa(S11) u ||T||
    kappa = o.ts.col.qr.nu[0] / o.ts.col.qr.nu[ko - 1]
    assert np.linalg.norm(np64(r1.T) - o.T) <= 1e2 * kappa * U64 * max(1.0, np.linalg.norm(o.T))
    r2 = curid.tsid(cuda(A), 0, tol=tol)
    assert r2.k == ko and list(npi(r2.I)) == list(o.I)
    assert r2.TW.shape == (ko, 500 - ko)
    r3 = curid.cur(cuda(A), 0, tol=tol, want_c=True, want_r=True)
    assert r3.k == ko and r3.U.shape == (ko, ko) and r3.C.shape == (500, ko)
    Ah = np64(A)
    assert np.array_equal(np64(r3.C), Ah[:, npi(r3.J)[:ko]])
    eg = O.rel_err_fro(Ah, np64(r3.C), np64(r3.U), np64(r3.R))
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    # the stop bounds the ID residual; the CUR error may exceed tol (Lemma 3.1)
    assert id_residual(Ah, npi(r1.J), np64(r1.T), ko) <= tol * 1.05
    # U = V* R^+ solves with R, whose condition is about kappa(S11): each side's
    # CUR error carries rounding of order kappa u (2.6e-6 vs 3.2e-6 at 1e-10)
    assert abs(eg - eo) <= max(1e-12, 1e2 * kappa * U64), (eg, eo)


def test_adaptive_rank_zero_and_unsupported():
    Z = torch.zeros((60, 50), dtype=torch.float64, device="cuda:0")
    r = curid.cur(Z, 0, tol=1e-8)
    assert r.k == 0 and list(npi(r.J)) == list(range(50)) and list(npi(r.I)) == list(range(60))
    A = cuda(syn.spectrum_matrix(200, 150, syn.exp_decay(150, 8.0), 24))
    # with a sketch the rank is searched (tests/test_gpu_adaptive_sketch.py);
    # BF16 storage has no deterministic method to adapt
    with pytest.raises(curid.CuridError) as e:
        curid.cur(A.to(torch.bfloat16), 0, tol=1e-6)
    assert e.value.status == 8
