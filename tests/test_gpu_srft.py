"""Structured sampling matrix of the accelerated randomized scheme (Section
5.2, Eq. (5.2)), real form: Omega = sqrt(m/l) R F D with F the orthonormal
DCT-II and D random signs.  The device-built Omega against the oracle's (rows
and signs drawn on the host and passed to both), the device draw of rows and
signs by its properties, and randomized CUR-IDs with this Omega against the
FP64 oracle, up to the benchmark size with l = 2k and no power step."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from parity import U64, gap_allows_exact, id_residual, np64, npi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def host_draw(m, l, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(m, l, replace=False), rng.choice([-1, 1], m)


def to_dev(rows, signs):
    return (torch.tensor(rows, dtype=torch.int32, device=DEV),
            torch.tensor(signs, dtype=torch.int8, device=DEV))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,l", [(37, 9), (1000, 17), (2049, 300), (8000, 400)])
def test_srft_omega_matches_oracle(dtype, m, l):
    rows, signs = host_draw(m, l, m + l)
    if m > 1000:
        rows[0] = 0  # the f = 0 row has its own scale
    Om = np64(curid.srft_omega(*to_dev(rows, signs), dtype=dtype))
    which = list(range(l)) if l <= 40 else list(range(0, l, max(1, l // 25))) + [l - 1]
    ref = O.srft_omega_rows(m, rows, signs, which=which)
    amp = np.sqrt(2.0 / l)
    atol = 1e-14 * amp if dtype == torch.float64 else 6.1e-8 * amp
    np.testing.assert_allclose(Om[which], ref, atol=atol, rtol=0)
    if dtype == torch.float64:
        np.testing.assert_allclose(Om @ Om.T, (m / l) * np.eye(l), atol=1e-12 * m / l, rtol=0)


@pytest.mark.parametrize("m,l", [(1, 1), (2, 2), (3, 3), (17, 17), (8000, 400), (20000, 1000)])
def test_srft_draw_properties(m, l):
    rows, signs = curid.srft_draw(m, l, 77, device=0)
    r, s = npi(rows), npi(signs)
    assert len(set(r.tolist())) == l and r.min() >= 0 and r.max() < m
    assert set(s.tolist()) <= {-1, 1}
    if m >= 8000:
        neg = int((s < 0).sum())
        assert abs(neg - m / 2) <= 5 * np.sqrt(m / 4)
        # rows spread over [0, m): each quarter holds about l / 4 of them
        counts = np.bincount(r * 4 // m, minlength=4)
        assert np.all(np.abs(counts - l / 4) <= 5 * np.sqrt(l * 3 / 16))
    rows2, signs2 = curid.srft_draw(m, l, 77, device=0)
    assert torch.equal(rows, rows2) and torch.equal(signs, signs2)
    if m >= 17:
        rows3, signs3 = curid.srft_draw(m, l, 78, device=0)
        assert not torch.equal(rows, rows3) and not torch.equal(signs, signs3)


def test_srft_rejects_bad_arguments():
    with pytest.raises(curid.CuridError):
        curid.srft_draw(10, 11, 1, device=0)
    with pytest.raises(ValueError):
        curid.srft_omega(torch.zeros(3, dtype=torch.int64, device=DEV),
                         torch.ones(10, dtype=torch.int8, device=DEV))


@pytest.mark.parametrize("dtype,tf32", [(torch.float64, False), (torch.float32, False),
                                        (torch.float32, True)])
def test_srft_randomized_cur_vs_oracle(dtype, tf32):
    m, n, k = 1500, 1100, 50
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), 51, dtype)
    rows, signs = host_draw(m, l, 52)
    Om = curid.srft_omega(*to_dev(rows, signs), dtype=dtype)
    r = curid.cur(A.to(DEV), k, p=l - k, q=0, omega=Om, tf32=tf32, want_c=True, want_r=True,
                  want_t=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur(Ah, O.srft_omega_rows(m, rows, signs), k)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    if (dtype == torch.float64 and gap_allows_exact(o.ts.col.qr, k, U64)
            and gap_allows_exact(o.ts.row.qr, k, U64)):
        assert list(J) == list(o.J) and list(I) == list(o.I)
        assert abs(eg - eo) <= 1e-12
    else:
        assert eg <= 1.05 * eo, (eg, eo)
        assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)


def test_srft_full_size_tf32():
    """The benchmark matrix (float32 8000 x 6000, sigma_j = j^-2), k = 200,
    l = 2k = 400 (two row chunks in the tensor-core product), q = 0."""
    m, n, k = 8000, 6000, 200
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(n), 1413, torch.float32, DEV)
    rows, signs = host_draw(m, l, 1414)
    Om = curid.srft_omega(*to_dev(rows, signs), dtype=torch.float32)
    r = curid.cur(A, k, p=l - k, q=0, omega=Om, tf32=True, want_c=True, want_r=True,
                  want_t=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur(Ah, O.srft_omega_rows(m, rows, signs), k)
    J, I = npi(r.J), npi(r.I)
    assert sorted(J) == list(range(n)) and sorted(I) == list(range(m))
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)


# ---- the fast application (curid_srft_sketch): Y = Omega A without Omega ----

def fast_tol(dtype, ref):
    """float64: rounding of an O(m log m) transform; float32: the transform's
    single-precision rounding (measured below 3e-7 of max |Y| in a host run of
    the same arithmetic at m = 8000), with margin."""
    return (1e-12 if dtype == torch.float64 else 3e-6) * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("cols", ["2", "4"])
@pytest.mark.parametrize("m,n,lda,l", [(1000, 517, 520, 17), (2048, 130, 130, 300),
                                       (2835, 7, 9, 40), (1, 3, 3, 1), (7, 5, 5, 7),
                                       (12, 1, 1, 12)])
def test_srft_sketch_matches_oracle(monkeypatch, dtype, cols, m, n, lda, l):
    """Every entry of the fast Omega A against the oracle's DCT along the
    columns (Eq. (5.2)), rows and signs drawn on the host and passed to both.
    m = 1000 = 4 4 2 5 5 5 ... covers radices 4, 2, 5; 2835 = 3^4 5 7 covers
    3, 5, 7; n ragged against the 2 or 4 columns per CTA; padded lda; tiny m."""
    monkeypatch.setenv("CURID_SRFT_COLS", cols)
    rows, signs = host_draw(m, l, 7 * m + l)
    g = np.random.default_rng(m + n)
    Afull = g.standard_normal((m, lda))
    A = torch.from_numpy(Afull).to(dtype).to(DEV)[:, :n]
    Y = np64(curid.srft_sketch(A, *to_dev(rows, signs)))
    ref = O.srft_sketch(np64(A), rows, signs)
    np.testing.assert_allclose(Y, ref, atol=fast_tol(dtype, ref), rtol=0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_srft_sketch_periodic_rows(dtype):
    """Rows outside [0, m) read the periodic extension of F, as the explicit
    Omega does: the definition Omega(i, t) = s_i d_t cos(pi f_i (2t+1) / (2m))
    written out in float64 (s_i = sqrt(1/l) when f_i = 0 mod 4m, else
    sqrt(2/l)), including f = m (a zero row), 2m, 4m - 1 and negative f."""
    m, n = 60, 9
    rows = np.array([0, m, 2 * m, 4 * m - 1, -3, 5 * m + 7, 3 * m + 1, 4 * m, -4 * m, 11],
                    dtype=np.int64)
    l = len(rows)
    signs = np.random.default_rng(3).choice([-1, 1], m)
    A = torch.from_numpy(np.random.default_rng(4).standard_normal((m, n))).to(dtype).to(DEV)
    Y = np64(curid.srft_sketch(A, *to_dev(rows, signs)))
    t = np.arange(m)
    f = rows % (4 * m)
    s = np.where(f == 0, np.sqrt(1.0 / l), np.sqrt(2.0 / l))
    Om = s[:, None] * signs[None, :] * np.cos(np.pi * rows[:, None] * (2 * t[None, :] + 1) / (2 * m))
    ref = Om @ np64(A)
    np.testing.assert_allclose(Y, ref, atol=fast_tol(dtype, ref), rtol=0)
    assert np.abs(Y[1]).max() <= fast_tol(dtype, ref)


def test_srft_sketch_full_size_sampled():
    """The benchmark matrix, float32 8000 x 6000, l = 400: sampled rows of the
    fast Omega A against the oracle's rows of Omega applied one by one."""
    m, n, l = 8000, 6000, 400
    A = syn.spectrum_matrix(m, n, syn.power_decay(n), 1413, torch.float32, DEV)
    rows, signs = host_draw(m, l, 1414)
    Y = np64(curid.srft_sketch(A, *to_dev(rows, signs)))
    which = [0, 1, 57, 199, 398, 399]
    Om = O.srft_omega_rows(m, rows, signs, which=which)
    ref = Om @ np64(A)
    np.testing.assert_allclose(Y[which], ref, atol=fast_tol(torch.float32, ref), rtol=0)


def test_srft_sketch_unsupported_and_invalid():
    A = torch.randn(22, 8, device=DEV)  # 22 = 2 x 11: a prime factor above 7
    rows, signs = to_dev(np.arange(4), np.ones(22, dtype=np.int64))
    with pytest.raises(curid.CuridError) as e:
        curid.srft_sketch(A, rows, signs)
    assert e.value.status == 8
    Ab = torch.zeros(64, 64, dtype=torch.bfloat16, device=DEV)
    with pytest.raises(curid.CuridError) as e:
        curid.cur(Ab, 8, p=8, omega=curid.Srft(*to_dev(np.arange(16), np.ones(64))))
    assert e.value.status == 8
    with pytest.raises(curid.CuridError) as e:
        curid.cur(torch.randn(64, 64, device=DEV), 8, p=-1,
                  omega=curid.Srft(*to_dev(np.arange(16), np.ones(64))))
    assert e.value.status == 1


@pytest.mark.parametrize("dtype,tf32,q", [(torch.float64, False, 0), (torch.float32, True, 0),
                                          (torch.float32, False, 1)])
def test_fast_srft_randomized_cur_vs_oracle(dtype, tf32, q):
    """The decomposition with the structured Omega applied fast (omega =
    Srft(rows, signs)) against the FP64 oracle with the same Omega formed."""
    m, n, k = 1500, 1100, 50
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), 51, dtype)
    rows, signs = host_draw(m, l, 52)
    r = curid.cur(A.to(DEV), k, p=l - k, q=q, omega=curid.Srft(*to_dev(rows, signs)), tf32=tf32,
                  want_c=True, want_r=True, want_t=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur(Ah, O.srft_omega_rows(m, rows, signs), k, q=q)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    if (dtype == torch.float64 and gap_allows_exact(o.ts.col.qr, k, U64)
            and gap_allows_exact(o.ts.row.qr, k, U64)):
        assert list(J) == list(o.J) and list(I) == list(o.I)
        assert abs(eg - eo) <= 1e-12
    else:
        assert eg <= 1.05 * eo, (eg, eo)
        assert abs(eg - eo) <= 1e-5, (eg, eo)
        assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)


def test_fast_srft_full_size():
    """The benchmark matrix (float32 8000 x 6000, sigma_j = j^-2), k = 200,
    l = 400, q = 0, with the structured Omega applied fast: the CUR error
    within 1e-5 of the oracle's with the same Omega formed."""
    m, n, k = 8000, 6000, 200
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(n), 1413, torch.float32, DEV)
    rows, signs = host_draw(m, l, 1414)
    r = curid.cur(A, k, p=l - k, q=0, omega=curid.Srft(*to_dev(rows, signs)), tf32=True,
                  want_c=True, want_r=True, want_t=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur(Ah, O.srft_omega_rows(m, rows, signs), k)
    J = npi(r.J)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    assert abs(eg - eo) <= 1e-5, (eg, eo)
    assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)
