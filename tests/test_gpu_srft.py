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
