"""Randomized CUR-ID of a sparse A (curid_cur_sparse: sparse-times-dense
sketch and power products, gathers from the compressed rows and columns)
against the FP64 oracle on the same values held densely, and against the
dense GPU path; A is a sum of sparse non-negative rank-one terms shaped like
the A_1 / A_2 matrices of Section 6, up to their full 300000 x 300 size."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from oracle.philox import gaussian as philox_gaussian
from parity import U64, gap_allows_exact, id_residual, np64, npi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def check_against_oracle(As, dtype, k, p, q, seed, corrected=False):
    A = syn.to_torch_csr(As, dtype, DEV)
    r = curid.cur_sparse(A, k, p, q=q, seed=seed, corrected=corrected, want_c=True, want_r=True,
                         want_t=True)
    assert r.status == 0 and r.k == k
    Ah = torch.tensor(As.toarray()).to(dtype).double().numpy()  # the values the GPU holds
    m, n = Ah.shape
    Om = philox_gaussian(k + p, m, seed)
    if corrected:
        o, _ = O.randomized_cur_corrected(Ah, Om, k, q=q)
    else:
        o, _ = O.randomized_cur(Ah, Om, k, q=q)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    if (dtype == torch.float64 and gap_allows_exact(o.ts.col.qr, k, U64)
            and gap_allows_exact(o.ts.row.qr, k, U64)):
        assert list(J[:k]) == list(o.J[:k]) and list(I[:k]) == list(o.I[:k])
        assert abs(eg - eo) <= 1e-12, (eg, eo)
    else:
        assert eg <= 1.05 * eo, (eg, eo)
        assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)
    return r, eg


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("q", [0, 1])
def test_sparse_cur_matches_oracle(dtype, q):
    """4000 x 300, 300 terms at about 1 % density: some rows are empty."""
    As = syn.sparse_rank_sum(4000, 300, syn.a1_coeffs(), 201, dx=0.005, dy=0.03)
    assert np.any(np.diff(As.indptr) == 0)
    check_against_oracle(As, dtype, 20, 10, q, 202)


def test_sparse_cur_corrected_and_wide():
    """m < n (the CSC side has the long lists) and the error-corrected U."""
    As = syn.sparse_rank_sum(300, 2500, syn.a1_coeffs(terms=120, big=1000.0), 211,
                             dx=0.05, dy=0.01)
    _, e_plain = check_against_oracle(As, torch.float64, 15, 10, 0, 212)
    _, e_corr = check_against_oracle(As, torch.float64, 15, 10, 0, 212, corrected=True)
    assert e_corr <= e_plain * (1 + 1e-9)


def test_sparse_equals_dense_path():
    """The same values held densely through curid_cur (same seed, same
    Omega): the products differ only in summation order, so the skeletons
    agree where the oracle's pivot gaps are wide and the errors agree."""
    k = 12
    As = syn.sparse_rank_sum(3000, 300, syn.a1_coeffs(big=1000.0), 221, dx=0.004, dy=0.03)
    A = syn.to_torch_csr(As, torch.float64, DEV)
    Ad = torch.tensor(As.toarray(), dtype=torch.float64, device=DEV)
    rs = curid.cur_sparse(A, k, 10, q=1, seed=7, want_c=True, want_r=True)
    rd = curid.cur(Ad, k, p=10, q=1, seed=7, want_c=True, want_r=True)
    Ah = np64(Ad)
    o, _ = O.randomized_cur(Ah, philox_gaussian(k + 10, 3000, 7), k, q=1)
    if gap_allows_exact(o.ts.col.qr, k, U64) and gap_allows_exact(o.ts.row.qr, k, U64):
        assert torch.equal(rs.J[:k], rd.J[:k]) and torch.equal(rs.I[:k], rd.I[:k])
    es = O.rel_err_fro(Ah, np64(rs.C), np64(rs.U), np64(rs.R))
    ed = O.rel_err_fro(Ah, np64(rd.C), np64(rd.U), np64(rd.R))
    assert es <= 1.05 * ed and ed <= 1.05 * es, (es, ed)


def test_sparse_a1_full_size_f32():
    """A_1-shaped: 300000 x 300, 300 terms, about 1.07M stored entries;
    k = 40, p = 10, q = 2 (the power count of the paper's randomized
    comparisons), float32 against the FP64 oracle."""
    As = syn.sparse_rank_sum(300000, 300, syn.a1_coeffs(), 231)
    check_against_oracle(As, torch.float32, 40, 10, 2, 232)


def test_sparse_rejects_deterministic_and_dense_input():
    As = syn.sparse_rank_sum(500, 100, syn.a1_coeffs(terms=20), 241, dx=0.05, dy=0.2)
    A = syn.to_torch_csr(As, torch.float64, DEV)
    with pytest.raises(curid.CuridError):
        curid.cur_sparse(A, 5, -1)
    with pytest.raises(ValueError):
        curid.cur_sparse(A.to_dense(), 5, 5)
