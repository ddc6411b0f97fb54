"""GPU parity of the precision form with BF16 storage of A: the BF16
tensor-core products (sample operand split into two BF16 parts) and the
randomized CUR-ID around them, against float64 products and the FP64 oracle
on the same BF16 values."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from parity import id_residual, np64, npi

pytestmark = pytest.mark.gpu


def bf16_matrix(m, n, seed, scale=8.0):
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), scale), seed, torch.float32)
    return A.to(torch.bfloat16).to("cuda:0").contiguous()


@pytest.mark.parametrize("m,n,l", [(1024, 800, 64), (1200, 1000, 300), (1600, 1200, 520)])
def test_bf16_product_matches_float64(m, n, l):
    """Y = Omega A with A in BF16 (one, two and three sample chunks; ragged
    column and K tails) against the float64 product of the same values."""
    A = bf16_matrix(m, n, 61)
    Om = syn.gaussian(l, m, 62, torch.float32).to("cuda:0")
    Y = curid.sketch_matrix(A, Om, q=0)
    ref = np64(Om) @ np64(A.float())
    err = np.max(np.abs(np64(Y) - ref)) / np.max(np.abs(ref))
    assert err <= 2e-5, err


@pytest.mark.parametrize("m,n,l", [(1024, 800, 64), (1200, 1000, 300)])
def test_bf16_power_sketch_matches_oracle(m, n, l):
    """One power step: both operand orientations (X A and X A^T) and the
    orthonormalisation between them, against the oracle's sketch."""
    A = bf16_matrix(m, n, 63)
    Om = syn.gaussian(l, m, 64, torch.float32).to("cuda:0")
    Y = curid.sketch_matrix(A, Om, q=1)
    ref = O.sketch(np64(A.float()), np64(Om), q=1)
    err = np.max(np.abs(np64(Y) - ref)) / np.max(np.abs(ref))
    assert err <= 5e-3, err


@pytest.mark.parametrize("m,n,k,p,q", [(1200, 1000, 60, 20, 2), (1600, 1200, 300, 20, 2)])
def test_bf16_randomized_cur_vs_oracle(m, n, k, p, q):
    A = bf16_matrix(m, n, 65, scale=40.0)
    Om = syn.gaussian(k + p, m, 66, torch.float32).to("cuda:0")
    r = curid.cur(A, k, p=p, q=q, omega=Om, want_c=True, want_r=True, want_t=True)
    Ah = np64(A.float())
    o, _ = O.randomized_cur(Ah, np64(Om), k, q=q)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C.float()), np64(r.R.float()), np64(r.U), np64(r.T)
    assert r.C.dtype == torch.bfloat16 and r.T.dtype == torch.float32
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    assert id_residual(Ah, J, T, k) <= 1.05 * id_residual(Ah, o.J, o.T, k)


def test_bf16_requires_randomized_and_alignment():
    A = bf16_matrix(256, 200, 67)
    with pytest.raises(curid.CuridError) as e:
        curid.cur(A, 10, p=-1)
    assert e.value.status == 8
    B = torch.zeros((256, 203), dtype=torch.bfloat16, device="cuda:0")
    with pytest.raises(curid.CuridError) as e:
        curid.cur(B, 10, p=5, seed=1)
    assert e.value.status == 8


def rel_err_gpu(A, C, U, R):
    """||A - C U R||_F / ||A||_F in float64 on the GPU."""
    Ad = A.double()
    D = Ad - (C.double() @ U) @ R.double()
    return float(torch.linalg.norm(D) / torch.linalg.norm(Ad))


def check_against_oracle(A, k, p, q, Om):
    """Randomized CUR-ID of the BF16 matrix A on the GPU and in the FP64
    oracle on the same BF16 values with the same Omega: C and R exact copies
    of A's entries, the CUR error within 1.05x of the oracle's.  Returns both
    errors.  (The 1e-5 bar on the difference is the float32-storage
    criterion; here both errors sit on the BF16 storage floor near 5e-3,
    where a skeleton chosen in float32 arithmetic differs from the float64
    one by about 1 % in error.)"""
    m, n = A.shape
    r = curid.cur(A, k, p=p, q=q, omega=Om, want_c=True, want_r=True)
    assert r.status == 0 and r.k == k
    J, I = r.J.long(), r.I.long()
    assert torch.equal(r.C, A[:, J[:k]]) and torch.equal(r.R, A[I[:k], :])
    assert sorted(J.tolist()) == list(range(n)) and sorted(I.tolist()) == list(range(m))
    eb = rel_err_gpu(A, r.C, r.U, r.R)
    Ah = np64(A.float())
    o, _ = O.randomized_cur(Ah, np64(Om), k, q=q)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eb < 1e-2, eb
    assert eb <= 1.05 * eo, (eb, eo)
    return eb, eo


def test_bf16_c3_shape_vs_oracle():
    """The full workload's spectrum, rank and sketch (sigma_j = 10^(-6j/500)
    for j <= 500, floor 1e-7, k = 500, p = 20, q = 2: l = 520, three sample
    chunks, blocked Gram factorisations of order 520) on a 4096 x 4096 BF16
    matrix, against the FP64 oracle."""
    w = syn.workload_mixed_bf16(device="cuda:0", m=4096, n=4096)
    Om = curid.gaussian(w["k"] + w["p"], 4096, 72, torch.float32)
    check_against_oracle(w["A"], w["k"], w["p"], w["q"], Om)


def test_bf16_full_config():
    """A 20000 x 20000 BF16, sigma_j = 10^(-6j/500) (j <= 500), floor 1e-7,
    k = 500, p = 20, q = 2, against the FP64 oracle on the same values and
    the same Omega (the storage rounding of A bounds both errors near 5e-3)."""
    w = syn.workload_mixed_bf16(device="cuda:0")
    A, k, p, q = w["A"], w["k"], w["p"], w["q"]
    Om = curid.gaussian(k + p, A.shape[0], 71, torch.float32)
    check_against_oracle(A, k, p, q, Om)
