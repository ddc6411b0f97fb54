"""CUR-ID with U from the error-corrected system of Section 4.3, Eq. (4.3)
(U R = V* + C^+ E, i.e. U = C^+ A R^+), through curid_cur_corrected,
against the FP64 oracle's cur_corrected on the same inputs: randomized
skeletons in float64, float32 and TF32 up to the benchmark size with the
structured sketch, and the deterministic case where the correction vanishes."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from parity import U64, gap_allows_exact, np64, npi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu_err(A, r):
    return O.rel_err_fro(A, np64(r.C), np64(r.U), np64(r.R))


@pytest.mark.parametrize("dtype,tf32", [(torch.float64, False), (torch.float32, False),
                                        (torch.float32, True)])
@pytest.mark.parametrize("q", [0, 1])
def test_corrected_randomized_vs_oracle(dtype, tf32, q):
    m, n, k, p = 1500, 1100, 50, 10
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), 31, dtype)
    Om = syn.gaussian(k + p, m, 32, dtype)
    r = curid.cur(A.to(DEV), k, p=p, q=q, omega=Om.to(DEV), tf32=tf32, want_c=True,
                  want_r=True, want_t=True, corrected=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur_corrected(Ah, np64(Om), k, q=q)
    J, I = npi(r.J), npi(r.I)
    C, R, U, T = np64(r.C), np64(r.R), np64(r.U), np64(r.T)
    assert np.array_equal(C, Ah[:, J[:k]]) and np.array_equal(R, Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, C, U, R)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    # the FP64 corrected U on the GPU's own skeleton
    Uo = O.cur_middle_corrected(Ah, C, R, O.vstar(J, T, n))
    e_same = O.rel_err_fro(Ah, C, Uo, R)
    if (dtype == torch.float64 and gap_allows_exact(o.ts.col.qr, k, U64)
            and gap_allows_exact(o.ts.row.qr, k, U64)):
        assert list(J) == list(o.J) and list(I) == list(o.I)
        assert abs(eg - eo) <= 1e-12, (eg, eo)
    else:
        assert eg <= 1.05 * eo, (eg, eo)
        assert abs(eg - e_same) <= 1e-5, (eg, e_same)
    # never worse than U = V* R^+ on the same call's skeleton
    r0 = curid.cur(A.to(DEV), k, p=p, q=q, omega=Om.to(DEV), tf32=tf32, want_c=True,
                   want_r=True)
    assert npi(r0.J).tolist() == J.tolist()
    assert eg <= gpu_err(Ah, r0) * (1 + 1e-6)


def test_corrected_deterministic_equals_plain():
    """Deterministic column ID: C^+ E = 0, so both U agree to rounding."""
    A = syn.spectrum_matrix(400, 300, syn.exp_decay(300), 1412, torch.float64)
    k = 40
    a = curid.cur(A.to(DEV), k, want_c=True, want_r=True)
    b = curid.cur(A.to(DEV), k, want_c=True, want_r=True, corrected=True)
    assert b.status == 0
    assert torch.equal(a.J, b.J) and torch.equal(a.I, b.I)
    Ua, Ub = np64(a.U), np64(b.U)
    np.testing.assert_allclose(Ub, Ua, atol=1e-7 * np.abs(Ua).max(), rtol=0)
    Ah = np64(A)
    o = O.cur_corrected(Ah, k)
    assert abs(gpu_err(Ah, b) - O.rel_err_fro(Ah, o.C, o.U, o.R)) <= 1e-12


def test_corrected_srft_full_size_tf32():
    """The benchmark matrix with the structured sketch (l = 2k = 400, q = 0):
    the corrected U removes most of the gap to the q = 1 accuracy."""
    m, n, k = 8000, 6000, 200
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(n), 1413, torch.float32, DEV)
    rng = np.random.default_rng(1414)
    rows, signs = rng.choice(m, l, replace=False), rng.choice([-1, 1], m)
    Om = curid.srft_omega(torch.tensor(rows, dtype=torch.int32, device=DEV),
                          torch.tensor(signs, dtype=torch.int8, device=DEV), torch.float32)
    r = curid.cur(A, k, p=l - k, q=0, omega=Om, tf32=True, want_c=True, want_r=True,
                  want_t=True, corrected=True)
    assert r.status == 0 and r.k == k
    Ah = np64(A)
    o, _ = O.randomized_cur_corrected(Ah, O.srft_omega_rows(m, rows, signs), k)
    eg = gpu_err(Ah, r)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    assert eg <= 1.05 * eo, (eg, eo)
    J, T = npi(r.J), np64(r.T)
    Uo = O.cur_middle_corrected(Ah, np64(r.C), np64(r.R), O.vstar(J, T, n))
    assert abs(eg - O.rel_err_fro(Ah, np64(r.C), Uo, np64(r.R))) <= 1e-5


def test_corrected_rank_deficient():
    """Exact rank 10 asked for k = 15: the row ID's rank (10) bounds the
    solve with K, rows beyond it are zero, and the product still reproduces
    A to rounding."""
    rng = np.random.default_rng(3)
    A = torch.tensor(rng.standard_normal((300, 10)) @ rng.standard_normal((10, 200)))
    r = curid.cur(A.to(DEV), 15, want_c=True, want_r=True, corrected=True)
    assert r.status == 2  # RANK_DEFICIENT
    assert np.isfinite(np64(r.U)).all()
    assert gpu_err(np64(A), r) <= 1e-11
