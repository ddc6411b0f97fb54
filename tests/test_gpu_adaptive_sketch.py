"""Adaptive rank with a sketch (Algorithm 4 with the tolerance stop of
Section 3): k == 0, tol > 0, p >= 0.  The device searches the sample size
(l doubling from 64, Omega from the seed) and decomposes at the rank found;
the oracle runs the same search on the same Omega (its own Philox4x32-10,
pinned against the published known answers) and the same decomposition."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from oracle.philox import gaussian as philox_gaussian
from parity import U64, gap_allows_exact, np64, npi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("q", [0, 1])
def test_adaptive_sketch_f64_matches_oracle(q):
    m, n, p, tol, seed = 600, 450, 10, 1e-5, 424242
    A = syn.spectrum_matrix(m, n, syn.exp_decay(n, 6.0), 111, torch.float64)
    r = curid.cur(A.to(DEV), 0, p=p, q=q, seed=seed, tol=tol, want_c=True, want_r=True,
                  want_t=True)
    Ah = np64(A)
    Om = philox_gaussian(min(m, n), m, seed)
    k, l, Y = O.randomized_rank_adaptive(Ah, Om, tol, p, q=q)
    assert r.k == k, (r.k, k)
    o, _ = O.randomized_cur(Ah, Om[:l], k, q=q)
    J, I = npi(r.J), npi(r.I)
    assert np.array_equal(np64(r.C), Ah[:, J[:k]]) and np.array_equal(np64(r.R), Ah[I[:k], :])
    eg = O.rel_err_fro(Ah, np64(r.C), np64(r.U), np64(r.R))
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    if gap_allows_exact(o.ts.col.qr, k, U64) and gap_allows_exact(o.ts.row.qr, k, U64):
        assert list(J[:k]) == list(o.J[:k]) and list(I[:k]) == list(o.I[:k])
        assert abs(eg - eo) <= 1e-12
    else:
        assert eg <= 1.05 * eo


@pytest.mark.parametrize("dtype,tf32,tol", [(torch.float64, False, 1e-10),
                                            (torch.float32, False, 1e-4),
                                            (torch.float32, True, 1e-4)])
def test_adaptive_sketch_exact_rank(dtype, tf32, tol):
    """Exact rank 70: found in the second sample (l = 128), and A is
    reproduced to the working precision."""
    m, n, rk = 500, 400, 70
    rng = np.random.default_rng(121)
    A = torch.tensor(rng.standard_normal((m, rk)) @ rng.standard_normal((rk, n)), dtype=dtype)
    r = curid.cur(A.to(DEV), 0, p=10, q=0, seed=7, tol=tol, tf32=tf32, want_c=True, want_r=True)
    assert r.k == rk
    e = O.rel_err_fro(np64(A), np64(r.C), np64(r.U), np64(r.R))
    assert e <= (1e-11 if dtype == torch.float64 else 1e-4), e


def test_adaptive_sketch_id_col_and_tsid():
    m, n = 600, 450
    A = syn.spectrum_matrix(m, n, syn.exp_decay(n, 6.0), 131, torch.float64).to(DEV)
    a = curid.id_col(A, 0, p=10, q=1, seed=5, tol=1e-6)
    b = curid.tsid(A, 0, p=10, q=1, seed=5, tol=1e-6)
    c = curid.cur(A, 0, p=10, q=1, seed=5, tol=1e-6)
    assert a.k == b.k == c.k > 0
    assert torch.equal(a.J, b.J) and torch.equal(b.J, c.J)


def test_adaptive_sketch_rejects_given_omega():
    A = torch.randn(200, 150, dtype=torch.float64, device=DEV)
    Om = torch.randn(64, 200, dtype=torch.float64, device=DEV)
    with pytest.raises(curid.CuridError):
        curid.cur(A, 0, p=10, q=0, omega=Om, tol=1e-6)
