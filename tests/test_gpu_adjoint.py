"""GPU parity of the CUR adjoint with frozen skeletons (curid_cur_adjoint and
the torch.autograd.Function over it) against the FP64 oracle in
oracle/adjoint.py."""
import numpy as np
import pytest
import torch

import paper_1412_8447_gb300 as curid
import synthetic as syn
from oracle.adjoint import cur_adjoint as oracle_adjoint
from oracle.adjoint import cur_loss_grad
from parity import np64, npi

pytestmark = pytest.mark.gpu


def cuda(t):
    return t.to("cuda:0").contiguous()


def forward(A, k):
    r = curid.cur(A, k, want_c=True, want_r=True, want_t=True)
    n = A.shape[1]
    return r, r.T[:, :n - k]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m,n,k,seed", [(300, 200, 20, 1), (257, 333, 37, 2), (120, 40, 40, 3),
                                        (64, 600, 33, 4)])
def test_adjoint_f64_matches_oracle(m, n, k, seed):
    A = cuda(syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 8.0), seed))
    r, T = forward(A, k)
    g = np.random.default_rng(seed)
    Cb, Ub, Rb = g.standard_normal((m, k)), g.standard_normal((k, k)), g.standard_normal((k, n))
    Ab = curid.cur_adjoint(A, r.J, r.I, T, k, cuda(torch.tensor(Cb)), cuda(torch.tensor(Ub)),
                           cuda(torch.tensor(Rb)))
    ref = oracle_adjoint(np64(A), npi(r.J), npi(r.I), k, Cb, Ub, Rb)
    assert rel(np64(Ab), ref) <= 1e-9


@pytest.mark.parametrize("which", ["C", "U", "R"])
def test_adjoint_single_cotangent(which):
    m, n, k = 180, 150, 16
    A = cuda(syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 8.0), 5))
    r, T = forward(A, k)
    g = np.random.default_rng(6)
    Cb = g.standard_normal((m, k)) if which == "C" else np.zeros((m, k))
    Ub = g.standard_normal((k, k)) if which == "U" else np.zeros((k, k))
    Rb = g.standard_normal((k, n)) if which == "R" else np.zeros((k, n))
    t = lambda x, w: cuda(torch.tensor(x)) if which == w else None  # noqa: E731
    Ab = curid.cur_adjoint(A, r.J, r.I, T, k, t(Cb, "C"), t(Ub, "U"), t(Rb, "R"))
    ref = oracle_adjoint(np64(A), npi(r.J), npi(r.I), k, Cb, Ub, Rb)
    assert rel(np64(Ab), ref) <= 1e-9


def test_adjoint_f32_differentiable_config():
    """A 2048 x 1024 float32, sigma_j = exp(-j/20), k = 64, deterministic:
    FP32 gradient against the FP64 oracle on the same frozen skeletons."""
    m, n, k = 2048, 1024, 64
    A = cuda(syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 20.0), 51, torch.float32))
    r, T = forward(A, k)
    g = np.random.default_rng(52)
    Cb, Ub, Rb = g.standard_normal((m, k)), g.standard_normal((k, k)), g.standard_normal((k, n))
    Ab = curid.cur_adjoint(A, r.J, r.I, T, k, cuda(torch.tensor(Cb, dtype=torch.float32)),
                           cuda(torch.tensor(Ub)), cuda(torch.tensor(Rb, dtype=torch.float32)))
    ref = oracle_adjoint(np64(A), npi(r.J), npi(r.I), k, Cb, Ub, Rb)
    assert rel(np64(Ab), ref) <= 1e-4, rel(np64(Ab), ref)


@pytest.mark.parametrize("dtype,m,n,k,tol", [(torch.float64, 200, 150, 12, 1e-9),
                                             (torch.float32, 2048, 1024, 64, 1e-4)])
def test_autograd_loss_gradient(dtype, m, n, k, tol):
    """loss = 1/2 ||A - C U R||_F^2 through CURFunction: A.grad against the
    oracle's frozen-skeleton loss gradient."""
    A0 = cuda(syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 20.0), 53, dtype))
    A = A0.clone().requires_grad_(True)
    C, U, R, J, I = curid.cur_differentiable(A, k)
    Res = A.double() - C.double() @ U @ R.double()
    loss = 0.5 * (Res * Res).sum()
    loss.backward()
    ref, ref_loss = cur_loss_grad(np64(A0), npi(J), npi(I), k)
    assert abs(float(loss.detach()) - ref_loss) <= max(tol, 1e-12) * ref_loss * 10
    assert rel(np64(A.grad), ref) <= tol, rel(np64(A.grad), ref)


def test_adjoint_rejects_bad_arguments():
    A = cuda(syn.spectrum_matrix(300, 280, syn.exp_decay(280, 8.0), 7, torch.float32))
    J = torch.arange(280, dtype=torch.int32, device="cuda:0")
    I = torch.arange(300, dtype=torch.int32, device="cuda:0")
    T = torch.zeros((40, 240), dtype=torch.float32, device="cuda:0")
    with pytest.raises(curid.CuridError) as e:
        curid.cur_adjoint(A, J, I, T, 0)
    assert e.value.status == 1
    with pytest.raises(curid.CuridError) as e:
        curid.cur_adjoint(A, J, I, T, 281)
    assert e.value.status == 1
    big = torch.zeros((4100, 4100), dtype=torch.float32, device="cuda:0")
    Jb = torch.arange(4100, dtype=torch.int32, device="cuda:0")
    with pytest.raises(curid.CuridError) as e:
        curid.cur_adjoint(big, Jb, Jb, big[:4097, :3], 4097)
    assert e.value.status == 8
