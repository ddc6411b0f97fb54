"""Complex A (the paper works over C) through curid_cur_complex, which runs
the real pipeline on the real 2 x 2-block embedding and reads the complex
J, I, T, U off it; against the complex FP64 oracle (plain complex pivoted
Gram-Schmidt) on the same values, deterministic and with a sketch (the
complex Gaussian Omega from the seed, the oracle's own Philox)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
from oracle.philox import gaussian as philox_gaussian

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def complex_spectrum(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
    return U @ np.diag(np.exp(-np.arange(r) / decay)) @ V.conj().T


def rel_err(A, C, U, R):
    return np.linalg.norm(A - C @ U @ R) / np.linalg.norm(A)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("m,n,k", [(300, 200, 20), (150, 260, 24)])
def test_complex_deterministic(dtype, m, n, k):
    A = complex_spectrum(m, n, 6.0, m + n)
    Ad = torch.tensor(A, dtype=dtype, device=DEV)
    Ah = Ad.cpu().to(torch.complex128).numpy()  # the values the GPU holds
    r = curid.cur_complex(Ad, k, want_t=True)
    assert r.status == 0 and r.k == k
    o = O.cur_complex(Ah, k)
    J, I = r.J.cpu().numpy(), r.I.cpu().numpy()
    assert sorted(J.tolist()) == list(range(n)) and sorted(I.tolist()) == list(range(m))
    C, R = Ah[:, J[:k]], Ah[I[:k], :]
    eg = rel_err(Ah, C, r.U.cpu().numpy(), R)
    eo = rel_err(Ah, o["C"], o["U"], o["R"])
    if dtype == torch.complex128:
        assert list(J[:k]) == list(o["J"][:k]) and list(I[:k]) == list(o["I"][:k])
        T = r.T.cpu().numpy()
        np.testing.assert_allclose(T, o["T"], atol=1e-9 * np.abs(o["T"]).max(), rtol=0)
        assert abs(eg - eo) <= 1e-12, (eg, eo)
    else:
        assert eg <= 1.05 * eo, (eg, eo)


@pytest.mark.parametrize("dtype,tf32", [(torch.complex128, False), (torch.complex64, False),
                                        (torch.complex64, True)])
def test_complex_randomized(dtype, tf32):
    m, n, k, p, q, seed = 400, 300, 25, 10, 1, 777
    A = complex_spectrum(m, n, 8.0, 12)
    Ad = torch.tensor(A, dtype=dtype, device=DEV)
    Ah = Ad.cpu().to(torch.complex128).numpy()
    r = curid.cur_complex(Ad, k, p=p, q=q, seed=seed, tf32=tf32)
    assert r.status == 0 and r.k == k
    G = philox_gaussian(k + p, 2 * m, seed)
    Om = G[:, 0::2] + 1j * G[:, 1::2]
    o = O.cur_complex(Ah, k, Y=O.sketch_complex(Ah, Om, q=q))
    J, I = r.J.cpu().numpy(), r.I.cpu().numpy()
    eg = rel_err(Ah, Ah[:, J[:k]], r.U.cpu().numpy(), Ah[I[:k], :])
    eo = rel_err(Ah, o["C"], o["U"], o["R"])
    if dtype == torch.complex128:
        assert list(J[:k]) == list(o["J"][:k]) and list(I[:k]) == list(o["I"][:k])
        assert abs(eg - eo) <= 1e-12, (eg, eo)
    else:
        assert eg <= 1.05 * eo, (eg, eo)


def test_complex_real_input_matches_real_path():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 150)) @ np.diag(np.exp(-np.arange(150) / 7.0)) @ \
        np.linalg.qr(rng.standard_normal((150, 150)))[0]
    rc = curid.cur_complex(torch.tensor(A, dtype=torch.complex128, device=DEV), 12)
    rr = curid.cur(torch.tensor(A, device=DEV), 12)
    assert torch.equal(rc.J[:12], rr.J[:12]) and torch.equal(rc.I[:12], rr.I[:12])
    U = rc.U.cpu().numpy()
    np.testing.assert_allclose(U.real, rr.U.cpu().numpy(), atol=1e-8 * np.abs(U).max(), rtol=0)
    assert np.abs(U.imag).max() <= 1e-9 * np.abs(U).max()
