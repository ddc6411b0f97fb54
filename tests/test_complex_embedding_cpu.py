"""The identity the complex path rests on, checked on the CPU with the two
oracles: the real CUR-ID of the 2 x 2-block embedding E(A) (x + iy ->
[[x, -y], [y, x]]), read off pair by pair, is the complex CUR-ID of A.  The
real pivots come in pairs {2j, 2j + 1}; the complex T and U are the even /
odd rows of the real ones, taken in the order the pairs were selected."""
import numpy as np
import pytest

import oracle as O


def embed(A):
    m, n = A.shape
    E = np.zeros((2 * m, 2 * n))
    E[0::2, 0::2] = A.real
    E[0::2, 1::2] = -A.imag
    E[1::2, 0::2] = A.imag
    E[1::2, 1::2] = A.real
    return E


def read_off(Jp, Ip, Tp, Up, k, n):
    for t in range(k):
        assert Jp[2 * t] ^ 1 == Jp[2 * t + 1] and Ip[2 * t] ^ 1 == Ip[2 * t + 1]
    for c in range(n - k):
        assert Jp[2 * k + 2 * c] % 2 == 0 and Jp[2 * k + 2 * c + 1] == Jp[2 * k + 2 * c] + 1

    def ev(P, t):
        return 2 * t if P[2 * t] % 2 == 0 else 2 * t + 1

    def od(P, t):
        return 2 * t + 1 if P[2 * t] % 2 == 0 else 2 * t

    J = [Jp[2 * t] >> 1 for t in range(n)]
    I = [Ip[2 * s] >> 1 for s in range(k)]
    T = np.array([[Tp[ev(Jp, t), 2 * c] + 1j * Tp[od(Jp, t), 2 * c] for c in range(n - k)]
                  for t in range(k)])
    U = np.array([[Up[ev(Jp, t), ev(Ip, s)] + 1j * Up[od(Jp, t), ev(Ip, s)] for s in range(k)]
                  for t in range(k)])
    return J, I, T, U


def complex_spectrum(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
    return U @ np.diag(np.exp(-np.arange(r) / decay)) @ V.conj().T


@pytest.mark.parametrize("q", [None, 0, 1])
def test_embedding_read_off_equals_complex_cur(q):
    m, n, k = 70, 50, 8
    A = complex_spectrum(m, n, 4.0, 400)
    if q is None:
        r = O.cur(embed(A), 2 * k)
        c = O.cur_complex(A, k)
    else:
        G = np.random.default_rng(401).standard_normal((k + 6, 2 * m))
        Om = G[:, 0::2] + 1j * G[:, 1::2]
        r, _ = O.randomized_cur(embed(A), embed(Om), 2 * k, q=q)
        c = O.cur_complex(A, k, Y=O.sketch_complex(A, Om, q=q))
    J, I, T, U = read_off(r.J, r.I, r.T, r.U, k, n)
    assert J[:k] == list(c["J"][:k]) and I == list(c["I"][:k])
    np.testing.assert_allclose(T, c["T"], atol=1e-10 * np.abs(c["T"]).max(), rtol=0)
    np.testing.assert_allclose(U, c["U"], atol=1e-9 * np.abs(c["U"]).max(), rtol=0)
