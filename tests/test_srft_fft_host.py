"""The index logic of the fast structured-sample transform (srft_fft.cuh:
mixed-radix stages, digit-reversed read-out, Makhoul's reordering, two real
columns per complex transform, rows beyond [0, m)) built for the host by g++
and checked against the oracle's DCT of Eq. (5.2).  No GPU: the kernel's
own parity tests are in test_gpu_srft.py."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("srft") / "srft_fft_host")
    subprocess.run([gxx, "-O1", "-std=c++17", "-o", exe, os.path.join(HERE, "srft_fft_host.cpp")],
                   check=True)
    return exe


def run(exe, A, signs, rows, prec):
    m, nc = A.shape
    text = " ".join([f"{m} {nc} {len(rows)} {prec}"] + [repr(float(v)) for v in A.ravel()]
                    + [str(int(v)) for v in signs] + [str(int(v)) for v in rows])
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    if out.strip() == "unsupported":
        return None
    return np.array([[float(x) for x in line.split()] for line in out.strip().splitlines()])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nc", [2, 4])
@pytest.mark.parametrize("m,l", [(1, 1), (2, 2), (3, 3), (5, 5), (7, 7), (8, 8), (12, 12),
                                 (210, 40), (1000, 30), (2835, 25), (4096, 20)])
def test_fast_transform_matches_oracle(harness, prec, nc, m, l):
    g = np.random.default_rng(m * 10 + nc + prec)
    A = g.standard_normal((m, nc))
    if prec:
        A = A.astype(np.float32).astype(np.float64)
    signs = g.choice([-1, 1], m)
    rows = g.choice(m, l, replace=False)
    Y = run(harness, A, signs, rows, prec)
    ref = O.srft_sketch(A, rows, signs)
    tol = (1e-12 if prec == 0 else 3e-6) * np.abs(ref).max()
    np.testing.assert_allclose(Y, ref, atol=tol, rtol=0)


def test_rows_beyond_the_range(harness):
    """Rows outside [0, m) follow F's periodic extension: the definition
    Omega(i, t) = s_i d_t cos(pi f_i (2t+1) / (2m)) written out, s_i = sqrt(1/l)
    for f_i = 0 mod 4m and sqrt(2/l) otherwise; row m is zero."""
    m = 60
    rows = np.array([0, m, 2 * m, 4 * m - 1, -3, 5 * m + 7, 3 * m + 1, 4 * m, -4 * m, 11])
    l = len(rows)
    g = np.random.default_rng(9)
    A = g.standard_normal((m, 4))
    signs = g.choice([-1, 1], m)
    Y = run(harness, A, signs, rows, 0)
    t = np.arange(m)
    s = np.where(rows % (4 * m) == 0, np.sqrt(1.0 / l), np.sqrt(2.0 / l))
    Om = s[:, None] * signs[None, :] * np.cos(np.pi * rows[:, None] * (2 * t[None, :] + 1) / (2 * m))
    np.testing.assert_allclose(Y, Om @ A, atol=1e-12 * np.abs(Om @ A).max(), rtol=0)
    assert np.abs(Y[1]).max() <= 1e-12 * np.abs(Om @ A).max()


def test_prime_factor_above_seven_is_unsupported(harness):
    A = np.ones((22, 2))
    assert run(harness, A, np.ones(22), np.arange(3), 0) is None
