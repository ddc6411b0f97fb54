"""GPU parity of the batched adaptive-rank column ID (curid_id_col_batched)
against the FP64 oracle's per-block column ID with the tolerance stop, on
Laplace kernel blocks (targets in the unit box at the origin, sources in the
unit box centred at (3, 0, 0), m_b and n_b uniform on 64..512)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1412_8447_gb300 as curid
import synthetic as syn
from parity import gap_allows_exact, npi

pytestmark = pytest.mark.gpu


def block(flat, shape, off):
    m, n = shape
    return flat[off:off + m * n].view(m, n)


def id_residual(A, J, T, k):
    """||A(:, J[k:]) - A(:, J[:k]) T||_F in float64."""
    A = np.asarray(A, dtype=np.float64)
    if k == 0:
        return np.linalg.norm(A)
    return np.linalg.norm(A[:, J[k:]] - A[:, J[:k]] @ np.asarray(T, dtype=np.float64))


def check_block(Ab, J, T, k, st, tol, u, exact_pivots=True):
    """One block against the oracle: rank, skeleton (where the pivot gaps
    exceed rounding), T, and the stopping criterion."""
    A = np.asarray(Ab.cpu(), dtype=np.float64)
    o = O.id_col(A, tol=tol)
    J, T = npi(J), np.asarray(T.cpu(), dtype=np.float64)
    assert st == 0, st
    normA = np.linalg.norm(A)
    # the GPU's skeleton meets the tolerance
    assert id_residual(A, J, T, k) <= tol * normA * 1.05 + 1e-300
    assert sorted(J.tolist()) == list(range(A.shape[1]))
    assert list(J[k:]) == sorted(J[k:].tolist())
    r = o.qr.resid
    margin = (o.k == 0 or r[o.k - 1] > tol * normA * (1 + 1e-6)) and r[o.k] < tol * normA * (1 - 1e-6)
    if exact_pivots and margin and gap_allows_exact(o.qr, o.k, u):
        assert k == o.k, (k, o.k)
        assert list(J) == list(o.J)
        if k:
            # both are backward-stable solves of S11 T = S12: their difference
            # is bounded by kappa(S11) u ||T|| (kappa ~ nu_1 / nu_k)
            kappa = o.qr.nu[0] / o.qr.nu[k - 1]
            assert np.linalg.norm(T - o.T) <= 1e2 * kappa * u * max(1.0, np.linalg.norm(o.T))
    else:
        assert abs(k - o.k) <= 1


@pytest.mark.parametrize("dtype,tol,u", [(torch.float64, 1e-8, 2.0 ** -53),
                                         (torch.float32, 1e-5, 2.0 ** -24)])
def test_batched_matches_oracle_small(dtype, tol, u):
    flat, shapes, offs = syn.laplace_batch(24, 1412 + 7, dtype, "cuda:0")
    B = curid.BatchedID(flat, shapes, offs, tol=tol, k_max=64)
    B.run()
    res = B.results()
    for b in range(len(shapes)):
        J, T, k, st = res[b]
        check_block(block(flat, shapes[b], offs[b]), J, T, k, st, tol, u,
                    exact_pivots=dtype == torch.float64)


def test_batched_fixed_rank_matches_oracle():
    """tol = 0: exactly min(m, n, k_max) steps, J and T as the oracle's fixed
    rank column ID."""
    flat, shapes, offs = syn.laplace_batch(6, 1412 + 8, torch.float64, "cuda:0", lo=40, hi=90)
    kmax = 12
    B = curid.BatchedID(flat, shapes, offs, tol=0.0, k_max=kmax)
    B.run()
    for b, (J, T, k, st) in enumerate(B.results()):
        A = block(flat, shapes[b], offs[b]).cpu().numpy()
        assert k == min(kmax, *shapes[b])
        o = O.id_col(A, k=k)
        if gap_allows_exact(o.qr, k, 2.0 ** -53):
            assert list(npi(J)) == list(o.J)
            kappa = o.qr.nu[0] / o.qr.nu[k - 1]
            assert (np.linalg.norm(T.cpu().numpy() - o.T)
                    <= 1e2 * kappa * 2.0 ** -53 * max(1, np.linalg.norm(o.T)))


def test_batched_edge_blocks():
    """A zero block (stops at k = 0), an exact rank-5 block (k = 5), a block
    holding a NaN (NONFINITE), a 1 x 1 block and a single-column block."""
    d = "cuda:0"
    mats = [torch.zeros(70, 50, dtype=torch.float64),
            syn.exact_rank(90, 80, 5, 3),
            syn.laplace_block(64, 64, 5),
            torch.tensor([[2.5]], dtype=torch.float64),
            syn.laplace_block(100, 1, 6)]
    mats[2][3, 7] = float("nan")
    offs, total = [], 0
    for M in mats:
        offs.append(total)
        total += (M.numel() + 1) // 2 * 2
    flat = torch.zeros(total, dtype=torch.float64)
    for M, o in zip(mats, offs):
        flat[o:o + M.numel()] = M.reshape(-1)
    flat = flat.to(d)
    shapes = [tuple(M.shape) for M in mats]
    B = curid.BatchedID(flat, shapes, offs, tol=1e-8, k_max=32)
    B.run()
    res = B.results()
    assert res[0][2] == 0 and res[0][3] == 0 and list(npi(res[0][0])) == list(range(50))
    assert res[1][2] == 5 and res[1][3] == 0
    o = O.id_col(mats[1].numpy(), tol=1e-8)
    assert list(npi(res[1][0])[:5]) == list(o.J[:5])
    assert res[2][3] == 4  # NONFINITE
    assert res[3][2] == 1 and res[3][3] == 0
    assert res[4][2] == 1 and res[4][3] == 0
    st, _ = curid.last_status(0)
    assert st == 4


def test_batched_graph_capture_and_autotune():
    """The launch captured into a CUDA graph and replayed gives the same
    results bit for bit; the autotuner picks a shape whose results still
    meet the tolerance with the same ranks."""
    flat, shapes, offs = syn.laplace_batch(96, 1412 + 9, torch.float64, "cuda:0")
    B = curid.BatchedID(flat, shapes, offs, tol=1e-8, k_max=64)
    B.run()
    torch.cuda.synchronize()
    J0, T0, k0 = B.Jflat.clone(), B.Tflat.clone(), B.k_out.clone()
    B.Jflat.zero_()
    B.Tflat.zero_()
    B.k_out.zero_()
    B.prepare()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.prepare()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.run()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(B.k_out, k0) and torch.equal(B.Jflat, J0) and torch.equal(B.Tflat, T0)
    threads, per_sm = B.autotune()
    assert threads in (128, 256, 512) and per_sm in (1, 2, 4)
    B.run()
    torch.cuda.synchronize()
    assert torch.equal(B.k_out, k0)
    for b, (J, T, k, st) in enumerate(B.results()):
        A = block(flat, shapes[b], offs[b]).cpu().numpy()
        assert id_residual(A, npi(J), T.cpu().numpy(), k) <= 1e-8 * np.linalg.norm(A) * 1.05


@pytest.mark.parametrize("dtype,tol,u", [(torch.float64, 1e-8, 2.0 ** -53),
                                         (torch.float32, 1e-5, 2.0 ** -24)])
def test_batched_full_config(dtype, tol, u):
    """4096 blocks, m_b, n_b on 64..512: every block meets the tolerance with
    a valid permutation; 12 sampled blocks against the oracle."""
    flat, shapes, offs = syn.laplace_batch(4096, 1412 + 4, dtype, "cuda:0")
    B = curid.BatchedID(flat, shapes, offs, tol=tol, k_max=64)
    B.run()
    torch.cuda.synchronize()
    k = B.k_out.cpu().numpy()
    st = B.block_status.cpu().numpy()
    assert (st == 0).all()
    assert (k >= 1).all() and (k <= 64).all()
    res = B.results()
    g = np.random.default_rng(17)
    for b in g.choice(len(shapes), 12, replace=False):
        J, T, kb, sb = res[b]
        check_block(block(flat, shapes[b], offs[b]), J, T, kb, sb, tol, u,
                    exact_pivots=dtype == torch.float64)
