"""Failure statuses driven on the GPU without faulting it (Section 2.3 for
rank deficiency): a wait between the blocks of the
persistent CPQR kernel that runs out (a one-cycle bound set on the handle),
a non-finite input, an exactly rank-deficient input, and a zero sample whose
row orthonormalisation (Section 5.3) cannot proceed.  After each, the same
handle serves the next call normally."""
import pytest
import torch

import paper_1412_8447_gb300 as curid
import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("l,n", [(210, 6000), (250, 9728), (300, 157)])
def test_timeout_then_recover(l, n):
    """A one-cycle bound on the inter-block waits: the kernel gives up on its
    first wait, every block leaves, the call reports CURID_TIMEOUT, and with
    the default bound restored the same factorization succeeds bit for bit
    (register-resident slabs, and the shared-memory kernel for l = 300)."""
    A = syn.spectrum_matrix(l, n, syn.power_decay(min(l, n)), 736, torch.float32).to(DEV)
    k = min(100, l, n)
    ref = curid.cpqr(A, k=k)
    curid.set_timeout(1)
    try:
        with pytest.raises(curid.CuridError) as e:
            curid.cpqr(A, k=k)
        assert e.value.status == 5
    finally:
        curid.set_timeout(0)
    again = curid.cpqr(A, k=k)
    assert again.status == 0
    assert torch.equal(again.J, ref.J) and torch.equal(again.S, ref.S)


def test_timeout_rejects_negative():
    h = curid._binding.handle(0)
    assert h.lib.curid_set_timeout(h.h, -1) == 1


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_rank_deficient_status(dtype):
    """Exact rank r < k: CURID_RANK_DEFICIENT and k_out = r (Section 2.3)."""
    r0, k = 23, 40
    A = syn.exact_rank(210, 3000, r0, 734, dtype)
    r = curid.cpqr(A.to(DEV), k=k)
    assert r.status == 2 and r.k == r0


def test_nonfinite_status():
    A = syn.spectrum_matrix(120, 3000, syn.exp_decay(120, 6.0), 735, torch.float32)
    A[37, 1234] = float("nan")
    with pytest.raises(curid.CuridError) as e:
        curid.cpqr(A.to(DEV), k=20)
    assert e.value.status == 4
    B = syn.spectrum_matrix(120, 3000, syn.exp_decay(120, 6.0), 735, torch.float32)
    assert curid.cpqr(B.to(DEV), k=20).status == 0


def test_breakdown_of_zero_sample():
    """A = 0 with a power step: the Gram matrix of the zero sample has trace
    zero, every shifted Cholesky attempt fails, and the call reports
    CURID_BREAKDOWN (the orthonormalisation of Section 5.3 cannot proceed)."""
    Z = torch.zeros((300, 200), dtype=torch.float32, device=DEV)
    with pytest.raises(curid.CuridError) as e:
        curid.cur(Z, 10, p=5, q=1, seed=3)
    assert e.value.status == 3
    A = syn.spectrum_matrix(300, 200, syn.exp_decay(200, 10.0), 737, torch.float32).to(DEV)
    r = curid.cur(A, 10, p=5, q=1, seed=3)
    assert r.status == 0
