"""HostStream: decompositions of host matrices with the copy of the next
matrix overlapped with the current decomposition.  Its results must be the
ones the plain device call gives on the same matrices and seeds (the same
kernels on the same inputs), and the copy-in of a buffer must not overtake
the decomposition still reading it (checked by alternating distinct
matrices through the buffers), with one decomposition in flight and with
three on three streams."""
import pytest
import torch

import paper_1412_8447_gb300 as curid
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tf32,inflight", [(False, 1), (True, 1), (True, 3)])
def test_host_stream_matches_device_calls(tf32, inflight):
    m, n, k, p, q = 1500, 1100, 60, 10, 1
    mats = [syn.spectrum_matrix(m, n, syn.power_decay(n), 1412 + i, torch.float32, "cpu")
            for i in range(5)]
    hosts = [a.pin_memory() for a in mats]
    seeds = [9000 + i for i in range(5)]
    hs = curid.HostStream(m, n, k, torch.float32, 0, p=p, q=q, tf32=tf32, inflight=inflight)
    res = hs.host_results(5)
    hs.run(hosts, res, seeds)
    torch.cuda.synchronize()
    for i in range(5):
        r = curid.cur(mats[i].to("cuda:0"), k, p=p, q=q, seed=seeds[i], tf32=tf32)
        torch.cuda.synchronize()
        assert r.status == 0
        J, I, U = res[i]
        assert torch.equal(J, r.J.cpu()), i
        assert torch.equal(I, r.I.cpu()), i
        assert torch.equal(U, r.U.cpu()), i


def test_host_stream_rejects_short_results():
    hs = curid.HostStream(64, 48, 8, torch.float32, 0, p=4, q=0)
    with pytest.raises(ValueError):
        hs.run([torch.zeros(64, 48).pin_memory()] * 2, hs.host_results(1))
