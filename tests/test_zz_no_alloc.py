"""The allocation-free collision batch (stp_check_edges_noalloc).

Some callers cannot allocate device memory while they run (a control loop that
must not block in the driver's allocator, a process whose device-memory budget
is fixed after start-up). For them the library offers a variant of the
collision batch whose scratch lives in one static device array. This test calls
it through the C ABI twice in a row, on different edge sets, and checks that its
verdicts equal those of stp_check_edges (the same kernel on the same inputs,
so they must agree exactly). The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu


def test_noalloc_batch_matches_check_edges_on_two_calls():
    import torch
    from paper_2609_30533_gb300 import build as B
    B.build()
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.ur5e(0)
    P = stp.problem_from(prob, prm, precision=0, max_iters=1)
    L = stp.lib()
    dev = torch.device("cuda:0")
    for call, n in enumerate((40000, 12345)):
        qa, ta, qb, tb = WL.microbench_edges(prob, n, prm.eta, prm.H, seed=100 + call)
        ref, _, _ = P.check_edges(qa, ta, qb, tb)
        t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in (qa, ta, qb, tb)]
        ver = torch.full((n,), 7, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        s = L.stp_check_edges_noalloc(P.handle, n, C.c_void_p(t[0].data_ptr()), C.c_void_p(t[1].data_ptr()),
                                      C.c_void_p(t[2].data_ptr()), C.c_void_p(t[3].data_ptr()),
                                      C.c_void_p(ver.data_ptr()))
        assert s == stp.STP_OK, stp.status_string(s)
        torch.cuda.synchronize()
        got = ver.cpu().numpy()
        assert np.array_equal(got, ref), int((got != ref).sum())
        assert 0 < got.mean() < 1
    # Beyond the stated maximum the call refuses with a clear status.
    n_big = 65536 + 1
    s = L.stp_check_edges_noalloc(P.handle, n_big, C.c_void_p(t[0].data_ptr()), C.c_void_p(t[1].data_ptr()),
                                  C.c_void_p(t[2].data_ptr()), C.c_void_p(t[3].data_ptr()),
                                  C.c_void_p(ver.data_ptr()))
    assert s == stp.STP_ERR_CAPACITY
    P.close()
