"""Failure detection without a GPU fault: every device wait in the library is
bounded, and an expired wait records CPG_ERR_TIMEOUT in the workspace's status
word instead of hanging.  The self-test entry point runs that exact bounded
wait on a barrier nothing completes; the host reads the status, and the
context stays usable for the next call.  A singular normal-equation matrix
(CPG_ERR_SINGULAR) is covered in test_gpu_parity.py."""
import numpy as np
import pytest

import cpsynth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as m
    return m


def test_expired_wait_is_reported_and_the_context_survives(cg):
    ws = cg.Workspace(torch.device("cuda"))
    assert cg.cpg_device_status(ws) == 0
    cg.selftest_timeout(4096, workspace=ws)
    assert cg.cpg_device_status(ws) == 6          # CPG_ERR_TIMEOUT
    assert cg.cpg_device_status(ws) == 0          # read and cleared
    # the same workspace and context still compute correct gradients
    I, R = [14, 18, 11, 16], 7
    y = cpsynth.random_tensor(I, seed=51)
    A = cpsynth.random_factors(I, R, seed=51)
    Ad = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).cuda()) for a in A]
    G = cg.cp_gradient_all(torch.from_numpy(y).cuda(), I, Ad, workspace=ws)
    torch.cuda.synchronize()
    want = oracle.cp_gradient_all(y.astype(np.float64), I, A)
    for n in range(len(I)):
        got = G[n].double().cpu().numpy()
        assert np.linalg.norm(got - want[n]) <= 1e-5 * np.linalg.norm(want[n])
    assert cg.cpg_device_status(ws) == 0
