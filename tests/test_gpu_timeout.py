"""Failure detection: a bounded device wait that runs out becomes HIF_ETIMEOUT.

The dependency-driven sweep of the upper levels (HIFCN_FLOW=1) makes each
work unit wait, with an iteration limit, for the completion flags of the
units it depends on.  hif_inject_flow_stall (host-side failure injection)
makes one unit skip publishing its flag, so its dependents' waits expire: a
flag that nothing sets, no GPU fault.  The solve must then report
HIF_ETIMEOUT, and after the injection is lifted the same handle must solve
again to the oracle's bar (1e-9 at CG tolerance 1e-10).
"""

import numpy as np
import pytest

import workloads as W
from parity import rel_err
from oracle import export, grid, hif, pcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_flow_wait_expiry_reports_timeout_and_handle_recovers(H, precision, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_FLOW", "1")
    w = W.small_variable_2d(n=64, m=8, dim=2, eps=1e-6, contrast=1e2, dt=1.0, corr_len=0.1, seed=11)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, w.n, 2, w.leaf, w.eps)
    opt = H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10)
    h = H.hif_import_factor(2, w.n, w.leaf, export.export_blob(F, w.dt), w.dt,
                            torch.from_numpy(w.a_nodes).cuda(), opt)
    b = np.random.default_rng(3).standard_normal(w.N)
    bt = torch.from_numpy(b).cuda()
    x_ref, _, _, _ = pcg.pcg(A, b, lambda v: hif.apply_inverse(F, v), tol=1e-10)

    H.hif_inject_flow_stall(h, 0, 4096)  # unit 0 never publishes; waits give up after 4096 polls
    with pytest.raises(H.HifError) as exc:
        H.pcg_solve(h, bt)
    assert exc.value.status == H.HIF_ETIMEOUT
    assert b"bounded device wait" in H.lib().hif_last_error()
    # the same handle, injection lifted: solves to the oracle's bar
    H.hif_inject_flow_stall(h, -1, 0)
    for _ in range(2):
        x, it, rr = H.pcg_solve(h, bt)
        assert rr <= 1.05e-10
        assert rel_err(x.cpu().numpy(), x_ref) <= 1e-9
    # and a CN step after it
    u1, it = H.cn_step(h, torch.from_numpy(w.u0.ravel().copy()).cuda())
    assert it >= 1
    h.close()


def test_inject_refused_without_flow_sweep(H, monkeypatch):
    import torch
    monkeypatch.delenv("HIFCN_FLOW", raising=False)
    w = W.small_variable_2d(n=32, m=8, dim=2, eps=1e-6, contrast=1e2, dt=1.0, corr_len=0.1)
    h = H.hif_setup(2, w.n, w.leaf, torch.from_numpy(w.a_nodes).cuda(), w.dt,
                    H.default_options(eps=w.eps))
    with pytest.raises(H.HifError) as exc:
        H.hif_inject_flow_stall(h, 0, 16)
    assert exc.value.status == H.HIF_EINVAL
    h.close()
