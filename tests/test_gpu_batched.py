"""cn_step_batched: independent CN steps of several operators at once.

Handles with the FP32 apply take the merged steps (one launch per step for
all of them): a handle's result there does not depend on the rest of the
batch (bit for bit the same alone and in any mix), and equals its single
cn_step result to the CG tolerance (1e-9 relative at tol 1e-10, iterations
+-1; the single path applies the leaf levels in another, equivalent form).
FP64 handles, and a handle listed twice, take per-handle streams and equal
their single steps bit for bit.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _mk(H, dim, n, m, seed, precision):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, seed=seed, contrast=1e3, dt=0.5,
                            corr_len=0.1)
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_setup(dim, n, m, a, w.dt, H.default_options(eps=1e-6, precision=precision))
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    return h, u


def _close(a, b, tol=1e-9):
    import torch
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= tol


def test_batched_equals_individual_steps(H):
    import torch
    specs = [(2, 64, 8, 1, 0), (2, 128, 16, 2, 1), (3, 16, 4, 3, 0), (2, 256, 16, 4, 1),
             (2, 32, 8, 5, 0), (3, 16, 4, 6, 1), (2, 64, 8, 7, 1)]
    hs, us = zip(*[_mk(H, *s) for s in specs])
    prec = [s[4] for s in specs]
    ref = []
    ref_it = []
    for h, u in zip(hs, us):
        o, it = H.cn_step(h, u)
        ref.append(o)
        ref_it.append(it)
    outs, its = H.cn_step_batched(list(hs), list(us))
    torch.cuda.synchronize()
    for o, r, i, ri, pr in zip(outs, ref, its, ref_it, prec):
        if pr == 0:
            assert torch.equal(o, r) and i == ri
        else:
            assert _close(o, r) and abs(i - ri) <= 1
    # merged results do not depend on the batch: each FP32 handle alone
    for h, u, o, pr in zip(hs, us, outs, prec):
        if pr == 1:
            alone, _ = H.cn_step_batched([h], [u])
            assert torch.equal(alone[0], o)
    # a second batched step from the first step's results
    outs2, _ = H.cn_step_batched(list(hs), outs)
    for h, o, o2, pr in zip(hs, outs, outs2, prec):
        single = H.cn_step(h, o)[0]
        assert torch.equal(single, o2) if pr == 0 else _close(o2, single)


def test_batched_repeated_handle_and_caller_reaction(H):
    import torch
    h, u = _mk(H, 2, 64, 8, 7, 0)
    h2, u2 = _mk(H, 2, 128, 16, 8, 1)
    r = (u * (1.0 - u)).contiguous()
    a1, _ = H.cn_step(h, u, r=r)
    b1, _ = H.cn_step(h2, u2)
    a2, _ = H.cn_step(h, a1, r=r)
    # the same handle twice: its steps run in list order on its own buffers
    outs, its = H.cn_step_batched([h, h2, h], [u, u2, a1], rs=[r, None, r])
    assert torch.equal(outs[0], a1) and _close(outs[1], b1) and torch.equal(outs[2], a2)
    assert len(its) == 3 and all(i >= 1 for i in its)
    # empty batch is a no-op
    assert H.cn_step_batched([], []) == ([], [])

