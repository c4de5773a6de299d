"""Serving: CN-step requests over resident operators with continuous batching.

The same operator must follow the same trajectory, bit for bit, whether it is
stepped alone (a batch of one) or served in a mix of operators of different
sizes and dimensions whose requests arrive from several clients while other
batches run, and after being evicted (HBM budget: the factor is offloaded to
host memory) and reloaded.
"""

import random
import threading
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    import paper_2004_05566_gb300.serve as S
    assert torch.cuda.is_available()
    return H, S


def _specs(S):
    out = {}
    for k, (dim, n, m) in enumerate([(2, 64, 8), (2, 128, 16), (2, 256, 16), (2, 32, 8), (3, 16, 4)]):
        w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, seed=40 + k, contrast=1e3,
                                dt=0.5, corr_len=0.1)
        out[f"op{k}"] = S.OperatorSpec(dim, n, m, w.a_nodes, w.dt, w.eps, w.u0, (1, 1.0, 1.0))
    return out


def _alone(H, spec, steps):
    import torch
    a = torch.from_numpy(spec.a_nodes).cuda()
    h = H.hif_setup(spec.dim, spec.n, spec.leaf, a, spec.dt,
                    H.default_options(eps=spec.eps, precision=spec.precision, cg_tol=1e-10))
    H.hif_set_reaction(h, *spec.reaction)
    u = torch.from_numpy(np.array(spec.u0).ravel().copy()).cuda()
    for _ in range(steps):  # a batch of one: the same kernels as in any served batch
        outs, _ = H.cn_step_batched([h], [u])
        u = outs[0]
    out = u.cpu().numpy()
    h.close()
    return out


@pytest.mark.parametrize("budget_mb,max_batch", [(4096, 256), (1, 2)])
def test_served_trajectories_equal_alone(mods, budget_mb, max_batch):
    H, S = mods
    specs = _specs(S)
    steps = 4
    ref = {oid: _alone(H, sp, steps) for oid, sp in specs.items()}
    # a 1 MB budget holds no operator, and batches of at most 2 leave the other
    # operators idle, so every admission evicts and operators are re-factored
    srv = S.CNServer(hbm_budget_bytes=budget_mb << 20, max_batch=max_batch)
    for oid, sp in specs.items():
        srv.register(oid, sp)
    futures = []
    lock = threading.Lock()

    def client(seed, ids):
        rng = random.Random(seed)
        for _ in range(steps):
            for oid in ids:
                f = srv.submit(oid)
                with lock:
                    futures.append(f)
                time.sleep(rng.random() * 0.002)

    ids = list(specs)
    ts = [threading.Thread(target=client, args=(i, ids[i::3])) for i in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    results = [f.result(timeout=120) for f in futures]
    try:
        for oid in ids:
            assert srv.step_count(oid) == steps
            assert np.array_equal(srv.state(oid), ref[oid]), oid
        assert all(r.latency_s > 0 and r.iters >= 1 for r in results)
        if max_batch > len(ids):
            assert srv.batches < len(results)  # several requests shared a batch
        else:
            assert srv.evictions > 0
            # evicted operators come back by reloading their offloaded factor
            assert any(srv.reload_count(oid) > 0 for oid in ids)
            assert all(srv.setups(oid) == 1 for oid in ids)
    finally:
        srv.close()
