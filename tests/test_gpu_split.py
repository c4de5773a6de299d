"""Split launches for large separator entities and large roots.

Levels whose entities exceed a size threshold apply those entities by row
blocks (forward) or column blocks (backward) over many CTAs after gathering
the entity inputs; roots above a threshold go through a row-block and a
column-block launch.  The thresholds are lowered here (environment variables
read when the factor is built) so that small problems take these paths: the
FP64 apply must equal the unsplit apply to 1e-13 (the same sums, in another
order in the backward column blocks), and CN steps must match the oracle to
1e-9 as everywhere else.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import pcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _setup(H, w, precision, env):
    import torch
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return H.hif_setup(w.dim, w.n, w.leaf, torch.from_numpy(w.a_nodes).cuda(), w.dt,
                           H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


SPLIT = {"HIFCN_SPLIT_DOFS": "16", "HIFCN_ROOT_SPLIT_DOFS": "16"}
CASES = [(2, 128, 8, 1e-6, 1.0), (3, 32, 4, 1e-4, 0.1)]


@pytest.mark.parametrize("dim,n,m,eps,dt", CASES, ids=["2d_n128_m8", "3d_n32_m4"])
def test_split_apply_equals_unsplit(H, dim, n, m, eps, dt):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=23)
    hs = _setup(H, w, 0, SPLIT)
    hu = _setup(H, w, 0, {})
    b = torch.from_numpy(np.random.default_rng(6).standard_normal(w.N)).cuda()
    ys = H.hif_apply(hs, b).cpu().numpy()
    yu = H.hif_apply(hu, b).cpu().numpy()
    assert np.linalg.norm(ys - yu) <= 1e-13 * np.linalg.norm(yu)


@pytest.mark.parametrize("dim,n,m,eps,dt", CASES, ids=["2d_n128_m8", "3d_n32_m4"])
@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32", "bf16top"])
def test_split_cn_steps_match_oracle(H, dim, n, m, eps, dt, precision):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=29)
    ref, _, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 2, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10)
    h = _setup(H, w, precision, SPLIT)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    for _ in range(2):
        u, _ = H.cn_step(h, u)
    assert np.linalg.norm(u.cpu().numpy() - ref.ravel()) <= 1e-9 * np.linalg.norm(ref)
