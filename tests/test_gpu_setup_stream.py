"""The factorization's memory plan does not change the factor.

* Fronts assembled and eliminated in chunks of cells through one reusable
  buffer, and the Jacobi and skeletonization scratch cut into several launches
  (budgets forced down to 64 KB: one cell or entity per chunk at these sizes),
  give a factor identical byte for byte to the one-chunk setup (the exported
  FP64 blobs are compared).
* A streaming setup (each finished level cast to FP32 / BF16 and its FP64
  values dropped, forced with HIFCN_LEAN_SETUP=1) gives reduced-precision
  applies and CN steps identical bit for bit to the handle that kept its FP64
  values, holds fewer device bytes, and refuses what needs the FP64 factor
  (an FP64 apply, an export) like a handle after hif_release_fp64.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CASES = [(2, 128, 8, 1e-6, 1.0), (3, 32, 4, 1e-4, 0.1), (3, 32, 8, 1e-4, 0.1)]
IDS = [f"{c[0]}d_n{c[1]}_m{c[2]}" for c in CASES]


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _setup(H, case, precision, **kw):
    import torch
    dim, n, m, eps, dt = case
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=17)
    opt = H.default_options(eps=eps, precision=precision, **kw)
    return w, H.hif_setup(dim, n, m, torch.from_numpy(w.a_nodes).cuda(), w.dt, opt)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_chunked_setup_is_bitwise_the_same(H, case, monkeypatch):
    _, ha = _setup(H, case, H.HIF_FP64)
    blob_a = H.hif_export_factor(ha)
    monkeypatch.setenv("HIFCN_SETUP_FRONT_BYTES", "65536")
    monkeypatch.setenv("HIFCN_SETUP_SCRATCH_BYTES", "65536")
    _, hb = _setup(H, case, H.HIF_FP64)
    blob_b = H.hif_export_factor(hb)
    assert len(blob_a) == len(blob_b)
    assert blob_a == blob_b
    ha.close()
    hb.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16top"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_streaming_setup_is_bitwise_the_same(H, case, precision, monkeypatch):
    import torch
    prec = H.HIF_FP32 if precision == "fp32" else H.HIF_FP32_BF16TOP
    kw = {} if precision == "fp32" else {"bf16_top_levels": 1}
    monkeypatch.setenv("HIFCN_LEAN_SETUP", "0")
    w, hk = _setup(H, case, prec, **kw)
    monkeypatch.setenv("HIFCN_LEAN_SETUP", "1")
    _, hl = _setup(H, case, prec, **kw)
    monkeypatch.delenv("HIFCN_LEAN_SETUP")
    qk, ql = H.hif_query(hk), H.hif_query(hl)
    assert qk["factor_entries"] == ql["factor_entries"]
    assert ql["device_bytes"] < qk["device_bytes"]
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal(w.N)).cuda()
    yk = H.hif_apply(hk, x, precision=prec).cpu().numpy()
    yl = H.hif_apply(hl, x, precision=prec).cpu().numpy()
    assert np.array_equal(yk, yl)
    H.hif_set_reaction(hk, 1, 1.0, 1.0)
    H.hif_set_reaction(hl, 1, 1.0, 1.0)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    uk, itk = H.cn_step(hk, u0)
    ul, itl = H.cn_step(hl, u0)
    assert itk == itl
    assert np.array_equal(uk.cpu().numpy(), ul.cpu().numpy())
    with pytest.raises(H.HifError):
        H.hif_apply(hl, x, precision=H.HIF_FP64)
    with pytest.raises(H.HifError):
        H.hif_export_factor(hl)
    H.hif_release_fp64(hl)  # already released: a no-op
    hk.close()
    hl.close()
