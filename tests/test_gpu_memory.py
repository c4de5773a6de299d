"""Memory of resident operators: FP64 values released, large allocations
offloaded to host memory and reloaded at the same device addresses.

* hif_release_fp64 frees the FP64 copy of an FP32 / BF16TOP factor: the
  solves read only the reduced copy, so CN steps are bit-identical with and
  without it, the handle's device bytes drop by at least the 8 bytes per
  stored value, and the FP64-only calls refuse.
* hif_offload / hif_reload move the large allocations to host memory and
  back at the same addresses: the device memory is returned (free memory
  grows), the handle refuses solves while offloaded, and the trajectory after
  the reload is bit-identical to one that was never offloaded (captured
  solve graphs included).
"""

import ctypes

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


def _setup(H, w, precision):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_setup(w.dim, w.n, w.leaf, a, w.dt,
                    H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10))
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    return h


def _steps(H, h, u, k):
    out = []
    for _ in range(k):
        u, it = H.cn_step(h, u)
        out.append((u.clone(), it))
    return out


CASES = [(2, 256, 16), (3, 32, 8)]


@pytest.mark.parametrize("dim,n,m", CASES, ids=[f"{d}d_n{n}" for d, n, m in CASES])
def test_release_fp64_keeps_fp32_solves(H, dim, n, m):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, contrast=1e3, dt=1.0, corr_len=0.1, seed=3)
    ha, hb = _setup(H, w, H.HIF_FP32), _setup(H, w, H.HIF_FP32)
    before = H.hif_query(hb)
    H.hif_release_fp64(hb)
    after = H.hif_query(hb)
    assert before["device_bytes"] - after["device_bytes"] >= 8 * before["factor_entries"]
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    ra, rb = _steps(H, ha, u0, 3), _steps(H, hb, u0, 3)
    for (ua, ia), (ub, ib) in zip(ra, rb):
        assert ia == ib and torch.equal(ua, ub)
    x = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(H.HifError) as e:
        H.hif_apply(hb, x, y, precision=H.HIF_FP64)
    assert e.value.status == H.HIF_EINVAL
    assert H.lib().hif_apply_noalloc(hb.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     None) == H.HIF_EINVAL
    with pytest.raises(H.HifError):
        H.hif_export_factor(hb)
    h64 = _setup(H, w, H.HIF_FP64)
    with pytest.raises(H.HifError):
        H.hif_release_fp64(h64)
    for h in (ha, hb, h64):
        h.close()


@pytest.mark.parametrize("precision", [1, 2], ids=["fp32", "fp32_bf16top"])
@pytest.mark.parametrize("dim,n,m", CASES, ids=[f"{d}d_n{n}" for d, n, m in CASES])
def test_offload_reload_continues_bit_identically(H, dim, n, m, precision):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, contrast=1e3, dt=1.0, corr_len=0.1, seed=4)
    ha, hb = _setup(H, w, precision), _setup(H, w, precision)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    ref = _steps(H, ha, u0, 4)
    first = _steps(H, hb, u0, 2)
    held = H.hif_query(hb)["device_bytes"]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    H.hif_offload(hb)
    free1, _ = torch.cuda.mem_get_info()
    low = H.hif_query(hb)["device_bytes"]
    assert low < 0.5 * held and free1 - free0 >= 0.5 * (held - low)
    with pytest.raises(H.HifError) as e:
        H.cn_step(hb, first[-1][0])
    assert e.value.status == H.HIF_EINVAL
    H.hif_reload(hb)
    assert H.hif_query(hb)["device_bytes"] == held
    rest = _steps(H, hb, first[-1][0], 2)
    for (ua, ia), (ub, ib) in zip(ref, first + rest):
        assert ia == ib and torch.equal(ua, ub)
    ha.close()
    hb.close()
