"""The C-ABI library loads and exports every entry point declared in include/*.h (CPU)."""

import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    return H.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hif_setup", "hif_apply", "pcg_solve", "cn_step", "hif_import_factor",
              "hif_export_factor", "hif_query", "hif_destroy", "hif_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names(lib):
    import paper_2004_05566_gb300.hifcn as H
    for n in _declared():
        if n in ("hif_strerror", "hif_last_error", "hif_default_options"):
            continue
        assert hasattr(H, n), n


def test_host_side_validation_without_gpu(lib):
    """Argument checks that run before any device call."""
    import ctypes
    import paper_2004_05566_gb300.hifcn as H
    out = ctypes.c_void_p()
    bad = H.HifGrid(2, 100, 16)  # 100 is not 16 * 2^L
    assert lib.hif_setup(ctypes.byref(bad), ctypes.c_void_p(1), 1.0, None, None,
                         ctypes.byref(out)) == H.HIF_EINVAL
    assert lib.hif_strerror(H.HIF_EINVAL) == b"invalid argument"
    o = H.default_options()
    assert abs(o.eps - 1e-6) < 1e-20 and o.true_res_period == 50 and o.cg_maxit == 1000
    assert o.theta == 0.5 and o.x0_mode == 0 and o.solver == 0
    good = H.HifGrid(2, 32, 8)
    for field, value in (("theta", 0.0), ("theta", 1.5), ("x0_mode", 2), ("solver", -1),
                         ("cg_maxit", -1)):
        ob = H.default_options()
        setattr(ob, field, value)
        assert lib.hif_setup(ctypes.byref(good), ctypes.c_void_p(1), 1.0, ctypes.byref(ob), None,
                             ctypes.byref(out)) == H.HIF_EINVAL, field


def test_binding_refuses_host_and_mistyped_tensors():
    """The binding marshals CUDA float64 tensors only: a host tensor, another
    dtype or a wrong length is refused before any library call."""
    import torch
    import paper_2004_05566_gb300.hifcn as H
    with pytest.raises(TypeError):
        H._vec(torch.zeros(9, dtype=torch.float64), 9, "x")
    with pytest.raises(TypeError):
        H._vec(torch.zeros(9, dtype=torch.float32), 9, "x")
    with pytest.raises(TypeError):
        H._vec([0.0] * 9, 9, "x")


def test_product_never_reaches_the_oracle():
    """No file of the package (Python or CUDA/C++) imports, includes or names
    the oracle package or the shared input generators."""
    import ast
    pkg = os.path.join(ROOT, "paper_2004_05566_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read(), path)
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        mods = [a.name for a in node.names]
                    elif isinstance(node, ast.ImportFrom):
                        mods = [node.module or ""]
                    else:
                        continue
                    for m in mods:
                        assert not m.split(".")[0] in ("oracle", "workloads"), (path, m)
            elif f.endswith((".cu", ".cuh", ".h", ".cpp", ".c")):
                src = open(path).read()
                assert "oracle/" not in src and "#include \"oracle" not in src, path


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library the binding raises: there is no CPU path."""
    import paper_2004_05566_gb300.hifcn as H
    monkeypatch.setattr(H, "_lib", None)
    monkeypatch.setattr(H, "_LIB_PATH", str(tmp_path / "libhifcn.so"))
    with pytest.raises(RuntimeError, match="not built"):
        H.lib()
    with pytest.raises(RuntimeError, match="not built"):
        H.default_options()
