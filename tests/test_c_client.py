"""The boundary is a C ABI: a C99 program that includes only include/hifcn.h
compiles with gcc -std=c99 -pedantic, links libhifcn.so and runs every check
that needs no GPU (tests/c_abi_client.c: defaults, status messages, and the
argument and option checks each entry point makes before touching the device)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdir():
    import __graft_entry__
    __graft_entry__.build()
    d = os.path.join(ROOT, "paper_2004_05566_gb300", "_lib")
    assert os.path.exists(os.path.join(d, "libhifcn.so"))
    return d


def test_plain_c_client(libdir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_client")
    build = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O1",
                            "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "c_abi_client.c"),
                            "-L", libdir, "-lhifcn", "-Wl,-rpath," + libdir, "-lm", "-o", exe],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert run.stdout.startswith("ok ")
