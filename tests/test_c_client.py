"""The C ABI from plain C: a C99 program that includes only include/rhg.h and
links only the library builds with -Wall -Werror -pedantic and passes its
host-side checks (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c99_client_builds_and_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import paper_1606_09481_gb300 as rhg
    lib = rhg.build()
    exe = str(tmp_path / "c_client")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c_client.c"), "-o", exe, os.path.abspath(lib),
           "-Wl,-rpath," + os.path.dirname(os.path.abspath(lib))]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr
    assert "c client ok" in run.stdout
