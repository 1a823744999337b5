"""The boundary is usable from plain C: tests/c/abi_host.c is compiled with the system C compiler
against include/mr.h, linked with libmrmod.so and run (host-only calls; no device needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB_DIR = os.path.join(ROOT, "paper_1305_3699_gb300", "lib")


def test_c_client_host_calls(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(LIB_DIR, "libmrmod.so")):
        pytest.skip("libmrmod.so not built")
    exe = str(tmp_path / "abi_host")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", LIB_DIR, "-lmrmod",
                    "-Wl,-rpath," + LIB_DIR, "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
