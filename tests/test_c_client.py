"""The C ABI from plain C: tests/c_client/stp_c_client.c compiles as pedantic
C99 against include/stp.h, links against the library, and (without a GPU)
reports STP_ERR_CUDA from stp_create_problem and exits 0: the library has no
CPU fallback."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_builds_and_refuses_without_a_device(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: this test covers the no-device path")
    from paper_2609_30533_gb300 import build as B
    lib = B.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "stp_c_client")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client", "stp_c_client.c"), "-L", libdir, "-lstp",
           "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "create: STP_ERR_CUDA" in r.stdout
