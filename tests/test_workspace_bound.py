"""deconv_workspace_size returns one layout plus a bound for the arrays that
differ between launch tunings; this test builds the exact layout of every
tuning a plan can be retuned to and checks the bound covers each (no GPU:
host code only, compiled with nvcc against the library's sources)."""
import glob
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1602_01410_gb300")


def test_workspace_bound_covers_every_tuning(tmp_path):
    from paper_1602_01410_gb300 import build as b
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    b.build()
    objs = [o for o in glob.glob(os.path.join(PKG, "_build", "*.o")) if os.path.basename(o) != "plan.o"]
    exe = str(tmp_path / "workspace_bound")
    cmd = [b.nvcc(), *b.ARCH, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(PKG, "csrc"), os.path.join(ROOT, "tests", "harness", "workspace_bound.cu"), *objs, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert r.stdout.count(" ok") >= 7
