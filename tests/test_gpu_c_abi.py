"""The C ABI from plain C, without Python (needs a GPU).

tests/c_abi/uniform_flow.c is compiled with gcc against include/lcs.h and
linked with liblcs.so and the CUDA runtime; it advances particles released
with the fluid velocity of a uniform flow through 50 steps with migration
between 2x2x2 subdomains and a cell sort every 5 steps, and checks that each
ends at X0 + n dt U0 (the exact solution of Eqs. 5-6 for U - V = 0) with an
unchanged velocity, and that ids and segments are intact.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def cuda_lib_dir(cuda: str) -> str:
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(cuda, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    pytest.skip("libcudart.so not found")


def test_uniform_flow_from_c(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_11008_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc") or pytest.skip("gcc not found")
    cuda = os.path.dirname(os.path.dirname(build.nvcc()))
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "uniform_flow")
    subprocess.run([gcc, "-std=c11", "-O2", os.path.join(ROOT, "tests", "c_abi", "uniform_flow.c"),
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    "-L", libdir, "-llcs", "-L", cuda_lib_dir(cuda), "-lcudart", "-lm",
                    "-Wl,-rpath," + libdir, "-Wl,-rpath," + cuda_lib_dir(cuda), "-o", exe],
                   check=True)
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.startswith("ok"), run.stdout
