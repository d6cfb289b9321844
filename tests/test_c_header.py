"""include/tn.h is a self-contained C header: a C99 program compiled with gcc against it and
linked to libtnq.so plans a circuit on the host (no device) and frees it."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2108_06831_gb300")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c99_program_against_header(tmp_path):
    lib = os.path.join(PKG, "libtnq.so")
    if not os.path.exists(lib):
        pytest.skip("libtnq.so is not built")
    exe = str(tmp_path / "host_plan")
    cuda_inc = "/usr/local/cuda/include"
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "host_plan.c"), "-o", exe, "-L", PKG, "-ltnq",
           f"-Wl,-rpath,{PKG}"]
    if os.path.isdir(cuda_inc):
        cmd[5:5] = ["-I", cuda_inc]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
