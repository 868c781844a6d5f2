"""The library from plain C: a C99 program that includes only include/rf.h,
compiled with -Wall -Wextra -pedantic -Werror and linked against librf.so,
runs the entry points that need no GPU (defaults, argument checks, the device
query, the tuner's host model).  No compute call is made."""
import os
import shutil
import subprocess

import pytest

from paper_1809_10895_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NO_GPU = not __import__("torch").cuda.is_available()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_client_builds_and_runs():
    lib = B.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(libdir, "rf_c_client")
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "client.c"),
                           "-o", exe, "-L", libdir, "-lrf", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"])
    r = subprocess.run([exe] + (["--no-device"] if NO_GPU else []), capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
