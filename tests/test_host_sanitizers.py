"""The host-side setup code of the library (nodes, Q, its eigen-decomposition,
DG matrices, slab and node-set transfers: csrc/st_setup.cpp) built with
AddressSanitizer and UndefinedBehaviorSanitizer and driven over every node
count and pair of node sets; any memory or undefined-behaviour error fails
the run.  CPU only."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_12883_gb300", "csrc")


def test_setup_code_under_asan_and_ubsan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "setup_sanitize"
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(CSRC, "st_setup.cpp"), os.path.join(ROOT, "tests", "host", "setup_sanitize_main.cpp"),
           "-o", str(exe)]
    build = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if build.returncode != 0 and "sanitize" in build.stdout and ("cannot find" in build.stdout or "-lasan" in build.stdout):
        pytest.skip("sanitizer runtimes not installed")
    assert build.returncode == 0, build.stdout
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, env=env,
                         timeout=300)
    assert run.returncode == 0 and run.stdout.strip().endswith("ok"), run.stdout
