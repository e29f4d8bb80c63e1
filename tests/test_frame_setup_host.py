"""The per-pixel reconstruction frame in FP32 (float-float set-up) against
the FP64 set-up, on the host: the library's device header compiled with the
host C++ compiler (no contraction), random absorber sets with and without
the moment bias.  Pixels whose Hankel matrix is near-singular take the FP64
path; the others must give the frame parameters (1/s, -mu/s, skewness, 1/d)
within a few float32 ulps of FP64 and the same kind of frame."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_float_float_frame_matches_fp64(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "frame_setup_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           "-I", os.path.join(ROOT, "paper_2501_12581_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "frame_setup_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    n32, n64, kind = int(out[0]), int(out[1]), int(out[2])
    worst = [float(x) for x in out[3:7]]
    assert n32 > 100000 and n64 > 0          # both paths taken
    assert kind == 0
    assert worst[0] <= 8 and worst[1] <= 8 and worst[3] <= 8, worst
    assert worst[2] <= 64, worst             # skewness, relative to max(1, |g|)
