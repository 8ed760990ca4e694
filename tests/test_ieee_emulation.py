"""The integer-pipe binary64 routines of the CUDA library (csrc/vc_ieee.cuh:
division by a constant, subtraction, 1 - x, the PLCM step, and the sine's
argument reduction: floor(RN(u + 1/2)), RN(t - k*PIO2_HI) and small integers
as binary64) compiled as host code and compared with the host CPU's IEEE-754
round-to-nearest-even arithmetic on millions of operands (PLCM-like and
arbitrary normal ranges, near-ties, half-integers, multiples of PIO2_HI)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_binary64_matches_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ieee_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2302_07411_gb300", "csrc"),
                           "-o", exe, os.path.join(ROOT, "tests", "ieee_emulation_check.cu")])
    out = subprocess.run([exe, "3000000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "div checked" in out.stdout and "kround checked" in out.stdout and "t-kHI checked" in out.stdout
