"""The packed-byte background band test of the CUDA path (csrc/hmi_band.h),
built with g++ on the CPU: exhaustive over (c', lo, hi) byte triples in every
byte lane, and on random 16-pixel chunks at random gains against a plain
per-channel loop of the band test (Sec. 3.1 (i): background iff every
gain-corrected channel lies in [lo, hi])."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_04393_gb300", "csrc")


def test_packed_band_test_matches_definition(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    exe = str(tmp_path / "band_swar_main")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC,
                    os.path.join(ROOT, "tests", "native", "band_swar_main.cpp"), "-o", exe],
                   check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
