"""CPU check of the CUDA library's Stockham FFT core: the radix-2/3/4/5/8/16 butterflies and stage
indexing of fft_core.cuh, compiled as host C++ (g++), against a direct long-double DFT."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_stockham_core_matches_direct_dft():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fftchk")
        subprocess.run(["g++", "-O2", "-std=c++17", "-x", "c++", os.path.join(HERE, "fft_core_check.cpp"),
                        "-o", exe], check=True)
        sizes = [str(n) for n in (1, 2, 3, 4, 5, 6, 8, 9, 12, 15, 16, 20, 25, 27, 32, 48, 60, 64, 80, 96,
                                  100, 125, 128, 144, 160, 192, 243, 250, 256, 384, 512, 1000, 1024)]
        r = subprocess.run([exe, *sizes], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
        r = subprocess.run([exe, "ct"], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
