"""The oracle's Philox4x32-10 against cuRAND's Philox4x32-10 block function, run on the GPU
(an implementation independent of both the oracle and this library)."""
import os
import subprocess

import pytest

import oracle
from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_oracle_philox_matches_curand(tmp_path):
    src = os.path.join(ROOT, "tests", "cuda", "curand_philox_check.cu")
    exe = str(tmp_path / "curand_philox_check")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", src, "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    for i in range(1024):
        ctr = [i, (7 * i) & 0xFFFFFFFF, (13 * i) & 0xFFFFFFFF, (17 * i) & 0xFFFFFFFF]
        key = [i, i ^ 0xDEADBEEF]
        expect = " ".join(f"{int(x):08x}" for x in oracle.philox4x32_10(ctr, key))
        assert out[i] == expect, i
