"""The C ABI from plain C: tests/c/abi_client.c, compiled with gcc against include/ga.h and
linked with libga.so, must produce the same records and MRCA bounds as the Python binding
(and a checkpoint resumed through ga_load the same end state)."""
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from gpu_util import gpu_run
from paper_2405_03605_gb300.workloads import RunShape, ASYNC_SEQUENTIAL

pytestmark = pytest.mark.gpu


def fnv1a(data, h=1469598103934665603):
    for byte in bytes(data):
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_c_client_matches_binding(tmp_path):
    from paper_2405_03605_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_client")
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_client.c"), "-o", exe,
                    os.path.dirname(lib) + "/libga.so", "-Wl,-rpath," + os.path.dirname(lib)],
                   check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    out = dict(line.split() for line in res.stdout.strip().split("\n"))

    shape = RunShape(rows=16, cols=16, seed=1234, run_id=7)
    g = gpu_run(shape)
    g.step(120)
    rec = g.snapshot()
    assert int(out["sync"], 16) == fnv1a(rec.tobytes())
    assert out["resume"] == out["sync"]
    ids = np.array([i * 127 % shape.n_agents for i in range(64)], np.uint32)
    lo, hi = g.mrca_bounds(ids)
    assert int(out["mrca"], 16) == fnv1a(hi.tobytes(), fnv1a(lo.tobytes()))

    a = gpu_run(shape.with_(mode=ASYNC_SEQUENTIAL, async_window=4))
    a.step(40)
    assert int(out["async"], 16) == fnv1a(a.snapshot().tobytes())
