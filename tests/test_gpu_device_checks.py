"""Device index checks (the pool has no compute-sanitizer): the device-check build of the
library, libga_debug.so (GA_DEVICE_CHECKS=1), tests every global index in every kernel and
records GA_EBOUNDS instead of making an out-of-range access.  A worker process drives that
build through synchronous runs of every island size and record size (tori from 1x1 up,
migration every 1 and 3 generations, MRCA), asynchronous runs on the sequential schedule
(both handoff protocols, windows 1 and 4), free-running asynchronous runs with the
mixed-counter MRCA and a mixed batch: every status must stay clean and every result must
still equal the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_check_fails():
    from paper_2405_03605_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, PAPER_2405_03605_GB300_LIB=lib)
    res = subprocess.run([sys.executable, os.path.join(HERE, "device_checks_worker.py")],
                         env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "device checks clean" in res.stdout
