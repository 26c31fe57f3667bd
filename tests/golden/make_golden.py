"""Write tests/golden/small_torus.json from the CPU oracle alone.

The 32x32-island torus of 32-agent islands (16-byte records: steady curation over 64 1-bit
sites), tournament size 5, p_del = 0.01, one migrant per direction every generation, seed
42, run for 1,000 generations in the adaptive (p_ben = 0.01) and purifying-only
(p_ben = 0) treatments of Sec. 3.  Stored: SHA-256 of the canonical end-state records and
a few summary values.  Run: python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleRun  # noqa: E402

CASES = {
    "adaptive": dict(p_ben=0.01, run_id=0),
    "purifying": dict(p_ben=0.0, run_id=1),
}
BASE = dict(rows=32, cols=32, island_size=32, tournament_size=5, p_del=0.01,
            surface_sites=64, differentia_bits=1, curation=0, migrate_every=1, seed=42)
GENERATIONS = 1000


def compute():
    out = {"generations": GENERATIONS, "base": BASE, "cases": {}}
    for name, kw in CASES.items():
        run = OracleRun(**BASE, **kw, threads=4)
        run.step(GENERATIONS)
        rec = run.snapshot()
        t = run.traits()
        out["cases"][name] = {
            **kw,
            "sha256": hashlib.sha256(rec.tobytes()).hexdigest(),
            "trait_sum": int(t.astype("int64").sum()),
            "trait_min": int(t.min()),
            "trait_max": int(t.max()),
        }
    return out


if __name__ == "__main__":
    data = compute()
    with open(os.path.join(HERE, "small_torus.json"), "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(data, indent=1))
