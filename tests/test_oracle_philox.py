"""Oracle Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
import os

import numpy as np

import oracle


def load_kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors(golden_dir):
    rows = load_kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, expect in rows:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == expect


def test_output_bits_balanced():
    # 4,096 counters -> 16,384 words; every bit position is set about half the time
    words = np.array([oracle.philox4x32_10([i, 7, 3 | (1 << 16), 0], [42, 0])
                      for i in range(4096)]).reshape(-1)
    for bit in range(32):
        frac = ((words >> bit) & 1).mean()
        assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(words.size)
