"""The C-ABI library builds, loads and exports every entry point include/ga.h declares; host-only
calls (configuration checks and sizes) work without a GPU."""
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2405_03605_gb300 import build, ga
    build.build()
    return ga.load_library()


def declared_functions():
    with open(os.path.join(ROOT, "include", "ga.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ga_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_exported(lib):
    from paper_2405_03605_gb300 import ga
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ga.EXPORTED)


def test_config_checks(lib):
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS, variant_shapes, PAPER_ADAPTIVE
    assert ga.config_check(SMALL_TORUS) == 0
    assert ga.config_check(PAPER_ADAPTIVE) == 0
    for n in (16, 32, 64):
        for shape in variant_shapes(n).values():
            assert ga.config_check(shape) == 0
    assert ga.config_check(SMALL_TORUS.with_(island_size=24)) == -1
    assert ga.config_check(SMALL_TORUS.with_(tournament_size=0)) == -1
    assert ga.config_check(SMALL_TORUS.with_(tournament_size=9)) == -1
    assert ga.config_check(SMALL_TORUS.with_(p_ben=0.6, p_del=0.5)) == -1
    assert ga.config_check(SMALL_TORUS.with_(differentia_bits=3)) == -1
    assert ga.config_check(SMALL_TORUS.with_(surface_sites=512)) == -1
    assert ga.config_check(SMALL_TORUS.with_(surface_sites=4, curation=2)) == -1
    assert ga.config_check(SMALL_TORUS.with_(rows=0)) == -1
    # valid but no kernel compiled for 256-agent islands
    assert ga.config_check(SMALL_TORUS.with_(island_size=256)) == -6


def test_async_config_checks(lib):
    """Asynchronous modes: kernels for islands of 8 to 128 agents, every record size and
    both genome models; unknown modes are invalid."""
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS, ASYNC, ASYNC_SEQUENTIAL, \
        MODEL_FITNESS
    for mode in (ASYNC, ASYNC_SEQUENTIAL):
        for n in (8, 16, 32, 64, 128):
            for sites, bits in ((64, 1), (128, 1), (256, 1), (32, 8)):
                shape = SMALL_TORUS.with_(mode=mode, island_size=n, surface_sites=sites,
                                          differentia_bits=bits)
                assert ga.config_check(shape) == 0, (mode, n, sites, bits)
            # the float-fitness model has kernels for 16, 32 and 64 agents in every mode
            want = 0 if n in (16, 32, 64) else -6
            assert ga.config_check(SMALL_TORUS.with_(mode=mode, island_size=n,
                                                     model=MODEL_FITNESS, p_del=0.33)) == want
        assert ga.config_check(SMALL_TORUS.with_(mode=mode, island_size=4)) == -6
    assert ga.config_check(SMALL_TORUS.with_(mode=3)) == -1


def test_async_workspace_sizes(lib):
    """16-byte records travel through 16-byte buffers, larger ones through a 16-byte flag
    word plus the record: four per island, after the two population buffers.  The synchronous
    run of 16-byte records carries the resident mailboxes there instead (256 bytes plus two
    parities of four 16-byte mailboxes per island)."""
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS, ASYNC
    for sites, rb in ((64, 16), (128, 32), (256, 48)):
        sync = SMALL_TORUS.with_(surface_sites=sites)
        extra = ga.workspace_bytes(sync.with_(mode=ASYNC)) - ga.workspace_bytes(sync)
        per_buffer = 16 if rb == 16 else 16 + rb
        want = sync.n_islands * 4 * per_buffer
        if rb == 16:
            want -= 256 + sync.n_islands * 128
        assert want <= extra < want + 256, (sites, extra, want)


def test_resident_state_sizes(lib):
    """Resident mailboxes are part of the workspace of synchronous 16-byte-record runs of at
    most 8,192 islands, and of no other run."""
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS
    def ws(**kw):
        return ga.workspace_bytes(SMALL_TORUS.with_(**kw))
    n16 = SMALL_TORUS.with_(rows=64, cols=128)  # 8,192 islands
    base = ws(rows=64, cols=128, surface_sites=128) - 2 * n16.n_agents * 32
    assert ws(rows=64, cols=128) - 2 * n16.n_agents * 16 == base + 256 + 8192 * 128
    over = SMALL_TORUS.with_(rows=64, cols=129)
    assert ws(rows=64, cols=129) - 2 * over.n_agents * 16 == base


def test_sizes(lib):
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS, variant_shapes, PAPER_ADAPTIVE
    assert ga.record_bytes(SMALL_TORUS) == 16
    v = variant_shapes(32)
    assert ga.record_bytes(v["steady256x1"]) == 48
    assert ga.record_bytes(v["tilted32x8"]) == 48
    assert ga.record_bytes(v["hybrid64x1"]) == 16
    assert ga.record_bytes(SMALL_TORUS.with_(surface_sites=128)) == 32
    n = PAPER_ADAPTIVE.n_agents
    assert n == 16777216
    ws = ga.workspace_bytes(PAPER_ADAPTIVE)
    assert 2 * n * 16 < ws <= 2 * n * 16 + 65536


def test_strerror(lib):
    from paper_2405_03605_gb300 import ga
    assert ga.strerror(0) == "ok"
    assert "invalid" in ga.strerror(-1)
    for code in range(-8, 0):  # every GA_E* code of ga.h has its own message
        assert ga.strerror(code) != "unknown error", code
    assert "index check" in ga.strerror(-8)
    assert ga.strerror(-99) == "unknown error"


def test_record_layout_matches_oracle(lib):
    import oracle
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS
    for S, b in ((64, 1), (256, 1), (32, 8), (128, 1), (16, 2), (4, 1)):
        assert ga.record_bytes(SMALL_TORUS.with_(surface_sites=S, differentia_bits=b)) == \
            oracle.record_bytes(S, b)


def test_product_path_has_no_oracle_reference():
    """The library and its binding never load the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2405_03605_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    text = f.read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "ga_oracle" not in text and "orc_" not in text, fn
