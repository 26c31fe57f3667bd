"""ctypes wrapper around the C oracle (test infrastructure only)."""
import ctypes as C
import numpy as np

from .build import build

STEADY, TILTED, HYBRID = 0, 1, 2
MODEL_TRAIT, MODEL_FITNESS = 0, 1

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    u32p = C.POINTER(C.c_uint32)
    i64p = C.POINTER(C.c_int64)
    lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.orc_philox4x32_10.restype = None
    for name in ("orc_site", ):
        getattr(lib, name).argtypes = [C.c_uint32, C.c_uint32, C.c_uint64]
        getattr(lib, name).restype = C.c_int64
    for name in ("orc_site_steady", "orc_site_tilted", "orc_site_hybrid"):
        getattr(lib, name).argtypes = [C.c_uint32, C.c_uint64]
        getattr(lib, name).restype = C.c_int64
    lib.orc_site_table.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, i64p]
    lib.orc_site_table.restype = None
    lib.orc_validate.argtypes = [C.c_void_p]
    lib.orc_validate.restype = C.c_int
    lib.orc_create.argtypes = [C.c_void_p]
    lib.orc_create.restype = C.c_void_p
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_destroy.restype = None
    lib.orc_step.argtypes = [C.c_void_p, C.c_uint32]
    lib.orc_step.restype = None
    lib.orc_migrate.argtypes = [C.c_void_p, u32p]
    lib.orc_migrate.restype = None
    lib.orc_reproduce.argtypes = [C.c_void_p, u32p]
    lib.orc_reproduce.restype = None
    lib.orc_generation.argtypes = [C.c_void_p]
    lib.orc_generation.restype = C.c_uint64
    lib.orc_agent_count.argtypes = [C.c_void_p]
    lib.orc_agent_count.restype = C.c_uint32
    lib.orc_record_bytes.argtypes = [C.c_void_p]
    lib.orc_record_bytes.restype = C.c_uint32
    lib.orc_snapshot.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_snapshot.restype = None
    lib.orc_load.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64]
    lib.orc_load.restype = None
    lib.orc_mrca_margin.argtypes = [C.c_uint32]
    lib.orc_mrca_margin.restype = C.c_uint32
    lib.orc_site_ranks.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, i64p]
    lib.orc_site_ranks.restype = None
    lib.orc_mrca_bounds.argtypes = [C.c_void_p, C.c_uint32, u32p, C.c_uint32, C.c_uint32,
                                    C.c_uint32, C.c_uint32, C.c_uint64, u32p, u32p]
    lib.orc_mrca_bounds.restype = C.c_int
    lib.orc_normal.argtypes = [C.c_uint32, C.c_uint32]
    lib.orc_normal.restype = C.c_float
    lib.orc_unit_log.argtypes = [C.c_float]
    lib.orc_unit_log.restype = C.c_float
    lib.orc_turn_cos.argtypes = [C.c_uint32]
    lib.orc_turn_cos.restype = C.c_float
    lib.orc_mrca_bounds_mixed.argtypes = [C.c_void_p, C.c_uint32, u32p, C.c_uint32, C.c_uint32,
                                          C.c_uint32, C.c_uint32, u32p, u32p]
    lib.orc_mrca_bounds_mixed.restype = C.c_int
    lib.orc_step_async.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p]
    lib.orc_step_async.restype = C.c_int
    lib.orc_track_lineage.argtypes = [C.c_void_p]
    lib.orc_track_lineage.restype = C.c_int
    lib.orc_divergence.argtypes = [C.c_void_p, u32p, C.c_uint32, u32p]
    lib.orc_divergence.restype = C.c_int
    lib.orc_openmp_enabled.argtypes = []
    lib.orc_openmp_enabled.restype = C.c_int
    _lib = lib
    return lib


class OracleConfig(C.Structure):
    """Mirror of the C ``orc_config`` struct."""
    _fields_ = [
        ("rows", C.c_uint32), ("cols", C.c_uint32),
        ("island_size", C.c_uint32), ("tournament_size", C.c_uint32),
        ("p_ben", C.c_double), ("p_del", C.c_double),
        ("surface_sites", C.c_uint32), ("differentia_bits", C.c_uint32),
        ("curation", C.c_uint32), ("migrate_every", C.c_uint32),
        ("seed", C.c_uint64), ("run_id", C.c_uint32), ("threads", C.c_uint32),
        ("model", C.c_uint32), ("effect_scale", C.c_double),
    ]


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint32))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key; returns 4 uint32."""
    lib = _load()
    c, cp = _u32(ctr)
    k, kp = _u32(key)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(cp, kp, out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def site(policy, S, T):
    """Site that the deposit of rank T overwrites, or -1 when it is not stored."""
    return int(_load().orc_site(policy, S, T))


def site_table(policy, S, t0, count):
    """Sites of ranks t0 .. t0 + count - 1 as an int64 array (-1: not stored)."""
    out = np.zeros(count, np.int64)
    _load().orc_site_table(policy, S, t0, count, out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def site_ranks(policy, S, T):
    """Rank held by every site at time T (-1: never written)."""
    out = np.zeros(S, np.int64)
    _load().orc_site_ranks(policy, S, T, out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def mrca_margin(b):
    return int(_load().orc_mrca_margin(b))


def record_bytes(surface_sites, differentia_bits):
    words = (surface_sites * differentia_bits + 31) // 32
    return (8 + 4 * words + 15) // 16 * 16


def mrca_bounds(records, ids, policy, S, b, T):
    """Pairwise (lo, hi) bounds for the sampled agents, row-major upper triangle."""
    lib = _load()
    records = np.ascontiguousarray(records, dtype=np.uint8)
    rb = record_bytes(S, b)
    ids_a, idp = _u32(ids)
    n = len(ids_a)
    npairs = n * (n - 1) // 2
    lo = np.zeros(npairs, np.uint32)
    hi = np.zeros(npairs, np.uint32)
    rc = lib.orc_mrca_bounds(records.ctypes.data, rb, idp, n, policy, S, b, T,
                             lo.ctypes.data_as(C.POINTER(C.c_uint32)),
                             hi.ctypes.data_as(C.POINTER(C.c_uint32)))
    if rc != 0:
        raise ValueError(f"oracle mrca_bounds failed ({rc})")
    return lo, hi


def normal(a, b):
    """Standard normal deviate from two 32-bit words (Box-Muller in IEEE single)."""
    return float(_load().orc_normal(a, b))


def unit_log(x):
    return float(_load().orc_unit_log(x))


def turn_cos(k):
    """cos(2 pi k / 2^24) for a 24-bit k."""
    return float(_load().orc_turn_cos(k))


def mrca_bounds_mixed(records, ids, policy, S, b):
    """Pairwise (lo, hi) bounds from each agent's own counter (counters may differ)."""
    lib = _load()
    records = np.ascontiguousarray(records, dtype=np.uint8)
    rb = record_bytes(S, b)
    ids_a, idp = _u32(ids)
    n = len(ids_a)
    npairs = n * (n - 1) // 2
    lo = np.zeros(npairs, np.uint32)
    hi = np.zeros(npairs, np.uint32)
    rc = lib.orc_mrca_bounds_mixed(records.ctypes.data, rb, idp, n, policy, S, b,
                                   lo.ctypes.data_as(C.POINTER(C.c_uint32)),
                                   hi.ctypes.data_as(C.POINTER(C.c_uint32)))
    if rc != 0:
        raise ValueError(f"oracle mrca_bounds_mixed failed ({rc})")
    return lo, hi


def openmp_enabled():
    return bool(_load().orc_openmp_enabled())


class OracleRun:
    """One GA run held by the C oracle: synchronous generations (step, migrate, reproduce)
    or the asynchronous mode on its sequential schedule (step_async)."""

    def __init__(self, rows, cols, island_size=32, tournament_size=5, p_ben=0.01, p_del=0.01,
                 surface_sites=64, differentia_bits=1, curation=STEADY, migrate_every=1,
                 seed=42, run_id=0, threads=1, model=MODEL_TRAIT, effect_scale=1.0):
        self._lib = _load()
        self.cfg = OracleConfig(rows, cols, island_size, tournament_size, p_ben, p_del,
                                surface_sites, differentia_bits, curation, migrate_every,
                                seed, run_id, threads, model, effect_scale)
        self._st = self._lib.orc_create(C.byref(self.cfg))
        if not self._st:
            raise ValueError("invalid oracle config")
        self.n_agents = int(self._lib.orc_agent_count(self._st))
        self.n_islands = rows * cols
        self.record_bytes = int(self._lib.orc_record_bytes(self._st))

    def close(self):
        if self._st:
            self._lib.orc_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def generation(self):
        return int(self._lib.orc_generation(self._st))

    def step(self, n_gens):
        self._lib.orc_step(self._st, n_gens)

    def step_async(self, n_gens, window=16):
        """Asynchronous mode on the sequential schedule: windows of `window` generations
        (the last one shorter), each run island by island in index order.  Returns the
        number of arrivals per (island, direction) as an (n_islands, 4) array."""
        arrivals = np.zeros((self.n_islands, 4), np.uint64)
        left = int(n_gens)
        while left > 0:
            w = min(window, left)
            rc = self._lib.orc_step_async(self._st, w, arrivals.ctypes.data)
            if rc != 0:
                raise MemoryError("oracle: out of memory")
            left -= w
        return arrivals

    def track_lineage(self):
        """Record every birth from now on (call at generation 0) so that divergence() can
        report true divergence ranks."""
        if self._lib.orc_track_lineage(self._st) != 0:
            raise MemoryError("oracle: out of memory")

    def divergence(self, ids):
        """True divergence rank D of each pair (i < j, row-major) of the given agents: the
        number of births their lineages share."""
        ids_a, idp = _u32(ids)
        n = len(ids_a)
        out = np.zeros(n * (n - 1) // 2, np.uint32)
        if self._lib.orc_divergence(self._st, idp, n,
                                    out.ctypes.data_as(C.POINTER(C.c_uint32))) != 0:
            raise ValueError("lineage tracking is off")
        return out

    def migrate(self):
        """Apply this generation's migration; return the source id of every slot."""
        src = np.zeros(self.n_agents, np.uint32)
        self._lib.orc_migrate(self._st, src.ctypes.data_as(C.POINTER(C.c_uint32)))
        return src

    def reproduce(self):
        """Selection, mutation and deposit of this generation; return winner slots."""
        par = np.zeros(self.n_agents, np.uint32)
        self._lib.orc_reproduce(self._st, par.ctypes.data_as(C.POINTER(C.c_uint32)))
        return par

    def snapshot(self):
        """Canonical records as a (n_agents, record_bytes) uint8 array."""
        out = np.zeros((self.n_agents, self.record_bytes), np.uint8)
        self._lib.orc_snapshot(self._st, out.ctypes.data)
        return out

    def load(self, records, generation):
        records = np.ascontiguousarray(records, dtype=np.uint8)
        assert records.shape == (self.n_agents, self.record_bytes)
        self._lib.orc_load(self._st, records.ctypes.data, generation)

    def traits(self):
        return self.snapshot()[:, 0:4].copy().view(np.int32).reshape(-1)

    def fitness(self):
        return self.snapshot()[:, 0:4].copy().view(np.float32).reshape(-1)

    def counters(self):
        return self.snapshot()[:, 4:8].copy().view(np.uint32).reshape(-1)

    def surfaces(self):
        words = (self.cfg.surface_sites * self.cfg.differentia_bits + 31) // 32
        return self.snapshot()[:, 8:8 + 4 * words].copy().view(np.uint32).reshape(
            self.n_agents, words)

    def mrca_bounds(self, ids):
        return mrca_bounds(self.snapshot(), ids, self.cfg.curation, self.cfg.surface_sites,
                           self.cfg.differentia_bits, self.generation)
