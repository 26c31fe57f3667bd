"""Thin ctypes binding of libga (include/ga.h): argument marshalling only.

Every step of the island GA and of the MRCA bounds runs in the library's CUDA kernels;
PyTorch supplies device memory (the run's workspace) and the CUDA stream.  The library must
have been built (``__graft_entry__.build()`` or ``python paper_2405_03605_gb300/build.py``);
``load_library`` raises if it is missing -- there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

from .workloads import RunShape

# The library built in-tree; PAPER_2405_03605_GB300_LIB may name another build of it.
LIB_PATH = os.environ.get("PAPER_2405_03605_GB300_LIB") or os.path.join(
    os.path.dirname(os.path.abspath(__file__)), "libga.so")

GA_OK = 0
STEADY, TILTED, HYBRID = 0, 1, 2
MODEL_TRAIT, MODEL_FITNESS = 0, 1
SYNC, ASYNC, ASYNC_SEQUENTIAL = 0, 1, 2
RESIDENT_AUTO, RESIDENT_OFF, RESIDENT_ON = 0, 1, 2

EXPORTED = (
    "ga_config_default", "ga_config_check", "ga_record_bytes", "ga_workspace_bytes",
    "ga_create", "ga_migrate_policy", "ga_step", "ga_sync", "ga_generation",
    "ga_launch_count", "ga_population", "ga_snapshot", "ga_snapshot_device", "ga_load",
    "ga_mrca_bounds", "ga_mrca_bounds_device", "ga_destroy", "ga_strerror", "ga_reset",
    "ga_curation_sites", "ga_mrca_bounds_noalloc", "ga_batch_create", "ga_batch_add",
    "ga_batch_remove", "ga_batch_size", "ga_batch_step", "ga_batch_sync",
    "ga_batch_launch_count", "ga_batch_autotune", "ga_batch_class_warps", "ga_batch_destroy",
    "ga_async_window", "ga_int_peak", "ga_resident_policy", "ga_inject_lost_migrants",
)


class GaError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class GaConfig(C.Structure):
    """Mirror of ``ga_config``."""
    _fields_ = [
        ("rows", C.c_uint32), ("cols", C.c_uint32),
        ("island_size", C.c_uint32), ("tournament_size", C.c_uint32),
        ("p_ben", C.c_double), ("p_del", C.c_double),
        ("surface_sites", C.c_uint32), ("differentia_bits", C.c_uint32),
        ("curation", C.c_uint32), ("mode", C.c_uint32),
        ("seed", C.c_uint64), ("run_id", C.c_uint32), ("model", C.c_uint32),
        ("stream", C.c_void_p), ("effect_scale", C.c_double),
    ]


_lib = None


def load_library(path=LIB_PATH):
    """Load libga.so and declare its signatures.  Raises when the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libga.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, u32, u64, sz = C.c_void_p, C.c_uint32, C.c_uint64, C.c_size_t
    u32p = C.POINTER(C.c_uint32)
    cfgp = C.POINTER(GaConfig)
    sig = {
        "ga_config_default": ([cfgp], C.c_int),
        "ga_config_check": ([cfgp], C.c_int),
        "ga_record_bytes": ([cfgp, u32p], C.c_int),
        "ga_workspace_bytes": ([cfgp, C.POINTER(sz)], C.c_int),
        "ga_create": ([cfgp, vp, sz, C.POINTER(vp)], C.c_int),
        "ga_migrate_policy": ([vp, u32, u32], C.c_int),
        "ga_step": ([vp, u32], C.c_int),
        "ga_sync": ([vp], C.c_int),
        "ga_generation": ([vp, C.POINTER(u64)], C.c_int),
        "ga_launch_count": ([vp, C.POINTER(u64)], C.c_int),
        "ga_population": ([vp, C.POINTER(vp), C.POINTER(sz)], C.c_int),
        "ga_snapshot": ([vp, vp, sz, C.POINTER(sz)], C.c_int),
        "ga_snapshot_device": ([vp, vp, sz, C.POINTER(sz)], C.c_int),
        "ga_load": ([vp, vp, sz, u64], C.c_int),
        "ga_mrca_bounds": ([vp, vp, u32, vp, vp], C.c_int),
        "ga_mrca_bounds_device": ([vp, vp, u32, vp, vp], C.c_int),
        "ga_destroy": ([vp], C.c_int),
        "ga_strerror": ([C.c_int], C.c_char_p),
        "ga_reset": ([vp], C.c_int),
        "ga_curation_sites": ([u32, u32, u32, u32, vp, vp], C.c_int),
        "ga_batch_create": ([vp, C.POINTER(vp)], C.c_int),
        "ga_batch_add": ([vp, vp], C.c_int),
        "ga_batch_remove": ([vp, vp], C.c_int),
        "ga_batch_size": ([vp, C.POINTER(u32)], C.c_int),
        "ga_batch_step": ([vp, u32], C.c_int),
        "ga_batch_sync": ([vp], C.c_int),
        "ga_batch_launch_count": ([vp, C.POINTER(u64)], C.c_int),
        "ga_batch_autotune": ([vp, u32, C.POINTER(u32)], C.c_int),
        "ga_batch_class_warps": ([vp, u32, C.POINTER(u32), C.POINTER(u32)], C.c_int),
        "ga_batch_destroy": ([vp], C.c_int),
        "ga_async_window": ([vp, u32], C.c_int),
        "ga_int_peak": ([u32, u32, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
        "ga_resident_policy": ([vp, u32, u32], C.c_int),
        "ga_inject_lost_migrants": ([vp, u32], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def strerror(code):
    return load_library().ga_strerror(code).decode()


def _check(rc, what):
    if rc != GA_OK:
        raise GaError(rc, what)


def make_config(shape: RunShape, stream=0):
    cfg = GaConfig()
    load_library().ga_config_default(C.byref(cfg))
    for k in ("rows", "cols", "island_size", "tournament_size", "p_ben", "p_del",
              "surface_sites", "differentia_bits", "curation", "seed", "run_id", "model",
              "effect_scale", "mode"):
        setattr(cfg, k, getattr(shape, k))
    cfg.stream = stream or None
    return cfg


def config_check(shape: RunShape):
    return load_library().ga_config_check(C.byref(make_config(shape)))


def workspace_bytes(shape: RunShape):
    n = C.c_size_t()
    _check(load_library().ga_workspace_bytes(C.byref(make_config(shape)), C.byref(n)),
           "ga_workspace_bytes")
    return n.value


def record_bytes(shape: RunShape):
    n = C.c_uint32()
    _check(load_library().ga_record_bytes(C.byref(make_config(shape)), C.byref(n)),
           "ga_record_bytes")
    return n.value


class Run:
    """One GA run on the current CUDA device.

    workspace: "torch" (default) allocates the device workspace as a torch uint8 tensor and
    hands it to the library; "library" lets the library cudaMalloc it.  stream: a
    torch.cuda.Stream (default: the current stream).
    """

    def __init__(self, shape: RunShape, stream=None, workspace="torch"):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.shape = shape
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.cfg = make_config(shape, self.stream.cuda_stream)
        self.record_bytes = record_bytes(shape)
        self.n_agents = shape.n_agents
        self._ws = None
        ptr, nbytes = None, 0
        if workspace == "torch":
            nbytes = workspace_bytes(shape)
            with torch.cuda.stream(self.stream):
                self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            self._ws_off = (-base) % 256
            ptr = base + self._ws_off
        h = C.c_void_p()
        _check(self.lib.ga_create(C.byref(self.cfg), ptr, nbytes, C.byref(h)), "ga_create")
        self._h = h
        _check(self.lib.ga_migrate_policy(h, 1 if shape.migrate_every else 0,
                                          max(1, shape.migrate_every)), "ga_migrate_policy")
        if shape.mode != SYNC:
            self.async_window(shape.async_window)

    # -- lifecycle ------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self.lib.ga_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping -------------------------------------------------------------------------
    def reset(self):
        _check(self.lib.ga_reset(self._h), "ga_reset")

    def migrate_policy(self, per_neighbor, every_k):
        _check(self.lib.ga_migrate_policy(self._h, per_neighbor, every_k), "ga_migrate_policy")

    def async_window(self, window):
        """Generations each launch runs in the asynchronous modes (1..256)."""
        _check(self.lib.ga_async_window(self._h, window), "ga_async_window")

    def resident_policy(self, mode, wait_limit_us=1_000_000):
        """RESIDENT_AUTO / RESIDENT_OFF / RESIDENT_ON and the mailbox wait limit (us)."""
        _check(self.lib.ga_resident_policy(self._h, mode, wait_limit_us), "ga_resident_policy")

    def inject_lost_migrants(self, island=0xFFFFFFFF):
        """Fault injection: in resident launches `island` never sends (0xFFFFFFFF: off)."""
        _check(self.lib.ga_inject_lost_migrants(self._h, island), "ga_inject_lost_migrants")

    def step(self, n_gens):
        _check(self.lib.ga_step(self._h, n_gens), "ga_step")

    def sync(self):
        _check(self.lib.ga_sync(self._h), "ga_sync")

    @property
    def generation(self):
        g = C.c_uint64()
        _check(self.lib.ga_generation(self._h, C.byref(g)), "ga_generation")
        return g.value

    @property
    def launches(self):
        n = C.c_uint64()
        _check(self.lib.ga_launch_count(self._h, C.byref(n)), "ga_launch_count")
        return n.value

    # -- state ----------------------------------------------------------------------------
    def snapshot(self, out=None):
        """Canonical records as a host (n_agents, record_bytes) uint8 array (optionally a
        caller-supplied, e.g. pinned, array of that shape)."""
        if out is None:
            out = np.empty((self.n_agents, self.record_bytes), np.uint8)
        assert out.dtype == np.uint8 and out.flags.c_contiguous
        assert out.nbytes == self.n_agents * self.record_bytes
        w = C.c_size_t()
        _check(self.lib.ga_snapshot(self._h, out.ctypes.data, out.nbytes, C.byref(w)),
               "ga_snapshot")
        return out

    def snapshot_device(self, out=None):
        """Canonical records copied into a device uint8 tensor (asynchronous)."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.n_agents, self.record_bytes), dtype=torch.uint8,
                              device="cuda")
        w = C.c_size_t()
        _check(self.lib.ga_snapshot_device(self._h, out.data_ptr(), out.numel(), C.byref(w)),
               "ga_snapshot_device")
        return out

    def population_ptr(self):
        p, n = C.c_void_p(), C.c_size_t()
        _check(self.lib.ga_population(self._h, C.byref(p), C.byref(n)), "ga_population")
        return p.value, n.value

    def load(self, records, generation):
        records = np.ascontiguousarray(records, dtype=np.uint8)
        _check(self.lib.ga_load(self._h, records.ctypes.data, records.nbytes, generation),
               "ga_load")

    # -- MRCA -----------------------------------------------------------------------------
    def mrca_bounds(self, ids, lo=None, hi=None):
        """Host ids -> host (lo, hi) uint32 arrays over pairs i < j, row-major (optionally
        caller-supplied, e.g. pinned, output arrays)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        n = ids.size
        pairs = n * (n - 1) // 2
        lo = np.empty(pairs, np.uint32) if lo is None else lo
        hi = np.empty(pairs, np.uint32) if hi is None else hi
        assert lo.dtype == np.uint32 and hi.dtype == np.uint32
        assert lo.size == pairs and hi.size == pairs
        _check(self.lib.ga_mrca_bounds(self._h, ids.ctypes.data, n, lo.ctypes.data,
                                       hi.ctypes.data), "ga_mrca_bounds")
        return lo, hi

    def mrca_bounds_device(self, ids, lo=None, hi=None):
        """Device ids tensor (int32/uint32 storage) -> device (lo, hi) tensors, async."""
        torch = self._torch
        n = ids.numel()
        pairs = n * (n - 1) // 2
        if lo is None:
            lo = torch.empty(pairs, dtype=torch.int32, device="cuda")
        if hi is None:
            hi = torch.empty(pairs, dtype=torch.int32, device="cuda")
        _check(self.lib.ga_mrca_bounds_device(self._h, ids.data_ptr(), n, lo.data_ptr(),
                                              hi.data_ptr()), "ga_mrca_bounds_device")
        return lo, hi


def curation_sites(policy, surface_sites, t0, count, stream=None):
    """Device int32 tensor of curation sites for ranks t0 .. t0 + count - 1 (-1: not stored)."""
    import torch
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().ga_curation_sites(policy, surface_sites, t0, count, out.data_ptr(),
                                            st or None), "ga_curation_sites")
    return out


def mrca_bounds_noalloc(records_ptr, record_bytes, n_agents, curation, surface_sites,
                        differentia_bits, generation, ids, lo, hi, stream=None):
    """ga_mrca_bounds_noalloc: MRCA bounds for callers that cannot allocate device memory.
    records_ptr: device address of the canonical records; ids, lo, hi: contiguous device
    tensors with 32-bit elements, caller-allocated, lo and hi distinct and holding at least
    n (n - 1) / 2 elements each (ValueError otherwise).  Synchronous; raises GaError when the
    library reports a failure."""
    import torch
    n = ids.numel()
    pairs = n * (n - 1) // 2
    for name, t, need in (("ids", ids, n), ("lo", lo, pairs), ("hi", hi, pairs)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
                and t.element_size() == 4):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of 4-byte elements")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} elements, {need} needed")
    if lo.data_ptr() == hi.data_ptr():
        raise ValueError("lo and hi must be distinct tensors")
    lib = load_library()
    f = lib.ga_mrca_bounds_noalloc
    f.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                  C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(f(records_ptr, record_bytes, n_agents, curation, surface_sites, differentia_bits,
             generation, ids.data_ptr(), n, lo.data_ptr(), hi.data_ptr(), st or None),
           "ga_mrca_bounds_noalloc")


PEAK_LOP3, PEAK_IMAD, PEAK_MIX = 0, 1, 2


def int_peak(kind, iters=2048, stream=None):
    """ga_int_peak: (operations per second, seconds) of one timed launch of the integer-pipe
    probe on the current device."""
    import torch
    rate, sec = C.c_double(), C.c_double()
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().ga_int_peak(kind, iters, st or None, C.byref(rate), C.byref(sec)),
           "ga_int_peak")
    return rate.value, sec.value


class Batch:
    """Several runs advanced by shared launches (``ga_batch_*``).  Member results are
    bit-identical to stepping each run alone.  stream: a torch.cuda.Stream (default: one the
    batch creates)."""

    def __init__(self, runs=(), stream=None):
        self.lib = load_library()
        self.stream = stream
        h = C.c_void_p()
        _check(self.lib.ga_batch_create(stream.cuda_stream if stream is not None else None,
                                        C.byref(h)), "ga_batch_create")
        self._h = h
        self.runs = []
        for r in runs:
            self.add(r)

    def add(self, run):
        _check(self.lib.ga_batch_add(self._h, run._h), "ga_batch_add")
        self.runs.append(run)

    def remove(self, run):
        _check(self.lib.ga_batch_remove(self._h, run._h), "ga_batch_remove")
        self.runs.remove(run)

    def step(self, n_gens):
        _check(self.lib.ga_batch_step(self._h, n_gens), "ga_batch_step")

    def sync(self):
        _check(self.lib.ga_batch_sync(self._h), "ga_batch_sync")

    def autotune(self, trial_gens=16):
        chunk = C.c_uint32()
        _check(self.lib.ga_batch_autotune(self._h, trial_gens, C.byref(chunk)),
               "ga_batch_autotune")
        warps = []
        i = 0
        while True:
            n, w = C.c_uint32(), C.c_uint32()
            if self.lib.ga_batch_class_warps(self._h, i, C.byref(n), C.byref(w)) != GA_OK:
                break
            warps.append((n.value, w.value))
            i += 1
        return {"chunk": chunk.value, "class_warps": warps}

    @property
    def launches(self):
        n = C.c_uint64()
        _check(self.lib.ga_batch_launch_count(self._h, C.byref(n)), "ga_batch_launch_count")
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            self.lib.ga_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
