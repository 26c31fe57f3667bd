"""CPU oracle for the synchronous trackable island-model GA (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
package.  It is a plain C restatement of the method (``ga_oracle.c``) behind ctypes, and
shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    OracleConfig,
    OracleRun,
    STEADY,
    TILTED,
    HYBRID,
    MODEL_TRAIT,
    MODEL_FITNESS,
    normal,
    unit_log,
    turn_cos,
    philox4x32_10,
    site,
    site_table,
    site_ranks,
    mrca_margin,
    mrca_bounds,
    mrca_bounds_mixed,
    record_bytes,
    openmp_enabled,
)
