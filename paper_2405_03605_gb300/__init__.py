"""GB300-native trackable island-model GA (synchronous island step + MRCA bounds).

The compute path is the C-ABI library ``libga.so`` built from ``csrc/`` for sm_103a; the
Python layer in ``ga.py`` only marshals arguments to it.  Importing this package does not
load the library: ``ga.load_library()`` does, on first use, and raises when it is missing.
"""
from .workloads import RunShape  # noqa: F401

__all__ = ["RunShape"]
