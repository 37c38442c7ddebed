"""nsort — a GB300-native (sm_103a) merge sort for 32-bit keys and key/value
pairs, after "A Hybrid Vectorized Merge Sort on ARM NEON" (NEON-MS).

The sort itself is CUDA in ``csrc/`` built into ``libnsort.so`` behind a C ABI
(``include/nsort.h``).  ``nsort`` is the thin ctypes binding with the same
names; it loads the library on first use and raises if it is missing (there
is no CPU fallback).  ``inputs`` draws the seeded synthetic workloads.
"""
__all__ = ["nsort", "inputs"]
