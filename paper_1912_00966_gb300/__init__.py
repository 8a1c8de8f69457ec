"""Earliest-arrival-time queries on GB300: Cluster-AP fixpoint in hand-written sm_103a CUDA.

The compute lives in libeat.so (C ABI in include/eat.h); `eat` is its ctypes binding.
Importing `paper_1912_00966_gb300.eat` fails loudly when libeat.so has not been built.
"""
