"""GB300-native batched range minimum queries (block-based sparse table).

The compute path is the CUDA library ``librmq_gb300.so`` built from ``csrc/``
for sm_103a; ``rmq`` is its thin ctypes binding (argument marshalling only).
``workloads`` holds the seeded input generators.
"""
__all__ = ["rmq", "workloads"]
