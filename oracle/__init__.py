"""FP64 CPU oracle of the 3DGS tile-splatting path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and
the two share no code.
"""
