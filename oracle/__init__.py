"""FP64 CPU oracle for the Tersoff potential -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA path in
``paper_1710_00882_gb300`` never imports it and shares none of its code.
"""
