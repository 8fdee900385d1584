"""Plain, slow CPU oracles of the paper's method (test infrastructure only).

``oracle.sph`` -- FP64 C implementation of the SPH sloshing model (Section 3).
``oracle.lpv`` -- FP64 NumPy implementation of the LPV surrogate (Section 4)
               and of its closed-loop use (Sections 5.1.1, 5.4).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
