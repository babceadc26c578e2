"""FP64 CPU oracle for the SNAP energy/force path (test infrastructure only).

The oracle is the slow, plain reference the CUDA library is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does.  It shares no code
with the CUDA path.  See ``snap_oracle.c`` for the definitions it follows.
"""
