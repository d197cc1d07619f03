"""FP64 CPU oracle for the FDTD hot path. Test infrastructure only: imported by
tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference legs of
``bench.py``; never by the CUDA library."""
