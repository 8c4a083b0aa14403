"""FP64 CPU oracle for the Zakharov / HOS wave step.

Test infrastructure only. ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers; the CUDA product path
never imports it and the two share no code (only the seeded input generators
of ``paper_2608_25203_b300.seas`` feed both, as data).
"""
from .dft import dft, dft_matrix, fwd2, inv2  # noqa: F401
from .zakharov import Grid, Oracle, mode_index, padded_size, run, sigma_box  # noqa: F401
