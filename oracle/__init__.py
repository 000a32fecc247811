"""FP64 CPU oracle for the particle-based BP update of "Soft-Coherent Direct
Multipath SLAM" (arXiv 2604.19723).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, helpers or constant
tables); the only common module is the seeded input generator
``paper_2604_19723_gb300.workload``, which holds none of the method's
arithmetic.

Every function cites the passage of the paper it follows (section, equation
or supplementary section).  The oracle is plain and slow on purpose:
complex-Gaussian messages are evaluated by their definition (explicit
Nz x Nz covariance, Cholesky, log-density) in ``messages_dense``; the
low-rank forms of Supplementary Sec. S-V live separately in
``messages_woodbury`` and are pinned against the dense definition.

Parity status of each function is listed in the module headers; the one
function with no independent pin is the particle-pairing choice itself
(reading R1), which is marked "parity unpinned" where it is used.
"""
