"""FP64 CPU oracle for the chordally decomposed ADMM (test infrastructure).

This package is the independent reference the CUDA library is checked
against.  It is plain, slow and written from the paper:
  chordal.py  chordal extension and maximal cliques (Section 2.1, Section 7.1.1)
  psd.py      cyclic Jacobi eigensolver, PSD projection (Eq. XkUpdate),
              Daleckii-Krein adjoint of the projection (not in the paper)
  admm.py     Algorithms 1, 2 and 3 in the paper's full vec() form.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference arms may import it.  The CUDA library and its Python binding never
do, and the oracle imports nothing from them.
"""
