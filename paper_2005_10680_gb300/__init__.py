"""GB300 (sm_103a) SpAMM with strict error control and SP2 purification.

A thin ctypes binding over the C ABI declared in ``include/spamm.h``; every
step of the computation runs in the CUDA library built from ``csrc/``. There
is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

    import paper_2005_10680_gb300 as sp
    ctx = sp.Context()
    A = ctx.from_dense(a_numpy_or_cuda_tensor, bs=64)
    C, rep = ctx.multiply(A, A, delta=1e-6)          # ||C - A A||_F < 1e-6
    D, prep = ctx.purify(F, n_occ, eps=1e-5, n_iter=60, homo=..., lumo=...)
"""
from ._lib import (  # noqa: F401
    SpammError, Context, Matrix, load_library, library_path, N_TAU, tau_table,
    FP64, MIXED, TRUNCMUL, APPROX, HYBRID,
)
