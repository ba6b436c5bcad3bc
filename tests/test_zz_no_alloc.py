"""The allocation-free tau search (spamm_cse_search_noalloc), for callers that
cannot allocate device memory, against the regular entry point spamm_multiply.

Inputs and outputs are buffers the caller already owns (here: torch CUDA
tensors); the entry point itself allocates nothing and keeps its scratch in a
fixed device array. Two calls in a row must both reproduce the tau index, tau
and bound that spamm_multiply selects for the same operands and delta."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _call(lib, na, nbm, nb, delta, out_i, out_t, out_b, stream):
    return lib.spamm_cse_search_noalloc(ctypes.c_void_p(na.data_ptr()),
                                        ctypes.c_void_p(nbm.data_ptr()), nb, delta,
                                        ctypes.c_void_p(out_i.data_ptr()),
                                        ctypes.c_void_p(out_t.data_ptr()),
                                        ctypes.c_void_p(out_b.data_ptr()), stream)


def test_noalloc_search_matches_spamm_multiply_twice():
    import torch

    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    lib = sp.load_library()
    # the last case has nb = 200 leaf blocks per side: its first fold fills every
    # entry of the scratch's first level buffer and it folds one level more
    cases = [(synth.banded_decay(1000, 31, length=40.0), 64, 1e-6),
             (synth.random_decaying(700, 32, length=30.0), 32, 1e-4),
             (synth.banded_decay(6400, 33, length=40.0), 32, 1e-6),
             (synth.lattice_fock_blocks(2048, seed=34, bs=32, cutoff=1.5).to_dense(), 32, 1e-6)]
    for X, bs, delta in cases:
        G = ctx.from_dense(X, bs)
        _, rep = ctx.multiply(G, G, delta, prec="fp64")
        nrm = torch.from_numpy(G.block_norms()).cuda().contiguous()
        nb = nrm.shape[0]
        for _ in range(2):
            out_i = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            out_t = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            out_b = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            assert _call(lib, nrm, nrm, nb, delta, out_i, out_t, out_b, stream) == 0
            torch.cuda.synchronize()
            assert int(out_i.item()) == rep["tau_index"]
            assert float(out_t.item()) == rep["tau"]
            assert float(out_b.item()) == pytest.approx(rep["bound"], rel=1e-12, abs=0)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    import paper_2005_10680_gb300 as sp
    lib = sp.load_library()
    big = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.spamm_cse_search_noalloc(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                      300, 1e-6, None, ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == 1
    assert b"256" in lib.spamm_last_error()
