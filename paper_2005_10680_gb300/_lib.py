"""ctypes marshalling for the C ABI (``include/spamm.h``). Argument
marshalling only: no step of the method runs here."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
N_TAU = 350
FP64, MIXED = 0, 1
TRUNCMUL, APPROX, HYBRID = 1, 4, 5
_PREC = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}


class SpammError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class Report(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tau_index", ctypes.c_int32),
                ("cse_evals", ctypes.c_int32), ("bound", ctypes.c_double),
                ("bound_round", ctypes.c_double), ("lmax", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("candidates", ctypes.c_int64),
                ("kept", ctypes.c_int64), ("formed", ctypes.c_int64),
                ("pipe_flops", ctypes.c_double),
                ("nnzb_out", ctypes.c_int64),
                ("fro_out", ctypes.c_double), ("trace_out", ctypes.c_double),
                ("idem", ctypes.c_double), ("removed_sq", ctypes.c_double),
                ("removed_blocks", ctypes.c_int64), ("ms", ctypes.c_float * 8)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms"}
        d["ms"] = list(self.ms)
        return d


class TuneResult(ctypes.Structure):
    _fields_ = [("bs", ctypes.c_int32), ("prec", ctypes.c_int), ("ms", ctypes.c_float * 4),
                ("cached", ctypes.c_int32)]


class PurifyOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("prec", ctypes.c_int), ("homo", ctypes.c_double),
                ("lumo", ctypes.c_double), ("have_bounds", ctypes.c_int),
                ("lmin", ctypes.c_double), ("lmax", ctypes.c_double)]


_PD = ctypes.POINTER(ctypes.c_double)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)


class PurifyReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("idem", ctypes.c_double), ("trace", ctypes.c_double),
                ("lmin", ctypes.c_double), ("lmax", ctypes.c_double),
                ("kept_total", ctypes.c_int64), ("formed_total", ctypes.c_int64),
                ("pipe_flops_total", ctypes.c_double),
                ("cand_total", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_phase", ctypes.c_double * 8),
                ("step_delta", _PD), ("step_tau", _PD), ("step_trace", _PD),
                ("step_idem", _PD), ("step_branch", _PI32), ("step_nnzb", _PI64),
                ("step_lmax", _PI32), ("step_ms", ctypes.POINTER(ctypes.c_float))]


_lib = None


def library_path() -> str:
    return os.path.join(HERE, "_build", "libspamm_gb300.so")


def load_library(build_if_stale: bool = True):
    """Load the CUDA library (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        from . import build as _build
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run python -m paper_2005_10680_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "spamm_create": ([P(vp), i32, vp], i32),
        "spamm_destroy": ([vp], None),
        "spamm_strerror": ([i32], ctypes.c_char_p),
        "spamm_last_error": ([], ctypes.c_char_p),
        "spamm_ctx_launches": ([vp], i64),
        "spamm_prec_supported": ([vp, i32, i32], i32),
        "spamm_mat_from_dense": ([vp, vp, i64, i64, i32, d, i32, P(vp)], i32),
        "spamm_mat_to_dense": ([vp, vp, vp, i64, i32], i32),
        "spamm_mat_to_blocks": ([vp, vp, _PI32, _PI32, vp, i32], i32),
        "spamm_mat_get_blocks": ([vp, vp, i64, _PI32, _PI32, vp, _PI32], i32),
        "spamm_mat_from_blocks": ([vp, i64, i32, i64, P(i32), P(i32), vp, i32, P(vp)], i32),
        "spamm_mat_info": ([vp, P(i64), P(i32), P(i64)], i32),
        "spamm_mat_block_norms": ([vp, vp, _PD], i32),
        "spamm_mat_block_map": ([vp, vp, _PI32], i32),
        "spamm_mat_free": ([vp], None),
        "spamm_cse": ([vp, vp, vp, _PD, i32, _PD], i32),
        "spamm_multiply": ([vp, vp, vp, d, i32, P(vp), P(Report)], i32),
        "spamm_multiply_tau": ([vp, vp, vp, d, i32, P(vp), P(Report)], i32),
        "spamm_sp2_step": ([vp, vp, i32, d, d, i32, P(vp), P(Report)], i32),
        "spamm_truncate": ([vp, vp, d, i32, P(Report)], i32),
        "spamm_purify": ([vp, vp, i64, d, i32, P(PurifyOpts), P(vp), P(PurifyReport)], i32),
        "spamm_cse_search_noalloc": ([vp, vp, i64, d, vp, vp, vp, vp], i32),
        "spamm_autotune": ([vp, vp, d, i32, P(TuneResult)], i32),
        "spamm_set_bound": ([vp, i32], i32),
        "spamm_debug_fail_alloc": ([i64], i32),
        "spamm_set_tau_table": ([vp, d, d], i32),
        "spamm_purify_batched": ([vp, i32, P(vp), P(i64), d, i32, P(PurifyOpts), i32, P(vp),
                                  P(PurifyReport), P(ctypes.c_int32)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str, allow=()):
    if st != 0 and st not in allow:
        lib = load_library(False)
        raise SpammError(st, where, lib.spamm_strerror(st).decode() + ": " +
                         lib.spamm_last_error().decode())
    return st


def tau_table() -> np.ndarray:
    t = np.empty(N_TAU)
    t[0] = 1.0
    for i in range(1, N_TAU):
        t[i] = 0.9 * t[i - 1]
    return t


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Matrix:
    """A block-sparse float64 matrix resident on the GPU (owns its handle)."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.spamm_mat_free(h)
            self.handle = None

    def free(self):
        self.__del__()

    def info(self):
        n, bs, nnzb = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(_lib.spamm_mat_info(self.handle, ctypes.byref(n), ctypes.byref(bs),
                                   ctypes.byref(nnzb)), "spamm_mat_info")
        return n.value, bs.value, nnzb.value

    @property
    def n(self):
        return self.info()[0]

    @property
    def bs(self):
        return self.info()[1]

    @property
    def nnzb(self):
        return self.info()[2]

    @property
    def nb(self):
        n, bs, _ = self.info()
        return -(-n // bs)

    def to_numpy(self) -> np.ndarray:
        n = self.n
        out = np.empty((n, n))
        _check(_lib.spamm_mat_to_dense(self.ctx.handle, self.handle, out.ctypes.data, n, 0),
               "spamm_mat_to_dense")
        return out

    def to_torch(self, device="cuda"):
        import torch
        n = self.n
        out = torch.empty((n, n), dtype=torch.float64, device=device)
        self.ctx.sync_torch()
        _check(_lib.spamm_mat_to_dense(self.ctx.handle, self.handle, out.data_ptr(), n, 1),
               "spamm_mat_to_dense")
        return out

    def to_blocks(self, out=None):
        """The stored leaf blocks, row-major: (brow, bcol, tiles) with tiles of shape
        (nnzb, bs, bs) (the inverse of Context.from_blocks). `out` (optional): a host
        buffer (numpy array or CPU torch tensor, ideally pinned) of at least
        nnzb * bs * bs float64 to write the tiles into; the returned tiles then view it."""
        n, bs, nnzb = self.info()
        brow = np.empty(nnzb, dtype=np.int32)
        bcol = np.empty(nnzb, dtype=np.int32)
        if out is None:
            tiles = np.empty((nnzb, bs, bs))
            ptr = tiles.ctypes.data
        else:
            size = out.numel() if _is_torch(out) else out.size
            if size < nnzb * bs * bs:
                raise ValueError(f"to_blocks: buffer of {size} entries, {nnzb * bs * bs} needed")
            ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
            tiles = (out.reshape(-1)[: nnzb * bs * bs].reshape(nnzb, bs, bs))
        _check(_lib.spamm_mat_to_blocks(self.ctx.handle, self.handle,
                                        brow.ctypes.data_as(_PI32), bcol.ctypes.data_as(_PI32),
                                        ptr, 0), "spamm_mat_to_blocks")
        return brow, bcol, tiles

    def get_blocks(self, brow, bcol):
        """Selected leaf blocks (bs x bs each, zeros where absent) and a flag per block
        saying whether it is stored."""
        brow = np.ascontiguousarray(brow, dtype=np.int32)
        bcol = np.ascontiguousarray(bcol, dtype=np.int32)
        count = len(brow)
        bs = self.bs
        tiles = np.empty((count, bs, bs))
        present = np.empty(count, dtype=np.int32)
        _check(_lib.spamm_mat_get_blocks(self.ctx.handle, self.handle, count,
                                         brow.ctypes.data_as(_PI32), bcol.ctypes.data_as(_PI32),
                                         tiles.ctypes.data, present.ctypes.data_as(_PI32)),
               "spamm_mat_get_blocks")
        return tiles, present.astype(bool)

    def to_host(self, out):
        """Write densely into a host buffer (numpy array or CPU torch tensor,
        ideally pinned), n x n float64 C-contiguous."""
        n = self.n
        ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
        assert tuple(out.shape) == (n, n)
        _check(_lib.spamm_mat_to_dense(self.ctx.handle, self.handle, ptr, n, 0),
               "spamm_mat_to_dense")
        return out

    def block_norms(self) -> np.ndarray:
        nb = self.nb
        out = np.empty((nb, nb))
        _check(_lib.spamm_mat_block_norms(self.ctx.handle, self.handle,
                                          out.ctypes.data_as(_PD)), "spamm_mat_block_norms")
        return out

    def block_map(self) -> np.ndarray:
        nb = self.nb
        out = np.empty((nb, nb), dtype=np.int32)
        _check(_lib.spamm_mat_block_map(self.ctx.handle, self.handle,
                                        out.ctypes.data_as(_PI32)), "spamm_mat_block_map")
        return out.astype(bool)


class Context:
    """Owns a spamm_ctx: device, CUDA stream, tau table and device scalars."""

    def __init__(self, device: int = 0, stream=None):
        load_library()
        h = ctypes.c_void_p()
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.stream = stream
        _check(_lib.spamm_create(ctypes.byref(h), device, sptr), "spamm_create")
        self.handle = h
        self.device = device

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.spamm_destroy(h)
            self.handle = None

    def supports(self, prec="mixed", bs: int = 64) -> bool:
        return bool(_lib.spamm_prec_supported(self.handle, _PREC[prec], bs))

    def launches(self) -> int:
        """Kernels launched through this context so far."""
        return int(_lib.spamm_ctx_launches(self.handle))

    def sync_torch(self):
        """Order the library's stream after torch work on the current stream."""
        try:
            import torch
            if torch.cuda.is_available() and self.stream is None:
                torch.cuda.current_stream(self.device).synchronize()
        except ImportError:
            pass

    # ------------------------------------------------------------ matrices
    def from_dense(self, a, bs: int = 64, drop: float = 0.0) -> Matrix:
        out = ctypes.c_void_p()
        if _is_torch(a):
            import torch
            assert a.dtype == torch.float64 and a.dim() == 2 and a.shape[0] == a.shape[1]
            a = a.contiguous()
            if a.is_cuda:
                self.sync_torch()
                st = _lib.spamm_mat_from_dense(self.handle, ctypes.c_void_p(a.data_ptr()), a.shape[0],
                                               a.stride(0), bs, drop, 1, ctypes.byref(out))
            else:
                a = a.numpy()
                st = _lib.spamm_mat_from_dense(self.handle, a.ctypes.data, a.shape[0], a.shape[0],
                                               bs, drop, 0, ctypes.byref(out))
        else:
            a = np.ascontiguousarray(a, dtype=np.float64)
            assert a.ndim == 2 and a.shape[0] == a.shape[1]
            st = _lib.spamm_mat_from_dense(self.handle, a.ctypes.data, a.shape[0], a.shape[0], bs,
                                           drop, 0, ctypes.byref(out))
        _check(st, "spamm_mat_from_dense")
        return Matrix(self, out.value)

    # ----------------------------------------------------------- operations
    def cse(self, A: Matrix, B: Matrix, taus=None) -> np.ndarray:
        taus = tau_table() if taus is None else np.ascontiguousarray(taus, dtype=np.float64)
        err = np.empty(len(taus))
        _check(_lib.spamm_cse(self.handle, A.handle, B.handle, taus.ctypes.data_as(_PD), len(taus),
                              err.ctypes.data_as(_PD)), "spamm_cse")
        return err

    def multiply(self, A: Matrix, B: Matrix, delta: float, prec="fp64"):
        out, rep = ctypes.c_void_p(), Report()
        _check(_lib.spamm_multiply(self.handle, A.handle, B.handle, float(delta), _PREC[prec],
                                   ctypes.byref(out), ctypes.byref(rep)), "spamm_multiply")
        return Matrix(self, out.value), rep.as_dict()

    def multiply_tau(self, A: Matrix, B: Matrix, tau: float, prec="fp64"):
        out, rep = ctypes.c_void_p(), Report()
        _check(_lib.spamm_multiply_tau(self.handle, A.handle, B.handle, float(tau), _PREC[prec],
                                       ctypes.byref(out), ctypes.byref(rep)), "spamm_multiply_tau")
        return Matrix(self, out.value), rep.as_dict()

    def sp2_step(self, X: Matrix, branch: int, delta: float = 0.0, tau: float = 0.0, prec="fp64"):
        out, rep = ctypes.c_void_p(), Report()
        _check(_lib.spamm_sp2_step(self.handle, X.handle, int(branch), float(delta), float(tau),
                                   _PREC[prec], ctypes.byref(out), ctypes.byref(rep)),
               "spamm_sp2_step")
        return Matrix(self, out.value), rep.as_dict()

    def truncate(self, X: Matrix, delta: float, symmetric: bool = True):
        rep = Report()
        _check(_lib.spamm_truncate(self.handle, X.handle, float(delta), int(bool(symmetric)),
                                   ctypes.byref(rep)), "spamm_truncate")
        return rep.as_dict()

    def purify(self, F: Matrix, n_occ: int, eps: float, n_iter: int, homo: float, lumo: float,
               variant: int = HYBRID, prec="fp64", lmin=None, lmax=None, strict: bool = True):
        opts = PurifyOpts(variant, _PREC[prec], float(homo), float(lumo),
                          int(lmin is not None and lmax is not None),
                          float(lmin or 0.0), float(lmax or 0.0))
        logs = {k: np.zeros(n_iter) for k in ("delta", "tau", "trace", "idem")}
        br = np.zeros(n_iter, dtype=np.int32)
        nz = np.zeros(n_iter, dtype=np.int64)
        lm = np.zeros(n_iter, dtype=np.int32)
        sms = np.zeros(n_iter, dtype=np.float32)
        rep = PurifyReport()
        rep.step_delta = logs["delta"].ctypes.data_as(_PD)
        rep.step_tau = logs["tau"].ctypes.data_as(_PD)
        rep.step_trace = logs["trace"].ctypes.data_as(_PD)
        rep.step_idem = logs["idem"].ctypes.data_as(_PD)
        rep.step_branch = br.ctypes.data_as(_PI32)
        rep.step_nnzb = nz.ctypes.data_as(_PI64)
        rep.step_lmax = lm.ctypes.data_as(_PI32)
        rep.step_ms = sms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        out = ctypes.c_void_p()
        st = _lib.spamm_purify(self.handle, F.handle, int(n_occ), float(eps), int(n_iter),
                               ctypes.byref(opts), ctypes.byref(out), ctypes.byref(rep))
        _check(st, "spamm_purify", allow=() if strict else (5,))
        it = rep.iters
        r = {"iters": it, "converged": bool(rep.converged), "idem": rep.idem, "trace": rep.trace,
             "lmin": rep.lmin, "lmax": rep.lmax, "kept_total": rep.kept_total,
             "formed_total": rep.formed_total, "pipe_flops_total": rep.pipe_flops_total,
             "cand_total": rep.cand_total, "ms_total": rep.ms_total,
             "ms_phase": list(rep.ms_phase), "status": st,
             "deltas": logs["delta"][:it].tolist(), "taus": logs["tau"][:it].tolist(),
             "traces": logs["trace"][:it].tolist(), "idems": logs["idem"][:it].tolist(),
             "branches": br[:it].tolist(), "nnzb": nz[:it].tolist(),
             "step_lmax": lm[:it].tolist(), "step_ms": sms[:it].tolist()}
        return Matrix(self, out.value), r

    def purify_batched(self, Fs, n_occ, eps: float, n_iter: int, homo, lumo, variant: int = HYBRID,
                       prec="fp64", workers: int = 8):
        """Purify independent problems concurrently (see spamm_purify_batched)."""
        count = len(Fs)
        FA = (ctypes.c_void_p * count)(*[F.handle.value for F in Fs])
        NO = (ctypes.c_int64 * count)(*[int(x) for x in n_occ])
        OP = (PurifyOpts * count)(*[PurifyOpts(variant, _PREC[prec], float(h), float(l), 0, 0.0, 0.0)
                                    for h, l in zip(homo, lumo)])
        DA = (ctypes.c_void_p * count)()
        RE = (PurifyReport * count)()
        ST = (ctypes.c_int32 * count)()
        st = _lib.spamm_purify_batched(self.handle, count, FA, NO, float(eps), int(n_iter), OP,
                                       int(workers), DA, RE, ST)
        _check(st, "spamm_purify_batched", allow=(5,))
        out = []
        for i in range(count):
            r = RE[i]
            out.append((Matrix(self, DA[i]), {"iters": r.iters, "converged": bool(r.converged),
                                              "status": int(ST[i]), "idem": r.idem,
                                              "trace": r.trace, "ms_total": r.ms_total,
                                              "kept_total": r.kept_total}))
        return out

    def autotune(self, X: Matrix, delta: float, allow_mixed: bool = True):
        """Fastest leaf size / arithmetic for X (see spamm_autotune)."""
        r = TuneResult()
        _check(_lib.spamm_autotune(self.handle, X.handle, float(delta), int(bool(allow_mixed)),
                                   ctypes.byref(r)), "spamm_autotune")
        return {"bs": r.bs, "prec": "mixed" if r.prec == MIXED else "fp64",
                "ms": {"fp64_bs32": r.ms[0], "fp64_bs64": r.ms[1], "fp64_bs128": r.ms[2],
                       "mixed_bs64": r.ms[3]}, "cached": bool(r.cached)}

    def set_bound(self, bound: str = "alg3"):
        """Bound for later searches on this context: "alg3" (Algorithm 3), "flat" (one
        level) or "spectral" (certifies the spectral norm of the error)."""
        _check(_lib.spamm_set_bound(self.handle, {"alg3": 0, "flat": 1, "spectral": 2}[bound]),
               "spamm_set_bound")

    def set_tau_table(self, start: float = 1.0, ratio: float = 0.9):
        """tau candidates tau_1 = start, tau_i = ratio tau_{i-1} for later searches."""
        _check(_lib.spamm_set_tau_table(self.handle, float(start), float(ratio)),
               "spamm_set_tau_table")

    def from_blocks(self, n: int, bs: int, brow, bcol, tiles) -> Matrix:
        """Matrix from a list of leaf blocks: tiles[t] (bs x bs) at block (brow[t], bcol[t]).
        tiles: numpy array (host) or CUDA torch tensor (device), float64, contiguous."""
        brow = np.ascontiguousarray(brow, dtype=np.int32)
        bcol = np.ascontiguousarray(bcol, dtype=np.int32)
        out = ctypes.c_void_p()
        if _is_torch(tiles):
            ptr, on_dev, keep = ctypes.c_void_p(tiles.data_ptr()), int(tiles.is_cuda), tiles
        else:
            keep = np.ascontiguousarray(tiles, dtype=np.float64)
            ptr, on_dev = keep.ctypes.data_as(ctypes.c_void_p), 0
        _check(_lib.spamm_mat_from_blocks(self.handle, int(n), int(bs), len(brow),
                                          brow.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          bcol.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          ptr, on_dev, ctypes.byref(out)), "spamm_mat_from_blocks")
        del keep
        return Matrix(self, out.value)
