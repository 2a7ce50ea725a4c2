"""Block smoothed-aggregation AMG + PCG for 3D elasticity on GB300 (sm_103a).

Thin ctypes binding of the C ABI declared in ``include/amg_gb300.h``.  It only
marshals arguments: every step of setup and solve runs in the library's CUDA
kernels.  PyTorch supplies device memory (its caching allocator, passed to the
library as an ``amg_allocator``, holds every hierarchy buffer) and the current
CUDA stream.  There is no CPU fallback: without the compiled library every
call raises.

Method: Demidov (2022), Alg. 1 (setup), Alg. 2 (V-cycle), Sec. 3 (block
arithmetic with rigid-body modes), Sec. 4 (CG, relative residual 1e-8).
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

AMG_OK, AMG_NOT_CONVERGED = 0, 1
AMG_ERR_ARG, AMG_ERR_CUDA, AMG_ERR_BREAKDOWN, AMG_ERR_COARSE, AMG_ERR_LIMIT, AMG_ERR_STATE = \
    -1, -2, -3, -4, -5, -6
_ERRORS = {-1: "bad argument", -2: "CUDA error", -3: "CG breakdown",
           -4: "coarsest matrix not positive definite", -5: "size limit", -6: "bad state"}
PREC_FP64, PREC_FP32, PREC_BF16, PREC_DF64 = 0, 1, 2, 3
STORAGE_BLOCK, STORAGE_SCALAR = 0, 1
AGG_GREEDY, AGG_MIS2 = 0, 1
SMOOTH_SPAI0, SMOOTH_ILU0, SMOOTH_BJACOBI = 0, 1, 2
SETUP_BLOCK, SETUP_SCALAR = 0, 1


class AmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_ERRORS.get(status, status)} ({status}): {msg}")
        self.status = status


class Bsr(ctypes.Structure):
    _fields_ = [("nbrows", ctypes.c_int32), ("nbcols", ctypes.c_int32),
                ("bs_r", ctypes.c_int32), ("bs_c", ctypes.c_int32), ("nnzb", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                            ctypes.c_void_p)


class Allocator(ctypes.Structure):
    """amg_allocator: the device memory supplier of a hierarchy."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("eps_strong", ctypes.c_double), ("relax", ctypes.c_double),
                ("smooth_relax", ctypes.c_double), ("coarse_enough", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("npre", ctypes.c_int32),
                ("npost", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("aggregation", ctypes.c_int32), ("smoother", ctypes.c_int32),
                ("ilu_sweeps", ctypes.c_int32), ("setup", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("allocator", ctypes.c_void_p)]


def _torch_alloc(ctx, nbytes, stream):
    import torch
    try:
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
    except Exception:  # the library reports the failure (NULL) as an error status
        return None


def _torch_free(ctx, ptr, nbytes, stream):
    if sys.is_finalizing():  # the process is ending: its memory goes with it
        return
    import torch
    torch.cuda.caching_allocator_delete(int(ptr))


def _finalizing() -> bool:
    """Handles still alive while the interpreter shuts down are not freed
    through the library: the allocator callbacks can no longer run Python,
    and the process exit returns the device memory anyway."""
    return sys.is_finalizing()


_TORCH_ALLOCATOR = None


def torch_allocator() -> Allocator:
    """PyTorch's CUDA caching allocator as an amg_allocator: the hierarchy's
    buffers then count in torch.cuda.memory_allocated() and obey its limits.
    The struct and its callbacks live for the whole process."""
    global _TORCH_ALLOCATOR
    if _TORCH_ALLOCATOR is None:
        _TORCH_ALLOCATOR = Allocator(_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free), None)
    return _TORCH_ALLOCATOR


def _with_allocator(params: Params, allocator) -> Params:
    """allocator: "torch" (PyTorch's caching allocator), None (the library's
    own cudaMallocAsync) or an Allocator the caller keeps alive."""
    if allocator == "torch":
        allocator = torch_allocator()
    params.allocator = None if allocator is None else ctypes.addressof(allocator)
    return params


class LevelDesc(ctypes.Structure):
    _fields_ = [("nbrows", ctypes.c_int32), ("bs", ctypes.c_int32), ("nnzb_A", ctypes.c_int64),
                ("nnzb_P", ctypes.c_int64), ("nagg", ctypes.c_int32),
                ("is_coarsest", ctypes.c_int32), ("eps", ctypes.c_double),
                ("omega", ctypes.c_double), ("rho", ctypes.c_double),
                ("smoother_lambda", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int32), ("coarse_n", ctypes.c_int32),
                ("setup_seconds", ctypes.c_double), ("bytes_matrices", ctypes.c_int64),
                ("bytes_total", ctypes.c_int64), ("operator_complexity", ctypes.c_double),
                ("learned", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("learned_lambda", ctypes.c_double), ("spai0_lambda", ctypes.c_double),
                ("bytes_solve", ctypes.c_int64), ("setup_phase_seconds", ctypes.c_double * 7)]

SETUP_PHASES = ("input", "strength_aggregation", "transfer", "galerkin", "smoothers", "coarse",
                "solve_copies")


class BatchDesc(ctypes.Structure):
    _fields_ = [("ninst", ctypes.c_int32), ("nrhs_total", ctypes.c_int32),
                ("nlevels", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("setup_seconds", ctypes.c_double), ("dofs_total", ctypes.c_int64),
                ("bytes_total", ctypes.c_int64), ("rhs_tile", ctypes.c_int32 * 48),
                ("cta_threads", ctypes.c_int32 * 48), ("ctas_per_sm", ctypes.c_int32 * 48),
                ("setup_phase_seconds", ctypes.c_double * 4)]


EXPORTED = ["amg_params_default", "amg_setup", "amg_apply_vcycle", "amg_solve", "amg_get_stats",
            "amg_level_info", "amg_level_export", "amg_free", "amg_last_error", "amg_bsr_spmv",
            "amg_bsr_spmv_dot", "amg_kernel_launches", "amg_level_spmv", "amg_level_padding",
            "amg_level_galerkin",
            "amg_batch_setup", "amg_batch_solve", "amg_batch_info", "amg_batch_free",
            "amg_set_learned_smoother", "amg_clear_learned_smoother", "amg_trainer_create",
            "amg_trainer_add_samples", "amg_trainer_add_generated", "amg_trainer_eval",
            "amg_trainer_step", "amg_trainer_params", "amg_trainer_free", "amg_fp64_fma_rate"]

LEARNED_NPARAM = 1222   # W1 [64][12], b1 [64], W2 [6][64], b2 [6]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library missing: {_build.LIB} (run the build)")
    lib = ctypes.CDLL(_build.LIB)
    P, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    sig = {
        "amg_params_default": ([P], ctypes.c_int),
        "amg_setup": ([P, P, i32, P, P, P], ctypes.c_int),
        "amg_apply_vcycle": ([P, P, P, P], ctypes.c_int),
        "amg_solve": ([P, P, P, d, i32, P, P, P], ctypes.c_int),
        "amg_get_stats": ([P, P], ctypes.c_int),
        "amg_level_info": ([P, i32, P], ctypes.c_int),
        "amg_level_export": ([P, i32, i32, P, P, P], ctypes.c_int),
        "amg_free": ([P], None),
        "amg_last_error": ([], ctypes.c_char_p),
        "amg_bsr_spmv": ([P, P, P, P], ctypes.c_int),
        "amg_bsr_spmv_dot": ([P, P, P, P, P], ctypes.c_int),
        "amg_kernel_launches": ([], ctypes.c_int64),
        "amg_level_spmv": ([P, i32, i32, P, P, P], ctypes.c_int),
        "amg_level_padding": ([P, i32, P], ctypes.c_int),
        "amg_level_galerkin": ([P, i32, i32, P, P], ctypes.c_int),
        "amg_batch_setup": ([i32, P, P, P, P, P, P], ctypes.c_int),
        "amg_batch_solve": ([P, P, P, d, i32, P, P, P], ctypes.c_int),
        "amg_batch_info": ([P, P], ctypes.c_int),
        "amg_batch_free": ([P], None),
        "amg_set_learned_smoother": ([P, P, P, P], ctypes.c_int),
        "amg_clear_learned_smoother": ([P], ctypes.c_int),
        "amg_trainer_create": ([P, d, P, P], ctypes.c_int),
        "amg_trainer_add_samples": ([P, P, P, i32, P], ctypes.c_int),
        "amg_trainer_add_generated": ([P, P, i32, ctypes.c_uint64, P], ctypes.c_int),
        "amg_trainer_eval": ([P, P, P, P], ctypes.c_int),
        "amg_trainer_step": ([P, i32, P, P], ctypes.c_int),
        "amg_trainer_params": ([P, P], ctypes.c_int),
        "amg_trainer_free": ([P], None),
        "amg_fp64_fma_rate": ([P, ctypes.c_int64, i32, P, P, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status, allow_not_converged=False):
    if status == AMG_OK or (allow_not_converged and status == AMG_NOT_CONVERGED):
        return status
    msg = load().amg_last_error()
    raise AmgError(status, msg.decode() if msg else "")


def _stream(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dptr(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def make_bsr(row_ptr, col, val, nbcols=None) -> Bsr:
    """BSR view of CUDA tensors: int32 row_ptr, int32 col, float64 val [nnzb, br, bc]."""
    import torch
    br, bc = int(val.shape[1]), int(val.shape[2])
    nbr = int(row_ptr.shape[0]) - 1
    return Bsr(nbr, nbr if nbcols is None else int(nbcols), br, bc, int(col.shape[0]),
               _dptr(row_ptr, torch.int32, "row_ptr"), _dptr(col, torch.int32, "col"),
               _dptr(val, torch.float64, "val"))


def default_params(**kw) -> Params:
    p = Params()
    load().amg_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().amg_kernel_launches())


def fp64_fma_rate(iters: int = 20000, stream=None) -> dict:
    """Measured FP64 FMA rate of the current device: {"fma_per_s", "tflops"
    (2 flops per FMA), "seconds" (the timed launch), "num_sms"}."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(2048 * sms, dtype=torch.float64, device="cuda")
    rate, sec, nsm = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int32(0)
    _check(load().amg_fp64_fma_rate(sink.data_ptr(), sink.numel(), int(iters), ctypes.byref(rate),
                                    ctypes.byref(sec), ctypes.byref(nsm), _stream(stream)))
    return {"fma_per_s": rate.value, "tflops": 2.0 * rate.value / 1e12, "seconds": sec.value,
            "num_sms": nsm.value}


def bsr_spmv(row_ptr, col, val, x, y=None, nbcols=None, stream=None):
    """y = A x (block SpMV kernel) on CUDA tensors."""
    import torch
    A = make_bsr(row_ptr, col, val, nbcols)
    if y is None:
        y = torch.empty(A.nbrows * A.bs_r, dtype=torch.float64, device=x.device)
    _check(load().amg_bsr_spmv(ctypes.byref(A), _dptr(x, torch.float64, "x"),
                               _dptr(y, torch.float64, "y"), _stream(stream)))
    return y


def bsr_spmv_dot(row_ptr, col, val, x, y=None, stream=None):
    """(y = A x, x . y) with the deterministic fused reduction."""
    import torch
    A = make_bsr(row_ptr, col, val)
    if y is None:
        y = torch.empty(A.nbrows * A.bs_r, dtype=torch.float64, device=x.device)
    d = ctypes.c_double(0.0)
    _check(load().amg_bsr_spmv_dot(ctypes.byref(A), _dptr(x, torch.float64, "x"),
                                   _dptr(y, torch.float64, "y"), ctypes.byref(d),
                                   _stream(stream)))
    return y, d.value


class AMG:
    """Hierarchy handle: setup (Alg. 1) on construction, V-cycle and PCG solve."""

    def __init__(self, row_ptr, col, val, B, params: Params | None = None, stream=None,
                 allocator="torch", **kw):
        import torch
        self._lib = load()
        self.params = params if params is not None else default_params(**kw)
        _with_allocator(self.params, allocator)
        A = make_bsr(row_ptr, col, val)
        self.n = A.nbrows * A.bs_r
        self.ns = int(B.shape[1])
        self.device = val.device
        h = ctypes.c_void_p()
        _check(self._lib.amg_setup(ctypes.byref(A), _dptr(B, torch.float64, "B"),
                                   int(B.shape[1]), ctypes.byref(self.params),
                                   _stream(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            if not _finalizing():
                self._lib.amg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vcycle(self, r, z=None, stream=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(self._lib.amg_apply_vcycle(self._h, _dptr(r, torch.float64, "r"),
                                          _dptr(z, torch.float64, "z"), _stream(stream)))
        return z

    def solve(self, f, u=None, tol=1e-8, maxiter=1000, stream=None):
        """(u, iterations, relative true residual, status)."""
        import torch
        if u is None:
            u = torch.zeros_like(f)
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0.0)
        st = _check(self._lib.amg_solve(self._h, _dptr(f, torch.float64, "f"),
                                        _dptr(u, torch.float64, "u"), float(tol), int(maxiter),
                                        ctypes.byref(it), ctypes.byref(res), _stream(stream)),
                    allow_not_converged=True)
        return u, it.value, res.value, st

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.amg_get_stats(self._h, ctypes.byref(s)))
        out = {k: getattr(s, k) for k, _ in Stats._fields_}
        out["setup_phase_seconds"] = dict(zip(SETUP_PHASES, list(s.setup_phase_seconds)))
        return out

    def level_info(self, l: int) -> dict:
        d = LevelDesc()
        _check(self._lib.amg_level_info(self._h, l, ctypes.byref(d)))
        return {k: getattr(d, k) for k, _ in LevelDesc._fields_}

    def set_learned_smoother(self, params, stream=None) -> int:
        """Use the network's 3x3 blocks on level 0.  Returns 0, or the reason it
        kept SPAI0: 1 a singular block, 2 lambda_max(M A) >= max(1.9, SPAI0's)."""
        w = np.ascontiguousarray(params, dtype=np.float32)
        if w.size != LEARNED_NPARAM:
            raise ValueError(f"expected {LEARNED_NPARAM} parameters")
        fb = ctypes.c_int32(0)
        _check(self._lib.amg_set_learned_smoother(self._h, w.ctypes.data, ctypes.byref(fb),
                                                  _stream(stream)))
        return int(fb.value)

    def clear_learned_smoother(self):
        _check(self._lib.amg_clear_learned_smoother(self._h))

    def learned_blocks(self) -> np.ndarray:
        info = self.level_info(0)
        out = np.empty((info["nbrows"], 3, 3))
        _check(self._lib.amg_level_export(self._h, 0, 7, None, None, out.ctypes.data))
        return out

    def level_spmv(self, l: int, which: int, x, y, stream=None):
        """y = op x with the solve's own kernel; which = 0 (A), 1 (P), 2 (R);
        3, 4, 5: the same in the FP32-pair copies of a PREC_DF64 hierarchy."""
        import torch
        _check(self._lib.amg_level_spmv(self._h, l, which, _dptr(x, torch.float64, "x"),
                                        _dptr(y, torch.float64, "y"), _stream(stream)))
        return y

    def galerkin_timing(self, l: int, storage: int = STORAGE_BLOCK) -> tuple:
        """(seconds, relative difference) of A_{l+1} = R_l (A_l P_l) recomputed in
        block or scalar storage, against the hierarchy's A_{l+1}."""
        sec, diff = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self._lib.amg_level_galerkin(self._h, l, storage, ctypes.byref(sec),
                                            ctypes.byref(diff)))
        return sec.value, diff.value

    def padding(self, l: int) -> tuple:
        out = (ctypes.c_double * 3)()
        _check(self._lib.amg_level_padding(self._h, l, out))
        return tuple(out)

    @property
    def nlevels(self) -> int:
        return self.stats()["nlevels"]

    def ilu_factor(self, l: int):
        """Host copies of level l's block ILU(0): (factor values on A's block
        pattern [nnzb, b, b], L below and U on/above the diagonal; inverses of
        U's diagonal blocks [nbrows, b, b])."""
        info = self.level_info(l)
        nbr, bs, nnz = info["nbrows"], info["bs"], info["nnzb_A"]
        F = np.empty((max(nnz, 1), bs, bs))
        D = np.empty((max(nbr, 1), bs, bs))
        _check(self._lib.amg_level_export(self._h, l, 8, None, None, F.ctypes.data))
        _check(self._lib.amg_level_export(self._h, l, 9, None, None, D.ctypes.data))
        return F[:nnz], D[:nbr]

    def export(self, l: int) -> dict:
        """Host copies of level l: A, P, R (BSR), aggregates, smoother, B, strength flags."""
        info = self.level_info(l)
        nbr, bs = info["nbrows"], info["bs"]
        out = {"info": info}

        def bsr(which, nrows, nnz, br, bc):
            rp = np.empty(nrows + 1, np.int32)
            cl = np.empty(max(nnz, 1), np.int32)
            vl = np.empty((max(nnz, 1), br, bc))
            _check(self._lib.amg_level_export(self._h, l, which, rp.ctypes.data, cl.ctypes.data,
                                              vl.ctypes.data))
            return rp, cl[:nnz], vl[:nnz]

        out["A"] = bsr(0, nbr, info["nnzb_A"], bs, bs)
        if not info["is_coarsest"]:
            out["P"] = bsr(1, nbr, info["nnzb_P"], bs, self.ns)
            out["R"] = bsr(2, info["nagg"], info["nnzb_P"], self.ns, bs)
            agg = np.empty(nbr, np.int32)
            _check(self._lib.amg_level_export(self._h, l, 3, agg.ctypes.data, None, None))
            out["agg"] = agg
            M = np.empty(nbr * bs)
            _check(self._lib.amg_level_export(self._h, l, 4, None, None, M.ctypes.data))
            out["M"] = M
            if self.params.smoother == SMOOTH_BJACOBI:
                Mb = np.empty((nbr, bs, bs))
                _check(self._lib.amg_level_export(self._h, l, 7, None, None, Mb.ctypes.data))
                out["Mb"] = Mb
            strong = np.empty(max(info["nnzb_A"], 1), np.uint8)
            _check(self._lib.amg_level_export(self._h, l, 6, strong.ctypes.data, None, None))
            out["strong"] = strong[:info["nnzb_A"]]
        B = np.empty((nbr * bs, self.ns))
        _check(self._lib.amg_level_export(self._h, l, 5, None, None, B.ctypes.data))
        out["B"] = B
        return out


class AMGBatch:
    """Batched form: independent instances, each with several right-hand sides,
    one hierarchy per instance and one graph-launched solve for all of them."""

    def __init__(self, mats, Bs, nrhs, params: Params | None = None, stream=None,
                 allocator="torch", **kw):
        import torch
        self._lib = load()
        self.params = params if params is not None else default_params(**kw)
        _with_allocator(self.params, allocator)
        n = len(mats)
        if not (len(Bs) == len(nrhs) == n):
            raise ValueError("mats, Bs and nrhs must have the same length")
        self._keep = [m for m in mats] + list(Bs)
        arr = (Bsr * n)(*[make_bsr(*m) for m in mats])
        bptr = (ctypes.c_void_p * n)(*[_dptr(b, torch.float64, "B") for b in Bs])
        k = (ctypes.c_int32 * n)(*[int(x) for x in nrhs])
        self.nrhs = [int(x) for x in nrhs]
        self.ndof = [int(m[0].shape[0] - 1) * 3 for m in mats]
        h = ctypes.c_void_p()
        _check(self._lib.amg_batch_setup(n, arr, bptr, k, ctypes.byref(self.params),
                                         _stream(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            if not _finalizing():
                self._lib.amg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, F, U=None, tol=1e-8, maxiter=1000, stream=None):
        """F: list of CUDA tensors [nrhs_i, 3 n_i]; returns (U, iters, resid, status)."""
        import torch
        n = len(F)
        if U is None:
            U = [torch.zeros_like(f) for f in F]
        fp = (ctypes.c_void_p * n)(*[_dptr(f, torch.float64, "F") for f in F])
        up = (ctypes.c_void_p * n)(*[_dptr(u, torch.float64, "U") for u in U])
        tot = sum(self.nrhs)
        it = (ctypes.c_int32 * tot)()
        res = (ctypes.c_double * tot)()
        st = _check(self._lib.amg_batch_solve(self._h, fp, up, float(tol), int(maxiter), it, res,
                                              _stream(stream)), allow_not_converged=True)
        out_it, out_res, g = [], [], 0
        for k in self.nrhs:
            out_it.append(list(it[g:g + k]))
            out_res.append(list(res[g:g + k]))
            g += k
        return U, out_it, out_res, st

    def info(self) -> dict:
        d = BatchDesc()
        _check(self._lib.amg_batch_info(self._h, ctypes.byref(d)))
        out = {k: getattr(d, k) for k, _ in BatchDesc._fields_
               if k not in ("rhs_tile", "cta_threads", "ctas_per_sm", "setup_phase_seconds")}
        out["setup_phase_seconds"] = dict(zip(("instances", "operators", "coarse_and_state",
                                               "autotune"), list(d.setup_phase_seconds)))
        out["rhs_tile"] = [[d.rhs_tile[3 * l + j] for j in range(3)] for l in range(d.nlevels)]
        out["cta_threads"] = [[d.cta_threads[3 * l + j] for j in range(3)]
                              for l in range(d.nlevels)]
        out["ctas_per_sm"] = [[d.ctas_per_sm[3 * l + j] for j in range(3)]
                              for l in range(d.nlevels)]
        return out


def learned_init(seed: int = 0, scale: float = 0.3) -> np.ndarray:
    """Initial network: W1 seeded Gaussian / sqrt(12), everything else zero
    (the zero output layer makes the learned smoother equal to SPAI0)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(LEARNED_NPARAM, dtype=np.float32)
    w[:64 * 12] = (scale * rng.standard_normal(64 * 12) / np.sqrt(12)).astype(np.float32)
    return w


class Trainer:
    """Training of the smoother network on the device (own kernels, Adam)."""

    def __init__(self, params, lr=1e-3, stream=None):
        self._lib = load()
        w = np.ascontiguousarray(params, dtype=np.float32)
        t = ctypes.c_void_p()
        _check(self._lib.amg_trainer_create(w.ctypes.data, float(lr), _stream(stream),
                                            ctypes.byref(t)))
        self._t = t
        self._keep = []

    def close(self):
        if getattr(self, "_t", None):
            if not _finalizing():
                self._lib.amg_trainer_free(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_samples(self, solver: "AMG", R, stream=None):
        import torch
        self._keep.append(solver)
        _check(self._lib.amg_trainer_add_samples(self._t, solver._h, _dptr(R, torch.float64, "R"),
                                                 int(R.shape[0]), _stream(stream)))

    def add_generated(self, solver: "AMG", nsamples: int, seed: int = 0, stream=None):
        self._keep.append(solver)
        _check(self._lib.amg_trainer_add_generated(self._t, solver._h, int(nsamples),
                                                   ctypes.c_uint64(seed), _stream(stream)))

    def eval(self, stream=None):
        loss = ctypes.c_double(0.0)
        g = np.empty(LEARNED_NPARAM, dtype=np.float32)
        _check(self._lib.amg_trainer_eval(self._t, ctypes.byref(loss), g.ctypes.data,
                                          _stream(stream)))
        return loss.value, g

    def step(self, nsteps=1, stream=None) -> float:
        loss = ctypes.c_double(0.0)
        _check(self._lib.amg_trainer_step(self._t, int(nsteps), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def params(self) -> np.ndarray:
        w = np.empty(LEARNED_NPARAM, dtype=np.float32)
        _check(self._lib.amg_trainer_params(self._t, w.ctypes.data))
        return w
