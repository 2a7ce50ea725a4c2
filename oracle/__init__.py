"""ORACLE -- test infrastructure only.

A plain, slow, FP64 scalar-CSR smoothed-aggregation AMG + PCG written in C
(``sa_amg_oracle.c``) from the paper's Alg. 1 (setup), Alg. 2 (V-cycle) and
Sec. 4 (CG, relative residual 1e-8).  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA path and never imports it.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against what
the paper and the mathematics fix (worked example of Sec. 2, rigid-body
annihilation, orthonormality, Galerkin symmetry, dense direct solves, ...).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sa_amg_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

P = ctypes.c_void_p
i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, no FMA contraction) into an in-tree library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("eps_strong", ctypes.c_double), ("coarse_enough", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("npre", ctypes.c_int),
                ("npost", ctypes.c_int), ("relax", ctypes.c_double),
                ("smooth_relax", ctypes.c_double), ("ns", ctypes.c_int),
                ("smoother", ctypes.c_int), ("ilu_sweeps", ctypes.c_int),
                ("aggregation", ctypes.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i = ctypes.c_double, ctypes.c_int
    sig = {
        "orc_csr_free": ([P], None),
        "orc_csr_shape": ([P, P], None),
        "orc_csr_copy": ([P, P, P, P], None),
        "orc_csr_from": ([i64, i64, P, P, P], P),
        "orc_unblock": ([i64, i64, i, i, P, P, P], P),
        "orc_spmv": ([P, P, P], None),
        "orc_graph_free": ([P], None),
        "orc_graph_shape": ([P, P], None),
        "orc_graph_copy": ([P, P, P, P, P], None),
        "orc_strength": ([P, i, d], P),
        "orc_aggregate": ([P, P], i64),
        "orc_aggregate_mis2": ([P, P], i64),
        "orc_fmix32": ([ctypes.c_uint32], ctypes.c_uint32),
        "orc_tentative": ([i64, i, P, i64, P, i, P], P),
        "orc_jacobi_rho": ([P, P, P], None),
        "orc_spgemm": ([P, P], P),
        "orc_transpose": ([P], P),
        "orc_smooth_prolongation": ([P, P, d, P], P),
        "orc_spai0": ([P, P], None),
        "orc_cholesky": ([i64, P, P], i),
        "orc_cholesky_solve": ([i64, P, P, P, P], None),
        "orc_params_default": ([P], None),
        "orc_setup": ([P, i, P, P, P], P),
        "orc_ilu0": ([P, i], P),
        "orc_ilu_apply": ([P, i, P, P, P], None),
        "orc_ilu_shape": ([P, P], None),
        "orc_ilu_copy": ([P, P, P, P, P], None),
        "orc_ilu_free": ([P], None),
        "orc_free": ([P], None),
        "orc_vcycle": ([P, P, P], None),
        "orc_pcg": ([P, P, P, d, i, P], i),
        "orc_nlevels": ([P], i),
        "orc_level_info": ([P, i, P, P], None),
        "orc_level_matrix": ([P, i, i], P),
        "orc_level_graph": ([P, i], P),
        "orc_level_vectors": ([P, i, P, P, P, P], None),
        "orc_coarse_factor": ([P, P, P], None),
        "orc_set_block_smoother": ([P, i, P], i),
        "orc_level_blocks": ([P, i, P], i),
        "orc_block_jacobi": ([P, i, ctypes.c_double, P], i),
        "orc_block_jacobi_lambda": ([P, i, P, i], ctypes.c_double),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(P)


class CSR:
    """Scalar CSR owned by numpy arrays (int64 ptr, int32 col, float64 val)."""

    def __init__(self, ptr, col, val, shape):
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.shape = (int(shape[0]), int(shape[1]))

    @property
    def nnz(self):
        return int(self.col.shape[0])

    def to_dense(self):
        D = np.zeros(self.shape)
        rows = np.repeat(np.arange(self.shape[0]), np.diff(self.ptr))
        np.add.at(D, (rows, self.col), self.val)
        return D

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.ptr), shape=self.shape)

    # --- marshalling to and from the C side -----------------------------
    def _handle(self):
        return _load().orc_csr_from(self.shape[0], self.shape[1], _p(self.ptr), _p(self.col),
                                    _p(self.val))

    @staticmethod
    def _from_handle(h, free=True):
        lib = _load()
        s = np.zeros(3, dtype=np.int64)
        lib.orc_csr_shape(h, _p(s))
        ptr = np.empty(s[0] + 1, dtype=np.int64)
        col = np.empty(s[2], dtype=np.int32)
        val = np.empty(s[2])
        lib.orc_csr_copy(h, _p(ptr), _p(col), _p(val))
        if free:
            lib.orc_csr_free(h)
        return CSR(ptr, col, val, (s[0], s[1]))


class _Owned:
    """A CSR handle on the C side, freed with the Python object."""

    def __init__(self, csr: CSR):
        self.h = csr._handle()

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_csr_free(self.h)
            self.h = None


def unblock(row_ptr, col, val, br, bc, nbcols=None) -> CSR:
    """Block CSR (BSR, blocks br x bc row-major) -> scalar CSR (Sec. 2)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    nbr = row_ptr.shape[0] - 1
    if nbcols is None:
        nbcols = nbr
    h = _load().orc_unblock(nbr, nbcols, br, bc, _p(row_ptr), _p(col), _p(val))
    return CSR._from_handle(h)


def spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.shape[0])
    o = _Owned(A)
    _load().orc_spmv(o.h, _p(x), _p(y))
    return y


def strength(A: CSR, b: int, eps: float):
    """Node graph with squared block norms and strong flags."""
    lib = _load()
    o = _Owned(A)
    g = lib.orc_strength(o.h, b, eps)
    s = np.zeros(2, dtype=np.int64)
    lib.orc_graph_shape(g, _p(s))
    ptr = np.empty(s[0] + 1, dtype=np.int64)
    col = np.empty(s[1], dtype=np.int32)
    nrm = np.empty(s[1])
    strong = np.empty(s[1], dtype=np.uint8)
    lib.orc_graph_copy(g, _p(ptr), _p(col), _p(nrm), _p(strong))
    lib.orc_graph_free(g)
    return {"ptr": ptr, "col": col, "norm2": nrm, "strong": strong}


def aggregate(A: CSR, b: int, eps: float):
    """Strength + three-pass aggregation; returns (agg, nagg)."""
    lib = _load()
    o = _Owned(A)
    g = lib.orc_strength(o.h, b, eps)
    s = np.zeros(2, dtype=np.int64)
    lib.orc_graph_shape(g, _p(s))
    agg = np.empty(s[0], dtype=np.int32)
    nagg = lib.orc_aggregate(g, _p(agg))
    lib.orc_graph_free(g)
    return agg, int(nagg)


def aggregate_mis2(A: CSR, b: int, eps: float):
    """Strength + MIS-2 aggregation (greedy distance-2 independent set in
    descending fmix32 priority on the undirected strong graph); returns
    (agg, nagg)."""
    lib = _load()
    o = _Owned(A)
    g = lib.orc_strength(o.h, b, eps)
    s = np.zeros(2, dtype=np.int64)
    lib.orc_graph_shape(g, _p(s))
    agg = np.empty(s[0], dtype=np.int32)
    nagg = lib.orc_aggregate_mis2(g, _p(agg))
    lib.orc_graph_free(g)
    if nagg < 0:
        raise RuntimeError("MIS-2 aggregation: roots are not a maximal distance-2 set")
    return agg, int(nagg)


def fmix32(x: int) -> int:
    """MurmurHash3's 32-bit finaliser, the MIS-2 node priority."""
    return int(_load().orc_fmix32(x & 0xFFFFFFFF))


def tentative(nnodes: int, b: int, agg: np.ndarray, nagg: int, B: np.ndarray):
    """(P_tent, B_c) from the aggregates and the near-nullspace."""
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.float64)
    ns = B.shape[1]
    Bc = np.empty((nagg * ns, ns))
    h = _load().orc_tentative(nnodes, b, _p(agg), nagg, _p(B), ns, _p(Bc))
    return CSR._from_handle(h), Bc


def jacobi_rho(A: CSR):
    """(d, rho): diagonal of A and the Gershgorin bound of rho(D^-1 A)."""
    o = _Owned(A)
    d = np.empty(A.shape[0])
    rho = np.zeros(1)
    _load().orc_jacobi_rho(o.h, _p(d), _p(rho))
    return d, float(rho[0])


def spgemm(A: CSR, B: CSR) -> CSR:
    oa, ob = _Owned(A), _Owned(B)
    return CSR._from_handle(_load().orc_spgemm(oa.h, ob.h))


def transpose(A: CSR) -> CSR:
    o = _Owned(A)
    return CSR._from_handle(_load().orc_transpose(o.h))


def smooth_prolongation(A: CSR, d: np.ndarray, omega: float, Pt: CSR) -> CSR:
    oa, op = _Owned(A), _Owned(Pt)
    d = np.ascontiguousarray(d, dtype=np.float64)
    return CSR._from_handle(_load().orc_smooth_prolongation(oa.h, _p(d), omega, op.h))


def spai0(A: CSR) -> np.ndarray:
    o = _Owned(A)
    m = np.empty(A.shape[0])
    _load().orc_spai0(o.h, _p(m))
    return m


def block_jacobi(A: CSR, b: int, w: float = 2.0 / 3.0) -> np.ndarray:
    """Block damped Jacobi blocks M_I = w A_II^{-1} (zero rows and columns of
    A_II left out), [n / b, b, b]; raises on a non-positive pivot."""
    o = _Owned(A)
    Mb = np.empty((A.shape[0] // b, b, b))
    rc = _load().orc_block_jacobi(o.h, b, w, _p(Mb))
    if rc != 0:
        raise ValueError(f"non-positive pivot in node block {-rc - 1}")
    return Mb


def block_jacobi_lambda(A: CSR, b: int, W: np.ndarray, iters: int = 20) -> float:
    """Rayleigh-quotient estimate of lambda_max(D_b^{-1} A) after `iters`
    power iterations from the hashed start vector; W = block_jacobi(A, b, 1)."""
    o = _Owned(A)
    W = np.ascontiguousarray(W, dtype=np.float64)
    return float(_load().orc_block_jacobi_lambda(o.h, b, _p(W), iters))


def cholesky(Adense: np.ndarray):
    """(L, zero_row, status) of the dense Cholesky with the zero-row rule."""
    L = np.ascontiguousarray(Adense, dtype=np.float64).copy()
    n = L.shape[0]
    z = np.zeros(n, dtype=np.uint8)
    rc = _load().orc_cholesky(n, _p(L), _p(z))
    return L, z, rc


def cholesky_solve(L, zrow, f):
    n = L.shape[0]
    u = np.empty(n)
    f = np.ascontiguousarray(f, dtype=np.float64)
    _load().orc_cholesky_solve(n, _p(L), _p(zrow), _p(f), _p(u))
    return u


class ILU0:
    """Block ILU(0) of a scalar CSR matrix in b x b blocks (the level smoother
    of Sec. 4's experiments); apply() solves with `sweeps` Jacobi sweeps per
    triangular factor."""

    def __init__(self, A: CSR, b: int):
        self._A = _Owned(A)
        self.h = _load().orc_ilu0(self._A.h, b)
        if not self.h:
            raise RuntimeError("block ILU(0) breakdown")
        sh = np.zeros(3, dtype=np.int64)
        _load().orc_ilu_shape(self.h, _p(sh))
        self.nb, self.b, self.nnzb = (int(x) for x in sh)

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_ilu_free(self.h)
            self.h = None

    def factors(self):
        """(ptr, col, val [nnzb, b, b], dinv [nb, b, b]): L strictly below and
        U on and above the block diagonal; dinv = U_II^-1."""
        ptr = np.empty(self.nb + 1, dtype=np.int64)
        col = np.empty(max(self.nnzb, 1), dtype=np.int32)
        val = np.empty((max(self.nnzb, 1), self.b, self.b))
        dinv = np.empty((self.nb, self.b, self.b))
        _load().orc_ilu_copy(self.h, _p(ptr), _p(col), _p(val), _p(dinv))
        return ptr, col[:self.nnzb], val[:self.nnzb], dinv

    def apply(self, r: np.ndarray, sweeps: int) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.empty_like(r)
        work = np.empty(2 * len(r))
        _load().orc_ilu_apply(self.h, sweeps, _p(r), _p(out), _p(work))
        return out


class Hierarchy:
    """Alg. 1 on a scalar CSR matrix; V-cycle (Alg. 2) and PCG on top."""

    def __init__(self, A: CSR, bs: int, B: np.ndarray, *, eps_strong=0.08, coarse_enough=3000,
                 max_levels=15, npre=1, npost=1, relax=2.0, smooth_relax=0.8, smoother="spai0",
                 ilu_sweeps=2, aggregation="greedy"):
        lib = _load()
        B = np.ascontiguousarray(B, dtype=np.float64)
        self.ns = B.shape[1]
        prm = _Params(eps_strong, coarse_enough, max_levels, npre, npost, relax, smooth_relax,
                      self.ns, {"spai0": 0, "ilu0": 1, "bjacobi": 2}[smoother], ilu_sweeps,
                      {"greedy": 0, "mis2": 1}[aggregation])
        self._A = _Owned(A)
        st = ctypes.c_int(0)
        self.h = lib.orc_setup(self._A.h, bs, _p(B), ctypes.byref(prm), ctypes.byref(st))
        if not self.h:
            raise RuntimeError(f"oracle setup failed with status {st.value}")

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_free(self.h)
            self.h = None

    @property
    def nlevels(self) -> int:
        return _load().orc_nlevels(self.h)

    def level(self, l: int) -> dict:
        lib = _load()
        info = np.zeros(5, dtype=np.int64)
        sc = np.zeros(4)
        lib.orc_level_info(self.h, l, _p(info), _p(sc))
        n, b, nagg, hasP = (int(x) for x in info[:4])
        out = {"n": n, "b": b, "nagg": nagg, "eps": sc[0], "omega": sc[1], "rho": sc[2],
               "bj_lambda": sc[3]}
        out["A"] = CSR._from_handle(lib.orc_level_matrix(self.h, l, 0), free=False)
        agg = np.empty(n // b, dtype=np.int32) if hasP else None
        M = np.empty(n) if hasP else None
        B = np.empty((n, self.ns))
        d = np.empty(n) if hasP else None
        lib.orc_level_vectors(self.h, l, _p(agg), _p(M), _p(B), _p(d))
        out.update(agg=agg, M=M, B=B, d=d)
        Mb = np.empty((n // b, b, b)) if hasP else None
        if Mb is not None and lib.orc_level_blocks(self.h, l, _p(Mb)) != 0:
            Mb = None
        out["Mb"] = Mb
        if hasP:
            out["P"] = CSR._from_handle(lib.orc_level_matrix(self.h, l, 1), free=False)
            out["R"] = CSR._from_handle(lib.orc_level_matrix(self.h, l, 2), free=False)
        return out

    def graph(self, l: int):
        """Strength graph of level l (None on the coarsest level)."""
        lib = _load()
        g = lib.orc_level_graph(self.h, l)
        if not g:
            return None
        s = np.zeros(2, dtype=np.int64)
        lib.orc_graph_shape(g, _p(s))
        ptr = np.empty(s[0] + 1, dtype=np.int64)
        col = np.empty(s[1], dtype=np.int32)
        nrm = np.empty(s[1])
        strong = np.empty(s[1], dtype=np.uint8)
        lib.orc_graph_copy(g, _p(ptr), _p(col), _p(nrm), _p(strong))
        return {"ptr": ptr, "col": col, "norm2": nrm, "strong": strong}

    def set_block_smoother(self, l: int, Mb: np.ndarray):
        """Use symmetric 3x3 blocks [N, 3, 3] as the smoother of level l."""
        Mb = np.ascontiguousarray(Mb, dtype=np.float64)
        if _load().orc_set_block_smoother(self.h, l, _p(Mb)) != 0:
            raise ValueError("level has no 3x3 smoother")

    def coarse_factor(self):
        nc = self.level(self.nlevels - 1)["n"]
        L = np.empty((nc, nc))
        z = np.empty(nc, dtype=np.uint8)
        _load().orc_coarse_factor(self.h, _p(L), _p(z))
        return L, z

    def vcycle(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        u = np.empty_like(f)
        _load().orc_vcycle(self.h, _p(f), _p(u))
        return u

    def solve(self, f: np.ndarray, u0=None, tol=1e-8, maxiter=500):
        """(u, iterations, final true relative residual)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        u = np.zeros_like(f) if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).copy()
        rel = np.zeros(1)
        it = _load().orc_pcg(self.h, _p(f), _p(u), tol, maxiter, _p(rel))
        if it < 0:
            raise RuntimeError("oracle CG breakdown")
        return u, it, float(rel[0])


def from_problem(p) -> CSR:
    """Scalar CSR view of a q1elasticity Problem (unblocked 3x3 BSR)."""
    return unblock(p.row_ptr, p.col, p.val.reshape(-1, 9), 3, 3)
