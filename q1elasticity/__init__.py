"""Seeded synthetic 3D elasticity inputs (Q1 hexahedra on a box).

This module is the one piece shared by the CUDA path and the oracle: it builds
the linear system ``A u = f`` of the paper's Eq. 1, the six rigid-body modes
``B`` (the near-nullspace matrix of Sec. 2) and the element material field.
It holds none of the multigrid method's arithmetic.

The paper's own matrices (a connecting rod and a solid hook, Sec. 4) are not
available; these boxes stand in for them.  Workloads:

* ``cube(n)``: n^3 elements, E = 1, nu = 0.3, clamped at x = 0, uniform body
  load (0, 0, -1).
* ``inclusions(n)``: n^3 elements, matrix E = 1 with spheres (radius 0.1 of
  the unit cube, SplitMix64 seed 2202) of E = 1000 until 20 % of the elements
  are inside, nu = 0.3, clamped at x = 0, traction (0, 0, -1) on x = 1.
* ``batch(...)``: independent boxes with seeded sizes, Poisson ratios and
  load cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "q1gen.c")
_LIB = os.path.join(_HERE, "_q1gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i, d, u64, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
        lib.q1_element_stiffness.argtypes = [d, d, P]
        lib.q1_inclusions.argtypes = [i, i, i, d, d, d, d, d, u64, P]
        lib.q1_inclusions.restype = i
        lib.q1_pattern.argtypes = [i, i, i, i, P]
        lib.q1_pattern.restype = i64
        lib.q1_assemble.argtypes = [i, i, i, d, d, P, i, P, P, P]
        lib.q1_assemble.restype = i
        lib.q1_rigid_body_modes.argtypes = [i, i, i, d, P, P]
        lib.q1_load.argtypes = [i, i, i, d, P, P, i, P]
        lib.q1_splitmix64.argtypes = [u64, P]
        lib.q1_splitmix64.restype = u64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Problem:
    """One elasticity system as BSR with 3x3 blocks (node-major DOFs)."""
    shape: tuple            # (nx, ny, nz) elements
    h: float
    nu: float
    row_ptr: np.ndarray     # int32 [N+1]
    col: np.ndarray         # int32 [nnzb]
    val: np.ndarray         # float64 [nnzb, 3, 3]
    B: np.ndarray           # float64 [3N, 6] rigid-body modes
    f: np.ndarray           # float64 [3N] or [nrhs, 3N]
    coords: np.ndarray      # float64 [N, 3]
    E_el: np.ndarray        # float64 [nx*ny*nz]
    clamp: bool = True
    meta: dict = field(default_factory=dict)

    @property
    def nnodes(self) -> int:
        return self.row_ptr.shape[0] - 1

    @property
    def ndof(self) -> int:
        return 3 * self.nnodes

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])


def element_stiffness(h: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """24x24 Q1 element stiffness of a cube of side h with E = 1."""
    Ke = np.zeros((24, 24))
    _load().q1_element_stiffness(h, nu, _ptr(Ke))
    return Ke


def splitmix64(state: int) -> tuple[int, int]:
    """(output, next_state) of SplitMix64 from ``state``."""
    nxt = np.zeros(1, dtype=np.uint64)
    out = _load().q1_splitmix64(ctypes.c_uint64(state & 0xFFFFFFFFFFFFFFFF), _ptr(nxt))
    return int(out), int(nxt[0])


def splitmix64_uniform(state: int, n: int) -> tuple[np.ndarray, int]:
    """n uniforms in [0,1) (53 random bits each) and the next state."""
    out = np.empty(n)
    for k in range(n):
        z, state = splitmix64(state)
        out[k] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out, state


def material(shape, h, *, inclusion_frac=0.0, radius=0.1, E_mat=1.0, E_inc=1000.0,
             seed=2202) -> np.ndarray:
    nx, ny, nz = shape
    E_el = np.empty(nx * ny * nz)
    if inclusion_frac > 0.0:
        rc = _load().q1_inclusions(nx, ny, nz, h, radius, inclusion_frac, E_mat, E_inc,
                                   ctypes.c_uint64(seed), _ptr(E_el))
        if rc < 0:
            raise RuntimeError("inclusion placement did not reach the volume fraction")
    else:
        E_el.fill(E_mat)
    return E_el


def make_problem(shape, *, nu=0.3, clamp=True, body=None, traction=None,
                 inclusion_frac=0.0, radius=0.1, E_inc=1000.0, seed=2202,
                 h=None, E_el=None) -> Problem:
    """Assemble the box problem.  ``shape`` = n or (nx, ny, nz) elements.

    ``h`` defaults to 1/nx (so a cube is the unit cube).  ``body`` is a body
    force per unit volume, ``traction`` a surface load on the face x = nx h;
    several load vectors may be stacked as rows (multiple right-hand sides).
    """
    if np.isscalar(shape):
        shape = (int(shape),) * 3
    nx, ny, nz = (int(s) for s in shape)
    if min(nx, ny, nz) < 1:
        raise ValueError("need at least one element per direction")
    h = 1.0 / nx if h is None else float(h)
    lib = _load()
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    row_ptr = np.empty(nn + 1, dtype=np.int32)
    nnzb = lib.q1_pattern(nx, ny, nz, int(clamp), _ptr(row_ptr))
    if nnzb < 0:
        raise ValueError("too many blocks for int32 indices")
    col = np.empty(nnzb, dtype=np.int32)
    val = np.empty((nnzb, 3, 3))
    if E_el is None:
        E_el = material((nx, ny, nz), h, inclusion_frac=inclusion_frac, radius=radius,
                        E_inc=E_inc, seed=seed)
    E_el = np.ascontiguousarray(E_el, dtype=np.float64)
    if lib.q1_assemble(nx, ny, nz, h, nu, _ptr(E_el), int(clamp), _ptr(row_ptr),
                       _ptr(col), _ptr(val)) != 0:
        raise RuntimeError("assembly failed")
    coords = np.empty((nn, 3))
    B = np.empty((3 * nn, 6))
    lib.q1_rigid_body_modes(nx, ny, nz, h, _ptr(coords), _ptr(B))
    loads = []
    bodies = np.zeros((0, 3)) if body is None else np.atleast_2d(np.asarray(body, float))
    tracs = np.zeros((0, 3)) if traction is None else np.atleast_2d(np.asarray(traction, float))
    nrhs = max(len(bodies), len(tracs), 1)
    for r in range(nrhs):
        fb = np.ascontiguousarray(bodies[r]) if r < len(bodies) else None
        ft = np.ascontiguousarray(tracs[r]) if r < len(tracs) else None
        f = np.empty(3 * nn)
        lib.q1_load(nx, ny, nz, h, _ptr(fb), _ptr(ft), int(clamp), _ptr(f))
        loads.append(f)
    f = loads[0] if nrhs == 1 else np.stack(loads)
    return Problem((nx, ny, nz), h, nu, row_ptr, col, val, B, f, coords, E_el, clamp)


def cube(n: int, nu: float = 0.3) -> Problem:
    """n^3 elements, E = 1, clamped at x = 0, body load (0, 0, -1)."""
    return make_problem(n, nu=nu, body=(0.0, 0.0, -1.0))


def inclusions(n: int, nu: float = 0.3, seed: int = 2202, frac: float = 0.2) -> Problem:
    """n^3 elements, E = 1 matrix with E = 1000 spheres at ``frac`` volume,
    clamped at x = 0, traction (0, 0, -1) on the face x = 1."""
    return make_problem(n, nu=nu, traction=(0.0, 0.0, -1.0), inclusion_frac=frac,
                        radius=0.1, E_inc=1000.0, seed=seed)


def batch_specs(ninst: int = 64, seed: int = 2202, nmin: int = 20, nmax: int = 60,
                rhs_max: int = 16):
    """Seeded sizes, Poisson ratios and load directions of a batch of boxes.

    Instance i draws from SplitMix64 seeded with seed + i: n ~ U{nmin..nmax}
    elements per side, nu ~ U[0.2, 0.45], nrhs ~ U{1..rhs_max}, and for each
    right-hand side a unit body-force direction uniform on the sphere.
    """
    specs = []
    for i in range(ninst):
        u, st = splitmix64_uniform(seed + i, 3)
        n = nmin + min(int(u[0] * (nmax - nmin + 1)), nmax - nmin)
        nu = 0.2 + 0.25 * u[1]
        nrhs = 1 + min(int(u[2] * rhs_max), rhs_max - 1)
        dirs, st = splitmix64_uniform(st, 2 * nrhs)
        d = []
        for r in range(nrhs):
            z = 2.0 * dirs[2 * r] - 1.0
            phi = 2.0 * np.pi * dirs[2 * r + 1]
            s = np.sqrt(max(0.0, 1.0 - z * z))
            d.append((s * np.cos(phi), s * np.sin(phi), z))
        specs.append({"n": n, "nu": nu, "nrhs": nrhs, "body": np.array(d)})
    return specs


def bsr_to_dense(p: Problem) -> np.ndarray:
    """Dense copy of the matrix (tiny meshes only; test helper)."""
    n = p.nnodes
    A = np.zeros((3 * n, 3 * n))
    for I in range(n):
        for q in range(p.row_ptr[I], p.row_ptr[I + 1]):
            J = p.col[q]
            A[3 * I:3 * I + 3, 3 * J:3 * J + 3] = p.val[q]
    return A
