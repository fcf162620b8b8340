"""Python access to the plain FP64 CPU oracle (``bbmd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product library never
imports, links or calls it, and it shares no code with the CUDA path.

Every function cites the passage of the paper it follows (see ``bbmd_oracle.h``):
Eq. lj0 / sc0 / mod0 (Sec. 2.1) for the pair potential, Sec. 2.2 for the cell search
with Newton's third law, Sec. 2.3.2 for velocity Verlet, Sec. 3 for the canonical
benchmark runs and Sec. 4 for g(r).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbmd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

POT_LJ, POT_SOFT = 0, 1
SHIFT_NONE, SHIFT_ENERGY, SHIFT_FORCE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bbmd_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB, _SRC, "-lm"]
        # OpenMP serves only the all-core baseline form; without it that form runs serially
        if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("potential", C.c_int32),
        ("shift", C.c_int32),
        ("eps", (C.c_double * 2) * 2),
        ("sigma", (C.c_double * 2) * 2),
        ("rcut", (C.c_double * 2) * 2),
        ("mass", C.c_double * 2),
    ]


class Thermo(C.Structure):
    _fields_ = [("kind", C.c_int32), ("T_start", C.c_double), ("T_end", C.c_double),
                ("tau", C.c_double)]


class NH(C.Structure):
    _fields_ = [("xi", C.c_double), ("eta", C.c_double), ("step", C.c_int64)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _u8p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _u64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i64, i32 = C.c_double, C.c_int64, C.c_int
        pd, pi64, pu8 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint8)
        pP = C.POINTER(Params)
        L.orc_pair.argtypes = [pP, i32, i32, d, pd, pd]
        L.orc_pair.restype = i32
        L.orc_forces_brute.argtypes = [i64, pd, pu8, pd, pP, pd, pd, pd, pd]
        L.orc_forces_brute.restype = None
        L.orc_forces_cells.argtypes = [i64, pd, pu8, pd, pP, pd, pd, pd, pd]
        L.orc_forces_cells.restype = i32
        L.orc_forces_cells_full.argtypes = [i64, pd, pu8, pd, pP, pd, pd, pd]
        L.orc_forces_cells_full.restype = i32
        L.orc_threads.argtypes = []
        L.orc_threads.restype = i32
        L.orc_fix_exponent.argtypes = [pd]
        L.orc_fix_exponent.restype = i32
        L.orc_quantize.argtypes = [i64, pd, i32, pd, pi64]
        L.orc_quantize.restype = None
        L.orc_cell_grid.argtypes = [pd, i32, d, pi64, pi64]
        L.orc_cell_grid.restype = i32
        L.orc_bin.argtypes = [i64, pi64, pi64, pi64, pi64]
        L.orc_bin.restype = None
        L.orc_r2_fixed.argtypes = [pi64, pi64, pi64, i32]
        L.orc_r2_fixed.restype = d
        L.orc_neighbors_brute.argtypes = [i64, pd, i32, pi64, pu8, pd, pi64, pi64]
        L.orc_neighbors_brute.restype = None
        L.orc_neighbors_cells.argtypes = [i64, pd, i32, pi64, pu8, pd, d, pi64, pi64]
        L.orc_neighbors_cells.restype = i32
        L.orc_forces_subset.argtypes = [i64, pd, pu8, pd, pP, i64, pi64, pd, pd]
        L.orc_forces_subset.restype = i32
        L.orc_neighbors_subset.argtypes = [i64, pd, i32, pi64, pu8, pd, d, i64, pi64, pi64, pi64]
        L.orc_neighbors_subset.restype = i32
        L.orc_kinetic.argtypes = [i64, pu8, pd, pP, pd]
        L.orc_kinetic.restype = d
        L.orc_md_run.argtypes = [i64, pd, pu8, pP, pd, pd, C.POINTER(C.c_int32), pd, i32,
                                 C.POINTER(NH), i64, d, C.POINTER(Thermo), i32, pd]
        L.orc_md_run.restype = i32
        L.orc_sd_run.argtypes = [i64, pd, pu8, pP, pd, i64, d, d, i32]
        L.orc_sd_run.restype = i32
        L.orc_gr_counts.argtypes = [i64, pd, i32, pi64, pu8, i64, d, C.POINTER(C.c_uint64)]
        L.orc_gr_counts.restype = None
        L.orc_gr_normalize.argtypes = [i64, pd, pu8, i64, d, C.POINTER(C.c_uint64), pd]
        L.orc_gr_normalize.restype = None
        L.orc_msd_fs.argtypes = [i64, pd, pu8, pd, C.POINTER(C.c_int32), pd,
                                 C.POINTER(C.c_int32), d, pd, pd]
        L.orc_msd_fs.restype = None
        _lib = L
    return _lib


def ka_params(potential: int = POT_LJ, shift: int = SHIFT_ENERGY, rc_factor: float = 2.5,
              mass=(1.0, 1.0)) -> Params:
    """Binary mixture of the paper's benchmark suite (Sec. 3): eps_AA=1, eps_AB=1.5,
    eps_BB=0.5, sigma_AA=1, sigma_AB=0.8, sigma_BB=0.88, m=1; r_c = rc_factor*sigma."""
    p = Params()
    p.potential = potential
    p.shift = shift
    eps = ((1.0, 1.5), (1.5, 0.5))
    sig = ((1.0, 0.8), (0.8, 0.88))
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = eps[a][b]
            p.sigma[a][b] = sig[a][b]
            p.rcut[a][b] = rc_factor * sig[a][b]
    p.mass[0], p.mass[1] = mass
    return p


def _box(L):
    L = np.asarray(L, dtype=np.float64)
    return np.full(3, float(L)) if L.ndim == 0 else np.ascontiguousarray(L, dtype=np.float64)


def pair(p: Params, a: int, b: int, r2: float):
    V, f = C.c_double(), C.c_double()
    hit = lib().orc_pair(C.byref(p), a, b, r2, C.byref(V), C.byref(f))
    return bool(hit), V.value, f.value


def forces(pos, species, L, p: Params, method: str = "brute"):
    """Forces (n,3), per-particle energy u (n,), virial W, potential energy PE.  method:
    "brute" (O(N^2) definition), "cells" (linked cells, Newton's third law) or "cells_full"
    (every particle sums its own stencil on every core; W is not computed)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    n = pos.shape[0]
    Lb = _box(L)
    F = np.zeros((n, 3))
    u = np.zeros(n)
    W, PE = C.c_double(), C.c_double()
    if method == "brute":
        lib().orc_forces_brute(n, _dp(Lb), _u8p(sp), _dp(pos), C.byref(p), _dp(F), _dp(u),
                               C.byref(W), C.byref(PE))
    elif method == "cells_full":  # all-core form: no virial
        rc = lib().orc_forces_cells_full(n, _dp(Lb), _u8p(sp), _dp(pos), C.byref(p), _dp(F),
                                         _dp(u), C.byref(PE))
        if rc != 0:
            raise ValueError("box too small for the cell search")
        W.value = float("nan")
    else:
        rc = lib().orc_forces_cells(n, _dp(Lb), _u8p(sp), _dp(pos), C.byref(p), _dp(F),
                                    _dp(u), C.byref(W), C.byref(PE))
        if rc != 0:
            raise ValueError("box too small for the cell search")
    return F, u, W.value, PE.value


def forces_subset(pos, species, L, p: Params, idx):
    """Forces (m,3) and energies (m,) of particles idx only (cell search, Sec. 2.2)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((idx.size, 3))
    u = np.zeros(idx.size)
    if lib().orc_forces_subset(pos.shape[0], _dp(_box(L)), _u8p(sp), _dp(pos), C.byref(p),
                               idx.size, _ip(idx), _dp(F), _dp(u)) != 0:
        raise ValueError("box too small for the cell search")
    return F, u


def neighbors_subset(xfix, species, L, k, R2, idx, rcell):
    xfix = np.ascontiguousarray(xfix, dtype=np.int64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    R2 = np.ascontiguousarray(R2, dtype=np.float64)
    off = np.zeros(idx.size + 1, dtype=np.int64)
    Lb = _box(L)
    L_ = lib()
    if L_.orc_neighbors_subset(xfix.shape[0], _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), rcell,
                               idx.size, _ip(idx), _ip(off), None) != 0:
        raise ValueError("box too small for the cell grid")
    nbr = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
    L_.orc_neighbors_subset(xfix.shape[0], _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), rcell,
                            idx.size, _ip(idx), _ip(off), _ip(nbr))
    return off, nbr[: int(off[-1])]


def fix_exponent(L) -> int:
    return int(lib().orc_fix_exponent(_dp(_box(L))))


def quantize(pos, L, k=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    Lb = _box(L)
    if k is None:
        k = fix_exponent(Lb)
    out = np.zeros(pos.shape, dtype=np.int64)
    lib().orc_quantize(pos.shape[0], _dp(Lb), k, _dp(pos), _ip(out))
    return out, k


def dequantize(xfix, k):
    """Exact double value of quantized positions (multiples of 2^-k)."""
    return np.ldexp(np.asarray(xfix, dtype=np.float64), -k)


def cell_grid(L, k, rcell):
    Lb = _box(L)
    nc = np.zeros(3, dtype=np.int64)
    D = np.zeros(3, dtype=np.int64)
    if lib().orc_cell_grid(_dp(Lb), k, rcell, _ip(nc), _ip(D)) != 0:
        raise ValueError("fewer than 3 cells per axis")
    return nc, D


def bin_cells(xfix, nc, D):
    xfix = np.ascontiguousarray(xfix, dtype=np.int64)
    out = np.zeros(xfix.shape[0], dtype=np.int64)
    lib().orc_bin(xfix.shape[0], _ip(xfix), _ip(np.asarray(nc, np.int64)),
                  _ip(np.asarray(D, np.int64)), _ip(out))
    return out


def r2_fixed(xi, xj, L, k):
    Lf = np.array([int(np.ldexp(v, k)) for v in _box(L)], dtype=np.int64)
    return lib().orc_r2_fixed(_ip(np.ascontiguousarray(xi, np.int64)),
                              _ip(np.ascontiguousarray(xj, np.int64)), _ip(Lf), k)


def list_R2(p: Params, skin: float) -> np.ndarray:
    """(rc_ab + skin)^2 evaluated as the two IEEE operations it shows."""
    R2 = np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            R = p.rcut[a][b] + skin
            R2[a, b] = R * R
    return R2


def neighbors(xfix, species, L, k, R2, method: str = "brute", rcell: float | None = None):
    """Full neighbour sets as (offsets[n+1], nbr) with ascending j per i."""
    xfix = np.ascontiguousarray(xfix, dtype=np.int64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    n = xfix.shape[0]
    Lb = _box(L)
    R2 = np.ascontiguousarray(R2, dtype=np.float64)
    off = np.zeros(n + 1, dtype=np.int64)
    L_ = lib()
    if method == "brute":
        L_.orc_neighbors_brute(n, _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), _ip(off), None)
        nbr = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
        L_.orc_neighbors_brute(n, _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), _ip(off), _ip(nbr))
    else:
        if rcell is None:
            rcell = float(np.sqrt(R2.max()))
        if L_.orc_neighbors_cells(n, _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), rcell, _ip(off),
                                  None) != 0:
            raise ValueError("box too small for the cell grid")
        nbr = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
        L_.orc_neighbors_cells(n, _dp(Lb), k, _ip(xfix), _u8p(sp), _dp(R2), rcell, _ip(off),
                               _ip(nbr))
    return off, nbr[: int(off[-1])]


def kinetic(vel, species, p: Params):
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    P = np.zeros(3)
    K = lib().orc_kinetic(vel.shape[0], _u8p(sp), _dp(vel), C.byref(p), _dp(P))
    return K, P


class MDState:
    """FP64 state advanced by :func:`md_run` (positions wrapped into [0, L))."""

    def __init__(self, pos, vel, species, L, p: Params, image=None):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).copy()
        self.vel = np.ascontiguousarray(vel, dtype=np.float64).copy()
        self.species = np.ascontiguousarray(species, dtype=np.uint8)
        self.L = _box(L)
        self.p = p
        n = self.pos.shape[0]
        self.image = (np.zeros((n, 3), dtype=np.int32) if image is None
                      else np.ascontiguousarray(image, dtype=np.int32).copy())
        self.F = np.zeros((n, 3))
        self.F_valid = 0
        self.nh = NH()

    @property
    def n(self):
        return self.pos.shape[0]


def threads() -> int:
    """Threads of the all-core force form (1 when built without OpenMP)."""
    return int(lib().orc_threads())


def md_run(st: MDState, nsteps: int, dt: float, thermo=None, use_cells=False,
           log: bool = False):
    """Advance ``st`` by ``nsteps`` velocity-Verlet steps (NVE, or Nose-Hoover when
    ``thermo = (T_start, T_end, tau)``).  Forces by brute force, by linked cells
    (``use_cells=True``) or by the all-core full-stencil form (``use_cells="all_cores"``).
    Returns the per-step log (nsteps, 5) of {KE, PE, xi, eta, T_target} when ``log`` is
    set."""
    th = None
    if thermo is not None:
        th = Thermo(1, float(thermo[0]), float(thermo[1]), float(thermo[2]))
    lg = np.zeros((nsteps, 5)) if log else None
    rc = lib().orc_md_run(st.n, _dp(st.L), _u8p(st.species), C.byref(st.p), _dp(st.pos),
                          _dp(st.vel), _i32p(st.image), _dp(st.F), st.F_valid,
                          C.byref(st.nh), nsteps, dt, C.byref(th) if th else None,
                          2 if use_cells == "all_cores" else 1 if use_cells else 0,
                          _dp(lg) if log else None)
    if rc != 0:
        raise ValueError("oracle md_run failed (box too small for cells?)")
    st.F_valid = 1
    return lg


def sd_run(pos, species, L, p: Params, nsteps: int, hmax: float = 1e-3, dmax: float = 0.05,
           use_cells: bool = False):
    pos = np.ascontiguousarray(pos, dtype=np.float64).copy()
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    if lib().orc_sd_run(pos.shape[0], _dp(_box(L)), _u8p(sp), C.byref(p), _dp(pos), nsteps,
                        hmax, dmax, 1 if use_cells else 0) != 0:
        raise ValueError("oracle sd_run failed")
    return pos


def gr_counts(xfix, species, L, k, nbins=500, rmax=5.0):
    xfix = np.ascontiguousarray(xfix, dtype=np.int64)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    out = np.zeros((2, 2, nbins), dtype=np.uint64)
    lib().orc_gr_counts(xfix.shape[0], _dp(_box(L)), k, _ip(xfix), _u8p(sp), nbins, rmax,
                        _u64p(out))
    return out


def gr_normalize(counts, species, L, rmax=5.0):
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    nbins = counts.shape[-1]
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    g = np.zeros((2, 2, nbins))
    lib().orc_gr_normalize(sp.shape[0], _dp(_box(L)), _u8p(sp), nbins, rmax, _u64p(counts),
                           _dp(g))
    return g


def msd_fs(pos, image, pos0, image0, species, L, kvec=7.25):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    pos0 = np.ascontiguousarray(pos0, dtype=np.float64)
    im = np.ascontiguousarray(image, dtype=np.int32)
    im0 = np.ascontiguousarray(image0, dtype=np.int32)
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    msd = np.zeros(2)
    fs = np.zeros(2)
    lib().orc_msd_fs(pos.shape[0], _dp(_box(L)), _u8p(sp), _dp(pos), _i32p(im), _dp(pos0),
                     _i32p(im0), kvec, _dp(msd), _dp(fs))
    return msd, fs
