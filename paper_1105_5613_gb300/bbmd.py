"""Thin ctypes binding of libbbmd (include/bbmd.h): the same entry points, argument
marshalling only.  Every step of the hot path runs in the CUDA library; there is no CPU
fallback -- loading fails loudly when the library has not been built.

PyTorch supplies device memory (its caching allocator, passed as a bbmd_alloc) and the
CUDA stream; both are optional.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbbmd.so")

BBMD_OK = 0
ERRORS = {
    1: "BBMD_ERR_ARG", 2: "BBMD_ERR_BOX_TOO_SMALL", 3: "BBMD_ERR_OOM", 4: "BBMD_ERR_CUDA",
    5: "BBMD_ERR_LIST_OVERFLOW", 6: "BBMD_ERR_NUMERIC", 7: "BBMD_ERR_TIMEOUT", 8: "BBMD_ERR_STATE",
}
POT_LJ, POT_SOFT = 0, 1
SHIFT_NONE, SHIFT_ENERGY, SHIFT_FORCE = 0, 1, 2
PREC_MIXED, PREC_FP64 = 0, 1
NBR_VERLET, NBR_CELL = 0, 1
THERMO_NVE, THERMO_NH = 0, 1
OBS_ENERGY, OBS_VIRIAL, OBS_MOMENTUM, OBS_GR, OBS_MSD, OBS_FS, OBS_SET_REF = 1, 2, 4, 8, 16, 32, 64
BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2
MAX_ORIGINS = 16


class BBMDError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class bbmd_params(C.Structure):
    _fields_ = [
        ("potential", C.c_int32), ("shift", C.c_int32), ("precision", C.c_int32),
        ("nbr_mode", C.c_int32),
        ("eps", (C.c_double * 2) * 2), ("sigma", (C.c_double * 2) * 2),
        ("rcut", (C.c_double * 2) * 2), ("mass", C.c_double * 2), ("skin", C.c_double),
        ("list_capacity", C.c_int32), ("stencil_capacity", C.c_int32), ("block_z", C.c_int32),
        ("init_jitter", C.c_double),
    ]


class bbmd_thermostat(C.Structure):
    _fields_ = [("kind", C.c_int32), ("T_start", C.c_double), ("T_end", C.c_double),
                ("tau", C.c_double)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class bbmd_alloc(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class bbmd_obs_args(C.Structure):
    _fields_ = [("nbins", C.c_int32), ("rmax", C.c_double), ("k", C.c_double),
                ("origin", C.c_int32)]


class bbmd_obs(C.Structure):
    _fields_ = [
        ("ke", C.c_double), ("pe", C.c_double), ("virial", C.c_double), ("pressure", C.c_double),
        ("temperature", C.c_double), ("momentum", C.c_double * 3), ("xi", C.c_double),
        ("eta", C.c_double), ("conserved", C.c_double), ("step", C.c_int64),
        ("n_rebuilds", C.c_int64), ("gr_counts", C.POINTER(C.c_uint64)),
        ("gr", C.POINTER(C.c_double)), ("msd", C.c_double * 2), ("fs", C.c_double * 2),
    ]


class bbmd_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("fix_exponent", C.c_int32), ("nc", C.c_int32 * 3),
                ("cell_side_fix", C.c_int64 * 3), ("list_capacity", C.c_int32),
                ("stencil_capacity", C.c_int32), ("device_bytes", C.c_int64),
                ("block_z", C.c_int32), ("shape_force_ms", C.c_float * 4),
                ("shape_list_ms", C.c_float * 4)]


PHASES = ["integrate", "rebuild", "list", "force", "finalize"]

EXPORTS = ["bbmd_create", "bbmd_destroy", "bbmd_step", "bbmd_step_profiled", "bbmd_observe",
           "bbmd_minimize",
           "bbmd_get_state", "bbmd_set_state", "bbmd_get_forces", "bbmd_get_cells",
           "bbmd_get_neighbors", "bbmd_rebuild", "bbmd_get_info", "bbmd_last_error",
           "bbmd_gr_counts_noalloc", "bbmd_tune", "bbmd_get_forces_ids", "bbmd_create_batch", "bbmd_step_batch",
           "bbmd_batch_replica", "bbmd_batch_size", "bbmd_batch_set_branches",
           "bbmd_batch_set_mode", "bbmd_batch_set_wait_limit", "bbmd_batch_uses_persistent",
           "bbmd_destroy_batch",
           "bbmd_batch_last_error", "bbmd_fma_peak", "bbmd_smem_scatter_rate"]

_lib = None


def load(path: str | None = None):
    """Load libbbmd.so (raises if it has not been built).  The BBMD_LIB environment
    variable selects another build of the library."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("BBMD_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libbbmd.so not found at {path}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    P = C.POINTER
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    L.bbmd_create.argtypes = [P(bbmd_params), i64, P(d), P(C.c_uint8), P(d), P(d), d, C.c_uint64,
                              vp, P(bbmd_alloc), P(vp)]
    L.bbmd_create.restype = C.c_int
    L.bbmd_destroy.argtypes = [vp]
    L.bbmd_destroy.restype = None
    L.bbmd_step.argtypes = [vp, i64, d, P(bbmd_thermostat)]
    L.bbmd_step.restype = C.c_int
    L.bbmd_step_profiled.argtypes = [vp, i64, d, P(bbmd_thermostat), P(d), P(i64)]
    L.bbmd_step_profiled.restype = C.c_int
    L.bbmd_observe.argtypes = [vp, C.c_uint32, P(bbmd_obs_args), P(bbmd_obs)]
    L.bbmd_observe.restype = C.c_int
    L.bbmd_minimize.argtypes = [vp, i64, d, d]
    L.bbmd_minimize.restype = C.c_int
    L.bbmd_get_state.argtypes = [vp, P(d), P(d), P(C.c_int32)]
    L.bbmd_get_state.restype = C.c_int
    L.bbmd_set_state.argtypes = [vp, P(d), P(d), P(C.c_int32)]
    L.bbmd_set_state.restype = C.c_int
    L.bbmd_get_forces.argtypes = [vp, P(d), P(d)]
    L.bbmd_get_forces.restype = C.c_int
    L.bbmd_get_forces_ids.argtypes = [vp, P(i64), i64, P(d), P(d)]
    L.bbmd_get_forces_ids.restype = C.c_int
    L.bbmd_get_cells.argtypes = [vp, P(i64)]
    L.bbmd_get_cells.restype = C.c_int
    L.bbmd_get_neighbors.argtypes = [vp, P(i64), i64, P(i64), P(i64), i64]
    L.bbmd_get_neighbors.restype = C.c_int
    L.bbmd_tune.argtypes = [vp]
    L.bbmd_tune.restype = C.c_int
    L.bbmd_rebuild.argtypes = [vp]
    L.bbmd_rebuild.restype = C.c_int
    L.bbmd_get_info.argtypes = [vp, P(bbmd_info)]
    L.bbmd_get_info.restype = C.c_int
    L.bbmd_gr_counts_noalloc.argtypes = [vp, C.c_int32, d, P(C.c_uint64)]
    L.bbmd_gr_counts_noalloc.restype = C.c_int
    PP = C.POINTER(C.c_void_p)
    L.bbmd_create_batch.argtypes = [P(bbmd_params), C.c_int32, P(i64), P(d), PP, PP, PP, P(d),
                                    C.c_uint64, vp, P(bbmd_alloc), P(vp)]
    L.bbmd_create_batch.restype = C.c_int
    L.bbmd_step_batch.argtypes = [vp, i64, d, P(bbmd_thermostat)]
    L.bbmd_step_batch.restype = C.c_int
    L.bbmd_batch_replica.argtypes = [vp, C.c_int32]
    L.bbmd_batch_replica.restype = vp
    L.bbmd_batch_set_branches.argtypes = [vp, C.c_int32]
    L.bbmd_batch_set_branches.restype = C.c_int
    L.bbmd_batch_set_mode.argtypes = [vp, C.c_int32]
    L.bbmd_batch_set_mode.restype = C.c_int
    L.bbmd_batch_set_wait_limit.argtypes = [vp, C.c_uint64]
    L.bbmd_batch_set_wait_limit.restype = C.c_int
    L.bbmd_batch_uses_persistent.argtypes = [vp]
    L.bbmd_batch_uses_persistent.restype = C.c_int32
    L.bbmd_batch_size.argtypes = [vp]
    L.bbmd_batch_size.restype = C.c_int32
    L.bbmd_destroy_batch.argtypes = [vp]
    L.bbmd_destroy_batch.restype = None
    L.bbmd_batch_last_error.argtypes = [vp]
    L.bbmd_batch_last_error.restype = C.c_char_p
    L.bbmd_last_error.argtypes = [vp]
    L.bbmd_last_error.restype = C.c_char_p
    L.bbmd_fma_peak.argtypes = [C.c_int32, P(C.c_int32), P(d)]
    L.bbmd_fma_peak.restype = C.c_int
    L.bbmd_smem_scatter_rate.argtypes = [C.c_int32, P(d)]
    L.bbmd_smem_scatter_rate.restype = C.c_int
    _lib = L
    return L


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _check(h, rc):
    if rc != BBMD_OK:
        msg = load().bbmd_last_error(h).decode() if h else ""
        raise BBMDError(rc, msg)


def ka_params(potential=POT_LJ, shift=SHIFT_ENERGY, precision=PREC_MIXED, nbr_mode=NBR_VERLET,
              skin=0.3, rc_factor=2.5, mass=(1.0, 1.0), list_capacity=0, stencil_capacity=0,
              block_z=0, init_jitter=0.0):
    """Parameters of the binary mixture of the paper's benchmark suite (Sec. 3):
    eps_AA=1, eps_AB=1.5, eps_BB=0.5, sigma_AA=1, sigma_AB=0.8, sigma_BB=0.88, m=1."""
    p = bbmd_params()
    p.potential, p.shift, p.precision, p.nbr_mode = potential, shift, precision, nbr_mode
    eps = ((1.0, 1.5), (1.5, 0.5))
    sig = ((1.0, 0.8), (0.8, 0.88))
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = eps[a][b]
            p.sigma[a][b] = sig[a][b]
            p.rcut[a][b] = rc_factor * sig[a][b]
    p.mass[0], p.mass[1] = mass
    p.skin = skin
    p.list_capacity = list_capacity
    p.stencil_capacity = stencil_capacity
    p.block_z = block_z
    p.init_jitter = init_jitter
    return p


def fma_peak(precision=PREC_MIXED):
    """Measured peak FMA rate of the current device: (TFLOP/s, SM count)."""
    L = load()
    nsm = C.c_int32(0)
    tf = C.c_double(0.0)
    _check(None, L.bbmd_fma_peak(precision, C.byref(nsm), C.byref(tf)))
    return tf.value, nsm.value


def smem_scatter_rate(kind):
    """Measured shared-memory scatter-adds per second of the current device (kind 0: 64-bit
    fixed point from float, 1: 32-bit integer, 2: FP32)."""
    r = C.c_double(0.0)
    _check(None, load().bbmd_smem_scatter_rate(kind, C.byref(r)))
    return r.value


def torch_allocator(device=None):
    """bbmd_alloc backed by torch's CUDA caching allocator (keep the returned tuple alive)."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    a = bbmd_alloc(fa, ff, None)
    return a, (fa, ff)


class Sim:
    """Owner of one bbmd_sim handle; methods map one-to-one to the C entry points."""

    def __init__(self, params, n, box, species, pos=None, vel=None, T0=0.0, seed=0,
                 stream=None, use_torch_allocator=False):
        L = load()
        box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
        sp = np.ascontiguousarray(species, dtype=np.uint8)
        if sp.shape != (n,):
            raise ValueError("species must have n entries")
        pos = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64).reshape(n, 3)
        vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3)
        self._keep = None
        alloc = None
        if use_torch_allocator:
            alloc, self._keep = torch_allocator()
        h = C.c_void_p()
        stream_ptr = None if stream is None else C.c_void_p(int(stream))
        rc = L.bbmd_create(C.byref(params), int(n), _dp(box),
                           sp.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(pos), _dp(vel), float(T0),
                           C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), stream_ptr,
                           C.byref(alloc) if alloc is not None else None, C.byref(h))
        if rc != BBMD_OK:
            raise BBMDError(rc, "bbmd_create")
        self.h = h
        self.n = int(n)
        self.box = box
        self.params = params

    def close(self):
        if getattr(self, "_borrowed", False):  # a replica handle: owned by its batch
            self.h = None
            return
        if getattr(self, "h", None):
            load().bbmd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps, dt, thermostat=None):
        th = None
        if thermostat is not None:
            kind, T0, T1, tau = thermostat
            th = bbmd_thermostat(kind, T0, T1, tau)
        _check(self.h, load().bbmd_step(self.h, int(nsteps), float(dt),
                                        C.byref(th) if th is not None else None))

    def step_profiled(self, nsteps, dt, thermostat=None):
        """Per-phase device time (ms, summed over the steps) and the rebuild count."""
        th = None
        if thermostat is not None:
            kind, T0, T1, tau = thermostat
            th = bbmd_thermostat(kind, T0, T1, tau)
        ms = np.zeros(len(PHASES))
        nreb = C.c_int64()
        _check(self.h, load().bbmd_step_profiled(self.h, int(nsteps), float(dt),
                                                 C.byref(th) if th is not None else None,
                                                 _dp(ms), C.byref(nreb)))
        return dict(zip(PHASES, ms.tolist())), int(nreb.value)

    def observe(self, mask, nbins=500, rmax=5.0, k=7.25, origin=0):
        o = bbmd_obs()
        counts = g = None
        if mask & OBS_GR:
            counts = np.zeros((2, 2, nbins), dtype=np.uint64)
            g = np.zeros((2, 2, nbins))
            o.gr_counts = counts.ctypes.data_as(C.POINTER(C.c_uint64))
            o.gr = _dp(g)
        args = bbmd_obs_args(nbins, rmax, k, origin)
        _check(self.h, load().bbmd_observe(self.h, mask, C.byref(args), C.byref(o)))
        res = {f: getattr(o, f) for f in ("ke", "pe", "virial", "pressure", "temperature", "xi",
                                          "eta", "conserved", "step", "n_rebuilds")}
        res["momentum"] = np.array(o.momentum[:])
        res["msd"] = np.array(o.msd[:])
        res["fs"] = np.array(o.fs[:])
        if counts is not None:
            res["gr_counts"] = counts
            res["gr"] = g
        return res

    def gr_counts_noalloc(self, nbins=500, rmax=5.0):
        """g(r) pair counts (2, 2, nbins) through bbmd_gr_counts_noalloc: no device memory is
        allocated (host result array only)."""
        counts = np.zeros((2, 2, nbins), dtype=np.uint64)
        _check(self.h, load().bbmd_gr_counts_noalloc(
            self.h, int(nbins), float(rmax), counts.ctypes.data_as(C.POINTER(C.c_uint64))))
        return counts

    def minimize(self, nsteps, hmax=1e-3, dmax=0.05):
        _check(self.h, load().bbmd_minimize(self.h, int(nsteps), float(hmax), float(dmax)))

    def get_state(self, out=None):
        """(pos, vel, image) in id order; out: three arrays to fill instead (e.g. pinned)."""
        if out is not None:
            pos, vel, img = out
            assert pos.shape == (self.n, 3) and pos.dtype == np.float64 and pos.flags.c_contiguous
            assert vel.shape == (self.n, 3) and vel.dtype == np.float64 and vel.flags.c_contiguous
            assert img.shape == (self.n, 3) and img.dtype == np.int32 and img.flags.c_contiguous
        else:
            pos = np.zeros((self.n, 3))
            vel = np.zeros((self.n, 3))
            img = np.zeros((self.n, 3), dtype=np.int32)
        _check(self.h, load().bbmd_get_state(self.h, _dp(pos), _dp(vel),
                                             img.ctypes.data_as(C.POINTER(C.c_int32))))
        return pos, vel, img

    def set_state(self, pos, vel, image=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(self.n, 3)
        ip = None
        if image is not None:
            image = np.ascontiguousarray(image, dtype=np.int32).reshape(self.n, 3)
            ip = image.ctypes.data_as(C.POINTER(C.c_int32))
        _check(self.h, load().bbmd_set_state(self.h, _dp(pos), _dp(vel), ip))

    def get_forces(self, energies=False):
        F = np.zeros((self.n, 3))
        u = np.zeros(self.n) if energies else None
        _check(self.h, load().bbmd_get_forces(self.h, _dp(F), _dp(u)))
        return (F, u) if energies else F

    def get_forces_ids(self, ids, energies=False):
        """Forces (m, 3) (and energies (m,)) of the particles ids only."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        F = np.zeros((ids.size, 3))
        u = np.zeros(ids.size) if energies else None
        _check(self.h, load().bbmd_get_forces_ids(self.h, ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                                  int(ids.size), _dp(F), _dp(u)))
        return (F, u) if energies else F

    def get_cells(self):
        c = np.zeros(self.n, dtype=np.int64)
        _check(self.h, load().bbmd_get_cells(self.h, c.ctypes.data_as(C.POINTER(C.c_int64))))
        return c

    def get_neighbors(self, ids=None):
        """Verlet lists as id sets: (offsets, nbr) for all particles (id order) or for ids."""
        L = load()
        P = C.POINTER(C.c_int64)
        if ids is None:
            m, ip = self.n, None
        else:
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            m, ip = ids.size, ids.ctypes.data_as(P)
        off = np.zeros(m + 1, dtype=np.int64)
        _check(self.h, L.bbmd_get_neighbors(self.h, ip, m, off.ctypes.data_as(P), None, 0))
        nbr = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
        _check(self.h, L.bbmd_get_neighbors(self.h, ip, m, off.ctypes.data_as(P),
                                            nbr.ctypes.data_as(P), int(nbr.size)))
        return off, nbr[: int(off[-1])]

    def tune(self):
        """Re-pick the block shape by timing it on the current state (bbmd_tune)."""
        _check(self.h, load().bbmd_tune(self.h))

    def rebuild(self):
        _check(self.h, load().bbmd_rebuild(self.h))

    def info(self):
        i = bbmd_info()
        _check(self.h, load().bbmd_get_info(self.h, C.byref(i)))
        return {"n": i.n, "fix_exponent": i.fix_exponent, "nc": list(i.nc),
                "cell_side_fix": list(i.cell_side_fix), "list_capacity": i.list_capacity,
                "stencil_capacity": i.stencil_capacity, "device_bytes": i.device_bytes,
                "block_z": i.block_z, "shape_force_ms": list(i.shape_force_ms),
                "shape_list_ms": list(i.shape_list_ms)}


def _thermo_array(thermostats, n_rep):
    if thermostats is None:
        return None
    if len(thermostats) != n_rep:
        raise ValueError("one thermostat per replica")
    arr = (bbmd_thermostat * n_rep)()
    for r, (kind, T0, T1, tau) in enumerate(thermostats):
        arr[r] = bbmd_thermostat(kind, T0, T1, tau)
    return arr


class Batch:
    """Owner of a bbmd_batch: independent replicas stepped together (bbmd_step_batch).
    replica(r) returns a Sim view of replica r (owned by the batch)."""

    def __init__(self, params, ns, boxes, species, pos=None, vel=None, T0=None, seed=0,
                 stream=None, use_torch_allocator=False):
        L = load()
        ns = [int(v) for v in ns]
        n_rep = len(ns)
        boxes = np.asarray(boxes, np.float64)
        if boxes.ndim == 1:  # one cubic side per replica
            boxes = np.repeat(boxes[:, None], 3, axis=1)
        boxes = np.ascontiguousarray(boxes.reshape(n_rep, 3))
        self._arrays = []

        def ptrs(arrs, dtype, shape_of):
            if arrs is None:
                return None
            out = (C.c_void_p * n_rep)()
            for r, a in enumerate(arrs):
                if a is None:
                    out[r] = None
                    continue
                a = np.ascontiguousarray(a, dtype=dtype).reshape(shape_of(r))
                self._arrays.append(a)
                out[r] = a.ctypes.data
            return C.cast(out, C.POINTER(C.c_void_p))

        sp = ptrs(species, np.uint8, lambda r: (ns[r],))
        pp = ptrs(pos, np.float64, lambda r: (ns[r], 3))
        vp_ = ptrs(vel, np.float64, lambda r: (ns[r], 3))
        T0 = np.ascontiguousarray(np.broadcast_to(np.asarray(0.0 if T0 is None else T0,
                                                             np.float64), (n_rep,)))
        narr = np.asarray(ns, dtype=np.int64)
        self._keep = None
        alloc = None
        if use_torch_allocator:
            alloc, self._keep = torch_allocator()
        h = C.c_void_p()
        stream_ptr = None if stream is None else C.c_void_p(int(stream))
        rc = L.bbmd_create_batch(C.byref(params), n_rep, narr.ctypes.data_as(C.POINTER(C.c_int64)),
                                 _dp(boxes), sp, pp, vp_, _dp(T0),
                                 C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), stream_ptr,
                                 C.byref(alloc) if alloc is not None else None, C.byref(h))
        if rc != BBMD_OK:
            raise BBMDError(rc, "bbmd_create_batch")
        self.h = h
        self.ns = ns
        self.params = params
        self._reps = []
        for r in range(n_rep):
            v = Sim.__new__(Sim)
            v._borrowed = True
            v.h = C.c_void_p(L.bbmd_batch_replica(h, r))
            v.n = ns[r]
            v.box = boxes[r].copy()
            v.params = params
            v._keep = None
            self._reps.append(v)

    def __len__(self):
        return len(self.ns)

    def replica(self, r):
        return self._reps[r]

    def set_branches(self, k):
        """Graph branches of the batch step (groups of replicas run concurrently)."""
        rc = load().bbmd_batch_set_branches(self.h, int(k))
        if rc != BBMD_OK:
            raise BBMDError(rc, "bbmd_batch_set_branches")

    def set_mode(self, mode):
        """Step path: BATCH_AUTO (persistent when it applies), BATCH_GRAPH or
        BATCH_PERSISTENT (bbmd_batch_set_mode)."""
        rc = load().bbmd_batch_set_mode(self.h, int(mode))
        if rc != BBMD_OK:
            raise BBMDError(rc, "bbmd_batch_set_mode")

    def set_wait_limit(self, ns):
        """Limit of each dependency wait of the persistent step, in ns
        (bbmd_batch_set_wait_limit)."""
        rc = load().bbmd_batch_set_wait_limit(self.h, int(ns))
        if rc != BBMD_OK:
            raise BBMDError(rc, "bbmd_batch_set_wait_limit")

    def uses_persistent(self):
        return bool(load().bbmd_batch_uses_persistent(self.h))

    def step(self, nsteps, dt, thermostats=None):
        """thermostats: None (NVE) or one (kind, T_start, T_end, tau) per replica."""
        arr = _thermo_array(thermostats, len(self.ns))
        rc = load().bbmd_step_batch(self.h, int(nsteps), float(dt), arr)
        if rc != BBMD_OK:
            raise BBMDError(rc, load().bbmd_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            for v in self._reps:
                v.h = None
            load().bbmd_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

