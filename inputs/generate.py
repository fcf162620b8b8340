"""Seeded, counter-based synthetic initial conditions for the binary Lennard-Jones mixture.

Definition of the generator (implemented identically, from this text, by the CUDA
library's on-device initialiser; neither side imports the other):

* ``splitmix64`` is the published SplitMix64 output function (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014):
  ``z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
  z ^ (z >> 31)`` on unsigned 64-bit integers.
* The draw number ``c`` (0-based) of stream ``s`` under seed ``seed`` is
  ``splitmix64(seed + (((s << 40) | c) + 1) * 0x9E3779B97F4A7C15)`` (mod 2**64), i.e. the
  ``(s<<40|c)+1``-th output of a SplitMix64 sequence started at ``seed``.  Every draw is
  therefore addressable by its counter, so any index range can be produced in parallel.
* ``uniform01(z) = (z >> 11) * 2**-53`` in [0, 1).
* Gaussian number ``m`` of the velocity stream uses draws ``2m`` and ``2m+1``:
  ``u1 = ((z1 >> 11) + 1) * 2**-53`` in (0, 1], ``u2 = (z2 >> 11) * 2**-53``,
  ``g = sqrt(-2 ln u1) * cos(2 pi u2)`` (Box-Muller).  Particle ``i``, axis ``d``
  uses ``m = 3 i + d``.

Workloads follow the benchmark suite of the paper (Sec. 3): a 80:20 binary mixture at
number density 1.2, started from an FCC lattice (4 n^3 sites) or from random
sequential addition, with Maxwell-Boltzmann velocities.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

STREAM_SPECIES = 1
STREAM_VEL = 2
STREAM_RSA = 3
STREAM_REPLICA = 4
STREAM_JITTER = 5

_TWO_M53 = 2.0 ** -53


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Draw number ``counters`` of ``stream`` (see module docstring)."""
    c = (np.uint64(stream) << np.uint64(40)) | np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
    return splitmix64(z)


def uniform01(z: np.ndarray) -> np.ndarray:
    return (z >> np.uint64(11)).astype(np.float64) * _TWO_M53


def gaussian(seed: int, m: np.ndarray) -> np.ndarray:
    """Gaussian number(s) ``m`` of the velocity stream (Box-Muller, see module docstring)."""
    m = np.asarray(m, dtype=np.uint64)
    z1 = counter_u64(seed, STREAM_VEL, np.uint64(2) * m)
    z2 = counter_u64(seed, STREAM_VEL, np.uint64(2) * m + np.uint64(1))
    u1 = ((z1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * _TWO_M53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * _TWO_M53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def box_for(n: int, rho: float) -> float:
    """Cubic box side for ``n`` particles at number density ``rho``."""
    return (n / rho) ** (1.0 / 3.0)


_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_lattice(ncell: int, L: float) -> np.ndarray:
    """FCC sites of ``ncell**3`` cubic unit cells filling a periodic cube of side ``L``.

    Site ``i = 4*(ix + n*(iy + n*iz)) + b`` sits at ``((ix, iy, iz) + basis[b] + 1/4) * a``
    with ``a = L / n``; shape (4 n^3, 3), float64.
    """
    n = int(ncell)
    a = L / n
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + _FCC_BASIS[None, :, :] + 0.25) * a
    return pos.reshape(-1, 3)


def fcc_sites(ncell: int, L: float, idx: np.ndarray, jitter: float = 0.0,
              seed: int = 0) -> np.ndarray:
    """Positions of the FCC sites ``idx`` (same numbering and values as
    :func:`fcc_lattice`), without building the whole lattice.  With ``jitter > 0``
    coordinate ``d`` of site ``i`` is moved by ``jitter * (2 u - 1)``, ``u`` the uniform
    draw ``3 i + d`` of the jitter stream (evaluated as written, no fused multiply-add;
    the result may leave the box and is reduced into it by the quantisation)."""
    n = int(ncell)
    a = L / n
    idx = np.asarray(idx, dtype=np.int64)
    b = idx % 4
    c = idx // 4
    cells = np.stack([c % n, (c // n) % n, c // (n * n)], axis=1).astype(np.float64)
    pos = (cells + _FCC_BASIS[b] + 0.25) * a
    if jitter > 0.0:
        ctr = (3 * idx[:, None] + np.arange(3)[None, :]).astype(np.uint64)
        u = uniform01(counter_u64(seed, STREAM_JITTER, ctr))
        pos = pos + float(jitter) * (2.0 * u - 1.0)
    return pos


def assign_species(n: int, n_b: int, seed: int) -> np.ndarray:
    """Seeded random choice of which ``n_b`` of ``n`` particles are species B (label 1).

    Particle ``i`` gets key ``counter_u64(seed, STREAM_SPECIES, i)``; the ``n_b``
    particles with the smallest ``(key, i)`` are B.  Sorting by random keys is a
    uniformly random shuffle, so this is a seeded shuffle of the labels.
    """
    sp = np.zeros(n, dtype=np.uint8)
    if n_b <= 0:
        return sp
    if n_b >= n:
        sp[:] = 1
        return sp
    key = counter_u64(seed, STREAM_SPECIES, np.arange(n, dtype=np.uint64))
    thr = np.partition(key, n_b - 1)[n_b - 1]
    below = key < thr
    sp[below] = 1
    need = n_b - int(below.sum())
    if need > 0:
        ties = np.flatnonzero(key == thr)[:need]
        sp[ties] = 1
    return sp


def maxwell_boltzmann(n: int, T: float, seed: int, masses: np.ndarray) -> np.ndarray:
    """Velocities at temperature ``T``: Gaussian draws scaled by sqrt(T/m), net momentum
    removed, then rescaled so that 2K/(3n-3) equals ``T`` exactly (shape (n, 3))."""
    m = np.asarray(masses, dtype=np.float64).reshape(n)
    g = gaussian(seed, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    v = g * np.sqrt(T / m)[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p / m.sum()
    if n > 1 and T > 0.0:
        ke = 0.5 * float((m[:, None] * v * v).sum())
        t_now = 2.0 * ke / (3 * n - 3)
        v *= math.sqrt(T / t_now)
    elif T == 0.0:
        v[:] = 0.0
    return v


def rsa_positions(n: int, L: float, dmin: float, seed: int, batch: int = 4096) -> np.ndarray:
    """Random sequential addition in a periodic cube: candidate ``t`` is the point
    ``L * (u_{3t}, u_{3t+1}, u_{3t+2})`` of the RSA stream; it is kept iff its
    minimum-image distance to every earlier kept point is >= ``dmin``.  Returns the
    first ``n`` kept points (shape (n, 3)).

    Candidates are examined in batches: a k-d tree of the points kept so far and one of the
    batch's own survivors propose the pairs closer than ``dmin`` (with a small margin), and
    every proposed pair is decided by the definition's own distance; candidates are then
    accepted in their order, so the result is the sequential definition's."""
    from scipy.spatial import cKDTree

    d2 = dmin * dmin
    rq = dmin * (1.0 + 1e-9) + 1e-12 * L

    def close(a, b):
        dx = a - b
        dx -= L * np.round(dx / L)
        return (dx * dx).sum(axis=-1) < d2

    kept = np.empty((n, 3), dtype=np.float64)
    nk = 0
    t0 = 0
    base = batch
    while nk < n:
        # later batches grow with the points still missing (fewer tree builds); the
        # candidate order, and so the result, does not depend on the batch sizes
        batch = max(base, min(1 << 20, 4 * (n - nk)))
        cnt = np.arange(3 * t0, 3 * (t0 + batch), dtype=np.uint64)
        cand = uniform01(counter_u64(seed, STREAM_RSA, cnt)).reshape(batch, 3) * L
        t0 += batch
        wrapped = np.where(cand >= L, cand - L, cand)  # tree coordinates only
        ok = np.ones(batch, dtype=bool)
        if nk > 0:
            tree = cKDTree(np.where(kept[:nk] >= L, kept[:nk] - L, kept[:nk]), boxsize=L)
            dist, _ = tree.query(wrapped, k=1, distance_upper_bound=rq)
            ok = dist > rq
            # clearly closer than dmin: rejected; within the margin: the definition decides
            ok &= ~(dist < dmin * (1.0 - 1e-9))
            for i in np.flatnonzero(~ok & (dist >= dmin * (1.0 - 1e-9)) & (dist <= rq)):
                lst = tree.query_ball_point(wrapped[i], rq)
                ok[i] = not close(kept[lst], cand[i]).any()
        idx = np.flatnonzero(ok)
        m = idx.size
        lo = hi = np.zeros(0, dtype=np.int64)
        if m > 1:
            pairs = cKDTree(wrapped[idx], boxsize=L).query_pairs(rq, output_type="ndarray")
            if pairs.size:
                lo = np.minimum(pairs[:, 0], pairs[:, 1])
                hi = np.maximum(pairs[:, 0], pairs[:, 1])
                exact = close(cand[idx[lo]], cand[idx[hi]])
                lo, hi = lo[exact], hi[exact]
        # acceptance in candidate order among the survivors: j is accepted iff none of its
        # earlier conflicting survivors is; decided in rounds, each round settling every
        # survivor whose earlier partners are all settled
        state = np.zeros(m, dtype=np.int8)  # 0 open, 1 accepted, -1 rejected
        has_earlier = np.zeros(m, dtype=bool)
        has_earlier[hi] = True
        state[~has_earlier] = 1
        while (state == 0).any():
            acc_partner = np.zeros(m, dtype=bool)
            acc_partner[hi[state[lo] == 1]] = True
            open_partner = np.zeros(m, dtype=bool)
            open_partner[hi[state[lo] == 0]] = True
            op = state == 0
            state[op & acc_partner] = -1
            state[op & ~acc_partner & ~open_partner] = 1
        take = idx[state == 1][: n - nk]
        kept[nk:nk + take.size] = cand[take]
        nk += take.size
    return kept


def replica_sizes(n_rep: int, nmin: int, nmax: int, seed: int, multiple: int = 5) -> list[int]:
    """Sizes of a replica batch: replica ``r`` takes draw ``r`` of the replica stream,
    ``n = nmin + (z mod (nmax - nmin + 1))``, rounded down to a multiple of ``multiple``
    (and raised to ``nmin`` rounded up if that falls below ``nmin``)."""
    z = counter_u64(seed, STREAM_REPLICA, np.arange(n_rep, dtype=np.uint64))
    span = np.uint64(nmax - nmin + 1)
    out = []
    for v in (z % span).astype(np.int64):
        n = nmin + int(v)
        n -= n % multiple
        if n < nmin:
            n += multiple
        out.append(n)
    return out


def replica_batch(n_rep: int, nmin: int, nmax: int, seed: int, rho: float = 1.2,
                  dmin: float = 0.7, frac_b: float = 0.2):
    """Random-sequential-addition mixtures of uneven size (80:20 at density ``rho``):
    sizes from :func:`replica_sizes`; replica ``r`` draws its positions and species under
    seed ``seed + r``.  Returns (sizes, boxes, positions, species)."""
    ns = replica_sizes(n_rep, nmin, nmax, seed)
    boxes, pos, sp = [], [], []
    for r, n in enumerate(ns):
        L = box_for(n, rho)
        boxes.append(L)
        pos.append(rsa_positions(n, L, dmin, seed + r))
        sp.append(assign_species(n, int(round(frac_b * n)), seed + r))
    return ns, boxes, pos, sp


@dataclass
class Workload:
    """One synthetic mixture: positions, velocities, species and box."""

    name: str
    n: int
    L: float
    species: np.ndarray
    pos: np.ndarray | None
    vel: np.ndarray | None
    T0: float
    seed: int
    ncell_fcc: int | None = None
    extra: dict = field(default_factory=dict)


def workload(kind: str, seed: int = 0, ncell: int | None = None, rho: float = 1.2,
             T0: float = 2.0, frac_b: float = 0.2, with_state: bool = True) -> Workload:
    """FCC-started mixtures of the paper's benchmark suite (Sec. 3, 80:20 at rho=1.2).

    ``kind``: ``"fcc"`` with ``ncell`` unit cells per side (N = 4 ncell^3).
    ``with_state=False`` skips positions/velocities (the library can build the same
    lattice and velocities on the device from the seed).
    """
    if kind != "fcc":
        raise ValueError(kind)
    n = 4 * ncell ** 3
    L = box_for(n, rho)
    n_b = int(round(frac_b * n))
    sp = assign_species(n, n_b, seed)
    pos = vel = None
    if with_state:
        pos = fcc_lattice(ncell, L)
        vel = maxwell_boltzmann(n, T0, seed, np.ones(n))
    return Workload(name=f"fcc{ncell}", n=n, L=L, species=sp, pos=pos, vel=vel, T0=T0,
                    seed=seed, ncell_fcc=ncell)
