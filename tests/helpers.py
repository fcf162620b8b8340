"""Shared helpers for the GPU parity tests: seeded inputs from ``inputs``, the oracle on
the same quantised positions, and the error metrics of the parity bar."""
import re
import os

import numpy as np

import oracle
from inputs import generate as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    """Entry points declared in include/bbmd.h."""
    txt = open(os.path.join(ROOT, "include", "bbmd.h")).read()
    return sorted(set(re.findall(r"\b(bbmd_[a-z_]+)\s*\(", txt)))


def mixture(ncell, seed=0, T=2.0, shake=0.0, rho=1.2, frac_b=0.2):
    """FCC mixture (optionally displaced by a seeded uniform shake), velocities at T."""
    n = 4 * ncell ** 3
    L = gen.box_for(n, rho)
    pos = gen.fcc_lattice(ncell, L)
    if shake > 0:
        rng = np.random.default_rng(seed + 1000)
        pos = (pos + rng.uniform(-shake, shake, pos.shape)) % L
    sp = gen.assign_species(n, int(round(frac_b * n)), seed)
    vel = gen.maxwell_boltzmann(n, T, seed, np.ones(n))
    return n, L, pos, vel, sp


def quantized(pos, L):
    """Positions exactly as the library holds them (documented quantisation rule)."""
    xfix, k = oracle.quantize(pos, L)
    return oracle.dequantize(xfix, k), xfix, k


def force_errors(F, Fo):
    """e_i = |F_i - F_i^ora| / max(|F_i^ora|, 0.1 RMS|F^ora|)."""
    rms = float(np.sqrt((Fo ** 2).sum(1).mean()))
    den = np.maximum(np.linalg.norm(Fo, axis=1), 0.1 * rms)
    return np.linalg.norm(F - Fo, axis=1) / den


def oracle_params(bp):
    """Oracle parameter block with the same values as a binding parameter block."""
    p = oracle.Params()
    p.potential, p.shift = bp.potential, bp.shift
    for a in range(2):
        p.mass[a] = bp.mass[a]
        for b in range(2):
            p.eps[a][b] = bp.eps[a][b]
            p.sigma[a][b] = bp.sigma[a][b]
            p.rcut[a][b] = bp.rcut[a][b]
    return p


def min_image_rms(a, b, L):
    d = a - b
    d -= L * np.round(d / L)
    return float(np.sqrt((d * d).sum(1).mean()))
