"""Argument checks of the C ABI that run on the host before any device work (no GPU
needed): every malformed request is refused with BBMD_ERR_ARG and no handle."""
import ctypes as C

import numpy as np
import pytest

from inputs import generate as gen


@pytest.fixture(scope="module")
def lib():
    from paper_1105_5613_gb300 import bbmd
    from paper_1105_5613_gb300 import build as b

    b.build()
    bbmd._lib = None
    return bbmd, bbmd.load()


def create(bbmd, L, params, n, box, species, pos=None, T0=1.0):
    h = C.c_void_p()
    boxa = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
    sp = None if species is None else np.ascontiguousarray(species, dtype=np.uint8)
    posa = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64)
    rc = L.bbmd_create(C.byref(params), int(n), boxa.ctypes.data_as(C.POINTER(C.c_double)),
                       None if sp is None else sp.ctypes.data_as(C.POINTER(C.c_uint8)),
                       None if posa is None else posa.ctypes.data_as(C.POINTER(C.c_double)),
                       None, float(T0), C.c_uint64(0), None, None, C.byref(h))
    return rc, h.value


def good(bbmd):
    n = 4 * 8 ** 3
    return n, gen.box_for(n, 1.2), np.zeros(n, np.uint8)


@pytest.mark.parametrize("case", ["n1", "n0", "box0", "boxnan", "pot", "shift", "prec", "nbr",
                                  "skin", "mass", "sigma", "asym", "lcap", "scap", "bz",
                                  "species2", "nospecies", "T0", "posnan", "notfcc"])
def test_create_refuses_malformed_requests(lib, case):
    bbmd, L = lib
    n, box, sp = good(bbmd)
    p = bbmd.ka_params()
    pos = None
    T0 = 1.0
    if case == "n1":
        n, sp = 1, sp[:1]
    elif case == "n0":
        n, sp = 0, sp[:0]
    elif case == "box0":
        box = 0.5
    elif case == "boxnan":
        box = float("nan")
    elif case == "pot":
        p.potential = 7
    elif case == "shift":
        p.shift = 3
    elif case == "prec":
        p.precision = 2
    elif case == "nbr":
        p.nbr_mode = 5
    elif case == "skin":
        p.skin = -0.1
    elif case == "mass":
        p.mass[1] = 0.0
    elif case == "sigma":
        p.sigma[0][0] = 0.0
    elif case == "asym":
        p.eps[0][1] = 2.0
    elif case == "lcap":
        p.list_capacity = 5000
    elif case == "scap":
        p.stencil_capacity = 70000
    elif case == "bz":
        p.block_z = 3
    elif case == "species2":
        sp = sp.copy()
        sp[17] = 2
    elif case == "nospecies":
        sp = None
    elif case == "T0":
        T0 = -1.0
    elif case == "posnan":
        pos = gen.fcc_lattice(8, box)
        pos[5, 1] = np.nan
    elif case == "notfcc":  # device lattice needs n = 4 m^3
        n, sp = n - 4, sp[:-4]
    rc, h = create(bbmd, L, p, n, box, sp, pos, T0)
    assert rc == 1 and not h  # BBMD_ERR_ARG, no handle


def test_null_handles_are_refused(lib):
    bbmd, L = lib
    assert L.bbmd_step(None, 1, 0.005, None) == 1
    assert L.bbmd_rebuild(None) == 1
    assert L.bbmd_tune(None) == 1
    assert L.bbmd_last_error(None) == b""
    L.bbmd_destroy(None)
    L.bbmd_destroy_batch(None)
    assert L.bbmd_batch_size(None) == 0
    assert L.bbmd_batch_replica(None, 0) is None
    out = C.c_void_p()
    p = bbmd.ka_params()
    assert L.bbmd_create_batch(C.byref(p), 0, None, None, None, None, None, None, 0, None, None,
                               C.byref(out)) == 1
