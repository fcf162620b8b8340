"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/bbmd.h declares (no compute calls)."""
import ctypes

import pytest

from tests.helpers import declared_symbols


def test_library_builds_and_exports_all_declared_symbols():
    from paper_1105_5613_gb300 import build as b
    from paper_1105_5613_gb300 import bbmd

    lib = b.build()
    L = ctypes.CDLL(lib)
    decl = declared_symbols()
    assert len(decl) >= 12
    for name in decl:
        assert hasattr(L, name), name
    assert set(bbmd.EXPORTS) == set(decl)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1105_5613_gb300 import bbmd

    with pytest.raises(RuntimeError):
        bbmd.load(str(tmp_path / "missing.so")) if bbmd._lib is None else (_ for _ in ()).throw(
            RuntimeError("already loaded"))


def test_params_struct_layout_matches_header():
    from paper_1105_5613_gb300 import bbmd

    # 4 int32 + 3*4 doubles + 2 doubles + 1 double + 2 int32
    assert ctypes.sizeof(bbmd.bbmd_params) == 16 + 12 * 8 + 2 * 8 + 8 + 16 + 8
    p = bbmd.ka_params()
    assert p.eps[0][1] == 1.5 and p.sigma[1][1] == 0.88 and p.rcut[0][1] == 2.0


def test_oracle_is_not_imported_by_the_product():
    import os

    root = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1105_5613_gb300")
    for dirpath, _, files in os.walk(root):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "bbmd_oracle" not in txt, f


def test_observe_args_layout_and_origin_count_match_header():
    import os
    import re

    from paper_1105_5613_gb300 import bbmd

    # int32 (+4 padding), 2 doubles, int32 (+4 padding)
    assert ctypes.sizeof(bbmd.bbmd_obs_args) == 32
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "bbmd.h")).read()
    assert int(re.search(r"#define BBMD_MAX_ORIGINS (\d+)", hdr).group(1)) == bbmd.MAX_ORIGINS
    assert int(re.search(r"BBMD_BATCH_PERSISTENT = (\d+)", hdr).group(1)) == bbmd.BATCH_PERSISTENT
