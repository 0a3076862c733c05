"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/lbm.h declares; argument validation that happens before
any CUDA call is checked here too (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lbm_create", "lbm_set_bc", "lbm_step", "lbm_fields", "lbm_destroy",
              "lbm_set_fields", "lbm_batch_create", "lbm_batch_step", "lbm_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2506_03905_gb300 as pkg
    L = pkg.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_create_rejects_bad_configs_before_touching_the_gpu():
    import paper_2506_03905_gb300 as pkg
    import lbm_cases as C
    good = C.channel_3d(nx=8, ny=8, nz=4)
    bad = [
        pkg.config_from_case(good.replace(nx=0)),
        pkg.config_from_case(good.replace(nu=-1.0)),
        pkg.config_from_case(good.replace(mach=0.0)),
    ]
    c = pkg.config_from_case(good)
    c.lattice = 27
    bad.append(c)
    c = pkg.config_from_case(good)
    c.collision = 7
    bad.append(c)
    c = pkg.config_from_case(good.replace(lattice="D2Q9", nz=1))
    c.nz = 2
    bad.append(c)
    for cfg in bad:
        h = ctypes.c_void_p()
        st = pkg.lib().lbm_create(ctypes.byref(cfg), ctypes.byref(h))
        assert st == pkg.LBM_EINVAL and not h.value
        assert pkg.lbm_last_error(None)
    # NULL handles are rejected, destroy(NULL) is a no-op
    assert pkg.lib().lbm_step(None, 1) == pkg.LBM_EINVAL
    assert pkg.lib().lbm_fields(None, 0, None, 0) == pkg.LBM_EINVAL
    pkg.lib().lbm_destroy(None)
