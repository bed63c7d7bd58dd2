"""The C-ABI library loads on the CPU and exports every symbol include/*.h declares.

No compute call is made (there is no GPU here); this only checks the boundary.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(pfsp_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("pfsp_load_instance", "pfsp_free_instance", "pfsp_bound_batch", "pfsp_stats",
                     "pfsp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2012_09511_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2012_09511_gb300 import pfsp
    for name in declared_functions():
        if name in ("pfsp_solve_batch_dev",):
            continue
        assert hasattr(pfsp, name) or hasattr(pfsp.lib(), name), name


def test_host_side_validation_without_gpu():
    # argument checks that run before any device work
    from paper_2012_09511_gb300 import pfsp
    import numpy as np
    with pytest.raises(pfsp.PfspError) as e:
        pfsp.pfsp_load_instance(np.zeros((0, 3), dtype=np.int32))
    assert e.value.code == pfsp.PFSP_ERR_INVALID
    with pytest.raises(pfsp.PfspError) as e:
        pfsp.pfsp_load_instance(-np.ones((3, 3), dtype=np.int32))
    assert e.value.code == pfsp.PFSP_ERR_INVALID
    with pytest.raises(pfsp.PfspError) as e:
        pfsp.pfsp_load_instance(np.ones((65, 3), dtype=np.int32))
    assert e.value.code == pfsp.PFSP_ERR_UNSUPPORTED
    with pytest.raises(pfsp.PfspError) as e:
        pfsp.pfsp_load_instance(np.ones((5, 33), dtype=np.int32))
    assert e.value.code == pfsp.PFSP_ERR_UNSUPPORTED
    with pytest.raises(pfsp.PfspError) as e:
        pfsp.pfsp_load_instance(np.full((5, 3), 1 << 23, dtype=np.int32))
    assert e.value.code == pfsp.PFSP_ERR_UNSUPPORTED


def test_entry_points_reject_null_instances_without_gpu():
    # the instance check runs before any device work, for every entry point
    # that takes one
    from paper_2012_09511_gb300 import pfsp
    import ctypes
    lib = pfsp._lib
    buf = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    assert lib.pfsp_bound_batch(None, 3, 1, buf, buf, buf, out, out) == pfsp.PFSP_ERR_INVALID
    assert lib.pfsp_bound_reduce(None, 2, 1, buf, buf, buf, 100, out) == pfsp.PFSP_ERR_INVALID
    assert lib.pfsp_bound_reduce_dev(None, 2, 1, buf, buf, buf, 100, out, None) == pfsp.PFSP_ERR_INVALID
    o = pfsp.pfsp_default_options()
    best = ctypes.c_int32()
    oc = ctypes.c_int()
    assert lib.pfsp_solve(None, ctypes.byref(o), ctypes.byref(best), out, ctypes.byref(oc)) == pfsp.PFSP_ERR_INVALID
    assert pfsp.SUMMARY_DTYPE.itemsize == 48
