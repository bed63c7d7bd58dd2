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
