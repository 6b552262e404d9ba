"""The C-ABI library loads and exports every function declared in include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(zeta_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    z = pytest.importorskip("paper_2602_24155_gb300")
    lib = ctypes.CDLL(z.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert names == set(z.EXPORTS)


def test_device_entry_points_fail_cleanly_without_a_gpu():
    z = pytest.importorskip("paper_2602_24155_gb300")
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(z.ZetaError) as e:
        z.zeta_create(0)
    assert e.value.status == 5  # ZETA_ERR_DEVICE: no CPU fallback
