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


def test_vector_executor_stays_within_its_register_budget():
    """k_execute (CUDA-core path) must use <= 96 registers and no local spills: above that a 160-thread block takes
    more than a quarter of the register file and the quintic batch loses a resident block per SM (about 40 %)."""
    import re
    import shutil
    import subprocess
    import tempfile
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(ROOT, "paper_2602_24155_gb300", "csrc", "zeta_kernels.cu")
    with tempfile.TemporaryDirectory() as tmp:
        out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xptxas", "-v",
                              "-c", src, "-o", os.path.join(tmp, "k.o")], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stderr.splitlines()
    seen = 0
    for i, line in enumerate(lines):
        if "Compiling entry function" in line and "k_executeILi4ELb" in line and "ELb0EE" in line:
            block = " ".join(lines[i:i + 4])
            regs = int(re.search(r"Used (\d+) registers", block).group(1))
            spills = re.search(r"(\d+) bytes spill stores", block)
            assert regs <= 96, (line, regs)
            assert spills is None or int(spills.group(1)) == 0
            seen += 1
    assert seen == 2


def test_int8_tensor_mma_is_not_available_on_sm_103a():
    """The exact-integer tensor path takes fp16 digits (tcgen05.mma kind::f16) because ptxas refuses
    kind::i8 (INT8 x INT8 -> INT32) for sm_103a; the same instruction assembles for sm_100a."""
    import shutil
    import subprocess
    import tempfile
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    src = r'''
#include <cstdint>
__global__ void k(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
'''
    results = {}
    with tempfile.TemporaryDirectory() as tmp:
        for kind in ("i8", "f16"):
            for arch in ("103a", "100a"):
                path = os.path.join(tmp, "mma_%s.cu" % kind)
                open(path, "w").write(src.replace("KIND", kind))
                out = subprocess.run([nvcc, "-c", "-gencode", "arch=compute_%s,code=sm_%s" % (arch, arch), path, "-o",
                                      os.path.join(tmp, "o.o")], capture_output=True, text=True, timeout=300)
                results[(kind, arch)] = (out.returncode, out.stderr)
    assert results[("i8", "103a")][0] != 0 and "not supported" in results[("i8", "103a")][1]
    assert results[("i8", "100a")][0] == 0
    assert results[("f16", "103a")][0] == 0
