"""The C-ABI library loads and exports every function include/cvq.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cvq_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["cvq_init_sector", "cvq_set_pool", "cvq_apply_H", "cvq_screen_pool", "cvq_apply_ansatz",
              "cvq_energy_and_grad", "cvq_workspace_bytes", "cvq_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2606_05297_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_shares_no_code_with_cuda_path():
    """The oracle neither imports the product package's compute modules nor
    includes its headers, and vice versa (only workloads is shared)."""
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                for line in src.splitlines():
                    if line.strip().startswith("#include"):
                        assert "cvq" not in line.split("#include", 1)[1].replace("cvq_oracle", ""), (f, line)
                    if "paper_2606_05297_gb300" in line and "import" in line:
                        assert "workloads" in line, (f, line)
    pkg = os.path.join(ROOT, "paper_2606_05297_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "from oracle" not in src and "import oracle" not in src, f


def test_status_of_cuda_errors():
    """CUDA errors that leave the context unusable map to CVQ_EDEVICE (5), an
    allocation failure to CVQ_ENOMEM (2), everything else to CVQ_ECUDA (3);
    host only, no device needed.  Values are cudaError_t codes of CUDA 13."""
    from paper_2606_05297_gb300 import build
    lib = ctypes.CDLL(build.build())
    f = lib.cvq_status_from_cuda
    f.argtypes, f.restype = [ctypes.c_int], ctypes.c_int
    assert f(0) == 0                      # cudaSuccess
    assert f(1) == 3                      # cudaErrorInvalidValue
    assert f(2) == 2                      # cudaErrorMemoryAllocation
    for code in (700, 710, 715, 716, 719, 214):  # illegal address, assert, illegal instruction, misaligned, launch failure, ECC
        assert f(code) == 5, code
