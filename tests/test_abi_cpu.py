"""CPU-side checks of the boundary: libntf.so loads without a GPU and exports
every function that include/ntf.h declares; the binding knows them all."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ntf.h")


def declared():
    names = []
    with open(HEADER) as fh:
        for line in fh:
            m = re.match(r"^NTF_API .*?\b(ntf_\w+)\(", line)
            if m:
                names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2001_04321_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = set(declared())
    for required in ("ntf_mttkrp", "ntf_gram", "ntf_bcd_update", "ntf_her_step", "ntf_objective", "ntf_solve",
                     "ntf_hadamard_grams", "ntf_her_extrapolate", "ntf_residual_sq", "ntf_tensor_to_bf16",
                     "ntf_tensor_norm_sq", "ntf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path]).decode()
    exported = set(re.findall(r"\bT (ntf_\w+)", out))
    missing = set(declared()) - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binding_matches_header(lib_path):
    import paper_2001_04321_gb300 as ntf
    L = ntf.load(lib_path)
    for name in declared():
        assert hasattr(L, name)
    assert set(ntf.EXPORTED) == set(declared())


def test_host_side_validation_without_gpu(lib_path):
    # argument checks run before any CUDA call: no GPU needed
    import ctypes as C
    import paper_2001_04321_gb300 as ntf
    L = ntf.load(lib_path)
    d = ntf._Tensor()
    d.order = 9                                  # order outside [2, 8]
    assert L.ntf_mttkrp(C.byref(d), None, 4, 0, None, None, 0, None) == 1
    assert b"order" in L.ntf_last_error()
    d.order = 3
    d.dims[0] = d.dims[1] = d.dims[2] = 4
    d.dtype = 0
    d.data = 16
    d.ld = 3                                     # ld < dims[N-1]
    assert L.ntf_mttkrp(C.byref(d), None, 4, 0, None, None, 0, None) == 1
    d.ld = 5                                     # 20-byte rows: not 16-byte aligned
    assert L.ntf_mttkrp(C.byref(d), None, 4, 0, None, None, 0, None) == 1
    assert b"16 bytes" in L.ntf_last_error()
    assert L.ntf_mttkrp_workspace_bytes(C.byref(d), 4, 0) == 0
    o = ntf._Opts()
    L.ntf_opts_default(C.byref(o))
    assert (o.her, o.inner_max, o.beta0, o.gamma, o.gamma_bar, o.eta) == (1, 1, 0.5, 1.05, 1.01, 1.5)
    assert L.ntf_bf16_ld(C.byref(d)) == 8


def test_oracle_builds_and_is_separate():
    import oracle
    path = oracle.build()
    assert os.path.exists(path)
    src = open(os.path.join(ROOT, "oracle", "ntf_oracle.c")).read()
    includes = re.findall(r"#include\s*[<\"]([^>\"]+)", src)
    assert includes and all(h in ("math.h", "stdint.h", "stdlib.h", "string.h") for h in includes)
    # the oracle package imports neither the CUDA package nor torch
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2001_04321_gb300" not in py and "import torch" not in py
