"""CPU checks of the C ABI boundary: the library loads and exports every
function declared in include/superscs.h (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1903_06477_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(scs_[A-Za-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libsuperscs.so not built (run __graft_entry__.build())")
    L = ctypes.CDLL(binding.LIB_PATH)
    names = sorted(set(_declared("superscs.h")) | set(_declared("superscs_mlp.h")))
    assert len(names) >= 24
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every declared entry point
    assert sorted(n for n, _, _ in binding._SIGS) == sorted(names)


def test_struct_layouts_match_header():
    """Field counts of the ctypes mirrors equal the header's struct members."""
    txt = open(os.path.join(ROOT, "include", "superscs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)

    def members(struct_name):
        m = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct_name + r";", txt)
        body = m.group(1)
        count = 0
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            count += decl.count(",") + 1
        return count

    assert members("scs_settings") == len(binding.Settings._fields_)
    assert members("scs_info") == len(binding.Info._fields_)
    assert members("scs_cone") == len(binding.Cone._fields_)
    assert members("scs_data") == len(binding.Data._fields_)


def test_default_settings_without_gpu():
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libsuperscs.so not built")
    s = binding.default_settings()
    assert s.direction == binding.DIR_AA and s.mem == 10 and s.eps == 1e-5
    assert s.c0 == 0.99 and s.sigma == 1e-2 and s.lam == 1.0 and s.ls_max == 20


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(binding.SCSError):
        binding.lib()


def test_mlp_gemm_entries_reject_bad_arguments_without_gpu():
    """Argument checks run before any device call, so they hold on a host
    without a GPU: an unknown kernel, a row stride that is not a multiple of
    8, a stride below K, a missing output, misaligned operands."""
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libsuperscs.so not built")
    L = binding.lib()
    p = ctypes.c_void_p(4096)  # never dereferenced: every call below fails its checks first
    bad = [
        (7, 4, 4, 8, p, 8, p, 8, p, 4),      # unknown kernel
        (0, 4, 4, 8, p, 12, p, 8, p, 4),     # lda not a multiple of 8
        (1, 4, 4, 16, p, 8, p, 16, p, 4),    # lda < K
        (1, 4, 4, 8, p, 8, p, 8, None, 4),   # no output
        (1, 4, 4, 8, ctypes.c_void_p(4100), 8, p, 8, p, 4),  # A not 16-byte aligned
        (0, 4, 5, 8, p, 8, p, 8, p, 4),      # ldc < N
        (0, -1, 4, 8, p, 8, p, 8, p, 4),     # negative M
    ]
    for args in bad:
        assert L.scs_mlp_gemm_nt(*args, None) == binding.SCS_EINVAL, args
    assert L.scs_mlp_set_gemm(None, 1) == binding.SCS_EINVAL
