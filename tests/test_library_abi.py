"""The C-ABI library loads and exports every entry point include/nao.h declares (CPU only:
no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "nao.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nao_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nao_init", "nao_destroy", "nao_last_error", "nao_bloch_sum", "nao_gen_eig", "nao_density_matrix"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1402_4247_gb300 import build as b
    if b.is_stale():
        try:
            b.build()
        except RuntimeError as e:  # pragma: no cover - no nvcc
            pytest.skip(str(e))
    lib = ctypes.CDLL(b.LIB)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1402_4247_gb300 import nao
    assert set(nao.EXPORTS) == set(_declared())


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1402_4247_gb300 import nao
    with pytest.raises(ValueError):
        nao._ptr(torch.zeros(3))
