"""The C ABI library builds for sm_103a, loads, and exports exactly what the header declares.

No GPU work is done here: only the shared library's symbol table is inspected.
"""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared(header: Path):
    text = header.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ph_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1708_04710_gb300 import build

    return build.build()


def test_header_declarations_exported(lib_path):
    declared = []
    for h in sorted((ROOT / "include").glob("*.h")):
        declared += _declared(h)
    assert declared, "no declarations found"
    lib = ctypes.CDLL(str(lib_path))
    for name in declared:
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_binding_covers_header(lib_path):
    from paper_1708_04710_gb300 import native

    declared = set()
    for h in sorted((ROOT / "include").glob("*.h")):
        declared |= set(_declared(h))
    assert declared == set(native.SIGNATURES), declared ^ set(native.SIGNATURES)


def test_context_fails_loudly_without_gpu(lib_path):
    import torch

    from paper_1708_04710_gb300 import native

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        native.Context()
