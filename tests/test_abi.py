"""The C ABI library builds for sm_103a, loads, and exports exactly what the header declares.

No GPU work is done here: only the shared library's symbol table and the sources are
inspected.
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


@pytest.mark.parametrize("cname,pyname", [("ph_opts", "PhOpts"), ("ph_stats", "PhStats"),
                                          ("ph_allocator", "PhAllocator")])
def test_struct_layout_matches_binding(tmp_path, cname, pyname):
    # the C compiler's view of the header (size and every field's offset) against ctypes'
    import shutil
    import subprocess

    from paper_1708_04710_gb300 import native

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    py = getattr(native, pyname)
    names = [f[0] for f in py._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ph_gb300.h"',
             "int main(void) {", f'  printf("%zu\\n", sizeof({cname}));']
    lines += [f'  printf("%zu\\n", offsetof({cname}, {n}));' for n in names]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [ctypes.sizeof(py)] + [getattr(py, n).offset for n in names]
    assert got == want, (cname, list(zip(["sizeof"] + names, got, want)))


def test_no_alloc_entry_point_source_allocates_nothing():
    """ph_beta_static's translation unit calls no allocation routine: no cudaMalloc* /
    cudaFree* (runtime or driver), no library context and none of its allocator hooks."""
    src = (ROOT / "paper_1708_04710_gb300" / "csrc" / "ph_noalloc.cu").read_text()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    banned = [r"\bcu(da)?Malloc\w*", r"\bcu(da)?Free\w*", r"\bcu(da)?MemAlloc\w*",
              r"\bcuMemCreate\b", r"\bdalloc\b", r"\bdfree\b", r"\balloc_n\b", r"\bph_ctx\b",
              r"\bnew\s+[A-Za-z_]", r"\bmalloc\s*\("]
    for pat in banned:
        assert not re.search(pat, code), f"ph_noalloc.cu matches {pat}"
    # the scratch is a file-scope device array, and host code passes its looked-up address
    assert re.search(r"__device__\s+__align__\(256\)\s+int32_t\s+g_left_scratch\[", code)
    assert "cudaGetSymbolAddress" in code


def _code_files(folder: Path):
    return [p for p in sorted(folder.rglob("*"))
            if p.suffix in (".py", ".cu", ".cuh", ".h", ".c") and "_build" not in p.parts]


def test_product_and_oracle_share_nothing():
    """The package and the header never import, load or include the oracle, the test tree or
    working files, and the oracle never uses the package: the two implementations meet only
    in the tests."""
    product = _code_files(ROOT / "paper_1708_04710_gb300") + _code_files(ROOT / "include")
    assert any(p.name == "ph_reduce.cu" for p in product)
    banned = [r"^\s*(import|from)\s+(oracle|tests|helpers|shard_cpu)\b", r"libph_oracle",
              r"ph_oracle\.[ch]", r"#\s*include\s*[<\"][^>\"]*oracle", r"\b_work\b"]
    for p in product:
        text = p.read_text()
        for pat in banned:
            assert not re.search(pat, text, flags=re.M), f"{p.relative_to(ROOT)} matches {pat}"
    for p in _code_files(ROOT / "oracle"):
        text = p.read_text()
        for pat in [r"paper_1708_04710_gb300", r"libph_gb300", r"ph_gb300\.h", r"ph_internal"]:
            assert not re.search(pat, text), f"{p.relative_to(ROOT)} matches {pat}"
