"""The C-ABI library loads and exports exactly the entry points include/gim.h declares.

No compute call is made here, so this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gim_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2009_07325_gb300 import build
    build.build()
    from paper_2009_07325_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("gim_create", "gim_destroy", "gim_graph_load", "gim_sample_rr", "gim_select_seeds", "gim_imm",
                 "gim_rr_export", "gim_coverage_export", "gim_reset_rr", "gim_last_error_string"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_no_undeclared_exports(lib):
    """Every gim_* symbol the library exports is declared in include/ (no undocumented entry points)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2009_07325_gb300 import binding
    out = subprocess.run([nm, "-D", "--defined-only", lib._name], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("gim_") and " T " in ln}
    assert exported, "no gim_* exports found"
    assert exported == _declared(), (sorted(exported - _declared()), sorted(_declared() - exported))


def test_binding_covers_every_declared_symbol():
    from paper_2009_07325_gb300 import binding
    assert set(binding.SIGNATURES) == _declared()


def test_library_has_no_oracle_dependency():
    """The product library and binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2009_07325_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gim_oracle" not in text and "orc_" not in text, f


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.gim_create(ctypes.byref(h), 0, None) != 0
    assert not h.value


def test_build_covers_every_translation_unit_for_sm_103a():
    from paper_2009_07325_gb300 import build
    cus = {f for f in os.listdir(build.CSRC) if f.endswith(".cu")}
    assert set(build.SOURCES) == cus and len(build.SOURCES) == len(cus)
    f = build.flags()
    assert "arch=compute_103a,code=sm_103a" in f and f[f.index("arch=compute_103a,code=sm_103a") - 1] == "-gencode"
    assert "-lineinfo" in f and not any(x.startswith("-march") for x in f)
    assert sum(1 for x in f if x == "-gencode") == 1       # one target: GB300 only


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libgim.so the binding raises instead of computing anything."""
    from paper_2009_07325_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="libgim.so not found"):
        binding.load_library(str(tmp_path / "libgim.so"))
