"""The C-ABI library builds, loads and exports every entry point include/zfact.h declares.
CPU only: no compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "zfact.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zfact_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_19163_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_expected_api():
    syms = declared_symbols()
    for s in ("zfact_create", "zfact_refine", "zfact_refine_batched", "zfact_propose", "zfact_destroy",
              "zfact_last_error"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    cdll, path = lib
    for s in declared_symbols():
        assert hasattr(cdll, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (zfact_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_covers_every_symbol():
    from paper_2404_19163_gb300 import zfact
    assert set(zfact.EXPORTED) == set(declared_symbols())


def test_default_opts_without_gpu(lib):
    from paper_2404_19163_gb300 import zfact
    o = zfact.make_opts()
    assert o.nmax == 50 and o.stop_rule == 0 and o.fixed_iters == 0 and o.final_residual == 1


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2404_19163_gb300 import Context, ZfactError
    with pytest.raises(ZfactError):
        Context(0)


def test_binding_raises_when_library_missing(tmp_path):
    from paper_2404_19163_gb300 import zfact
    saved = zfact._lib
    zfact._lib = None
    try:
        with pytest.raises(ImportError):
            zfact.load(str(tmp_path / "nope.so"))
    finally:
        zfact._lib = saved


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2404_19163_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "zfact_oracle" not in txt and "liboracle" not in txt, f


def header_enum(prefix):
    src = open(os.path.join(ROOT, "include", "zfact.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {name: int(val) for name, val in re.findall(r"\b(%s[A-Z0-9_]+)\s*=\s*(\d+)" % prefix, src)}


@pytest.mark.parametrize("table,prefix", [("PRECISION", "ZFACT_P_"), ("REFINE_MODE", "ZFACT_R_"),
                                          ("EMULATION", "ZFACT_EMU_")])
def test_binding_names_match_header_enums(table, prefix):
    """The binding's name -> value tables are the header's enumerators, value for value."""
    from paper_2404_19163_gb300 import zfact
    enum = header_enum(prefix)
    mapping = getattr(zfact, table)
    assert enum and {prefix + k.upper(): v for k, v in mapping.items()} == enum
