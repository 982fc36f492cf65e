"""The C interface: the library builds for sm_103a, loads without a GPU and
exports every entry point the header declares; the Python binding keeps the
C names and has no CPU fallback."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2203_06117_gb300 as gs

HEADER = os.path.join(gs.INCLUDE, "gatspi.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gatspi_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    return gs.build()


def test_header_declares_the_interface():
    names = declared_functions()
    for core in ["gatspi_load_netlist", "gatspi_load_delays", "gatspi_set_stimulus",
                 "gatspi_simulate", "gatspi_saif"]:
        assert core in names
    assert sorted(gs.EXPORTS) == names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(gatspi_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_is_built_for_sm_103a_only(built):
    # every translation unit is compiled with exactly one -gencode, for sm_103a
    flags = gs.NVCC_FLAGS
    gencodes = [flags[i + 1] for i, f in enumerate(flags) if f == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]
    assert not any(f.startswith(("-arch", "--gpu-architecture")) for f in flags)


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = gs.lib().gatspi_create(ctypes.byref(h), 0, 0)
    assert rc in (gs.EINVAL, gs.ECUDA)
    assert not h.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(gs, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(gs, "_lib", None)
    with pytest.raises(ImportError):
        gs.lib()


def test_product_code_never_touches_the_oracle():
    pkg = os.path.dirname(gs.__file__)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "event_sim" not in src and "osim_" not in src, f
