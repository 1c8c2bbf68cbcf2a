"""The C-ABI library loads without a GPU and exports every entry point of include/femamg.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "femamg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)
    keep = {n for n in names if n.startswith(("fem_", "amg_", "pcg_", "bddc_"))}
    return sorted(keep)


@pytest.fixture(scope="module")
def lib():
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as fa
    return fa.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["fem_assemble", "amg_setup", "pcg_solve", "fem_system_destroy",
                     "amg_hier_destroy", "fem_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2102_03515_gb300 import _binding
    assert set(_declared_functions()) == set(_binding.SIGNATURES)


def test_no_cpu_fallback_in_package():
    # the package never imports the oracle and has no CPU compute path
    pkg = os.path.join(ROOT, "paper_2102_03515_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracle is", ""), f


def test_version_and_error_strings_without_gpu(lib):
    import paper_2102_03515_gb300 as fa
    assert "sm_103a" in fa.fem_version()
    assert isinstance(fa.fem_last_error(), str)


def test_autotuner_pins_and_clears_without_a_gpu(lib):
    # the tuner's table is host state: pinning, unpinning, clearing and the JSON report need
    # no device
    import paper_2102_03515_gb300 as fa
    fa.fem_autotune_clear()
    rep = fa.fem_autotune_report()
    assert rep["entries"] == [] and rep["pins"] == {}
    fa.fem_autotune_pin("csr_f64", 3)
    fa.fem_autotune_pin("stencil_f32", 1)
    fa.fem_autotune_pin("csr_f64", 2)   # a second pin of a family replaces the first
    assert fa.fem_autotune_report()["pins"] == {"stencil_f32": 1, "csr_f64": 2}
    fa.fem_autotune_pin("stencil_f32", -1)
    assert fa.fem_autotune_report()["pins"] == {"csr_f64": 2}
    fa.fem_autotune_clear()
    assert fa.fem_autotune_report()["pins"] == {}
    from paper_2102_03515_gb300 import _binding as B
    assert lib.fem_autotune_pin(None, 0) == B.FEM_EINVAL


def test_build_targets_sm_103a_only_and_keeps_refinement_unfused():
    # every translation unit is compiled for sm_103a alone with line info; the refinement's
    # decisions are kept free of FMA contraction; every .cu file of the library is built
    from paper_2102_03515_gb300 import build as b
    srcs = sorted(f for f in os.listdir(b.SRC) if f.endswith(".cu"))
    assert sorted(b.SOURCES) == srcs
    for s in srcs:
        f = b._flags(s)
        gencodes = [f[i + 1] for i, t in enumerate(f) if t == "-gencode"]
        assert gencodes == ["arch=compute_103a,code=sm_103a"] and "-lineinfo" in f
        assert ("-fmad=false" in f) == (s in b.NO_FMAD)
    assert b.NO_FMAD == {"adapt.cu"}
