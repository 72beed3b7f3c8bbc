"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every entry point declared in include/wombat.h (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wombat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("wb_grid_create", "wb_load_state", "wb_compute_dt", "wb_advance",
                 "wb_read_state", "wb_conserved_totals", "wb_grid_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1701_07452_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_knows_every_symbol():
    from paper_1701_07452_gb300 import binding
    assert set(binding.EXPORTED) == set(declared_functions())


def test_descriptor_validation_without_gpu():
    from paper_1701_07452_gb300 import binding
    d = binding.make_desc((32, 32, 32))
    assert binding.grid_bytes(d) > 11 * 42 ** 3 * 8
    bad = binding.make_desc((30, 32, 32), patches=(4, 1, 1))
    try:
        binding.grid_bytes(bad)
    except binding.WombatError as e:
        assert e.code == binding.WB_ERR_INVALID
    else:
        raise AssertionError("uneven patches accepted")
