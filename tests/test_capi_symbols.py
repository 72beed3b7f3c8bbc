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


def test_workspace_size_with_and_without_kept_stages():
    """Workspace bytes follow the documented count of intermediate arrays:
    54 doubles per padded zone when the corrector stages reuse the predictor
    arrays, 81 with keep_stages (state: 11)."""
    from paper_1701_07452_gb300 import binding
    n = (40, 40, 40)
    V = 50 ** 3
    lean = binding.grid_bytes(binding.make_desc(n))
    keep = binding.grid_bytes(binding.make_desc(n, keep_stages=True))
    assert abs((keep - lean) - (81 - 54) * 8 * V) < 4096   # the work region is rounded up
    assert (11 + 54) * 8 * V <= lean < (11 + 54) * 8 * V + (1 << 22)
    d = binding.make_desc(n)
    d.keep_stages = 2
    try:
        binding.grid_bytes(d)
    except binding.WombatError as e:
        assert e.code == binding.WB_ERR_INVALID
    else:
        raise AssertionError("keep_stages = 2 accepted")


def test_descriptor_edge_cases_rejected_without_gpu():
    """Empty, ragged and out-of-range descriptors fail with WB_ERR_INVALID
    before any device work (no GPU needed)."""
    from paper_1701_07452_gb300 import binding
    bad = [
        dict(n=(0, 8, 8)),                        # empty axis
        dict(n=(8, -4, 8)),
        dict(n=(30, 32, 32), patches=(4, 1, 1)),  # patches must divide n
        dict(n=(8, 8, 8), patches=(0, 1, 1)),
        dict(n=(8, 8, 8), length=(1.0, 0.0, 1.0)),
        dict(n=(8, 8, 8), gamma=1.0),
        dict(n=(8, 8, 8), gamma=2.5),
        dict(n=(8, 8, 8), cfl=0.0),
        dict(n=(8, 8, 8), eps=(0.1, 0.0, 0.5, 0.0, 0.1, 0.0, 0.1)),
        dict(n=(8, 8, 8), sweby=0.5),
        dict(n=(8, 8, 8), bc=(0, 2, 0)),
        dict(n=(8, 8, 8), batch_patches=-1),
        dict(n=(8, 8, 8), prot_rho=-1.0),
        dict(n=(8, 8, 8), rho_floor=-1.0),
        dict(n=(8, 8, 8), p_floor=float("nan")),
        dict(n=(20000, 20000, 20000)),            # beyond any device: refused, no overflow
    ]
    for kw in bad:
        kw = dict(kw)
        n = kw.pop("n")
        d = binding.make_desc(n, **kw)
        try:
            binding.grid_bytes(d)
        except binding.WombatError as e:
            assert e.code == binding.WB_ERR_INVALID, kw
        else:
            raise AssertionError(f"accepted: n={n} {kw}")
    # ragged (non-cubic, odd) sizes and one-zone axes are valid
    for n in ((7, 5, 3), (1, 1, 9), (33, 1, 1)):
        assert binding.grid_bytes(binding.make_desc(n)) > 0
