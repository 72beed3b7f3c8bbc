"""wb_step_noalloc: the one entry point that allocates no device memory.

Some callers of this library cannot call cudaMalloc: a plug-in inside a host
application that owns every device allocation, an embedding that is handed
device buffers and nothing else, or a real-time loop that may not take
cudaMalloc's implicit device synchronisation.  They cannot give a wb_grid its
workspace, so wb_step_noalloc advances a small single box by one CTU+CT step
with all intermediates in a static device array inside the library.  These
tests call it through the C ABI twice in a row on periodic, outflow and
one-plane (2D) boxes and check each result against the regular grid API
(wb_advance) with the parity tolerance the other GPU tests use, and check the
size limit at its boundary.  The file sorts last so that pytest collects it
last.
"""
import pytest

from parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("n,bc", [((14, 12, 10), (0, 0, 0)), ((13, 11, 9), (1, 0, 1)),
                                  ((20, 16, 1), (0, 0, 0))])
def test_noalloc_matches_grid_two_calls(wb, n, bc):
    import torch
    from paper_1701_07452_gb300.initial_conditions import random_box

    st = random_box(n, seed=17)
    ref = wb.Grid(n, length=st["length"], bc=bc)
    ref.load_state(st)
    U0, bx0, by0, bz0, _ = ref.read(on_device=True)
    dev = U0.device
    cur = [U0.clone(), bx0.clone(), by0.clone(), bz0.clone()]
    dt_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    for call in range(2):
        out = [torch.full_like(a, float("nan")) for a in cur]
        wb.step_noalloc(ref.desc, *cur, *out, dt_out=dt_dev)
        dt_ref_before = ref.dt()
        ref.advance(1)
        want = ref.read(on_device=True)
        torch.cuda.synchronize()
        assert abs(dt_dev.item() - dt_ref_before) <= 1e-14 * dt_ref_before
        for got, exp in zip(out, want[:4]):
            assert rel_err(got.cpu().numpy(), exp.cpu().numpy()) < 1e-11, call
        cur = out


def test_noalloc_size_limit_boundary(wb):
    """A 26^3 cube fits the 24 MiB array (and steps like the grid API); 27^3
    is refused with WB_ERR_INVALID and a message naming the limit."""
    import torch
    from paper_1701_07452_gb300.initial_conditions import random_box

    n = (26, 26, 26)
    st = random_box(n, seed=23)
    ref = wb.Grid(n, length=st["length"])
    ref.load_state(st)
    cur = [a.clone() for a in ref.read(on_device=True)[:4]]
    out = [torch.full_like(a, float("nan")) for a in cur]
    wb.step_noalloc(ref.desc, *cur, *out)
    ref.advance(1)
    want = ref.read(on_device=True)
    torch.cuda.synchronize()
    for got, exp in zip(out, want[:4]):
        assert rel_err(got.cpu().numpy(), exp.cpu().numpy()) < 1e-11
    d = wb.make_desc((27, 27, 27))
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(wb.WombatError) as ei:
        wb.step_noalloc(d, z, z, z, z, z, z, z, z)
    assert ei.value.code == wb.WB_ERR_INVALID
    assert "static limit" in str(ei.value)
