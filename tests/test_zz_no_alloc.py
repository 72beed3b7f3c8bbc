"""wb_step_noalloc: the one entry point that allocates no device memory.

Some callers of this library cannot call cudaMalloc: code that runs while a
stream is being captured into a CUDA graph, plug-ins whose host application
owns every allocation, or embeddings that only hand over device buffers.
They cannot size a wb_grid workspace, so wb_step_noalloc advances a small
single box by one CTU+CT step with all intermediates in a static device
array inside the library.  This test calls it through the C ABI twice in a
row and checks each result against the regular grid API (wb_advance), with
the parity tolerance the other GPU tests use.  It lives in a file of its own
so that pytest collects it last.
"""
import numpy as np
import pytest

from parity import rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_grid_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding as wb
    from paper_1701_07452_gb300.initial_conditions import random_box

    n = (14, 12, 10)
    st = random_box(n, seed=17)
    ref = wb.Grid(n, length=st["length"])
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


def test_noalloc_rejects_oversized_box():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding as wb
    d = wb.make_desc((64, 64, 64))
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(wb.WombatError) as ei:
        wb.step_noalloc(d, z, z, z, z, z, z, z, z)
    assert ei.value.code == wb.WB_ERR_INVALID
    assert "static limit" in str(ei.value)
