"""Second-order convergence of MHD waves oblique to the 3D grid (Sec. "Linear
Wave Convergence", the GS08 setup): a 2N x N x N periodic grid of size
(3, 3/2, 3/2), wave vector k = (1/3, 2/3, 2/3) (wavelength 1), background
rho = 1, P = 3/5, B = (1, sqrt 2, 1/2) in the wave frame and at rest, face
field from an edge potential.  After one wave period the L1 error vector
against the initial state must fall with a slope of at least 1.8 between
N = 64 and 128, for the fast, Alfven and slow modes.  This pins the
multi-dimensional parts of the step (transverse predictor states with the
div B source, corner EMFs, constrained transport) to second order at sizes
the oracle cannot reach; the GPU path equals the oracle on the same step
(test_gpu_parity.py)."""
import math

import numpy as np
import pytest

import linear_waves as lw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


def oblique_error(wb, mode, n):
    rest = (0.0, 0.0, 0.0)
    lam, U, bx, by, bz = lw.state_oblique(mode, n, v=rest)
    g = wb.Grid((2 * n, n, n), length=(3.0, 1.5, 1.5), gamma=lw.GAMMA)
    g.load(U, bx, by, bz)
    B0 = g.read()[4]
    T = 1.0 / abs(lam)
    assert abs(g.advance(10 ** 7, t_end=T) - T) < 1e-12
    assert g.counters()["unphysical"] == 0
    U1, _, _, _, B1 = g.read()
    return lw.l1_error(U1, U, B1, B0)


@pytest.mark.parametrize("mode", ["fast", "alfven", "slow"])
def test_oblique_wave_second_order(wb, mode):
    e64 = oblique_error(wb, mode, 64)
    e128 = oblique_error(wb, mode, 128)
    slope = math.log2(e64 / e128)
    assert slope >= 1.8, (mode, e64, e128, slope)
    assert e128 < 2.5e-8, e128      # the error itself is at the size of the 1D modes'
