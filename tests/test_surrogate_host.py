"""Host logic of the learned form (no GPU): the initial parameter vector follows the layout the
library documents for sbse_fno_set_params (lift W [width][2], lift b, per layer the spectral weights
[2m][2m][m][width][width] complex, the pointwise W and b, then the projection w and b)."""
import numpy as np

from paper_2205_06690_gb300 import surrogate as S


class _FakeNet:
    def __init__(self, width, modes, layers):
        self.width, self.modes, self.layers = width, modes, layers
        C, m = width, modes
        self.n_params = 2 * C + C + layers * (2 * (2 * m) * (2 * m) * m * C * C + C * C + C) + C + 1
        self.p = None

    def set_params(self, p):
        self.p = p


def test_init_params_layout():
    C, m, L = 6, 3, 2
    net = _FakeNet(C, m, L)
    p = S.init_params(net, seed=4)
    assert p.dtype == np.float32 and p.size == net.n_params and net.p is p
    o = 0
    lift_w = p[o:o + 2 * C]; o += 2 * C
    lift_b = p[o:o + C]; o += C
    assert np.all(lift_b == 0) and np.std(lift_w) > 0
    for _ in range(L):
        spec = p[o:o + 2 * (2 * m) * (2 * m) * m * C * C]; o += spec.size
        assert np.all(spec >= 0) and np.all(spec < 1.0 / (C * C))
        o += C * C  # pointwise W
        assert np.all(p[o:o + C] == 0); o += C
    o += C
    assert p[o] == 0 and o + 1 == p.size
    assert np.array_equal(S.init_params(_FakeNet(C, m, L), seed=4), p)  # seeded
