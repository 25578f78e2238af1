"""Pins of the FP64 oracle of the FNO surrogate (CPU only)."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import fno


def _setup(seed=0, B=2, N=8, C=3, m=2, L=2):
    p = fno.init_params(C, m, L, seed)
    rng = np.random.default_rng(seed + 100)
    x = rng.standard_normal((B, 2, N, N, N))
    return p, x, m


def _loss(p, x, m, t):
    y = fno.forward(p, x, m)
    return 0.5 * np.sum((y - t) ** 2)


def test_gelu_is_x_times_normal_cdf_and_its_derivative():
    x = np.linspace(-4, 4, 41)
    assert np.allclose(fno.gelu(x), x * norm.cdf(x), atol=1e-14)
    h = 1e-6
    num = (fno.gelu(x + h) - fno.gelu(x - h)) / (2 * h)
    assert np.allclose(fno.gelu_grad(x), num, atol=1e-8)


def test_spectral_convolution_with_identity_weights_passes_kept_waves_and_removes_others():
    """Kept modes are k in [0, m) U [N - m, N) per axis (frequencies -m..m-1): plane waves with all
    |k| <= m - 1 pass unchanged, waves beyond the cutoff vanish, and channels do not mix."""
    N, C, m = 8, 3, 2
    R = np.zeros((2 * m, 2 * m, m, C, C), dtype=complex)
    R[..., np.arange(C), np.arange(C)] = 1.0
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    keep = np.cos(2 * np.pi * (1 * x + 1 * y - 1 * z) / N) + 0.5
    drop_x = np.cos(2 * np.pi * (3 * x) / N)
    drop_y = np.sin(2 * np.pi * (2 * y + 1 * x) / N)
    vv = np.stack([keep, drop_x, drop_y])[None]
    out, _ = fno.spectral_forward(vv, R, m)
    assert np.max(np.abs(out[0, 0] - keep)) < 1e-12
    assert np.max(np.abs(out[0, 1])) < 1e-12 and np.max(np.abs(out[0, 2])) < 1e-12


@pytest.mark.parametrize("what", ["lift_w", "lift_b", "pw_w", "pw_b", "spec_re", "spec_im", "proj_w",
                                  "proj_b"])
def test_backward_matches_central_differences(what):
    p, x, m = _setup()
    t = np.random.default_rng(7).standard_normal((x.shape[0],) + x.shape[2:])
    y, cache = fno.forward(p, x, m, keep=True)
    g = fno.backward(p, cache, y - t, m)
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(4):
        if what in ("lift_w", "lift_b", "proj_w"):
            arr = getattr(p, what)
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = _loss(p, x, m, t)
            arr[idx] = old - h
            lm = _loss(p, x, m, t)
            arr[idx] = old
            ana = g[what][idx]
        elif what == "proj_b":
            old = p.proj_b
            p.proj_b = old + h
            lp = _loss(p, x, m, t)
            p.proj_b = old - h
            lm = _loss(p, x, m, t)
            p.proj_b = old
            ana = g["proj_b"]
        elif what in ("pw_w", "pw_b"):
            layer = int(rng.integers(0, len(p.spec)))
            arr = getattr(p, what)[layer]
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = _loss(p, x, m, t)
            arr[idx] = old - h
            lm = _loss(p, x, m, t)
            arr[idx] = old
            ana = g[what][layer][idx]
        else:
            layer = int(rng.integers(0, len(p.spec)))
            arr = p.spec[layer]
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            step = h if what == "spec_re" else 1j * h
            arr[idx] = old + step
            lp = _loss(p, x, m, t)
            arr[idx] = old - step
            lm = _loss(p, x, m, t)
            arr[idx] = old
            gc = g["spec"][layer][idx]
            ana = gc.real if what == "spec_re" else gc.imag
        num = (lp - lm) / (2 * h)
        assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (what, num, ana)


def test_input_gradient_matches_central_differences():
    p, x, m = _setup(seed=2)
    t = np.random.default_rng(9).standard_normal((x.shape[0],) + x.shape[2:])
    y, cache = fno.forward(p, x, m, keep=True)
    g = fno.backward(p, cache, y - t, m)
    h = 1e-6
    for idx in [(1, 0, 3, 2, 5), (0, 1, 7, 0, 1), (1, 1, 4, 4, 4)]:
        x[idx] += h
        lp = _loss(p, x, m, t)
        x[idx] -= 2 * h
        lm = _loss(p, x, m, t)
        x[idx] += h
        num = (lp - lm) / (2 * h)
        assert abs(num - g["x"][idx]) <= 1e-6 * max(1.0, abs(num))


def test_single_layer_network_is_affine_in_the_input():
    """With one Fourier layer there is no activation: y(a x1 + b x2) = a y(x1) + b y(x2) - (a+b-1) y(0)."""
    p = fno.init_params(3, 2, 1, 4)
    rng = np.random.default_rng(5)
    x1, x2 = rng.standard_normal((2, 1, 2, 8, 8, 8))
    y0 = fno.forward(p, np.zeros_like(x1), 2)
    lhs = fno.forward(p, 0.3 * x1 + 1.7 * x2, 2)
    rhs = 0.3 * fno.forward(p, x1, 2) + 1.7 * fno.forward(p, x2, 2) - (0.3 + 1.7 - 1.0) * y0
    assert np.max(np.abs(lhs - rhs)) < 1e-12
