"""The paper-scale grid edges 80 and 96 (Sec. III: the 520-electron system on ~0.85M points)
against the FP64 oracle, through the C ABI (GPU only).

In the mixed mode these grids run the lane-pair split FFT passes (one pencil over two lanes); in the
FP64 mode they run the generic shared-memory Stockham passes (no register FFT fits an FP64 pencil
of 80 or 96 points). Both are compared element-wise with the oracle on small windows of occupied
orbitals, short runs and every switch of the step (cleaning interval, coefficient law, feedback):
FP64 within 1e-10 relative, mixed within 2e-3 (the tolerances of the smaller grids)."""
import numpy as np
import pytest

import sbse_inputs as si
from oracle import tdh
from conftest import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


_SYS = {}


def _system(N):
    if N not in _SYS:
        p = si.model_system.Preset(f"g{N}", N=N, box=0.25 * N, n_wells=8, seed=N, n_occ=6, n_o=3, n_c=4)
        _SYS[N] = si.make_system(p)
    return _SYS[N]


def _run(B, s, precision, prm, pairs, n_occ=6, n_o=3, n_c=4, tma=1):
    with B.Context(0, precision) as c:
        B.sbse_set_option(c.h, B.SBSE_OPT_TMA_PLANES, tma)
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(n_occ, n_o, n_c, s.phi[:n_occ + n_c], s.eps[:n_occ + n_c], 0.5)
        return c.apply_W(prm, pairs, copy_out=True)


@pytest.mark.parametrize("N,M,dist,fb", [
    (80, 3, 0, 1),   # cleaning every 3 steps (0, 3, 6), Gaussian coefficients, TDH feedback
    (80, 0, 1, 0),   # no cleaning, +-1 signs, frozen potential
    (96, 4, 1, 1),   # cleaning every 4 steps, +-1 signs, feedback
    (96, 1, 0, 0),   # cleaning before every step, Gaussian, no feedback
])
def test_split_grids_match_oracle(B, N, M, dist, fb):
    s = _system(N)
    prm = B.TDHParams(n_s=3, n_steps=8, clean_every=M, dt=0.05, gamma=0.1, alpha=1e-4, seed=N + M,
                      coeff_dist=dist, feedback=fb)
    pairs = [(0, 0), (0, 2), (1, 2)]  # odd count: the last Poisson slot packs one density
    W64 = _run(B, s, B.SBSE_FP64, prm, pairs)
    W32 = _run(B, s, B.SBSE_MIXED, prm, pairs)
    # the z sweep with its columns staged by bulk tensor copies (default) or loaded by the threads:
    # the same arithmetic, the same result
    W32r = _run(B, s, B.SBSE_MIXED, prm, pairs, tma=0)
    assert np.array_equal(W32, W32r)
    coeff = tdh.stochastic_coefficients(prm.seed, prm.n_s, 6, "sign" if dist else "gaussian")
    op = tdh.TDHParams(n_steps=prm.n_steps, dt=prm.dt, gamma=prm.gamma, alpha=prm.alpha,
                       clean_every=M, feedback=bool(fb))
    ref = tdh.screened_potentials(tdh.Grid(N, s.box), s.v_loc, s.phi, 6, 3, coeff, op, pairs=pairs)
    for k, pr in enumerate(pairs):
        assert rel_err(W64[k].reshape(N, N, N), ref[pr]) < 1e-10
        assert rel_err(W32[k].reshape(N, N, N), ref[pr]) < 2e-3


def test_split_grid_exchange_and_excitons(B):
    """(ia|jb) through the Poisson passes of the split grid (mixed: FP32 FFTs + tensor-core grid
    sums) against the FP64 GPU path (generic passes + FP64 grid sums) and the oracle's exchange
    matrix on 96^3; then a whole short run's excitons, mixed vs FP64, within 5 meV."""
    s = _system(96)
    n_occ, n_o, n_c = 6, 3, 4
    K = {}
    for prec in (B.SBSE_FP64, B.SBSE_MIXED):
        with B.Context(0, prec) as c:
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(n_occ, n_o, n_c, s.phi[:n_occ + n_c], s.eps[:n_occ + n_c], 0.5)
            K[prec] = c.build_A(B.SBSE_EXCHANGE)
    phi_o, _, phi_c, _ = tdh.windows(s.phi, s.eps, n_occ, n_o, n_c)
    kref = tdh.exchange_K(tdh.Grid(96, s.box), phi_o, phi_c)
    off = lambda a: a - np.diag(np.diag(a))
    assert rel_err(off(K[B.SBSE_FP64]) / 2, off(kref)) < 1e-10
    assert rel_err(off(K[B.SBSE_MIXED]), off(K[B.SBSE_FP64])) < 1e-4
    prm = B.TDHParams(n_s=4, n_steps=30, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=5)
    ev = {}
    for prec in (B.SBSE_FP64, B.SBSE_MIXED):
        with B.Context(0, prec) as c:
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(n_occ, n_o, n_c, s.phi[:n_occ + n_c], s.eps[:n_occ + n_c], 0.5)
            c.apply_W(prm, tdh.pair_list(n_o))
            c.build_A()
            ev[prec] = c.spectrum(6)
    assert np.max(np.abs(ev[B.SBSE_MIXED] - ev[B.SBSE_FP64])) < 5.0 / 27211.386245988


def test_generic_passes_fp64_at_64(B):
    """FP64 at 64^3 takes the generic five-sweep passes (an FP64 register pencil of 64 does not
    fit): W against the oracle within 1e-10 on two pairs."""
    p = si.model_system.Preset("g64", N=64, box=16.0, n_wells=8, seed=64, n_occ=5, n_o=2, n_c=3)
    s = si.make_system(p)
    prm = B.TDHParams(n_s=3, n_steps=6, clean_every=4, dt=0.05, gamma=0.1, alpha=1e-4, seed=9)
    pairs = [(0, 1), (1, 1)]
    W = _run(B, s, B.SBSE_FP64, prm, pairs, n_occ=5, n_o=2, n_c=3)
    coeff = tdh.stochastic_coefficients(9, 3, 5, "gaussian")
    op = tdh.TDHParams(n_steps=6, dt=0.05, gamma=0.1, alpha=1e-4, clean_every=4)
    ref = tdh.screened_potentials(tdh.Grid(64, 16.0), s.v_loc, s.phi, 5, 2, coeff, op, pairs=pairs)
    for k, pr in enumerate(pairs):
        assert rel_err(W[k].reshape(64, 64, 64), ref[pr]) < 1e-10
