"""Chebyshev absorption spectrum (Sec. II.C) through the C ABI vs the FP64 oracle (GPU only)."""
import numpy as np
import pytest

from oracle import spectrum, tdh
from conftest import rel_err

pytestmark = pytest.mark.gpu

EV = 1.0 / 27.211386245988


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def tiny_case(tiny16):
    """tiny16 in FP64: the GPU context with A built, and the oracle's own A on the same inputs."""
    s = tiny16
    p = s.preset
    prm_kw = dict(n_steps=p.n_steps, clean_every=10, dt=p.dt, gamma=p.gamma, alpha=p.alpha)
    coeff = tdh.stochastic_coefficients(0, 10, p.n_occ, "gaussian")
    ref = tdh.run(tdh.Grid(s.N, s.box), s.v_loc, s.phi, s.eps, p.n_occ, p.n_o, p.n_c, p.scissor, coeff,
                  tdh.TDHParams(**prm_kw), p.n_exc)
    return s, prm_kw, ref["A"]


def _gpu_ctx(B, s, prm_kw):
    p = s.preset
    c = B.Context(0, B.SBSE_FP64)
    c.set_grid(s.N, s.box, s.v_loc)
    c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c], p.scissor)
    c.apply_W(B.TDHParams(n_s=10, seed=0, **prm_kw), tdh.pair_list(p.n_o))
    c.build_A()
    return c


@pytest.mark.parametrize("axis", [0, 2])
def test_absorption_matches_oracle_fp64(B, tiny_case, axis):
    """Residues R_n and sigma(omega) on 0.08 eV broadening, 2048 terms, 8 x 8 A of the 16^3 system;
    FP64 on both sides, so the agreement is set by the 1e-10 agreement of A."""
    s, prm_kw, A_ref = tiny_case
    p = s.preset
    n_terms, width = 2048, 0.08 * EV
    c0, w0 = spectrum.scaling(A_ref)
    omega = np.linspace(c0 - w0, c0 + w0, 401)
    grid = tdh.Grid(s.N, s.box)
    phi_o, _, phi_c, _ = tdh.windows(s.phi, s.eps, p.n_occ, p.n_o, p.n_c)
    sig_ref, R_ref, f0 = spectrum.absorption(grid, phi_o, phi_c, A_ref, axis, n_terms, width, omega)
    with _gpu_ctx(B, s, prm_kw) as c:
        sig, R = c.absorption(axis, n_terms, width, omega)
        sig2, R2 = c.absorption(axis, n_terms, width, omega)  # repeat: scratch reused
    assert abs(R[0] - f0 @ f0) < 1e-10 * (f0 @ f0)
    assert rel_err(R, R_ref) < 1e-8
    assert rel_err(sig, sig_ref) < 1e-8
    assert np.array_equal(sig, sig2) and np.array_equal(R, R2)
    # the expansion resolves the broadened lines: equal to the oracle's eigenpair sum
    assert rel_err(sig, spectrum.sigma_exact(A_ref, f0, omega, width)) < 1e-6


def test_absorption_argument_errors(B, tiny16):
    s = tiny16
    p = s.preset
    with B.Context(0, B.SBSE_FP64) as c:
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c], p.scissor)
        with pytest.raises(B.SbseError, match="NOT_READY"):
            c.absorption(0, 64, 0.01, [0.5])
        c.build_A(B.SBSE_EXCHANGE)
        for args in [(3, 64, 0.01), (0, 1, 0.01), (0, 64, 0.0), (0, 64, -1.0), (0, 1 << 17, 0.01)]:
            with pytest.raises(B.SbseError, match="INVALID_ARG"):
                c.absorption(*args, [0.5])
        sig, R = c.absorption(1, 2, 0.01, [0.5, 1.0])
        assert np.all(np.isfinite(sig)) and R.shape == (2,)


def _small(N, box, n_wells, seed, n_occ, n_o, n_c):
    import sbse_inputs as si
    return si.make_system(si.model_system.Preset(f"v{N}", N=N, box=box, n_wells=n_wells, seed=seed,
                                                 n_occ=n_occ, n_o=n_o, n_c=n_c))


@pytest.mark.parametrize("case", ["tiny16_k4", "tiny16_all", "n32_k10"])
def test_exciton_eigenvectors(B, tiny16, case):
    """sbse_spectrum with eigenvectors (FP64 A with the exchange term): A x_j = lambda_j x_j to
    1e-10 |A|, orthonormal to 1e-10, eigenvalues equal to those of numpy's eigh of the same matrix,
    vectors equal to eigh's up to the sign convention (largest component positive) wherever the
    eigenvalue is separated from its neighbours."""
    if case.startswith("tiny16"):
        s, n_occ, n_o, n_c = tiny16, 4, 2, 4
        k = 4 if case == "tiny16_k4" else 8
    else:
        s, n_occ, n_o, n_c, k = _small(32, 10.0, 6, 3, 8, 4, 8), 8, 4, 8, 10
    with B.Context(0, B.SBSE_FP64) as c:
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(n_occ, n_o, n_c, s.phi[:n_occ + n_c], s.eps[:n_occ + n_c], 0.5)
        A = c.build_A(B.SBSE_EXCHANGE)
        ev, X = c.spectrum(k, vectors=True)
        ev2, X2 = c.spectrum(k, vectors=True)
    n = n_o * n_c
    assert X.shape == (n, k) and np.array_equal(X, X2) and np.array_equal(ev, ev2)
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A @ X - X * ev[None, :])) < 1e-10 * scale
    assert np.max(np.abs(X.T @ X - np.eye(k))) < 1e-10
    E, U = np.linalg.eigh(0.5 * (A + A.T))
    assert np.max(np.abs(ev - E[:k])) < 1e-10 * scale
    for j in range(k):
        gap = min(abs(E[j] - E[q]) for q in range(n) if q != j)
        if gap > 1e-6 * scale:
            u = U[:, j] * np.sign(U[np.argmax(np.abs(U[:, j])), j])
            assert np.max(np.abs(X[:, j] - u)) < 1e-8
        assert X[np.argmax(np.abs(X[:, j])), j] > 0
