"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI (GPU only).

Tolerances: FP64 mode, 1e-10 relative (max-norm) on W_ij, A and the excitons; mixed mode (FP32
propagation), exciton energies within 5 meV = 1.8375e-4 Ha of the oracle and W within 2e-3
relative (the FP32 round-off of N_t split-operator steps, each ~6e-8 relative, grows like sqrt(N_t)
to ~1e-5 and the induced potential is a difference-form quantity, so 2e-3 leaves margin).
"""
import numpy as np
import pytest

import sbse_inputs as si
from oracle import tdh
from conftest import rel_err

pytestmark = pytest.mark.gpu

MEV = 1.0 / 27211.386245988


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def _small_system(N, box, n_wells, seed, n_occ, n_o, n_c):
    p = si.model_system.Preset(f"s{N}", N=N, box=box, n_wells=n_wells, seed=seed, n_occ=n_occ,
                               n_o=n_o, n_c=n_c)
    return si.make_system(p)


def _gpu(B, sys_, precision, prm, n_occ, n_o, n_c, scissor, k, pairs=None, terms=3):
    pairs = tdh.pair_list(n_o) if pairs is None else pairs
    with B.Context(0, precision) as c:
        c.set_grid(sys_.N, sys_.box, sys_.v_loc)
        c.set_orbitals(n_occ, n_o, n_c, sys_.phi[:n_occ + n_c], sys_.eps[:n_occ + n_c], scissor)
        W = c.apply_W(prm, pairs, copy_out=True)
        A = c.build_A(terms) if len(pairs) == n_o * (n_o + 1) // 2 else None
        ev = c.spectrum(k) if A is not None else None
    return W, A, ev


def _oracle(sys_, prm, n_occ, n_o, n_c, scissor, k, pairs=None):
    g = tdh.Grid(sys_.N, sys_.box)
    dist = "sign" if prm.coeff_dist == 1 else "gaussian"
    coeff = tdh.stochastic_coefficients(prm.seed, prm.n_s, n_occ, dist)
    op = tdh.TDHParams(n_steps=prm.n_steps, dt=prm.dt, gamma=prm.gamma, alpha=prm.alpha,
                       clean_every=prm.clean_every, feedback=bool(prm.feedback))
    return tdh.run(g, sys_.v_loc, sys_.phi, sys_.eps, n_occ, n_o, n_c, scissor, coeff, op, k,
                   pairs=pairs)


def test_fp64_full_path_tiny16(B, tiny16):
    """The smallest workload, whole path: 16^3 grid, 8 electrons, 3 pairs, 200 steps."""
    s = tiny16
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=p.n_steps, clean_every=10, dt=p.dt, gamma=p.gamma,
                      alpha=p.alpha, seed=0)
    W, A, ev = _gpu(B, s, B.SBSE_FP64, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    ref = _oracle(s, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    for k, pr in enumerate(tdh.pair_list(p.n_o)):
        assert rel_err(W[k].reshape(s.N, s.N, s.N), ref["W"][pr]) < 1e-10
    assert rel_err(A, ref["A"]) < 1e-10
    assert rel_err(ev, ref["excitons"]) < 1e-10


@pytest.mark.parametrize("N,box,n_occ,n_o,n_c,M,dist,fb,L", [
    (10, 6.0, 3, 3, 2, 7, 1, 1, 5),    # radix 2*5, 6 pairs, cleaning off the step grid, +-1 signs
    (12, 7.0, 4, 2, 3, 0, 0, 1, 3),    # radix 4*3, odd pair count, no cleaning
    (20, 8.0, 2, 1, 4, 1, 0, 0, 1),    # radix 4*5, one pair, clean every step, no feedback, L=1
    (24, 8.0, 5, 3, 1, 4, 1, 1, 7),    # radix 4*2*3, n_c = 1
])
def test_fp64_ragged_grids_and_switches(B, N, box, n_occ, n_o, n_c, M, dist, fb, L):
    s = _small_system(N, box, 3, N, n_occ, n_o, n_c)
    prm = B.TDHParams(n_s=L, n_steps=23, clean_every=M, dt=0.05, gamma=0.2, alpha=1e-4, seed=N,
                      coeff_dist=dist, feedback=fb)
    k = min(3, n_o * n_c)
    W, A, ev = _gpu(B, s, B.SBSE_FP64, prm, n_occ, n_o, n_c, 0.3, k)
    ref = _oracle(s, prm, n_occ, n_o, n_c, 0.3, k)
    for j, pr in enumerate(tdh.pair_list(n_o)):
        assert rel_err(W[j].reshape(N, N, N), ref["W"][pr]) < 1e-10
    assert rel_err(A, ref["A"]) < 1e-10
    assert rel_err(ev, ref["excitons"]) < 1e-10


def test_fp64_single_step_and_pair_subset(B, tiny16):
    s = tiny16
    prm = B.TDHParams(n_s=4, n_steps=1, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=3)
    W, _, _ = _gpu(B, s, B.SBSE_FP64, prm, 4, 2, 4, 0.5, 2, pairs=[(1, 1)])
    ref = _oracle(s, prm, 4, 2, 4, 0.5, 2, pairs=[(1, 1)])
    assert rel_err(W[0].reshape(16, 16, 16), ref["W"][(1, 1)]) < 1e-10


def test_mixed_precision_tiny16_excitons_within_5meV(B, tiny16):
    s = tiny16
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=p.n_steps, clean_every=10, dt=p.dt, gamma=p.gamma,
                      alpha=p.alpha, seed=0)
    W, A, ev = _gpu(B, s, B.SBSE_MIXED, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    ref = _oracle(s, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    for k, pr in enumerate(tdh.pair_list(p.n_o)):
        assert rel_err(W[k].reshape(s.N, s.N, s.N), ref["W"][pr]) < 2e-3
    assert np.max(np.abs(ev - ref["excitons"])) < 5 * MEV


def test_couplings_off_gives_energy_differences(B, tiny16):
    s = tiny16
    with B.Context(0, B.SBSE_MIXED) as c:
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(4, 2, 4, s.phi, s.eps, 0.5)
        A = c.build_A(0)
        ev = c.spectrum(8)
    d = np.array([s.eps[4 + a] - s.eps[2 + i] + 0.5 for i in range(2) for a in range(4)])
    assert np.array_equal(A, np.diag(d))
    assert np.max(np.abs(ev - np.sort(d))) < 1e-14


def test_call_order_and_argument_errors(B, tiny16):
    s = tiny16
    with B.Context(0, B.SBSE_FP64) as c:
        with pytest.raises(B.SbseError) as e:
            c.set_orbitals(4, 2, 4, s.phi, s.eps, 0.5)
        assert e.value.code == B.SBSE_ERR_NOT_READY
        with pytest.raises(B.SbseError) as e:
            c.set_grid(14, 8.0, np.zeros(14 ** 3))
        assert e.value.code == B.SBSE_ERR_SHAPE
        v = s.v_loc.copy()
        v[0, 0, 0] = np.nan
        with pytest.raises(B.SbseError) as e:
            c.set_grid(16, 8.0, v)
        assert e.value.code == B.SBSE_ERR_NUMERIC
        c.set_grid(16, 8.0, s.v_loc)
        c.set_orbitals(4, 2, 4, s.phi, s.eps, 0.5)
        with pytest.raises(B.SbseError) as e:
            c.spectrum(2)
        assert e.value.code == B.SBSE_ERR_NOT_READY
        with pytest.raises(B.SbseError) as e:
            c.build_A(B.SBSE_DIRECT)
        assert e.value.code == B.SBSE_ERR_NOT_READY
        prm = B.TDHParams(n_s=2, n_steps=2)
        for bad in ([(1, 0)], [(0, 2)], [(0, 1), (0, 1)]):
            with pytest.raises(B.SbseError) as e:
                c.apply_W(prm, bad)
            assert e.value.code == B.SBSE_ERR_INVALID_ARG
        with pytest.raises(B.SbseError) as e:
            c.apply_W(B.TDHParams(n_s=0), [(0, 0)])
        assert e.value.code == B.SBSE_ERR_INVALID_ARG
        c.build_A(B.SBSE_EXCHANGE)
        ev = np.empty(2)
        ec = np.empty(16)  # eigenvectors: (n_o n_c) x k = 8 x 2, row-major
        assert B.load().sbse_spectrum(c.h, 2, B._dptr(ev), B._dptr(ec)) == B.SBSE_OK
        X = ec.reshape(8, 2)
        assert np.max(np.abs(X.T @ X - np.eye(2))) < 1e-10
        assert B.load().sbse_spectrum(c.h, 0, B._dptr(ev), None) == B.SBSE_ERR_INVALID_ARG


@pytest.fixture(scope="module")
def mid48():
    return si.make_system(si.preset("mid48"))


def test_mid48_full_launch_sampled_pair_fp64_and_mixed(B, mid48):
    """The 48^3, 120-electron workload in the launch configuration of the benchmark (all 36 pairs
    in one call, L = 10, cleaning every 10 steps), shortened to 100 steps so that the oracle can
    recompute one sampled pair; plus the exciton energies of the two precision modes."""
    s = mid48
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=100, clean_every=10, dt=p.dt, gamma=p.gamma, alpha=p.alpha,
                      seed=1)
    W64, A64, ev64 = _gpu(B, s, B.SBSE_FP64, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    W32, A32, ev32 = _gpu(B, s, B.SBSE_MIXED, prm, p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc)
    pairs = tdh.pair_list(p.n_o)
    k = pairs.index((5, 7))
    g = tdh.Grid(s.N, s.box)
    coeff = tdh.stochastic_coefficients(1, 10, p.n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=100, dt=p.dt, gamma=p.gamma, alpha=p.alpha, clean_every=10)
    phi_o = s.phi[p.n_occ - p.n_o:p.n_occ]
    rho = phi_o[5] * phi_o[7]
    w_ref = tdh.coulomb_periodic(rho, g) + tdh.tdh_w_pol(g, s.v_loc, s.phi[:p.n_occ], rho, coeff, op)
    assert rel_err(W64[k].reshape(48, 48, 48), w_ref) < 1e-10
    assert rel_err(W32[k].reshape(48, 48, 48), w_ref) < 2e-3
    assert np.max(np.abs(A64 - A64.T)) < 1e-12
    assert np.max(np.abs(ev32 - ev64)) < 5 * MEV


@pytest.mark.parametrize("name", ["tiny16", "mid48"])
def test_tensor_core_exchange_contraction_matches_fp64(B, name, tiny16, mid48):
    """(ia|jb) by the tcgen05 BF16-split GEMM (mixed mode) against the FP64 CUDA-core GEMM and the
    oracle: the exchange matrix depends on the orbitals only, so the difference is the contraction
    arithmetic alone (expected ~1e-6 relative for three-term BF16 splitting with FP32 sums)."""
    s = tiny16 if name == "tiny16" else mid48
    p = s.preset
    K = {}
    for prec, tc in ((B.SBSE_FP64, 1), (B.SBSE_MIXED, 1), (B.SBSE_MIXED, 0)):
        with B.Context(0, prec) as c:
            B.sbse_set_option(c.h, B.SBSE_OPT_TENSOR_CORES, tc)
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c],
                           p.scissor)
            K[(prec, tc)] = c.build_A(B.SBSE_EXCHANGE)
    diag = np.diag(np.diag(K[(B.SBSE_FP64, 1)]))
    if name == "tiny16":
        phi_o, _, phi_c, _ = tdh.windows(s.phi, s.eps, p.n_occ, p.n_o, p.n_c)
        kref = tdh.exchange_K(tdh.Grid(s.N, s.box), phi_o, phi_c)
        assert rel_err((K[(B.SBSE_FP64, 1)] - np.diag(np.diag(K[(B.SBSE_FP64, 1)]))) / 2,
                       kref - np.diag(np.diag(kref))) < 1e-10
    ref = K[(B.SBSE_FP64, 1)] - diag
    assert rel_err(K[(B.SBSE_MIXED, 1)] - diag, ref) < 1e-4
    assert rel_err(K[(B.SBSE_MIXED, 0)] - diag, ref) < 1e-4


def test_pair_chunking_does_not_change_results(B, mid48):
    """Advancing the pairs in L2-sized chunks (SBSE_OPT_CHUNK_MB) runs the same kernels on the same
    items: the FP64 results are bitwise identical to advancing all pairs at once."""
    s = mid48
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=12, clean_every=5, dt=p.dt, gamma=p.gamma, alpha=p.alpha, seed=2)
    out = []
    for mb in (0, 20):
        with B.Context(0, B.SBSE_FP64) as c:
            B.sbse_set_option(c.h, B.SBSE_OPT_CHUNK_MB, mb)
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c],
                           p.scissor)
            out.append(c.apply_W(prm, tdh.pair_list(p.n_o)[:7], copy_out=True))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_step_matches_pass_kernels(B, mid48, prec):
    """The persistent step kernel runs the same tile arithmetic as the three pass kernels, only
    scheduled from a queue: results are bitwise identical (7 pairs, odd count; cleaning every 5)."""
    s = mid48
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=12, clean_every=5, dt=p.dt, gamma=p.gamma, alpha=p.alpha, seed=4)
    precision = B.SBSE_FP64 if prec == "fp64" else B.SBSE_MIXED
    out = []
    for persistent in (0, 1):
        with B.Context(0, precision) as c:
            B.sbse_set_option(c.h, B.SBSE_OPT_PERSISTENT, persistent)
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c],
                           p.scissor)
            out.append(c.apply_W(prm, tdh.pair_list(p.n_o)[3:10], copy_out=True))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("N,box", [(32, 10.0), (40, 12.0), (64, 16.0)])
def test_tma_streamed_inverse_pass_matches_plain_kernel(B, N, box):
    """The inverse plane pass fed by bulk asynchronous copies (SBSE_OPT_TMA_PLANES, mixed mode) runs
    the same transforms and density sums as the plain plane kernel: W agrees to FP32 round-off. Odd
    pair count (5) and L = 3, so that the persistent grid's last units are uneven; on 32^3 and 40^3
    W also matches the FP64 oracle within the mixed tolerance."""
    n_occ, n_o, n_c = 6, 3, 4
    s = _small_system(N, box, 5, N, n_occ, n_o, n_c)
    prm = B.TDHParams(n_s=3, n_steps=24, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=2)
    pairs = tdh.pair_list(n_o)[:5]
    out = []
    for tma in (0, 1):
        with B.Context(0, B.SBSE_MIXED) as c:
            B.sbse_set_option(c.h, B.SBSE_OPT_TMA_PLANES, tma)
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(n_occ, n_o, n_c, s.phi[:n_occ + n_c], s.eps[:n_occ + n_c], 0.5)
            out.append(c.apply_W(prm, pairs, copy_out=True))
    assert rel_err(out[1], out[0]) < 1e-6
    if N <= 40:
        coeff = tdh.stochastic_coefficients(prm.seed, prm.n_s, n_occ, "gaussian")
        op = tdh.TDHParams(n_steps=prm.n_steps, dt=prm.dt, gamma=prm.gamma, alpha=prm.alpha,
                           clean_every=prm.clean_every)
        ref = tdh.screened_potentials(tdh.Grid(N, box), s.v_loc, s.phi, n_occ, n_o, coeff, op,
                                      pairs=pairs)
        for k, pr in enumerate(pairs):
            assert rel_err(out[1][k].reshape(N, N, N), ref[pr]) < 2e-3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(B, prec):
    """SBSE_OPT_GRAPH: the captured time loop replayed on later calls gives the results of direct
    launches, bitwise; a new seed (coefficients are uploaded outside the graph) replays correctly,
    and a new step count is captured afresh. 32^3 system, 5 pairs, cleaning every 4 steps."""
    s = _small_system(32, 10.0, 5, 7, 6, 3, 4)
    precision = B.SBSE_FP64 if prec == "fp64" else B.SBSE_MIXED
    pairs = tdh.pair_list(3)[:5]

    def run(graph, seeds, steps):
        out = []
        with B.Context(0, precision) as c:
            B.sbse_set_option(c.h, B.SBSE_OPT_GRAPH, graph)
            c.set_grid(s.N, s.box, s.v_loc)
            c.set_orbitals(6, 3, 4, s.phi[:10], s.eps[:10], 0.5)
            for seed, n in zip(seeds, steps):
                prm = B.TDHParams(n_s=4, n_steps=n, clean_every=4, dt=0.05, gamma=0.1, alpha=1e-4, seed=seed)
                out.append(c.apply_W(prm, pairs, copy_out=True))
        return out

    seeds, steps = [1, 1, 2, 2], [14, 14, 14, 9]
    direct = run(0, seeds, steps)
    graph = run(1, seeds, steps)
    for a, b in zip(direct, graph):
        assert np.array_equal(a, b)
    assert np.array_equal(graph[0], graph[1]) and not np.array_equal(graph[1], graph[2])


def test_pair_shards_reassemble_the_single_run(B, tiny16):
    """The multi-GPU split of a system (paper_2205_06690_gb300.shard): blocks of pairs propagated by
    separate contexts (here two 'ranks' run in turn on one GPU), each contracting its own
    direct-element columns (sbse_get_direct); the gathered columns given to a context that holds no
    W at all (sbse_set_direct) give the A and excitons of one run over all pairs. FP64; the packing
    of two pair densities per Poisson transform differs between the runs, hence 1e-12, not bitwise.
    The W blocks themselves also reassemble (sbse_set_W)."""
    from paper_2205_06690_gb300 import shard
    s = tiny16
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=60, clean_every=10, dt=p.dt, gamma=p.gamma, alpha=p.alpha, seed=0)
    pairs = shard.pair_list(p.n_o)

    def ctx():
        c = B.Context(0, B.SBSE_FP64)
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi[:p.n_occ + p.n_c], s.eps[:p.n_occ + p.n_c], p.scissor)
        return c

    with ctx() as c:
        W_ref = c.apply_W(prm, pairs, copy_out=True)
        A_ref = c.build_A()
        ev_ref = c.spectrum(p.n_exc)
        D_ref = B.sbse_get_direct(c.h, pairs, p.n_c)
    blocks, cols = [], []
    for r in range(2):
        mine = [pairs[i] for i in shard.pair_block(len(pairs), r, 2)]
        with ctx() as c:
            blocks.append(c.apply_W(prm, mine, copy_out=True))
            cols.append(B.sbse_get_direct(c.h, mine, p.n_c))
    W = np.concatenate(blocks)
    assert rel_err(W, W_ref) < 1e-12
    D = np.concatenate(cols, axis=1)
    assert rel_err(D, D_ref) < 1e-12
    with ctx() as c:
        B.sbse_set_direct(c.h, D)
        A = c.build_A()
        ev = c.spectrum(p.n_exc)
    assert rel_err(A, A_ref) < 1e-12 and rel_err(ev, ev_ref) < 1e-12
    with ctx() as c:
        B.sbse_set_W(c.h, pairs, W)
        A = c.build_A()
    assert rel_err(A, A_ref) < 1e-12
