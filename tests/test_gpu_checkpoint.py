"""Checkpoint / resume of a propagation (GPU only): a run split into ranges, with the state saved to
host memory and loaded into a new context between them, gives the W of one uninterrupted run to
the bit, in FP64 and in the mixed mode (the partial FP32 time integral is part of the state); a
continuation without a matching state is refused."""
import numpy as np
import pytest

import sbse_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def _ctx(B, s, p, precision, persistent=0):
    c = B.Context(0, precision)
    B.sbse_set_option(c.h, B.SBSE_OPT_PERSISTENT, persistent)  # the persistent step kernel, where it exists
    c.set_grid(p.N, p.box, s.v_loc)
    c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, 0.5)
    return c


@pytest.mark.parametrize("N,precision_name,fb,persistent", [(16, "SBSE_FP64", 1, 0), (16, "SBSE_MIXED", 1, 0),
                                                            (20, "SBSE_MIXED", 0, 0), (80, "SBSE_MIXED", 1, 0),
                                                            (32, "SBSE_MIXED", 1, 1)])
def test_split_run_with_saved_state_matches_one_run(B, N, precision_name, fb, persistent):
    precision = getattr(B, precision_name)
    p = si.model_system.Preset(f"ck{N}", N=N, box=0.5 * N if N < 64 else 0.25 * N, n_wells=4, seed=N,
                               n_occ=6, n_o=3, n_c=2)
    s = si.make_system(p)
    prm = B.TDHParams(n_s=4, n_steps=37, clean_every=5, dt=0.05, gamma=0.1, alpha=1e-4, seed=9, feedback=fb)
    pairs = [(0, 1), (1, 1), (0, 2)]
    ng = N ** 3
    with _ctx(B, s, p, precision, persistent) as c:
        w_one = c.apply_W(prm, pairs, copy_out=True)
    # ranges ending inside a cleaning interval, on a cleaning step and at a flush boundary of the
    # FP32 time integral (16 steps)
    cuts = [0, 7, 15, 16, 30, 37]
    with _ctx(B, s, p, precision, persistent) as c:
        assert B.sbse_apply_W_range(c.h, prm, pairs, cuts[0], cuts[1]) is None
        B.sbse_apply_W_range(c.h, prm, pairs, cuts[1], cuts[2])
        state = B.sbse_save_state(c.h)
    with _ctx(B, s, p, precision, persistent) as c2:  # a fresh context, as after a restart
        B.sbse_load_state(c2.h, state)
        for a, b in zip(cuts[2:-2], cuts[3:-1]):
            B.sbse_apply_W_range(c2.h, prm, pairs, a, b)
        w_split = B.sbse_apply_W_range(c2.h, prm, pairs, cuts[-2], cuts[-1], n_g=ng)
        assert np.array_equal(w_split, w_one)
        # the finished run holds no state; a continuation is refused
        with pytest.raises(B.SbseError):
            B.sbse_apply_W_range(c2.h, prm, pairs, 30, 37)


def test_resume_needs_the_same_parameters_and_pairs(B):
    p = si.model_system.Preset("ck", N=16, box=8.0, n_wells=4, seed=3, n_occ=6, n_o=3, n_c=2)
    s = si.make_system(p)
    prm = B.TDHParams(n_s=4, n_steps=20, clean_every=5, dt=0.05, gamma=0.1, alpha=1e-4, seed=9)
    pairs = [(0, 1), (1, 1)]
    with _ctx(B, s, p, B.SBSE_MIXED) as c:
        B.sbse_apply_W_range(c.h, prm, pairs, 0, 8)
        for bad in (dict(n_begin=9), dict(pairs=[(0, 1)]), dict(prm=B.TDHParams(
                n_s=4, n_steps=20, clean_every=5, dt=0.05, gamma=0.1, alpha=1e-4, seed=10))):
            with pytest.raises(B.SbseError):
                B.sbse_apply_W_range(c.h, bad.get("prm", prm), bad.get("pairs", pairs), bad.get("n_begin", 8), 20)
        with pytest.raises(B.SbseError):
            B.sbse_apply_W_range(c.h, prm, pairs, 0, 21)  # past n_steps
        state = B.sbse_save_state(c.h)
        with pytest.raises(B.SbseError):
            B.sbse_load_state(c.h, state[:100])  # truncated
        B.sbse_apply_W_range(c.h, prm, pairs, 8, 20)  # the state left in the context continues
