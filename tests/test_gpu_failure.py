"""Failure paths of the library, made to happen without faulting or hanging the GPU (GPU only).

* A bounded device wait that runs out: the persistent step kernel waits for the tiles it depends on
  with an iteration limit; SBSE_OPT_WAIT_LIMIT = 1 makes those waits give up almost at once. The
  kernel skips the work of such tiles and still ends, sbse_apply_W reports SBSE_ERR_DEVICE_TIMEOUT,
  and the same context then runs correctly with the default limit and is destroyed normally.
* An allocation that fails: SBSE_OPT_MEM_LIMIT_MB caps the device memory a context may hold; a call
  that needs more fails with SBSE_ERR_OOM, and after the cap is lifted the same context runs.
"""
import numpy as np
import pytest

from oracle import tdh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def _ctx(B, s, precision):
    p = s.preset
    c = B.Context(0, precision)
    c.set_grid(s.N, s.box, s.v_loc)
    c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, p.scissor)
    return c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_timed_out_wait_reports_device_timeout_and_context_recovers(B, tiny16, prec):
    s = tiny16
    p = s.preset
    precision = B.SBSE_FP64 if prec == "fp64" else B.SBSE_MIXED
    prm = B.TDHParams(n_s=10, n_steps=12, clean_every=5, dt=p.dt, gamma=p.gamma, alpha=p.alpha, seed=4)
    pairs = tdh.pair_list(p.n_o)
    with _ctx(B, s, precision) as c:
        ref = c.apply_W(prm, pairs, copy_out=True)
    with _ctx(B, s, precision) as c:
        B.sbse_set_option(c.h, B.SBSE_OPT_PERSISTENT, 1)
        B.sbse_set_option(c.h, B.SBSE_OPT_WAIT_LIMIT, 1)
        with pytest.raises(B.SbseError) as e:
            c.apply_W(prm, pairs)
        assert e.value.code == B.SBSE_ERR_DEVICE_TIMEOUT
        B.sbse_set_option(c.h, B.SBSE_OPT_WAIT_LIMIT, 0)
        W = c.apply_W(prm, pairs, copy_out=True)
    assert np.array_equal(W, ref)


def test_memory_limit_reports_oom_and_context_recovers(B, tiny16):
    s = tiny16
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=8, clean_every=5, dt=p.dt, gamma=p.gamma, alpha=p.alpha, seed=1)
    pairs = tdh.pair_list(p.n_o)
    with _ctx(B, s, B.SBSE_MIXED) as c:
        ref = c.apply_W(prm, pairs, copy_out=True)
    with _ctx(B, s, B.SBSE_MIXED) as c:
        with pytest.raises(B.SbseError) as e:
            B.sbse_set_option(c.h, B.SBSE_OPT_MEM_LIMIT_MB, -1)
        assert e.value.code == B.SBSE_ERR_INVALID_ARG
        B.sbse_set_option(c.h, B.SBSE_OPT_MEM_LIMIT_MB, 1)  # the propagated orbitals alone need 2 MiB
        with pytest.raises(B.SbseError) as e:
            c.apply_W(prm, pairs)
        assert e.value.code == B.SBSE_ERR_OOM
        assert "memory limit" in B.sbse_last_error(c.h)
        B.sbse_set_option(c.h, B.SBSE_OPT_MEM_LIMIT_MB, 0)
        W = c.apply_W(prm, pairs, copy_out=True)
    assert np.array_equal(W, ref)
