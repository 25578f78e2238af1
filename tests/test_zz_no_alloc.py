"""The allocation-free eigensolver entry point against the context-based one (GPU only).

sbse_spectrum_noalloc serves callers that cannot allocate device memory: its scratch is a fixed
device array inside the library. This test builds A with a context, takes its eigenvalues with
sbse_spectrum, then calls the allocation-free variant twice in a row on the same matrix (held in a
device buffer that the test allocates) and checks both results against the first, within the
1e-10 relative tolerance of the FP64 parity tests; around the second call the device's free memory
must not change. It lives in its own file so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_context_spectrum_twice(tiny16):
    torch = pytest.importorskip("torch")
    from paper_2205_06690_gb300 import binding as B

    s = tiny16
    p = s.preset
    prm = B.TDHParams(n_s=10, n_steps=30, clean_every=10, dt=p.dt, gamma=p.gamma, alpha=p.alpha,
                      seed=5)
    pairs = [(i, j) for i in range(p.n_o) for j in range(i, p.n_o)]
    n = p.n_o * p.n_c
    k = 6
    with B.Context(0, B.SBSE_FP64) as c:
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, p.scissor)
        c.apply_W(prm, pairs)
        A = c.build_A()
        ref = c.spectrum(k)
    a_dev = torch.from_numpy(np.ascontiguousarray(A)).to("cuda:0")
    ev_dev = [torch.full((k,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in range(2)]
    for call in range(2):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        B.sbse_spectrum_noalloc(a_dev.data_ptr(), n, k, ev_dev[call].data_ptr(), 0)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the module (lazy loading); the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        got = ev_dev[call].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert torch.equal(a_dev.cpu(), torch.from_numpy(A))  # input not modified
    with pytest.raises(B.SbseError) as e:
        B.sbse_spectrum_noalloc(a_dev.data_ptr(), 513, k, ev_dev[0].data_ptr(), 0)
    assert e.value.code == B.SBSE_ERR_SHAPE
