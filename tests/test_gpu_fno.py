"""FNO surrogate kernels (CUDA) against the FP64 oracle of the same network (GPU only).

The CUDA kernels use BF16 copies of the spectral and pointwise weights and FP32 sums; the oracle is
given the same BF16-rounded weights, so the remaining differences are FP32 rounding (relative
1e-4 on outputs, 2e-3 on gradients, which sum O(B N^3) FP32 terms)."""
import numpy as np
import pytest

from oracle import fno as ofno
from conftest import rel_err

pytestmark = pytest.mark.gpu


def _bf16(a):
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _pack(p: ofno.FNOParams):
    out = [p.lift_w.ravel(), p.lift_b]
    for R, W, b in zip(p.spec, p.pw_w, p.pw_b):
        out += [np.stack([R.real, R.imag], axis=-1).ravel(), W.ravel(), b]
    out += [p.proj_w, np.array([p.proj_b])]
    return np.concatenate(out).astype(np.float32)


def _unpack(v, C, m, L, round_bf16=False):
    v = v.astype(np.float64)
    o = 0

    def take(n):
        nonlocal o
        r = v[o:o + n]
        o += n
        return r
    lw = take(2 * C).reshape(C, 2)
    lb = take(C)
    spec, W, b = [], [], []
    for _ in range(L):
        r = take(2 * 4 * m ** 3 * C * C).reshape(2 * m, 2 * m, m, C, C, 2)
        w = take(C * C).reshape(C, C)
        if round_bf16:
            r = _bf16(r)
            w = _bf16(w)
        spec.append(r[..., 0] + 1j * r[..., 1])
        W.append(w)
        b.append(take(C))
    pw = take(C)
    pb = float(take(1)[0])
    return ofno.FNOParams(lw, lb, spec, W, b, pw, pb)


@pytest.mark.parametrize("N,C,m,L,B", [(8, 4, 2, 2, 2), (12, 6, 3, 3, 1)])
def test_fno_forward_and_gradients_match_oracle(N, C, m, L, B):
    torch = pytest.importorskip("torch")
    from paper_2205_06690_gb300 import binding as Bd
    net = Bd.FNO(N, width=C, modes=m, layers=L, max_batch=B)
    p = ofno.init_params(C, m, L, seed=N)
    vec = _pack(p)
    net.set_params(vec)
    pr = _unpack(vec, C, m, L, round_bf16=True)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((B, 2, N, N, N)).astype(np.float32)
    dy = rng.standard_normal((B, N, N, N)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, N, N, N), dtype=torch.float32, device="cuda")
    net.forward(B, xd.data_ptr(), yd.data_ptr())
    y_ref, cache = ofno.forward(pr, x.astype(np.float64), m, keep=True)
    assert rel_err(yd.cpu().numpy(), y_ref) < 1e-4
    dyd = torch.from_numpy(dy).cuda()
    net.gradients(B, xd.data_ptr(), dyd.data_ptr())
    _, g = net.get_params()
    gref = ofno.backward(pr, cache, dy.astype(np.float64), m)
    gp = _unpack(g, C, m, L)
    assert rel_err(gp.lift_w, gref["lift_w"]) < 2e-3
    assert rel_err(gp.lift_b, gref["lift_b"]) < 2e-3
    assert rel_err(gp.proj_w, gref["proj_w"]) < 2e-3
    assert abs(gp.proj_b - gref["proj_b"]) < 2e-3 * max(1.0, abs(gref["proj_b"]))
    for l in range(L):
        assert rel_err(gp.pw_w[l], gref["pw_w"][l]) < 2e-3
        assert rel_err(gp.pw_b[l], gref["pw_b"][l]) < 2e-3
        assert rel_err(gp.spec[l], gref["spec"][l]) < 2e-3
    net.close()


def test_fno_training_reduces_loss_on_a_learnable_target():
    """Adam steps on a target produced by another network of the same shape: the loss must fall."""
    torch = pytest.importorskip("torch")
    from paper_2205_06690_gb300 import binding as Bd
    N, C, m, L, B = 12, 8, 3, 2, 4
    teacher = Bd.FNO(N, width=C, modes=m, layers=L, max_batch=B)
    teacher.set_params(_pack(ofno.init_params(C, m, L, seed=100)))
    student = Bd.FNO(N, width=C, modes=m, layers=L, max_batch=B)
    student.set_params(_pack(ofno.init_params(C, m, L, seed=7)))
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.standard_normal((B, 2, N, N, N)).astype(np.float32)).cuda()
    t = torch.empty((B, N, N, N), dtype=torch.float32, device="cuda")
    teacher.forward(B, x.data_ptr(), t.data_ptr())
    losses = [student.train_step(B, x.data_ptr(), t.data_ptr(), 3e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0]


def test_surrogate_trained_on_tdh_pairs_and_spot_checked():
    """End to end on small Gaussian-well systems (16^3, box 8): training pairs from the stochastic
    TDH, FNO training, then surrogate W for a held-out system with a spot check against fresh
    propagation. The trained network must beat the untrained one on held-out pairs, be much faster
    per pair than propagation, and the spot-checked pairs must carry the propagated W."""
    torch = pytest.importorskip("torch")
    import sbse_inputs as si
    from paper_2205_06690_gb300 import binding as Bd
    from paper_2205_06690_gb300 import surrogate as S

    N, box = 16, 8.0
    prm = Bd.TDHParams(n_s=10, n_steps=100, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=3)
    sc = S.Scales(s_rho=1.0 / box ** 3, s_v=1.0, s_w=1.0)
    xs, ts, systems = [], [], []
    for seed in range(1000, 1005):
        p = si.model_system.Preset(f"t{seed}", N=N, box=box, n_wells=4, seed=seed, n_occ=6, n_o=4, n_c=2)
        s = si.make_system(p)
        systems.append((p, s))
    for p, s in systems[:4]:
        with Bd.Context(0, Bd.SBSE_MIXED) as c:
            c.set_grid(N, box, s.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, 0.5)
            pairs = [(i, j) for i in range(p.n_o) for j in range(i, p.n_o)]
            x, t = S.training_pairs(c, prm, pairs, N ** 3, sc)
            xs.append(x)
            ts.append(t)
    x = torch.cat(xs)
    t = torch.cat(ts)
    sc.s_w = float(t.abs().max().item())
    t = t / sc.s_w
    net = Bd.FNO(N, width=12, modes=4, layers=4, max_batch=8)
    net.set_params(_pack(ofno.init_params(12, 4, 4, seed=0)))
    p, s = systems[4]
    pairs = [(i, j) for i in range(p.n_o) for j in range(i, p.n_o)]
    with Bd.Context(0, Bd.SBSE_MIXED) as c:
        c.set_grid(N, box, s.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, 0.5)
        w_ref = c.apply_W(prm, pairs, copy_out=True)

        def held_out_err():
            Bd.sbse_surrogate_W(c.h, net.h, pairs, sc.s_rho, sc.s_v, sc.s_w)
            w = Bd.sbse_get_W(c.h, pairs, N ** 3)
            return float(np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref))

        e0 = held_out_err()
        losses = S.train(net, x, t, steps=300, batch=8, lr=2e-3)
        e1 = held_out_err()
        rep = S.surrogate_apply_W(c, net, sc, prm, pairs, N ** 3, spot_frac=0.2, tol=0.5, seed=1)
        w_after = Bd.sbse_get_W(c.h, rep["spot_pairs"], N ** 3)
        idx = [pairs.index(q) for q in rep["spot_pairs"]]
        # same seed and parameters: the propagated W (up to the FP32 rounding of a different
        # Poisson packing partner) replaced the surrogate's for the spot-checked pairs
        assert np.linalg.norm(w_after - w_ref[idx]) <= 1e-4 * np.linalg.norm(w_ref[idx])
        A = c.build_A()
        assert np.all(np.isfinite(A))
    assert losses[-1] < 0.5 * losses[0]
    assert e1 < e0
    assert rep["surrogate_s_per_pair"] < rep["tdh_s_per_pair"]
