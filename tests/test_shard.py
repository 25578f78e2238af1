"""Pair sharding across ranks (paper_2205_06690_gb300.shard): partition, the all-gather of W and the
all-gather of the direct-element columns (the exchange of the sharded path: n_c^2 numbers per
pair), tested with gloo ranks on the CPU. The W of each block come from the FP64 oracle, so the
gathered sets and the A assembled from them must equal the single-process result exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2205_06690_gb300 import shard


def test_pair_blocks_partition_the_pairs():
    for n in (1, 3, 36, 136):
        for world in (1, 2, 3, 8):
            blocks = [shard.pair_block(n, r, world) for r in range(world)]
            flat = [i for b in blocks for i in b]
            assert flat == list(range(n))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert shard.pair_list(3) == [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    with pytest.raises(ValueError):
        shard.pair_block(5, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    """8^3 system (dense eigenpairs), 3 pairs, 20 TDH steps with cleaning every 5."""
    import sbse_inputs as si
    from oracle import tdh
    p = si.model_system.Preset("shard8", N=8, box=8.0, n_wells=4, seed=0, n_occ=2, n_o=2, n_c=2)
    v, eps, phi = si.dense_eigensystem(p)
    coeff = tdh.stochastic_coefficients(5, 4, 2, "gaussian")
    op = tdh.TDHParams(n_steps=20, dt=0.05, gamma=0.1, alpha=1e-4, clean_every=5)
    return tdh.Grid(8, 8.0), v, phi, eps, 2, 2, 2, coeff, op


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from oracle import tdh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, v, phi, eps, n_occ, n_o, n_c, coeff, op = _system()
        pairs = shard.pair_list(n_o)
        mine = [pairs[i] for i in shard.pair_block(len(pairs), rank, world)]
        w = tdh.screened_potentials(g, v, phi, n_occ, n_o, coeff, op, pairs=mine)
        w_local = np.array([w[p].reshape(-1) for p in mine]).reshape(len(mine), -1)
        w_all = shard.gather_W(w_local, len(pairs), rank, world)
        np.save(os.path.join(out_dir, f"w{rank}.npy"), w_all)
        # this rank's direct-element columns D[ab][pair] = dV sum_r phi_a phi_b W_ij, then their gather
        _, _, phi_c, _ = tdh.windows(phi, eps, n_occ, n_o, n_c)
        C = phi_c.reshape(n_c, -1)
        cols = np.array([((C[:, None, :] * C[None, :, :]).reshape(n_c * n_c, -1) @ w[p].reshape(-1)) * g.dV
                         for p in mine]).T.reshape(n_c * n_c, len(mine))
        np.save(os.path.join(out_dir, f"d{rank}.npy"), shard.gather_columns(cols, len(pairs), rank, world))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_W_and_A_equal_the_single_process_result(tmp_path, world):
    from oracle import tdh
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    g, v, phi, eps, n_occ, n_o, n_c, coeff, op = _system()
    pairs = shard.pair_list(n_o)
    ref = tdh.screened_potentials(g, v, phi, n_occ, n_o, coeff, op, pairs=pairs)
    ref_arr = np.array([ref[p].reshape(-1) for p in pairs])
    phi_o, eps_o, phi_c, eps_c = tdh.windows(phi, eps, n_occ, n_o, n_c)
    A_ref = tdh.assemble_A(eps_o, eps_c, 0.5, tdh.exchange_K(g, phi_o, phi_c), tdh.direct_D(g, phi_o, phi_c, ref))
    C = phi_c.reshape(n_c, -1)
    d_ref = np.array([((C[:, None, :] * C[None, :, :]).reshape(n_c * n_c, -1) @ ref[p].reshape(-1)) * g.dV
                      for p in pairs]).T
    for r in range(world):
        w_all = np.load(tmp_path / f"w{r}.npy")
        assert np.array_equal(w_all, ref_arr)
        d_all = np.load(tmp_path / f"d{r}.npy")
        assert np.array_equal(d_all, d_ref)
        # D[ia, jb] from the gathered columns equals the oracle's direct element
        Dm = np.zeros((n_o * n_c, n_o * n_c))
        for k, (i, j) in enumerate(pairs):
            blk = d_all[:, k].reshape(n_c, n_c)
            Dm[i * n_c:(i + 1) * n_c, j * n_c:(j + 1) * n_c] = blk
            Dm[j * n_c:(j + 1) * n_c, i * n_c:(i + 1) * n_c] = blk.T
        assert np.allclose(Dm, tdh.direct_D(g, phi_o, phi_c, ref), rtol=0, atol=1e-14)
        w_dict = {p: w_all[k].reshape(phi.shape[1:]) for k, p in enumerate(pairs)}
        A = tdh.assemble_A(eps_o, eps_c, 0.5, tdh.exchange_K(g, phi_o, phi_c), tdh.direct_D(g, phi_o, phi_c, w_dict))
        assert np.array_equal(A, A_ref)
