"""The sharded J-build and B rows on CPU: the partition of the unique pairs, and two gloo ranks that
each contract their rows of F_u (the oracle's factored form, eq. tensors and eq. ig1) and combine
them with all-reduces through paper_2210_13069_gb300.shard, against the oracle's single-process
factored J-build and Algorithm 1 B."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2210_13069_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("npair,world", [(1, 1), (5, 2), (210, 2), (1830, 3), (16290, 4), (300, 8), (3, 4)])
def test_pair_ranges_cover_once(npair, world):
    rr = shard.pair_ranges(npair, world)
    assert len(rr) == world
    covered = np.zeros(npair, dtype=int)
    for r0, r1 in rr:
        assert 0 <= r0 <= r1 <= npair
        covered[r0:r1] += 1
    assert np.all(covered == 1)
    assert [r0 for r0, _ in rr[1:]] == [r1 for _, r1 in rr[:-1]]
    if npair >= 128 * world * 4:
        assert all(r0 % 128 == 0 for r0, _ in rr)
        lens = [r1 - r0 for r0, r1 in rr]
        assert max(lens) - min(lens) <= 2 * 128  # each boundary within 64 of its exact place


def _mol():
    sys.path.insert(0, ROOT)
    from paper_2210_13069_gb300 import synth
    return synth.random_molecule(4201, natoms=2, cube=3.0, nprim=2, alpha_range=(0.2, 20.0), omega=0.4, n=6, P=6)


def _oracle_halves(o, D):
    """The two halves of the factored J-build from the oracle's factors (numpy)."""
    nb, n = o.nbf, o.n
    M = o.factor_M(threads=2)  # N_b^2 x n^3, row mu N_b + nu
    pairs = [(mu, nu) for mu in range(nb) for nu in range(mu, nb)]
    Fu = np.array([M[mu * nb + nu] for mu, nu in pairs])
    _, w = o.nodes()
    K = sum(w[p] * np.kron(o.cheb(0, p), np.kron(o.cheb(1, p), o.cheb(2, p))) for p in range(o.P))
    K *= o.omega / np.sqrt(np.pi)
    u = np.array([[D[q, mu, nu] * (1.0 if mu == nu else 2.0) for mu, nu in pairs] for q in range(D.shape[0])])

    def partial_x(r0, r1):
        return u[:, r0:r1] @ Fu[r0:r1]

    def apply_x(X, r0, r1):
        Y = X @ K  # K symmetric
        J = np.zeros_like(D)
        for r in range(r0, r1):
            mu, nu = pairs[r]
            J[:, mu, nu] = J[:, nu, mu] = Fu[r] @ Y.T
        return J

    return partial_x, apply_x, len(pairs)


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2210_13069_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = _mol()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(17, m.nbf, 3)
    partial_x, apply_x, npair = _oracle_halves(o, D)

    def allreduce(a):
        t = torch.as_tensor(np.ascontiguousarray(a))
        dist.all_reduce(t)
        return t.numpy()

    J = shard.jbuild_sharded(partial_x, apply_x, allreduce, npair, rank, world)
    pairs = [(mu, nu) for mu in range(o.nbf) for nu in range(mu, o.nbf)]
    r0, r1, rows = shard.b_rows_sharded(
        lambda a, b: o.B_rows([pairs[r][0] * o.nbf + pairs[r][1] for r in range(a, b)], threads=2), npair, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, J, r0, r1, rows))


def test_two_gloo_ranks_sum_to_the_single_rank_jbuild():
    import torch.multiprocessing as mp
    import oracle
    from paper_2210_13069_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m = _mol()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(17, m.nbf, 3)
    ref = o.jbuild_factored(D)
    for rank, J, _, _, _ in out:  # both ranks hold the all-reduced J
        assert np.max(np.abs(J - ref)) <= 1e-13 * np.abs(ref).max(), rank
    # the ranks' B rows together are the unique-pair rows of B, each once
    B = o.assemble_B()
    nb = o.nbf
    pairs = [(mu, nu) for mu in range(nb) for nu in range(mu, nb)]
    got = np.concatenate([rows for _, _, _, _, rows in out])
    assert [r0 for _, _, r0, _, _ in out] == [0, out[0][3]] and out[1][3] == len(pairs)
    want = np.array([B[mu * nb + nu] for mu, nu in pairs])
    assert np.max(np.abs(got - want)) <= 1e-13 * np.abs(want).max()
