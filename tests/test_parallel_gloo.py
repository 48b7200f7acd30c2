"""The multi-rank partition logic on CPU ranks (gloo, world size 2): sharded moments of one system
(atoms split over the ranks, global centre and radius, one all-reduce) equal the single-process
moments, and item shards cover every item once.  The per-rank geometry and moment functions are
the CPU oracle here; only the partition and reduction logic of the package is under test (the
library's per-rank route runs in tests/test_gpu_sharded.py)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_0704_1672_gb300 import parallel, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _packed(Q, L):
    out = np.zeros((L + 1) ** 2)
    for l in range(L + 1):
        out[l * l] = Q[l * l + l].real
        for m in range(1, l + 1):
            out[l * l + 2 * m - 1] = Q[l * l + l + m].real
            out[l * l + 2 * m] = Q[l * l + l + m].imag
    return out


def _oracle_fn(xyzq, L, c, a):
    import oracle
    Q = oracle.moments(xyzq.numpy(), c, L)
    return torch.tensor(_packed(Q, L))


def _oracle_center_sums(xyzq):
    import oracle
    n = len(xyzq)
    if n == 0:
        return np.zeros(4)
    c, _ = oracle.center_radius(xyzq.numpy())
    return np.array([c[0] * n, c[1] * n, c[2] * n, float(n)])


def _radius_about(xyzq, c):
    x = xyzq.numpy()
    return float(np.sqrt(((x[:, :3] - c) ** 2).sum(1).max())) if len(x) else 0.0


def _worker(rank, world, port, S, L, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = parallel.shard_range(len(S), rank, world)
        local = torch.tensor(S[lo:hi])
        q, c, a = parallel.sharded_moments(local, L, moment_fn=_oracle_fn, geom=(_oracle_center_sums, _radius_about))
        out[rank] = (q.numpy(), c, a)
    finally:
        torch.distributed.destroy_process_group()


def test_shard_ranges_cover_everything_once():
    for n in (0, 1, 7, 100, 101):
        for w in (1, 2, 3, 8):
            idx = np.concatenate([parallel.shard_items(n, r, w) for r in range(w)])
            assert np.array_equal(idx, np.arange(n))


def test_sharded_moments_equal_single_process():
    import oracle
    rng = np.random.default_rng(4)
    S = synth.pack(synth.uniform_ball(rng, 301, 6.0) + [1.0, -2.0, 0.5], synth.charges_normal_net_zero(rng, 301))
    L = 8
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), S, L, out), nprocs=world, join=True)
        res = dict(out)
    c_ref, a_ref = oracle.center_radius(S)
    q_ref = _packed(oracle.moments(S, c_ref, L), L)
    for r in range(world):
        q, c, a = res[r]
        assert np.allclose(c, c_ref, rtol=0, atol=1e-13) and abs(a - a_ref) < 1e-12
        assert np.max(np.abs(q - q_ref)) < 1e-11 * np.max(np.abs(q_ref))
    assert np.array_equal(res[0][0], res[1][0])
