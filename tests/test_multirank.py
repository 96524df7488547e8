"""World-size-2 checks of the multi-rank host logic on CPU (gloo): the timing
aggregation used by bench.py, and exactness of term sharding (partial
amplitudes of contiguous term ranges add up to the full sum)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1808_00128_gb300 import sharding


def test_shard_ranges_cover_exactly():
    for chi in (1, 7, 64, 1000, 2 ** 16 + 3):
        for world in (1, 2, 3, 8):
            spans = [sharding.shard_range(chi, r, world) for r in range(world)]
            assert spans[0][0] == 0
            for (a0, c0), (a1, _) in zip(spans, spans[1:]):
                assert a0 + c0 == a1
            assert spans[-1][0] + spans[-1][1] == chi
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle import decomp
    from oracle import estimators as E
    from paper_1808_00128_gb300 import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # timing aggregation: the job time is the slowest rank's
    t = sharding.max_over_ranks(10.0 + rank)
    # term sharding: each rank evaluates its range of a 24-term sparsified state
    n = 6
    ops = workloads.random_clifford_t(n, 40, 4, seed=31)
    chi = 24
    a0, c = sharding.shard_range(chi, rank, world)
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=chi, mode="sparsify", seed=3,
                                                 alphas=range(a0, a0 + c))
    part = torch.tensor([[E.amplitude(terms, coefs, x).real, E.amplitude(terms, coefs, x).imag]
                         for x in range(1 << n)], dtype=torch.float64)
    sharding.allreduce_sum(part)
    q.put((rank, t, part.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import decomp
    from oracle import estimators as E
    from paper_1808_00128_gb300 import workloads
    n = 6
    ops = workloads.random_clifford_t(n, 40, 4, seed=31)
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=24, mode="sparsify", seed=3)
    full = np.array([[E.amplitude(terms, coefs, x).real, E.amplitude(terms, coefs, x).imag]
                     for x in range(1 << n)])
    for rank, t, part in out:
        assert t == 11.0
        np.testing.assert_allclose(part, full, atol=1e-12)


class _OracleShard:
    """The five calls metropolis_sharded makes, answered by the oracle for one term
    range (CPU stand-in for a context on one GPU)."""

    def __init__(self, n, ops, chi_total, seed, a0, c):
        from oracle import decomp
        self.n = n
        self.terms, self.coefs, _ = decomp.build_decomposition(n, ops, chi=chi_total, mode="sparsify", seed=seed,
                                                               alphas=range(a0, a0 + c))

    def _amp(self, xs):
        import torch
        from oracle import estimators as E
        a = [E.amplitude(self.terms, self.coefs, int(x)) for x in xs]
        return torch.tensor([[v.real, v.imag] for v in a], dtype=torch.float64)

    def amplitude(self, x):
        return self._amp(x.tolist())

    def chains_init(self, x):
        self.cx = [int(v) for v in x.tolist()]

    def chains_set_amplitude(self, amp):
        self.cp = [float(a[0] ** 2 + a[1] ** 2) for a in amp.tolist()]

    def metropolis_propose(self, seed, step):
        from oracle import estimators as E
        self.y = [x ^ (1 << E.metropolis_draws(self.n, seed, c, step)[0]) for c, x in enumerate(self.cx)]
        return self._amp(self.y)

    def metropolis_accept(self, amp, seed, step, trace=None):
        from oracle import estimators as E
        for c, a in enumerate(amp.tolist()):
            py = a[0] ** 2 + a[1] ** 2
            _, r = E.metropolis_draws(self.n, seed, c, step)
            if py >= self.cp[c] or r < py / self.cp[c]:
                self.cx[c], self.cp[c] = self.y[c], py
        if trace is not None:
            trace[:] = torch_tensor(self.cx)


def torch_tensor(v):
    import torch
    return torch.tensor(v, dtype=torch.int64)


def _sharded_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_1808_00128_gb300 import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, chi, seed = 6, 24, 3
    ops = workloads.random_clifford_t(n, 40, 4, seed=31)
    a0, c = sharding.shard_range(chi, rank, world)
    shard = _OracleShard(n, ops, chi, seed, a0, c)
    x0 = torch.tensor([1, 5, 9, 33], dtype=torch.int64)
    sharding.chains_init_sharded([shard], x0, allreduce=sharding.allreduce_sum)
    T = 12
    trace = torch.zeros((T, 4), dtype=torch.int64)
    sharding.metropolis_sharded([shard], T, seed=8, trace=trace, allreduce=sharding.allreduce_sum)
    q.put((rank, trace.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sharded_metropolis():
    """Two ranks, each holding half of a 24-term decomposition, run the term-sharded
    chain (partial amplitudes all-reduced every step); both produce the oracle's
    single-process chain."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import decomp
    from oracle import estimators as E
    from paper_1808_00128_gb300 import workloads
    n = 6
    ops = workloads.random_clifford_t(n, 40, 4, seed=31)
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=24, mode="sparsify", seed=3)
    want = np.zeros((12, 4), np.int64)
    for c, x in enumerate([1, 5, 9, 33]):
        px = E.probability(terms, coefs, x)
        for t in range(12):
            x, px, *_ = E.metropolis_step(terms, coefs, x, px, n, seed=8, chain=c, step=t)
            want[t, c] = x
    assert len({int(r) for r, _ in out}) == 2
    assert (want[1:] != want[:-1]).any()        # the chains move
    for _, tr in out:
        np.testing.assert_array_equal(tr, want)
