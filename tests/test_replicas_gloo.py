"""Multi-rank form (replicas, no data-path collective) on CPU: two gloo ranks.

Each rank searches its contiguous shard of the sky directions with the oracle
(the GPU kernels do the same per rank on a GPU machine); rank 0 gathers the
candidate lists.  Checked: the shards partition the directions, the gathered
candidates equal a single-process search over all directions, and the timing
reduction returns the slowest rank's value.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1407_8333_gb300 import replicas, synth
        assert replicas.rank_world() == (rank, world)
        inp, pp = synth.random_case(61, n_fft=16, n_bins=40, n_fdot=9, n_dir=7, p=0.3)
        b, e = replicas.direction_shard(inp.sky.shape[0], rank, world)
        res = oracle.search(inp, pp, dirs=list(range(b, e))) if e > b else None
        part = (b, e, None if res is None else {k: res[k] for k in ("cell", "row", "count", "cr")})
        parts = replicas.gather_to_rank0(part)
        slowest = replicas.max_over_ranks(10.0 * (rank + 1))
        replicas.barrier()
        if rank == 0:
            full = oracle.search(inp, pp)
            spans = [(p[0], p[1]) for p in parts]
            ok = spans == [replicas.direction_shard(7, r, world) for r in range(world)]
            for k in ("cell", "row", "count", "cr"):
                got = np.concatenate([p[2][k] for p in parts if p[2] is not None])
                ok = ok and np.array_equal(got, full[k])
            q.put(("ok" if ok else "mismatch", slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_directions_and_gather():
    import multiprocessing as mp
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    status, slowest = q.get(timeout=10)
    assert status == "ok"
    assert slowest == 20.0


def test_direction_shards_partition():
    from paper_1407_8333_gb300 import replicas
    for n_dir in (0, 1, 5, 8, 257):
        for world in (1, 2, 3, 8):
            spans = [replicas.direction_shard(n_dir, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n_dir
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.direction_shard(4, 2, 2)
