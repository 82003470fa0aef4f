"""Two-rank (gloo, CPU) test of the sharded update chain: each rank draws its
own shard of a virtual batch and runs the oracle on it; the gathered shards
must equal the single-process result, and the timing reduction must return
the maximum over ranks.  No GPU, no data-path collective in the product."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle
import synth
from paper_1904_08555_b300 import shard

N, STEPS, PER_RANK, WORLD = 5, 16, 7, 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(WORLD), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    w, r, _ = shard.world()
    A = synth.uniform_np(synth.SEED_CHAIN_SWEEP, synth.STREAM_A + shard.element_offset(r, PER_RANK, N),
                         PER_RANK * N * N).reshape(PER_RANK, N, N)
    X = oracle.update_chain(A, STEPS)
    shard.barrier(w)
    elapsed = shard.max_over_ranks(w, float(10 + r))
    gathered = [torch.zeros(PER_RANK * N * N, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(gathered, torch.from_numpy(X.ravel()))    # test-side check only
    if r == 0:
        q.put((elapsed, torch.cat(gathered).numpy()))
    dist.destroy_process_group()


def test_two_rank_shards_reassemble_single_process_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    elapsed, got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert elapsed == 10.0 + WORLD - 1
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, WORLD * PER_RANK, N)
    np.testing.assert_array_equal(got.reshape(-1, N, N), oracle.update_chain(A, STEPS))


def test_offsets():
    assert shard.first_instance(3, 100) == 300
    assert shard.element_offset(2, 10, 4) == 320
    assert shard.max_over_ranks(1, 2.5) == 2.5
