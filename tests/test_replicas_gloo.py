"""The N > 1 path of the bench (independent replicas, one per rank), run as two gloo ranks on
the CPU.  Each rank takes its own slice of the seeded batch, the slowest rank's time sets the
job's time, and the rate counts every rank's evaluations.  The per-rank evaluation here is the
oracle's (the GPU step needs a device); what is checked is the host logic around it: disjoint,
covering slices that regenerate exactly the instances of the unsharded batch, the barrier, the
max-over-ranks reduction and the whole-job rate."""
import json
import os
import socket
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORLD = 2
PER_RANK = 2
SEED = 1002


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2601_09951_gb300 import workloads as W

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        idx = bench.replica_indices(rank, PER_RANK)
        insts = W.hea_batch(PER_RANK * world, seed=SEED, indices=idx)
        energies = [float(oracle.energy(inst)) for inst in insts]
        # Distinct per-rank timings: each entry's maximum sits on a different rank.
        local = [1.0 + rank, 2.0 - rank, 0.25 * (rank + 1)]
        dist.barrier()
        reduced = bench.max_over_ranks(local, dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, {"rank": rank, "idx": idx,
                                          "names": [i["name"] for i in insts],
                                          "energies": energies, "reduced": reduced})
        if rank == 0:
            rate = bench.whole_job_rate(PER_RANK, world, 10, reduced[0])
            with open(os.path.join(out_dir, "ranks.json"), "w") as f:
                json.dump({"ranks": gathered, "rate": rate}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_slices_are_disjoint_and_cover():
    import bench
    slices = [bench.replica_indices(r, 5) for r in range(4)]
    flat = [i for s in slices for i in s]
    assert sorted(flat) == list(range(20))
    assert len(set(flat)) == len(flat)


def test_whole_job_rate_counts_every_rank():
    import bench
    assert bench.whole_job_rate(4096, 8, 200, 2.0) == 4096 * 8 * 200 / 2.0
    assert bench.whole_job_rate(4096, 1, 200, 2.0) * 8 == bench.whole_job_rate(4096, 8, 200, 2.0)


def test_two_gloo_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle
    from paper_2601_09951_gb300 import workloads as W

    oracle.lib()  # build the oracle once before the ranks import it
    with tempfile.TemporaryDirectory() as out_dir:
        mp.start_processes(_rank_main, args=(WORLD, _free_port(), out_dir), nprocs=WORLD,
                           join=True, start_method="spawn")
        with open(os.path.join(out_dir, "ranks.json")) as f:
            res = json.load(f)

    ranks = sorted(res["ranks"], key=lambda r: r["rank"])
    idx = [i for r in ranks for i in r["idx"]]
    assert idx == list(range(WORLD * PER_RANK))
    full = W.hea_batch(WORLD * PER_RANK, seed=SEED)
    assert [n for r in ranks for n in r["names"]] == [i["name"] for i in full]
    # Sharding does not change any instance: energies equal the unsharded run's exactly.
    assert [e for r in ranks for e in r["energies"]] == [float(oracle.energy(i)) for i in full]
    # Maximum over ranks, element by element, seen identically by every rank.
    for r in ranks:
        assert r["reduced"] == [2.0, 2.0, 0.5]
    assert res["rate"] == PER_RANK * WORLD * 10 / 2.0
