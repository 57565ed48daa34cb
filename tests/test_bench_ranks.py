"""The benchmark's multi-rank plumbing on CPU: two gloo ranks (world size 2, 127.0.0.1) through
bench.py's own rendezvous, barrier and max-over-ranks timing, as `--gpus 2` under torchrun
uses them (there the backend is NCCL); and the reference arm, which only rank 0 runs."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # each rank's "time": the job's time is the slowest rank's
    t = bench.max_over_ranks(w, 10.0 + 5.0 * rank)
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(t))


def test_two_ranks_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)),
                             nprocs=world, start_method="spawn", join=False)
    assert ctx.join(timeout=120) or ctx.join(timeout=120)
    for r in range(world):
        assert float((tmp_path / f"rank{r}.txt").read_text()) == 15.0


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    old = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2"]
    try:
        args = bench.parse()
    finally:
        sys.argv = old
    # rank 1 of 2: no work, no output, exit status 0 (rank 0 alone times the oracle)
    assert bench.run_reference(args, 2, 1) == 0


def test_world_of_one_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup() == (1, 0, 0)
        assert bench.max_over_ranks(1, 3.5) == 3.5
        bench.barrier(1)
    finally:
        os.environ.update(env)


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
