"""The multi-rank (replica) logic of bench.py on CPU ranks over gloo.

Every rank runs an independent episode; the job's time is the slowest
rank's, and value counts the cells of all ranks. Only rank 0 prints the
reference arm. No GPU: the collectives run on the gloo backend.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.ranks_from_env()
        # rank r timed (r + 1) * 100 ms for its K steps
        dist.barrier()
        ms = bench.max_over_ranks(100.0 * (r + 1), w)
        val = bench.whole_job_value(w, 128 ** 3, 100, ms / 2)
        # the reference arm: rank 0 alone runs it and prints
        ref = bench.run_reference(None, r) if r != 0 else "rank0"
        out[r] = (w, r, lr, ms, val, ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_cells():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, lr, ms, val, ref) in res.items():
        assert (w, rr, lr) == (2, r, r)
        assert ms == 200.0                                   # the slower rank's time
        assert val == pytest.approx(2 * 128 ** 3 * 100 / 0.1)  # both ranks' cells
    assert res[1][5] is None                                 # rank 1 does no reference work


def test_single_rank_defaults():
    assert bench.ranks_from_env({}) == (1, 0, 0)
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_value(1, 1000, 10, 1000.0) == 10000.0


def test_cpu_baseline_one_thread_and_all_cores_on_a_small_sample():
    import argparse
    args = argparse.Namespace(cpu_n=10)
    one = bench.cpu_baseline(args)
    many = bench.cpu_baseline_all_cores(args, procs=2)
    assert one["cores"] == 1 and many["cores"] == 2
    assert one["value"] > 0 and many["value"] > 0
    assert one["kind"] == many["kind"] == "oracle"
    assert one["host_cpus"] == many["host_cpus"] == os.cpu_count()
    # value counts every copy's cells over the slowest copy's time (the
    # structure of the figure, not a timing ratio, which host load can skew)
    assert many["value"] == pytest.approx(2 * 10 ** 3 / many["seconds"])
    assert one["value"] == pytest.approx(10 ** 3 / one["seconds"])
    assert many["wall_seconds"] >= many["seconds"]


def test_smoother_roofline_counts_the_methods_full_sweep_bytes():
    # a full red-black sweep of the finest level must read x, b and the three
    # fraction arrays and write x once (FP32: 24 B/cell); a launch is a half
    # sweep, so it is charged 12 B/cell whatever the kernel itself re-reads
    assert bench.alg_bytes_per_cell("mg_smooth0", 2) == 12.0
    assert bench.alg_bytes_per_cell("mg_smooth0", 3) == 12.0
    # the other classes: their operands read and written once
    assert bench.alg_bytes_per_cell("apply_dot", 2) == 20
    assert bench.alg_bytes_per_cell("cg_xr", 2) == 24
    assert bench.alg_bytes_per_cell("unknown", 2) is None
