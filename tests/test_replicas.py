"""Multi-GPU runs are independent replicas: the host logic of bench.py under
two gloo ranks on CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank "timed" a different total; the job takes the slowest
    total_ms, e2e_s = bench.reduce_max([100.0 + 50.0 * rank, 0.02 * (rank + 1)], dist, "cpu")
    out.put((rank, total_ms, e2e_s, bench.replica_seed(7, rank),
             bench.job_rate(world, 10, total_ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_to_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, e2e_s, seed, rate in res:
        assert total_ms == pytest.approx(150.0)          # max over ranks
        assert e2e_s == pytest.approx(0.04)
        assert seed == 7 + rank                           # distinct pair per replica
        assert rate == pytest.approx(2 * 10 / 0.150)      # whole-job frames/s


def test_single_process_needs_no_collective():
    import bench
    assert bench.reduce_max([1.0, 2.0]) == [1.0, 2.0]
    assert bench.job_rate(1, 20, 400.0) == pytest.approx(50.0)


def test_schedule_labels_decode_the_tuner_encoding():
    # 0 = cluster; 8 v + d = depth d on footprint v (the fs_autotune encoding)
    import bench
    assert bench.schedule_label(0) == "cluster"
    assert bench.schedule_label(7) == "blocking x7 (64x64 footprints, 512 threads)"
    assert bench.schedule_label(16) == "blocking x8 (32x32 footprints, 256 threads)"
    assert bench.schedule_label(31) == "blocking x7 (64x64 footprints, 1024 threads)"
    assert bench.schedule_label(40) == "blocking x8 (32x32 footprints, 1024 threads)"
    assert bench.schedule_label(41) == "blocking x1 (32x32 footprints, 512 threads)"
    assert bench.schedule_label(49) == "blocking x9 (32x32 footprints, 1024 threads)"
    assert bench.schedule_label(55) == "blocking x15 (32x32 footprints, 1024 threads)"
    assert bench.schedule_label(56) == ("blocking x1 (64x64 footprints 48 columns apart, "
                                        "1024 threads, TMA-staged)")
    assert bench.schedule_label(63).startswith("blocking x8 (64x64 footprints 48 columns")
    assert bench.interior(bench.TMA_FOOTPRINT, 7) == (48, 50)
    assert bench.interior(3, 7) == (50, 50)
    # one label per footprint variant of the kernels, the TMA one last
    import os
    import re
    src = open(os.path.join(os.path.dirname(bench.__file__), "paper_1909_07545_gb300", "csrc",
                            "fs_kernels.h")).read()
    assert int(re.search(r"PD_TILE_COUNT = (\d+)", src).group(1)) + 2 == len(bench.FOOTPRINTS)
    assert "constexpr int PD_TILE_64_TMA = PD_TILE_COUNT;" in src
    assert "constexpr int PD_TILE_64x48_T768 = PD_TILE_COUNT + 1;" in src
    assert bench.schedule_label(70) == "blocking x7 (64x48 footprints, 768 threads)"
    assert bench.interior(7, 6) == (52, 36)
