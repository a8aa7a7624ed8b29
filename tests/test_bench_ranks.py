"""Multi-rank logic of bench.py on CPU: two gloo ranks (world size 2) agree on
the slowest rank's time, and the job value counts every rank's particles.
(The ranks' particles are coupled by the update through one all-gather per
iteration, covered by tests/test_sharded.py; this file covers the timing
reduction, the launch accounting and the oracle leg of the update workload.)"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, e = bench.reduce_over_ranks(100.0 + 50.0 * rank, 200.0 - 10.0 * rank, "cpu")
    out[rank] = (t, e, bench.job_value(600, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for rank in range(world):
        t, e, v = out[rank]
        assert t == 150.0 and e == 200.0
        assert v == pytest.approx(1200 / 0.150)


def test_launch_count_of_a_gradient_plan():
    # the wave kernel and the misfit reduction, plus the merge of per-item
    # gradients when several work items share a particle
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.fwi_gradient_launches({"sources_per_item": 2}, 20) == 3
    assert bench.fwi_gradient_launches({"sources_per_item": 20}, 20) == 2
    # and the fill launch on the idle SMs when the plan has one
    fill = {"cluster_ctas": 2, "rows_per_thread": 8, "threads": 288, "clusters": 4}
    assert bench.fwi_gradient_launches({"sources_per_item": 2, "fill": fill}, 20) == 4
    assert bench.SVGD_STEP_LAUNCHES == 20


def test_update_baseline_is_the_oracle_on_a_scaled_sample():
    # the oracle's update on min(n, 150) particles, its time scaled by (n / ns)^2
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    small = bench.update_cpu_baseline(12, 64, False)
    assert small["kind"] == "oracle" and small["unit"] == "ms" and small["value"] > 0
    assert "12 x 64" in small["sample"] and "(12 / 12)^2" in small["sample"]
    big = bench.update_cpu_baseline(300, 8, True)
    assert "ssvgd_step on 150 x 8" in big["sample"] and "(300 / 150)^2" in big["sample"]
