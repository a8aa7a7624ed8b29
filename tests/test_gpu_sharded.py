"""Particles split across two ranks on the one GPU (gloo, gathering through
host memory): the sharded update through the library's svgd_step /
ssvgd_step equals the single-process update of the concatenated ensemble bit
for bit (the ranks' kernels never wait on one another: each rank runs its own
independent update)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNTS = (50, 46)
D = 5000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    rng = np.random.default_rng(41)
    n = sum(COUNTS)
    return (rng.standard_normal((n, D)).astype(np.float32),
            rng.standard_normal((n, D)).astype(np.float32))


def _updates(vg):
    return {"svgd": lambda X, G: vg.svgd_step(X, G, 0.05, gscale=-1.0),
            "ssvgd": lambda X, G: vg.ssvgd_step(X, G, 0.05, seed=3, it=9, gscale=-1.0)}


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import paper_2310_13325_gb300 as vg
    from paper_2310_13325_gb300 import sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    X, G = _problem()
    a = sum(COUNTS[:rank])
    res = {}
    for name, fn in _updates(vg).items():
        Xl = torch.tensor(X[a:a + COUNTS[rank]], device="cuda:0")
        Gl = torch.tensor(G[a:a + COUNTS[rank]], device="cuda:0")
        sharded.sharded_update(Xl, Gl, fn)
        torch.cuda.synchronize()
        res[name] = Xl.cpu().numpy()
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def test_two_ranks_on_one_gpu_equal_the_single_process_update():
    import paper_2310_13325_gb300 as vg
    X, G = _problem()
    ref = {}
    for name, fn in _updates(vg).items():
        Xt, Gt = torch.tensor(X, device="cuda:0"), torch.tensor(G, device="cuda:0")
        fn(Xt, Gt)
        ref[name] = Xt.cpu().numpy()
    world = len(COUNTS)
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for rank in range(world):
        a = sum(COUNTS[:rank])
        for name in ("svgd", "ssvgd"):
            assert np.array_equal(out[rank][name], ref[name][a:a + COUNTS[rank]]), (rank, name)
