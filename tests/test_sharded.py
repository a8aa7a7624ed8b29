"""Particles split across two gloo ranks (CPU): the sharded update, which
all-gathers the particles and gradients and applies the coupled update of
Eq. 17 / Eq. 22-25 to the whole ensemble, equals the update of the
concatenated ensemble in one process. The update applied here is the FP64
oracle's (the library's is covered by the GPU test); ranks hold unequal
numbers of particles."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNTS = (5, 3)
D = 7


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    rng = np.random.default_rng(31)
    n = sum(COUNTS)
    return (rng.standard_normal((n, D)), rng.standard_normal((n, D)),
            rng.standard_normal((n, D)))


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import svgd as osvgd
    from paper_2310_13325_gb300 import sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, G, xi = _problem()
    a = sum(COUNTS[:rank])
    mine = slice(a, a + COUNTS[rank])
    counts, first = sharded.rank_rows(COUNTS[rank])
    assert counts == list(COUNTS) and first == a

    def svgd(Xf, Gf):
        new, _ = osvgd.svgd_step(Xf.numpy(), Gf.numpy(), 0.2, lo=-np.ones(D), hi=np.ones(D))
        Xf.copy_(torch.from_numpy(new))

    def ssvgd(Xf, Gf):
        new, _, _ = osvgd.ssvgd_step(Xf.numpy(), Gf.numpy(), 0.2, xi)
        Xf.copy_(torch.from_numpy(new))

    res = {}
    for name, fn in (("svgd", svgd), ("ssvgd", ssvgd)):
        Xl = torch.from_numpy(X[mine].copy())
        full = sharded.sharded_update(Xl, torch.from_numpy(G[mine].copy()), fn)
        res[name] = (Xl.numpy().copy(), full.numpy().copy())
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_update_equals_the_whole_ensemble_update():
    import sys
    sys.path.insert(0, ROOT)
    from oracle import svgd as osvgd
    X, G, xi = _problem()
    ref = {"svgd": osvgd.svgd_step(X, G, 0.2, lo=-np.ones(D), hi=np.ones(D))[0],
           "ssvgd": osvgd.ssvgd_step(X, G, 0.2, xi)[0]}
    world = len(COUNTS)
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for rank in range(world):
        a = sum(COUNTS[:rank])
        for name in ("svgd", "ssvgd"):
            mine, full = out[rank][name]
            assert np.array_equal(full, ref[name])
            assert np.array_equal(mine, ref[name][a:a + COUNTS[rank]])
