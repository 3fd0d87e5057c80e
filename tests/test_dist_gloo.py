"""Two CPU ranks (gloo): the data-parallel backward's only exchange -- the
sum of per-shard surfel gradients -- equals the gradient of the whole ray
batch. Gradients come from the FP64 oracle, so this runs without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_15867_gb300.dist import allreduce_grads, ray_shard

NAMES = ("means", "quats", "scales", "opacity", "features")


def test_ray_shard_covers_batch():
    for n in (0, 1, 7, 64, 1001):
        for w in (1, 2, 3, 8):
            parts = [ray_shard(n, w, r) for r in range(w)]
            idx = np.concatenate([np.arange(n)[p] for p in parts])
            assert np.array_equal(idx, np.arange(n))
            sizes = [p.stop - p.start for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ray_shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import oracle
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.tiny_scene(seed=500, n=48)
    sc.scales[:] *= 2.0
    ro, rd = synth.random_rays_through_scene(300, seed=501)
    gf, gd, go = synth.upstream_grads(300, 3, seed=502)
    sl = ray_shard(300, world, rank)
    g = oracle.trace_grad(sc, ro[sl], rd[sl], gf[sl], gd[sl], go[sl], oracle.Params(), n_threads=1)
    grads = {k: torch.from_numpy(g[k].copy()) for k in NAMES}
    allreduce_grads(grads)
    if rank == 0:
        np.savez(out_path, **{k: v.numpy() for k, v in grads.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce(tmp_path):
    import oracle
    import synth
    out = str(tmp_path / "g.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    sc = synth.tiny_scene(seed=500, n=48)
    sc.scales[:] *= 2.0
    ro, rd = synth.random_rays_through_scene(300, seed=501)
    gf, gd, go = synth.upstream_grads(300, 3, seed=502)
    ref = oracle.trace_grad(sc, ro, rd, gf, gd, go, oracle.Params(), n_threads=1)
    for k in NAMES:
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-10, atol=1e-12)
