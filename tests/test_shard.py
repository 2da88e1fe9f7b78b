"""Views of a mapping window sharded over two gloo ranks (CPU): each rank differentiates its
views with the FP64 oracle, the per-Gaussian gradients are summed over ranks and the pose
gradients gathered; the result equals the oracle's K-view gradients."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    from scenes import make_scene
    return make_scene("window500k", n=3000, K=5, W=64, H=48, f=50.0)


def _grads(s, cams):
    import oracle
    from scenes import random_image
    K = cams.shape[0]
    o = oracle.forward(s.params(), cams, s.W, s.H)
    # upstream gradients drawn for all 5 views, sliced to this rank's views
    gr_all = random_image(3, (5, 3, s.H, s.W)).astype(np.float64)
    gd_all = random_image(4, (5, s.H, s.W)).astype(np.float64)
    return o, gr_all, gd_all, K


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2509_06433_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _scene()
    a, b = shard.view_range(s.K, rank, world)
    cams = s.cams.reshape(-1, 16)[a:b]
    o, gr_all, gd_all, _ = _grads(s, cams)
    g = oracle.backward(s.params(), cams, s.W, s.H, o["lists"], gr_all[a:b], gd_all[a:b])
    grads = {k: torch.as_tensor(g[k]) for k in shard.NAMES}
    shard.allreduce_gaussian_grads(grads)
    pose = shard.gather_pose_grads(torch.as_tensor(g["pose"]), s.K)
    q.put((rank, {k: v.numpy() for k, v in grads.items()}, pose.numpy()))
    dist.destroy_process_group()


def test_view_range_partitions():
    from paper_2509_06433_gb300 import shard
    for K in (1, 5, 8, 16):
        for world in (1, 2, 3, 8):
            ranges = [shard.view_range(K, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == K
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_two_ranks_sum_to_the_k_view_gradients():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = _scene()
    cams = s.cams.reshape(-1, 16)
    o, gr_all, gd_all, _ = _grads(s, cams)
    ref = oracle.backward(s.params(), cams, s.W, s.H, o["lists"], gr_all, gd_all)
    for rank, grads, pose in out:
        for k, v in grads.items():
            np.testing.assert_allclose(v, ref[k], rtol=1e-9, atol=1e-12 * np.abs(ref[k]).max())
        np.testing.assert_allclose(pose, ref["pose"], rtol=1e-12, atol=1e-15)
    assert np.abs(ref["pose"]).max() > 0
