"""View-sharded training on CPU: two gloo ranks, each holding a replica of the Gaussians
and half of the views.  Each rank takes the FP64 oracle adjoint of its own views' pixels,
puts it in the trainer's flat gradient bucket and runs the bucket's all-reduce; the sum
must equal the adjoint of all views computed in one process (the gradient of a sum of
per-view terms is the sum of the per-view gradients), and the view shards must cover
every view exactly once.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PLANES = ("mean", "scale", "rot", "opacity", "sh", "sg_amp", "sg_axis", "sg_sharp")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    """The 2,000-Gaussian scene of the small workload seen by 4 orbit views at 32x32, and
    seeded per-pixel loss weights (all pixels of all views)."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2501_00342_b300 import inputs as I
    sc, _ = I.workload(0)
    cams = I.orbit_cameras(4, 32, 32, fov_x_deg=60.0, radius=4.0)
    pix = np.concatenate([O.all_pixels(c, v) for v, c in enumerate(cams)])
    w = np.random.default_rng(5).normal(size=(len(pix), 3))
    return sc, cams, pix, w


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2501_00342_b300.render import GaussianModel
    from paper_2501_00342_b300.train import GradientBucket, shard_views
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, cams, pix, w = _problem()
    mine = np.isin(pix[:, 0], list(shard_views(len(cams), world, rank)))
    g = O.adjoint_pixels(sc, cams, pix[mine], w[mine], threads=2)
    bucket = GradientBucket(GaussianModel.from_scene(sc, device="cpu"), dtype=torch.float64, device="cpu")
    for p in PLANES:
        if bucket.planes[p] is not None:
            bucket.planes[p].copy_(torch.from_numpy(g[p]))
    bucket.allreduce()
    out.put((rank, int(mine.sum()), {p: (None if t is None else t.numpy().copy()) for p, t in bucket.planes.items()}))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_every_view_once():
    sys.path.insert(0, ROOT)
    from paper_2501_00342_b300.train import shard_views
    for views in (1, 4, 7, 16):
        for world in (1, 2, 3, 4, 8):
            got = [v for r in range(world) for v in shard_views(views, world, r)]
            assert got == list(range(views))
            sizes = [len(shard_views(views, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_views(4, 2, 2)


def test_allreduced_shard_adjoints_equal_the_full_adjoint():
    import oracle as O
    sc, cams, pix, w = _problem()
    full = O.adjoint_pixels(sc, cams, pix, w, threads=4)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][1] + got[1][1] == len(pix) and got[0][1] > 0 and got[1][1] > 0
    for rank, _, planes in got:
        for p in PLANES:
            if full[p] is None or planes[p] is None:
                assert full[p] is None and planes[p] is None
                continue
            scale = max(np.abs(full[p]).max(), 1e-30)
            assert np.abs(full[p]).max() > 0, p
            # FP64 sums of the same terms in another grouping
            assert np.abs(planes[p] - full[p]).max() <= 1e-12 * scale, (rank, p)
