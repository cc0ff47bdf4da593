"""Data-parallel fine-tuning step (paper_2208_02705_gb300.dp) on CPU ranks with
the gloo backend, the gradient engine being the FP64 oracle: the summed
per-rank gradients (loss normalised by the global batch) equal the
single-process gradient of the union batch, and after the Adam step every
replica holds the same weights as the single process.  A rank that dies
before the all-reduce is detected by the survivor as an error (collective
timeout), not a hang."""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


class OracleEngine:
    """The dp_train_step engine interface backed by the FP64 oracle."""

    def __init__(self, wl, grid, weights, W, H):
        import fixtures as F
        self.wl, self.grid, self.W, self.H = wl, grid, W, H
        self.w = weights.astype(np.float64)
        self.m = np.zeros_like(self.w)
        self.v = np.zeros_like(self.w)
        self.cams = F.camera_array(wl.cams)
        self.last_grad = None

    def local_grad(self, cams, rays, target, opts, norm):
        import oracle as O
        loss, g, _, _ = O.loss_grad(self.grid, self.w.astype(np.float32), self.wl.affine, self.W, self.H,
                                    self.wl.sigma_scale, self.cams, rays, target, self.wl.delta, self.wl.n_max,
                                    loss_norm=norm)
        return torch.tensor([loss], dtype=torch.float64), torch.from_numpy(g)

    def adam_step(self, grad, lr, step):
        import oracle as O
        self.last_grad = grad.numpy().copy()
        w, m, v = O.adam(self.w, self.m, self.v, self.last_grad, lr, step)
        self.w, self.m, self.v = (a.reshape(self.w.shape) for a in (w, m, v))


def _setup(W=16, H=2, n=256):
    import fixtures as F
    import oracle as O
    wl = F.room32()
    grid = O.Grid(wl.scene, wl.part)
    weights = F.xavier_weights(1, F.ROLE_STUDENT, wl.part.n_fields, W, H, bias_scale=0.1)
    rays = F.ray_batch(1, wl.cams, n)
    target = np.random.default_rng(77).uniform(0, 1, (n, 3)).astype(np.float32)
    return wl, grid, weights, rays, target


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _dp_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2208_02705_gb300.dp import dp_train_step, lr_schedule
    wl, grid, weights, rays, target = _setup()
    eng = OracleEngine(wl, grid, weights, 16, 2)
    mine = np.arange(rank, rays.shape[0], world)          # disjoint shards of the batch
    n_global = rays.shape[0]
    losses = []
    for step in (1, 2):
        loss = dp_train_step(eng, None, rays[mine], target[mine], None, n_global, step, lr_schedule(step - 1, 10))
        losses.append(float(loss.item()))
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), w=eng.w, g=eng.last_grad, losses=np.array(losses))
    dist.destroy_process_group()


def test_dp_step_equals_single_process(tmp_path):
    world = 2
    mp.start_processes(_dp_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    from paper_2208_02705_gb300.dp import lr_schedule
    wl, grid, weights, rays, target = _setup()
    single = OracleEngine(wl, grid, weights, 16, 2)
    losses = []
    for step in (1, 2):
        loss, g = single.local_grad(None, rays, target, None, 3.0 * rays.shape[0])
        single.adam_step(g, lr_schedule(step - 1, 10), step)
        losses.append(float(loss.item()))
    r = [np.load(os.path.join(tmp_path, f"rank{k}.npz")) for k in range(world)]
    # every replica is identical (the all-reduced gradient is the same bits everywhere)
    assert np.array_equal(r[0]["w"], r[1]["w"])
    gmax = np.abs(single.last_grad).max()
    assert np.abs(r[0]["g"] - single.last_grad).max() <= 1e-12 * gmax
    assert np.abs(r[0]["w"] - single.w).max() <= 1e-9
    assert np.allclose(r[0]["losses"], losses, rtol=1e-12)


def _failing_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)                      # this rank dies between steps, before the collective
    t = torch.ones(4)
    try:
        dist.all_reduce(t)
        status = "completed"
    except Exception as e:               # the survivor learns of it from the collective
        status = "error: " + type(e).__name__
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(status)


def test_dead_rank_is_detected_not_hung(tmp_path):
    import multiprocessing
    world = 2
    ctx = multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=90)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a surviving rank hung"
    assert procs[1].exitcode == 3
    status = open(os.path.join(tmp_path, "rank0.txt")).read()
    assert status.startswith("error"), status
