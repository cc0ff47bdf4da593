"""Data-parallel fine-tuning step.

The paper fine-tunes with a batch of rays per process on several GPUs
(Sec. "Training Details and Parameters").  Every process renders its own
rays; because the L2 loss is normalised by the global batch (3 x the total
number of rays), the sum of the per-process gradients is the gradient of the
global batch, so one all-reduce (sum) per step followed by the same Adam
update on every process keeps the replicas identical.

`engine` is anything with `local_grad(cams, rays, target, opts, norm)` and
`adam_step(grad, lr, step)` -- the CUDA context (`paper_2208_02705_gb300.Roam`)
in production; the collective is torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def lr_schedule(step: int, total_steps: int, lr0: float = 1e-3, lr1: float = 5e-5) -> float:
    """Exponential decay from lr0 to lr1 over total_steps (Sec. "Training
    Details and Parameters")."""
    if total_steps <= 1:
        return lr0
    return lr0 * (lr1 / lr0) ** (min(step, total_steps - 1) / (total_steps - 1))


def dp_train_step(engine, cams, rays, target, opts, n_global: int, step: int, lr: float, group=None):
    """One data-parallel step; returns the global loss (a 1-element tensor)."""
    import torch.distributed as dist
    loss, grad = engine.local_grad(cams, rays, target, opts, norm=3.0 * n_global)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(loss, op=dist.ReduceOp.SUM, group=group)
    engine.adam_step(grad, lr=lr, step=step)
    return loss
