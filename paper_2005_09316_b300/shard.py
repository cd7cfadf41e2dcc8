"""Multi-GPU partitioning of the hot path: host logic for one process per GPU.

Predict and peel need no collective.
- A job of several independent observations is split by observation (weak scaling; what bench.py
  does under torchrun).
- One observation can be split by whole time steps: a rank takes rows t*B + b for t in its range
  and calls the single-GPU entry points on that slice.

The adjoint of a split observation has one exchange step. The loss and every gradient are sums over
visibility rows (L = sum |D - G V|^2), so the per-rank sums are added with one all-reduce. Step times
take the maximum over ranks. Everything here is torch.distributed calls plus index arithmetic; the
arithmetic of the method stays in the CUDA library.
"""
from __future__ import annotations

from dataclasses import replace


def time_partition(n_time: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous time-step range [t0, t1) of `rank`; sizes differ by at most one, earlier ranks larger."""
    if world < 1 or not 0 <= rank < world or n_time < 0:
        raise ValueError("bad partition request")
    base, extra = divmod(n_time, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def time_slice(obs, t0: int, t1: int):
    """The DeviceObs of time steps [t0, t1) of `obs` (a view: uvw[t0:t1], same channels and baselines)."""
    if not 0 <= t0 <= t1 <= obs.n_time:
        raise ValueError("time slice out of range")
    return replace(obs, n_time=t1 - t0, uvw=obs.uvw[t0:t1])


def max_over_ranks(x: float, group=None, device=None) -> float:
    """Maximum of a per-rank scalar (a step time) over the process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


GRAD_KEYS = ("flux", "alpha", "l", "m", "g_maj", "g_min", "g_pa", "s_beta1", "s_beta2", "s_pa", "s_coeff", "loss")


def allreduce_grads(grads: dict, group=None) -> dict:
    """Sum the gradient tensors (and the loss) of every rank in place, in a fixed key order."""
    import torch.distributed as dist
    for k in GRAD_KEYS:
        t = grads.get(k)
        if t is not None and t.numel():
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return grads


def sharded_predict_grad(ctx, obs, model, gains, data, world: int, rank: int, group=None) -> dict:
    """Adjoint of one observation split by time steps over the ranks of `group`.

    `data` is this rank's slice [t1 - t0][B][F]. `gains` is [Tg][Fg][A]: with Tg = n_time each rank
    passes the full table and the rows of its slice are taken here. Returns the summed gradients and
    loss; the residual stays local."""
    t0, t1 = time_partition(obs.n_time, world, rank)
    g = gains[t0:t1] if gains.shape[0] == obs.n_time and obs.n_time > 1 else gains
    local = ctx.predict_grad(time_slice(obs, t0, t1), model, g, data)
    return allreduce_grads(local, group)
