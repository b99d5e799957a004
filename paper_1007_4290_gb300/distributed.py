"""Multi-GPU use of the sweeping preconditioner: source sharding.

The setup and the apply are sequential over the layers (Algorithms 2.5/2.6), and one
layer is too small to split, so GPUs share the work by right-hand sides: every rank holds
its own factorisation (a replica, built locally) and solves its own slice of the sources.
The only exchange of the method is the sum over sources of the misfit and of its gradient
with respect to c, one all-reduce of n*n + 1 values.
"""
import torch
import torch.distributed as dist


def shard(count, world, rank):
    """Contiguous [lo, hi) slice of `count` items owned by `rank` (sizes differ by <= 1)."""
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _reduce_device(group=None):
    """The device of the all-reduce buffer, the same on every rank whatever its shard:
    this process's current CUDA device under NCCL, the host otherwise."""
    if dist.is_initialized() and dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def sharded_misfit_gradient(grad_fn, F, d, group=None):
    """Misfit and gradient summed over all sources when each rank owns a slice of them.

    grad_fn(F_local, d_local) -> (J_local, g_local) evaluates this rank's sources (for a
    handle h: lambda F, d: h.grad(F, rec_idx, d, tol)).  F and d hold ALL sources
    (identically on every rank); each rank evaluates its shard and one all-reduce adds
    the partial misfits and gradients.  Returns (J, g) on every rank.
    """
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    lo, hi = shard(F.shape[0], world, rank)
    if hi > lo:
        J, g = grad_fn(F[lo:hi], d[lo:hi])
        g = torch.as_tensor(g, dtype=torch.float64).reshape(-1)
    else:
        J, g = 0.0, None
    n_grad = int(F[0].numel()) if torch.is_tensor(F) else int(F[0].size)
    buf = torch.zeros(n_grad + 1, dtype=torch.float64, device=_reduce_device(group))
    if g is not None:
        buf[:n_grad] = g
    buf[n_grad] = float(J)
    if world > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[n_grad].item(), buf[:n_grad]
