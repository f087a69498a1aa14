"""Shot-sharded gradients across processes (one GPU per process).

The misfit and gradient are sums over shots (Sec. "Modelling and Inversion": the least-squares
misfit sums over sources and receivers), so shots are independent solves: rank k takes a
contiguous range of shots, computes its partial misfit and FP64 gradient, and one all-reduce
(sum) of [5][2][nz][nx] + 1 float64 values combines them.  This is the only exchange on the
path; the benchmark's replicas (independent problems per rank) need none.

The frequency-domain Born misfit of Schemes I/II is a sum over frequencies as well as over
shots (Sec. "Modelling and Inversion": the sum over w >= 0), so its gradient shards by
frequency the same way: rank k takes a contiguous range of frequencies (each rank builds the
Green tables of its own frequencies only) and one all-reduce of [2][nz][nx] + 1 values sums
the parts.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shot_range(ns: int, rank: int, world: int):
    """Contiguous [lo, hi) shots of `rank`: the first ns % world ranks take one extra shot."""
    base, extra = divmod(ns, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def sharded_gradient(local_gradient, src_xy, data, group=None):
    """Sum over ranks of local_gradient(src_xy[lo:hi], data[lo:hi]) -> (misfit, grads).

    local_gradient(src, data) returns (misfit: float, grads: [5][2][nz][nx] float64 tensor) for
    its shots (on any device).  The all-reduce runs on the device of the returned gradient
    (CPU tensors with gloo, CUDA tensors with NCCL)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = shot_range(src_xy.shape[0], rank, world)
    J, G = local_gradient(src_xy[lo:hi], data[lo:hi])
    G = torch.as_tensor(G, dtype=torch.float64)
    buf = torch.cat([G.reshape(-1), torch.tensor([float(J)], dtype=torch.float64, device=G.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[-1].item(), buf[:-1].reshape(G.shape)


def sharded_frequency_gradient(local_gradient, freqs, spectrum, data, group=None):
    """Sum over ranks of local_gradient(freqs[lo:hi], spectrum[lo:hi], data[lo:hi]) ->
    (misfit, grad) for the frequency-domain Born misfit; data is [nf][ns][nr].

    local_gradient returns (misfit: float, grad: [2][nz][nx] float64 tensor) for its
    frequencies (zero of them: (0, zeros)); the all-reduce runs on the gradient's device."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = shot_range(len(freqs), rank, world)
    J, G = local_gradient(freqs[lo:hi], spectrum[lo:hi], data[lo:hi])
    G = torch.as_tensor(G, dtype=torch.float64)
    buf = torch.cat([G.reshape(-1), torch.tensor([float(J)], dtype=torch.float64, device=G.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[-1].item(), buf[:-1].reshape(G.shape)
