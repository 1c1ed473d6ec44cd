"""Frequency sharding of E_c across processes (one GPU each).

E_c = (1/2pi) sum_m w_m sum_i g(lambda_i(omega_m)) (Eq. 10) is a sum over the quadrature
frequencies; with independent frequencies (no warm start, rpa_options.independent_frequencies)
every frequency's subspace iteration starts from the same V0 and the terms are independent.  A
rank evaluates a contiguous range of frequencies (rpa_options.omega_first / omega_count) and one
all-reduce of the per-frequency contributions and Ritz values (zero outside each rank's range)
gives every rank the E_c of the whole quadrature.  Host logic only: the partition and the
combination; the computation of each range is the library's.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import numpy as np


def frequency_partition(n_omega: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous, balanced range (first, count) of the ascending frequency indices for one rank;
    the first n_omega % world ranks take one frequency more.  count is 0 for ranks beyond
    n_omega."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_omega, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def combine(ec_per_omega: np.ndarray, lambdas: np.ndarray, group=None):
    """Sum the ranks' per-frequency contributions and Ritz values (each zero outside its rank's
    range) over the process group: returns (E_c, ec_per_omega, lambdas) of the whole quadrature,
    the same on every rank."""
    import torch
    import torch.distributed as dist
    buf = torch.from_numpy(np.concatenate([np.ravel(ec_per_omega), np.ravel(lambdas)]).astype(np.float64))
    if dist.is_available() and dist.is_initialized():
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
        t = buf.to(dev) if dev is not None else buf
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        buf = t.cpu()
    out = buf.numpy()
    n = np.size(ec_per_omega)
    ecm = out[:n].reshape(np.shape(ec_per_omega))
    lam = out[n:].reshape(np.shape(lambdas))
    return float(np.sum(ecm)), ecm, lam


def ec_sharded(evaluate: Callable[[int, int], Tuple[np.ndarray, np.ndarray]], n_omega: int, world: int, rank: int,
               group=None):
    """E_c over a frequency partition: evaluate(first, count) computes this rank's range and
    returns its (ec_per_omega, lambdas) arrays over all n_omega frequencies (zeros outside the
    range); the ranks' results are combined by one all-reduce."""
    first, count = frequency_partition(n_omega, world, rank)
    ecm, lam = evaluate(first, count)
    return combine(ecm, lam, group)


def library_evaluator(ctx, V0, options):
    """evaluate(first, count) for ec_sharded on a library context: runs rpa_ec on the range with
    independent frequencies (a rank with an empty range contributes zeros)."""
    import dataclasses

    def evaluate(first: int, count: int):
        nw = options.n_omega
        if count == 0:
            return np.zeros(nw), np.zeros((nw, V0.shape[0]))
        o = dataclasses.replace(options, independent_frequencies=1, omega_first=first, omega_count=count)
        ctx.set_options(o)
        res = ctx.ec(V0)
        ctx.set_options(options)
        return res.e_c_per_omega, res.lambdas

    return evaluate
