"""q-parallel G0W0 pass over the ranks of a torch.distributed group (one GPU per rank).

chi0(q), eps~(q), W^c(q) and the q term of Sigma_c (Eq. GW_selfe_element summed over q) are
independent for different q, so the q mesh is split across the ranks, every rank runs the q loop
of its own points through the C ABI (gw_g0w0_qset on its own plan, inputs replicated), and one
sum-reduction of Sigma_c [N_k][n_sigma][n_freq] over the ranks joins them. The QP solve then
runs on every rank with the same summed Sigma_c. Nothing else is exchanged.

Host-side logic only (the partition and the reduction); the arithmetic is in libgw.
"""
from __future__ import annotations

Q0_WEIGHT = 1.25   # q = 0 also builds the head and wings of eps~ (Eq. dielectric_func_gamma)


def q_partition(n_q, world, q0_weight=Q0_WEIGHT):
    """Disjoint lists of q points, one per rank, covering 0 .. n_q - 1: round-robin in q order,
    each point to the rank with the least work so far (q = 0 counts q0_weight, the others 1;
    ties go to the lowest rank). Each list is ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for q in range(n_q):
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(q)
        load[r] += q0_weight if q == 0 else 1.0
    return parts


def sum_over_ranks(t, group=None):
    """In-place sum of a (complex or real) tensor over the ranks of the group; a no-op for a
    single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return t
    v = torch.view_as_real(t) if t.is_complex() else t
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return t


def sharded_sigma(accumulate, n_k, n_sigma, n_freq, device, group=None):
    """Sigma_c of the whole mesh on every rank: accumulate(qs, acc) adds the q terms of this
    rank's points into acc [n_k][n_sigma][n_freq] (complex128, zeroed here); the ranks' partial
    sums are then added together."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    qs = q_partition(n_k, world)[rank]
    acc = torch.zeros((n_k, n_sigma, n_freq), dtype=torch.complex128, device=device)
    if qs:
        accumulate(qs, acc)
    return sum_over_ranks(acc, group)


def g0w0_sharded(gw, plan, sys, system, group=None):
    """One q-parallel G0W0 pass of `system` on the plan of this rank: returns (Sigma_c, e_qp, gap)."""
    nsig = system.sigma_hi - system.sigma_lo
    acc = sharded_sigma(lambda qs, a: gw.gw_g0w0_qset(plan, sys, qs, a), system.n_k, nsig, system.n_freq,
                        "cuda", group)
    e, gap, _ = gw.gw_qp(plan, sys, system.n_k, nsig, sigma=acc)
    return acc, e, gap
