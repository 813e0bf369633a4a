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
# cost of one q term of Sigma_c relative to chi0 + eps~ / W^c of one q (split precision, cfg1
# launch list: ~5.4 ms against ~16.5 ms)
SIGMA_SHARE = 0.33


def minus_q(nk, q):
    """Index of -q on the Gamma-centred mesh nk (index (i1 n2 + i2) n3 + i3)."""
    n1, n2, n3 = nk
    i1, r = divmod(q, n2 * n3)
    i2, i3 = divmod(r, n3)
    return ((-i1 % n1) * n2 + (-i2 % n2)) * n3 + (-i3 % n3)


def q_units(n_q, nk=None):
    """The units of work of the q loop: single q points, or with time reversal (nk given) the
    pairs {q, -q}, whose chi0, eps~ and W^c the q loop computes once (a point with -q = q stays
    alone). Ascending lists, ordered by their first point."""
    if nk is None:
        return [[q] for q in range(n_q)]
    if nk[0] * nk[1] * nk[2] != n_q:
        raise ValueError("nk does not match n_q")
    seen, units = set(), []
    for q in range(n_q):
        if q in seen:
            continue
        mq = minus_q(nk, q)
        u = sorted({q, mq})
        seen.update(u)
        units.append(u)
    return units


def unit_cost(u, q0_weight=Q0_WEIGHT, nk=None, sigma_share=SIGMA_SHARE):
    """Work of a unit: without pairing, q0_weight for q = 0 and 1 for the others; with pairing
    (nk given), one chi0 / screen evaluation (q0_weight at q = 0) plus one Sigma_c term per point."""
    if nk is None:
        return q0_weight if u == [0] else 1.0
    return (q0_weight if 0 in u else 1.0) + sigma_share * len(u)


def q_partition(n_q, world, q0_weight=Q0_WEIGHT, nk=None, sigma_share=SIGMA_SHARE):
    """Disjoint lists of q points, one per rank, covering 0 .. n_q - 1, each ascending.

    Without nk: round-robin in q order, each point to the rank with the least work so far (q = 0
    counts q0_weight, the others 1; ties go to the lowest rank). With nk (time-reversal pairing):
    the pairs {q, -q} stay on one rank, so that its q loop computes chi0, eps~ and W^c once per
    pair; the units go largest first to the least-loaded rank (costs from unit_cost)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    units = q_units(n_q, nk)
    if nk is not None:
        units = sorted(units, key=lambda u: (-unit_cost(u, q0_weight, nk, sigma_share), u[0]))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for u in units:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].extend(u)
        load[r] += unit_cost(u, q0_weight, nk, sigma_share)
    return [sorted(p) for p in parts]


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


def sharded_sigma(accumulate, n_k, n_sigma, n_freq, device, group=None, nk=None):
    """Sigma_c of the whole mesh on every rank: accumulate(qs, acc) adds the q terms of this
    rank's points into acc [n_k][n_sigma][n_freq] (complex128, zeroed here); the ranks' partial
    sums are then added together. nk: keep the time-reversal pairs {q, -q} on one rank."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    qs = q_partition(n_k, world, nk=nk)[rank]
    acc = torch.zeros((n_k, n_sigma, n_freq), dtype=torch.complex128, device=device)
    if qs:
        accumulate(qs, acc)
    return sum_over_ranks(acc, group)


def g0w0_sharded(gw, plan, sys, system, group=None, trs=None):
    """One q-parallel G0W0 pass of `system` on the plan of this rank: returns (Sigma_c, e_qp, gap).
    trs: the plan's time_reversal flag (default: the system's); with it the pairs {q, -q} stay
    on one rank."""
    nsig = system.sigma_hi - system.sigma_lo
    trs = bool(getattr(system, "trs", False)) if trs is None else bool(trs)
    acc = sharded_sigma(lambda qs, a: gw.gw_g0w0_qset(plan, sys, qs, a), system.n_k, nsig, system.n_freq,
                        "cuda", group, nk=tuple(system.nk) if trs else None)
    e, gap, _ = gw.gw_qp(plan, sys, system.n_k, nsig, sigma=acc)
    return acc, e, gap
