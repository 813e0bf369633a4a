"""Sigma_c at k points off the Gamma-centred mesh (band energies along lines through the zone).

Sigma_c(k) = sum over the q mesh of the q term of Eq. (GW_selfe_element), whose rows
C^mu_{nm}(k, k - q) need the KS states at k and at k - q. For a point k0 off the mesh, the points
k0 - q form the mesh shifted by k0, so a plan built on that shifted mesh (gw_problem.k_offset =
k0, the KS energies and vectors given there) holds those rows, while W^c(q) lives on the
unshifted q mesh of the ordinary plan. This module drives the C ABI: W^c(q) of the ordinary plan
(gw_chi0, gw_screen) feeds gw_sigma_ext on every shifted plan; the QP solve of a shifted plan
then gives the QP energies at its points. Argument marshalling only: the arithmetic is in libgw.
"""
from __future__ import annotations


def sigma_offmesh(gw, main_problem, shifted_problems, n_k, n_sigma, n_freq, n_aux, k_range=None):
    """Sigma_c [N_k][n_sigma][n_freq] on each shifted mesh (rows of k_range = (lo, hi) only; all by
    default) and its QP energies [N_k][n_sigma] (meaningful on k_range). main_problem: the
    ordinary plan's gw_problem; shifted_problems: gw_problems with k_offset set and the main
    system's chemical potential. Returns (list of device Sigma_c tensors, list of QP arrays)."""
    import torch
    lo, hi = (0, n_k) if k_range is None else k_range
    plan = gw.gw_plan_create(main_problem)
    plans = []
    try:
        for p in shifted_problems:
            plans.append(gw.gw_plan_create(p))
        W = torch.empty((n_freq, n_aux, n_aux), dtype=torch.complex128, device="cuda")
        accs = [torch.zeros((n_k, n_sigma, n_freq), dtype=torch.complex128, device="cuda") for _ in plans]
        for q in range(n_k):
            gw.gw_chi0(plan, 0, q)
            gw.gw_screen(plan, 0, q, W)
            for pl, acc in zip(plans, accs):
                gw.gw_sigma_ext(pl, 0, q, W, lo, hi, acc)
        qps = [gw.gw_qp(pl, 0, n_k, n_sigma, sigma=acc)[0] for pl, acc in zip(plans, accs)]
    finally:
        for pl in plans:
            gw.gw_plan_destroy(pl)
        gw.gw_plan_destroy(plan)
    return accs, qps
