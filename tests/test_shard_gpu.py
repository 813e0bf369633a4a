"""gw_g0w0_qset, the per-rank q loop of the q-parallel pass, on one GPU: the Sigma_c of the parts
of a q partition (as shard.q_partition gives for 3 ranks), each accumulated by its own plan as a
rank would, sum to gw_g0w0's Sigma_c; and the q list is checked."""
import numpy as np
import pytest

from paper_2011_01400_gb300.synth import make_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "3xbf16"])
def test_partition_terms_sum_to_the_whole_pass(prec):
    from paper_2011_01400_gb300 import gw, shard
    s = make_system("cfg0", seed=21)
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    shape = (s.n_k, nsig, s.n_freq)
    full = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_g0w0(plan, 0, full)
        e_full, gap_full, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=full)
    finally:
        gw.gw_plan_destroy(plan)
    parts = shard.q_partition(s.n_k, 3)
    total = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    for qs in parts:
        plan = gw.gw_plan_create(pb.prob)       # one plan per "rank"
        try:
            acc = torch.zeros(shape, dtype=torch.complex128, device="cuda")
            gw.gw_g0w0_qset(plan, 0, qs, acc)
            total += acc
        finally:
            gw.gw_plan_destroy(plan)
    f, t = full.cpu().numpy(), total.cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.abs(f - t).max() <= tol * np.abs(f).max()
    plan = gw.gw_plan_create(pb.prob)
    try:
        e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=total)
    finally:
        gw.gw_plan_destroy(plan)
    # the split path sums some products with float atomics: run-to-run noise ~1e-8 Ha
    tol_e = 1e-9 if prec == "fp64" else 1e-7
    assert abs(gap - gap_full) < tol_e and np.abs(e - e_full).max() < tol_e


def test_q_list_is_checked():
    from paper_2011_01400_gb300 import gw
    s = make_system("tiny", seed=22)
    pb = gw.Problem(s, "fp64")
    acc = torch.zeros((s.n_k, s.sigma_hi - s.sigma_lo, s.n_freq), dtype=torch.complex128, device="cuda")
    for bad in ([0, 0], [s.n_k], [-1]):
        plan = gw.gw_plan_create(pb.prob)
        try:
            with pytest.raises(gw.GwError) as ei:
                gw.gw_g0w0_qset(plan, 0, bad, acc)
            assert ei.value.status == gw.GW_ERR_ARG
        finally:
            gw.gw_plan_destroy(plan)
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_g0w0_qset(plan, 0, [], acc)          # no points: nothing added
        assert float(acc.abs().max()) == 0.0
    finally:
        gw.gw_plan_destroy(plan)
