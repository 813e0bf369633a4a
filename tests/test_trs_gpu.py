"""Time reversal in the q loop (gw_problem.time_reversal): for inputs with eps(-k) = eps(k),
c(-k) = conj(c(k)) and V(-q) = conj(V(q)), chi0(-q) = conj(chi0(q)) and W^c(-q) = conj(W^c(q)), so
gw_g0w0 computes chi0 / eps~ / W^c once per pair (q, -q). The pass must give the Sigma_c of the
pass without the symmetry, and the oracle's; inputs that break the symmetry are refused."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HA_MEV = 27211.386


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


def pass_sigma(s, prec, trs, qs=None):
    from paper_2011_01400_gb300 import gw
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec, trs=trs)
    plan = gw.gw_plan_create(pb.prob)
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        if qs is None:
            gw.gw_g0w0(plan, 0, acc)
        else:
            gw.gw_g0w0_qset(plan, 0, qs, acc)
        e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return acc.cpu().numpy(), e, gap


@pytest.mark.parametrize("hw", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("3xfp16", 1e-6), ("3xtf32", 1e-6)])
def test_pairs_give_the_full_pass(prec, tol, hw):
    """hw = 1: q -> 0 along one direction, which breaks k -> -k for Sigma_c, so only the q points are
    paired; hw = 2 (direction average): Sigma_c(-k) = Sigma_c(k) too, and the pass computes the
    target k <= -k only."""
    s = make_system("cfg0", seed=31, nk=(3, 2, 1), head_wings=hw)   # q and -q differ for 4 of the 6 q
    assert s.trs
    sig_t, e_t, gap_t = pass_sigma(s, prec, True)
    sig_f, e_f, gap_f = pass_sigma(s, prec, False)
    scale = np.abs(sig_f).max()
    assert np.abs(sig_t - sig_f).max() <= tol * scale
    ref = O.g0w0(s)
    err = np.abs(sig_t - ref["sigma"]).max() * HA_MEV
    print(f"{prec} head_wings={hw}: time reversal vs none {np.abs(sig_t - sig_f).max() / scale:.1e} rel, vs oracle {err:.2e} meV")
    assert err <= (1e-6 if prec == "fp64" else 1.0)
    assert abs(gap_t - ref["gap"]) * HA_MEV <= (1e-6 if prec == "fp64" else 1.0)


def test_pairs_inside_a_q_subset():
    s = make_system("cfg0", seed=32, nk=(3, 2, 1))
    parts = [[0, 2, 4], [1, 3, 5]]                         # 2 and 4 are a pair; 3 and 5 too
    tot_t = sum(pass_sigma(s, "fp64", True, qs)[0] for qs in parts)
    tot_f = sum(pass_sigma(s, "fp64", False, qs)[0] for qs in parts)
    assert np.abs(tot_t - tot_f).max() <= 1e-12 * np.abs(tot_f).max()


def test_broken_symmetry_is_refused():
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=33, nk=(3, 2, 1), trs=False)
    pb = gw.Problem(s, "fp64", trs=True)
    with pytest.raises(gw.GwError) as ei:
        gw.gw_plan_create(pb.prob)
    assert ei.value.status == gw.GW_ERR_ARG and "time_reversal" in str(ei.value)
