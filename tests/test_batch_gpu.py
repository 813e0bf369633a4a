"""Batch plans: several independent systems of uneven size (bands, occupations, ABFs, k mesh,
frequencies) in one plan, their whole q loops run concurrently on the GPU (gw_g0w0_batch).
Every system must give what its own single-system plan gives, and the oracle's Sigma_c / gap."""
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


def systems():
    return [make_system("tiny", seed=1),
            make_system("cfg0", seed=2, n_freq=12),
            make_system("cfg0", seed=3, n_bands=24, n_occ=6, n_freq=16, nk=(2, 2, 1), sigma=(4, 8)),
            make_system("tiny", seed=4, n_freq=10, head_wings=0)]


def single(gw, s, prec):
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    nsig = s.sigma_hi - s.sigma_lo
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_g0w0(plan, 0, acc)
        e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return acc.cpu().numpy(), e, gap


@pytest.mark.parametrize("prec,tol_same,tol_mev", [("fp64", 1e-12, 1e-6), ("3xtf32", 1e-6, 1.0), ("3xbf16", 1e-6, 1.0), ("3xfp16", 1e-6, 1.0)])
def test_batch_matches_single_plans_and_oracle(prec, tol_same, tol_mev):
    from paper_2011_01400_gb300 import gw
    ss = systems()
    pbs = [gw.Problem(s, prec) for s in ss]
    plan = gw.gw_plan_create([pb.prob for pb in pbs])
    accs = [torch.zeros((s.n_k, s.sigma_hi - s.sigma_lo, s.n_freq), dtype=torch.complex128, device="cuda")
            for s in ss]
    try:
        assert gw.gw_plan_n_sys(plan) == len(ss)
        gw.gw_g0w0_batch(plan, accs, n_threads=3)
        res = [gw.gw_qp(plan, i, s.n_k, s.sigma_hi - s.sigma_lo, sigma=accs[i]) for i, s in enumerate(ss)]
        # a per-system call on the batch plan is routed to that system
        f, _ = gw.gw_plan_freq(plan, ss[0].n_freq)
        assert len(f) == ss[0].n_freq
    finally:
        gw.gw_plan_destroy(plan)
    for i, s in enumerate(ss):
        sig = accs[i].cpu().numpy()
        sig1, e1, gap1 = single(gw, s, prec)
        ref = O.g0w0(s)
        scale = np.abs(sig1).max()
        assert np.abs(sig - sig1).max() <= tol_same * scale, f"system {i}: batch differs from its own plan"
        err = np.abs(sig - ref["sigma"]).max() * HA_MEV
        print(f"{prec} system {i} ({s.n_k} k, {s.n_bands} bands, {s.n_aux} ABF, {s.n_freq} w): "
              f"Sigma_c vs oracle {err:.2e} meV")
        assert err <= tol_mev
        e, gap, _ = res[i]
        if ref["gap"] is not None:
            assert abs(gap - ref["gap"]) * HA_MEV <= tol_mev


def test_batch_rejects_bad_system_index():
    from paper_2011_01400_gb300 import gw
    ss = systems()[:2]
    pbs = [gw.Problem(s, "fp64") for s in ss]
    plan = gw.gw_plan_create([pb.prob for pb in pbs])
    try:
        with pytest.raises(gw.GwError) as ei:
            gw.gw_chi0(plan, 2, 0)
        assert ei.value.status == gw.GW_ERR_ARG
        gw.gw_chi0(plan, 1, 0)   # in range: routed to system 1
    finally:
        gw.gw_plan_destroy(plan)
