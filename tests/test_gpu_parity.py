"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on identical seeded inputs.

Tolerances: FP64 method 1e-11 relative; split precision (3xTF32, 3xBF16, 3xFP16) relative
Frobenius error of chi0 <= 1e-6 per (q, w); Sigma_c and the QP gap within 1 meV. W^c has no target
of its own: W^c = V^1/2 (eps~^-1 - 1) V^1/2 is, at the top frequencies, a difference 1e-2..1e-3 of
its terms, so its relative error is the terms' rounding divided by that ratio; it is bounded at
1e-10 (FP64) and 1e-5 (split) here.
"""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system

HA_MEV = 27211.386
MEV = 1.0 / HA_MEV

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


def run_gpu(system, prec, qs=None, keep=False):
    from paper_2011_01400_gb300 import gw
    pb = gw.Problem(system, prec)
    plan = gw.gw_plan_create(pb.prob)
    N, nw = system.n_aux, system.n_freq
    out = dict(chi0={}, Wc={})
    try:
        qs = range(system.n_k) if qs is None else qs
        for q in qs:
            c = torch.empty((nw, N, N), dtype=torch.complex128, device="cuda") if keep else None
            w = torch.empty((nw, N, N), dtype=torch.complex128, device="cuda") if keep else None
            gw.gw_chi0(plan, 0, q, c)
            gw.gw_screen(plan, 0, q, w)
            gw.gw_sigma(plan, 0, q, None)
            if keep:
                out["chi0"][q] = c.cpu().numpy()
                out["Wc"][q] = w.cpu().numpy()
        nsig = system.sigma_hi - system.sigma_lo
        sig = torch.empty((system.n_k, nsig, nw), dtype=torch.complex128, device="cuda")
        # the plan's own accumulator is read back through gw_qp; also fetch it by re-running qp on a copy
        e, gap, nconv = gw.gw_qp(plan, 0, system.n_k, nsig)
        out.update(e_qp=e, gap=gap, nconv=nconv)
        out["freq"] = gw.gw_plan_freq(plan, nw)
        out["mu"] = gw.gw_plan_mu(plan)
    finally:
        gw.gw_plan_destroy(plan)
    return out


def run_gpu_sigma(system, prec, qs):
    """Sigma_c summed over qs into a caller-owned accumulator."""
    from paper_2011_01400_gb300 import gw
    pb = gw.Problem(system, prec)
    plan = gw.gw_plan_create(pb.prob)
    nsig = system.sigma_hi - system.sigma_lo
    acc = torch.zeros((system.n_k, nsig, system.n_freq), dtype=torch.complex128, device="cuda")
    try:
        for q in qs:
            gw.gw_chi0(plan, 0, q)
            gw.gw_screen(plan, 0, q)
            gw.gw_sigma(plan, 0, q, acc)
        e, gap, nconv = gw.gw_qp(plan, 0, system.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return acc.cpu().numpy(), e, gap, nconv


def rel_fro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def cfg0():
    s = make_system("cfg0", seed=0)
    ref = O.g0w0(s, keep=True)
    return s, ref


def test_frequency_grid_and_mu_match(cfg0):
    s, ref = cfg0
    out = run_gpu(s, "fp64", qs=[])
    f, w = out["freq"]
    assert np.abs(f - ref["omega"]).max() < 1e-12 * ref["omega"].max()
    assert np.abs(w - ref["g"]).max() < 1e-12 * ref["g"].max()
    assert abs(out["mu"] - ref["mu"]) < 1e-15


@pytest.mark.parametrize("prec,tol_chi,tol_w", [("fp64", 1e-11, 1e-10), ("3xtf32", 1e-6, 1e-5), ("3xbf16", 1e-6, 1e-5),
                                                ("3xfp16", 1e-6, 1e-5)])
def test_chi0_and_wc_cfg0(cfg0, prec, tol_chi, tol_w):
    s, ref = cfg0
    out = run_gpu(s, prec, keep=True)
    worst_c = worst_w = 0.0
    for q in range(s.n_k):
        for j in range(s.n_freq):
            worst_c = max(worst_c, rel_fro(out["chi0"][q][j], ref["per_q"][q]["chi0"][j]))
            worst_w = max(worst_w, rel_fro(out["Wc"][q][j], ref["per_q"][q]["Wc"][j]))
    print(f"{prec}: chi0 worst rel-Frobenius {worst_c:.3e}, W^c {worst_w:.3e}")
    assert worst_c <= tol_chi
    assert worst_w <= tol_w


@pytest.mark.parametrize("prec,tol_mev", [("fp64", 1e-6), ("3xtf32", 1.0), ("3xbf16", 1.0), ("3xfp16", 1.0)])
def test_sigma_qp_gap_cfg0(cfg0, prec, tol_mev):
    s, ref = cfg0
    sig, e, gap, nconv = run_gpu_sigma(s, prec, range(s.n_k))
    err_sig = np.abs(sig - ref["sigma"]).max() * HA_MEV
    err_e = np.abs(e - ref["e_qp"]).max() * HA_MEV
    err_gap = abs(gap - ref["gap"]) * HA_MEV
    print(f"{prec}: Sigma_c max err {err_sig:.3e} meV, E_qp {err_e:.3e} meV, gap {err_gap:.3e} meV")
    assert nconv == s.n_k * (s.sigma_hi - s.sigma_lo) and ref["converged"].all()
    assert err_sig <= tol_mev and err_e <= tol_mev and err_gap <= tol_mev


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "3xbf16", "3xfp16"])
def test_g0w0_driver_matches_per_q_calls(cfg0, prec):
    """gw_g0w0 (q groups, batched FP64 factorisations) gives the per-q result and the oracle's."""
    from paper_2011_01400_gb300 import gw
    s, ref = cfg0
    sig_q, e_q, gap_q, _ = run_gpu_sigma(s, prec, range(s.n_k))
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    nsig = s.sigma_hi - s.sigma_lo
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_g0w0(plan, 0, acc)
        e, gap, nconv = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
        ms, fl = gw.gw_plan_last_chi0_stats(plan)
    finally:
        gw.gw_plan_destroy(plan)
    sig = acc.cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-9
    assert np.abs(sig - sig_q).max() <= tol * np.abs(sig_q).max() * 100
    assert np.abs(sig - ref["sigma"]).max() * HA_MEV < (1e-6 if prec == "fp64" else 1.0)
    assert abs(gap - ref["gap"]) * HA_MEV < (1e-6 if prec == "fp64" else 1.0)
    assert ms > 0 and fl > 0


@pytest.mark.parametrize("prec,tol_mev", [("fp64", 1e-6), ("3xtf32", 1.0), ("3xbf16", 1.0)])
def test_sigma_x_cfg0(prec, tol_mev):
    """Exchange self-energy against the oracle (FP64 path to rounding; split paths use FP32 products)."""
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=0)
    ref = O.sigma_x(s)
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    try:
        out = torch.empty((s.n_k, s.sigma_hi - s.sigma_lo), dtype=torch.float64, device="cuda")
        gw.gw_sigma_x(plan, 0, out)
        gw.gw_sigma_x(plan, 0, out)      # overwritten, not accumulated
        got = out.cpu().numpy()
    finally:
        gw.gw_plan_destroy(plan)
    err = np.abs(got - ref).max() * HA_MEV
    print(f"{prec}: Sigma_x max err {err:.3e} meV (|Sigma_x| max {np.abs(ref).max() * HA_MEV:.0f} meV)")
    assert err <= tol_mev
    if prec == "fp64":
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("window", [(0, 4), (1, 3)])
def test_qp_gap_selection_hand_built(window):
    """gw_qp and gw_qp_static on the hand-built case of tests/qp_case.py (caller-owned Sigma_c
    and Sigma_x - v_xc): the QP energies, the indirect gap known by construction, and the
    midgap chemical potential."""
    import qp_case as C
    from paper_2011_01400_gb300 import gw
    s = C.system(window)
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, "fp64")
    plan = gw.gw_plan_create(pb.prob)
    try:
        f, _ = gw.gw_plan_freq(plan, s.n_freq)
        sig = torch.from_numpy(C.sigma_c(s, f)).cuda()
        dxv = torch.from_numpy(C.dxv(s)).cuda()
        for call in (gw.gw_qp, gw.gw_qp_static):
            e, gap, nconv = call(plan, 0, s.n_k, nsig, sigma=sig, dxv=dxv)
            assert nconv == s.n_k * nsig
            assert np.abs(e - C.e_expected(s)).max() < 1e-8
            assert abs(gap - C.GAP) < 1e-8
        assert abs(gw.gw_plan_mu(plan) - C.MU) < 1e-15
    finally:
        gw.gw_plan_destroy(plan)


@pytest.fixture(scope="module")
def cfg0_avg():
    s = make_system("cfg0", seed=0, head_wings=2)
    om, g = O.freq_grid(s.n_freq, s.omega0)
    chi = O.chi0(s, 0, om)
    _, W = O.screen(s, 0, chi, om)
    ref = O.g0w0(s)
    return s, W, ref


@pytest.mark.parametrize("prec,tol_w,tol_mev", [("fp64", 1e-10, 1e-6), ("3xbf16", 1e-5, 1.0), ("3xfp16", 1e-5, 1.0)])
def test_direction_averaged_q0(cfg0_avg, prec, tol_w, tol_mev):
    """head_wings = 2: W^c(0) from eps~^-1 - 1 averaged over the directions of q -> 0 (the oracle
    inverts eps~ for each of the 128 directions; the library uses the Schur-complement form on
    the inverse of the body), then the whole pass: Sigma_c and the gap against the oracle."""
    from paper_2011_01400_gb300 import gw
    s, W_ref, ref = cfg0_avg
    N, nw, nsig = s.n_aux, s.n_freq, s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    W = torch.empty((nw, N, N), dtype=torch.complex128, device="cuda")
    acc = torch.zeros((s.n_k, nsig, nw), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_chi0(plan, 0, 0)
        gw.gw_screen(plan, 0, 0, W)
        gw.gw_g0w0(plan, 0, acc)
        e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    W = W.cpu().numpy()
    ew = max(rel_fro(W[j], W_ref[j]) for j in range(nw))
    es = np.abs(acc.cpu().numpy() - ref["sigma"]).max() * HA_MEV
    eg = abs(gap - ref["gap"]) * HA_MEV
    print(f"{prec} averaged q=0: W^c {ew:.2e}, Sigma_c {es:.2e} meV, gap {eg:.2e} meV")
    assert ew <= tol_w and es <= tol_mev and eg <= tol_mev
