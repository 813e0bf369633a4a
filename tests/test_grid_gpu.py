"""A caller-supplied imaginary-frequency grid (gw_problem.freq / freq_w) through the C ABI, against the
FP64 oracle run on the same grid: the tangent-mapped midpoint rule w_j = w0 tan(t_j), a grid the
default construction never makes, in its natural and in reversed order.

Tolerances as for the default grid: FP64 Sigma_c, E_QP and the gap within 1e-6 meV; split
precision within 1 meV."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system

HA_MEV = 27211.386

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


def tan_midpoint(n, w0):
    t = (np.arange(n) + 0.5) * np.pi / (2 * n)
    return w0 * np.tan(t), w0 * (np.pi / (2 * n)) / np.cos(t) ** 2


def run(system, prec, grid):
    from paper_2011_01400_gb300 import gw
    pb = gw.Problem(system, prec, grid=grid)
    plan = gw.gw_plan_create(pb.prob)
    nsig = system.sigma_hi - system.sigma_lo
    acc = torch.zeros((system.n_k, nsig, system.n_freq), dtype=torch.complex128, device="cuda")
    try:
        f, w = gw.gw_plan_freq(plan, system.n_freq)
        for q in range(system.n_k):
            gw.gw_chi0(plan, 0, q)
            gw.gw_screen(plan, 0, q)
            gw.gw_sigma(plan, 0, q, acc)
        e, gap, nconv = gw.gw_qp(plan, 0, system.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return dict(freq=f, w=w, sigma=acc.cpu().numpy(), e_qp=e, gap=gap, nconv=nconv)


@pytest.fixture(scope="module")
def case():
    s = make_system("cfg0", seed=0)
    grid = tan_midpoint(s.n_freq, 2.0)
    rev = (grid[0][::-1].copy(), grid[1][::-1].copy())
    return s, grid, rev, O.g0w0(s, grid=grid), O.g0w0(s, grid=rev)


@pytest.mark.parametrize("prec,tol_mev", [("fp64", 1e-6), ("3xbf16", 1.0), ("3xfp16", 1.0)])
@pytest.mark.parametrize("order", ["ascending", "reversed"])
def test_caller_grid_matches_oracle(case, prec, tol_mev, order):
    s, grid, rev, ref_a, ref_r = case
    g, ref = (grid, ref_a) if order == "ascending" else (rev, ref_r)
    out = run(s, prec, g)
    assert np.array_equal(out["freq"], g[0]) and np.array_equal(out["w"], g[1])
    err_sig = np.abs(out["sigma"] - ref["sigma"]).max() * HA_MEV
    err_e = np.abs(out["e_qp"] - ref["e_qp"]).max() * HA_MEV
    err_gap = abs(out["gap"] - ref["gap"]) * HA_MEV
    print(f"{prec} {order}: Sigma_c {err_sig:.3e} meV, E_qp {err_e:.3e} meV, gap {err_gap:.3e} meV")
    assert out["nconv"] == s.n_k * (s.sigma_hi - s.sigma_lo) and ref["converged"].all()
    assert err_sig <= tol_mev and err_e <= tol_mev and err_gap <= tol_mev
