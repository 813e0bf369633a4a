"""gw_qp_static (QP solve with fixed device scratch, no allocation) against gw_qp.

Collected last on purpose: it must also hold after every other GPU test has run in the same
process (the scratch array is looked up once per device and then reused).
"""
import numpy as np
import pytest

from paper_2011_01400_gb300.synth import make_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_HA = 1e-12  # same kernel and inputs as gw_qp: agreement to rounding of the host copy


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_qp_static_matches_qp_twice(prec):
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=11)
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_g0w0(plan, 0)  # the plan's own Sigma_c accumulator
        e_ref, gap_ref, nc_ref = gw.gw_qp(plan, 0, s.n_k, nsig)
        for _ in range(2):
            e, gap, nc = gw.gw_qp_static(plan, 0, s.n_k, nsig)
            assert np.abs(e - e_ref).max() <= TOL_HA
            assert abs(gap - gap_ref) <= TOL_HA
            assert nc == nc_ref == s.n_k * nsig
        # caller-owned Sigma_c and a non-zero Sigma_x - v_xc shift
        acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
        gw.gw_g0w0(plan, 0, acc)
        dxv = torch.linspace(-0.05, 0.05, s.n_k * nsig, dtype=torch.float64, device="cuda").reshape(s.n_k, nsig)
        e_ref, gap_ref, nc_ref = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc, dxv=dxv)
        for _ in range(2):
            e, gap, nc = gw.gw_qp_static(plan, 0, s.n_k, nsig, sigma=acc, dxv=dxv)
            assert np.abs(e - e_ref).max() <= TOL_HA
            assert abs(gap - gap_ref) <= TOL_HA
            assert nc == nc_ref
    finally:
        gw.gw_plan_destroy(plan)
