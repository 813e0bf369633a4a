"""The declared failure statuses of the C ABI, produced on the GPU by inputs the host builds (no
fault, trap or hang is provoked):

- GW_ERR_NOT_PD: occupied levels at k lie above empty levels at k + q, so some transition
  energies D = eps_a(k+q) - eps_i(k) are negative, the Lorentzian weights 2D/(w^2 + D^2) change
  sign, chi0(q) is no longer negative semidefinite and eps~ = 1 - V^1/2 chi0 V^1/2 has negative
  eigenvalues (down to about -100 at the lowest frequency for this system). The FP64 Cholesky
  factorisation meets a non-positive pivot and the call reports it; the plan then stays in its
  error state. The surrogate's ridge fit reports the same status for x = 0 and ridge 0.
- GW_ERR_NOMEM: the workspace cap GW_WORKSPACE_LIMIT refuses an allocation before cudaMalloc.
GW_ERR_TIMEOUT is not produced here: every bounded wait of the tensor-core kernel guards a
pipeline whose bulk copies or MMAs are in flight, and no host-built input makes one of those
waits run out.
"""
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


def inverted_system():
    s = make_system("tiny", seed=7, nk=(2, 1, 1), head_wings=0, c_scale=1.0)
    s.eps = np.array([[0.80, 0.90, 1.00, 1.10, 1.20, 1.30],
                      [-0.90, -0.80, -0.70, -0.60, -0.50, -0.40]])
    return s


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "3xbf16"])
def test_indefinite_eps_reports_not_pd(prec):
    from paper_2011_01400_gb300 import gw
    s = inverted_system()
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_chi0(plan, 0, 1)
        with pytest.raises(gw.GwError) as ei:
            gw.gw_screen(plan, 0, 1)
        assert ei.value.status == gw.GW_ERR_NOT_PD
        with pytest.raises(gw.GwError) as ei:      # the error sticks until destroy
            gw.gw_chi0(plan, 0, 0)
        assert ei.value.status == gw.GW_ERR_STATE
    finally:
        gw.gw_plan_destroy(plan)
    plan = gw.gw_plan_create(pb.prob)
    try:
        with pytest.raises(gw.GwError) as ei:
            gw.gw_g0w0(plan, 0)
        assert ei.value.status == gw.GW_ERR_NOT_PD
    finally:
        gw.gw_plan_destroy(plan)
    # a regular system in a fresh plan still works afterwards
    ok = make_system("tiny", seed=1)
    pb2 = gw.Problem(ok, prec)
    plan = gw.gw_plan_create(pb2.prob)
    try:
        gw.gw_g0w0(plan, 0)
    finally:
        gw.gw_plan_destroy(plan)


def test_ridge_fit_of_zero_inputs_reports_not_pd():
    from paper_2011_01400_gb300 import gw
    from paper_2011_01400_gb300.synth import surrogate_init
    dims = (4, 16, 6)
    m = gw.gw_surrogate_create(*dims, torch.from_numpy(surrogate_init(*dims)).cuda())
    try:
        x = torch.zeros((32, dims[0]), device="cuda")
        y = torch.ones((32, dims[2]), device="cuda")
        with pytest.raises(gw.GwError) as ei:
            gw.gw_surrogate_fit_linear(m, x, y, 0.0)
        assert ei.value.status == gw.GW_ERR_NOT_PD
    finally:
        gw.gw_surrogate_destroy(m)


def test_workspace_limit_reports_nomem(monkeypatch):
    from paper_2011_01400_gb300 import gw
    s = make_system("tiny", seed=1)
    pb = gw.Problem(s, "3xbf16")
    monkeypatch.setenv("GW_WORKSPACE_LIMIT", "4096")
    with pytest.raises(gw.GwError) as ei:
        gw.gw_plan_create(pb.prob)
    assert ei.value.status == gw.GW_ERR_NOMEM
    assert "GW_WORKSPACE_LIMIT" in str(ei.value)
    monkeypatch.delenv("GW_WORKSPACE_LIMIT")
    plan = gw.gw_plan_create(pb.prob)
    gw.gw_plan_destroy(plan)
