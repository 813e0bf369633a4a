"""gw_qp_static (QP solve with fixed device scratch, no allocation) against gw_qp.

Some callers cannot allocate device memory at the moment they re-solve the QP equation: a
process whose device memory is held by a caching allocator, or a serving loop that cannot take
the device-wide synchronisation of cudaFree. gw_qp_static serves them with its scratch in a
fixed array of the library; these tests check that it gives gw_qp's results, that it makes no
device allocation and launches exactly its two kernels, that it refuses sizes beyond its
capacity before launching anything, and that calls on the systems of a batch plan, a larger
one followed by a smaller one, do not read stale scratch.

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


def static_calls_match(gw, plan, sys, n_k, nsig, **kw):
    """Two gw_qp_static calls in a row against gw_qp: same energies, gap and converged count,
    no device allocation, two kernel launches per call."""
    e_ref, gap_ref, nc_ref = gw.gw_qp(plan, sys, n_k, nsig, **kw)
    for _ in range(2):
        a0, l0 = gw.gw_device_allocations(), gw.gw_kernel_launches()
        e, gap, nc = gw.gw_qp_static(plan, sys, n_k, nsig, **kw)
        assert gw.gw_device_allocations() == a0
        assert gw.gw_kernel_launches() == l0 + 2
        assert np.abs(e - e_ref).max() <= TOL_HA
        assert abs(gap - gap_ref) <= TOL_HA
        assert nc == nc_ref
    return nc_ref


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_qp_static_matches_qp_twice(prec):
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=11)
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_g0w0(plan, 0)  # the plan's own Sigma_c accumulator
        assert static_calls_match(gw, plan, 0, s.n_k, nsig) == s.n_k * nsig
        # caller-owned Sigma_c and a non-zero Sigma_x - v_xc shift
        acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
        gw.gw_g0w0(plan, 0, acc)
        dxv = torch.linspace(-0.05, 0.05, s.n_k * nsig, dtype=torch.float64, device="cuda").reshape(s.n_k, nsig)
        static_calls_match(gw, plan, 0, s.n_k, nsig, sigma=acc, dxv=dxv)
    finally:
        gw.gw_plan_destroy(plan)


def test_qp_static_on_a_batch_plan_larger_then_smaller():
    from paper_2011_01400_gb300 import gw
    ss = [make_system("tiny", seed=12),                     # 4 k x 4 bands = 16 pairs
          make_system("cfg0", seed=13, n_freq=12)]          # 8 k x 4 bands = 32 pairs
    pbs = [gw.Problem(s, "3xtf32") for s in ss]
    plan = gw.gw_plan_create([pb.prob for pb in pbs])
    try:
        gw.gw_g0w0_batch(plan)
        for i in (1, 0):
            s = ss[i]
            static_calls_match(gw, plan, i, s.n_k, s.sigma_hi - s.sigma_lo)
    finally:
        gw.gw_plan_destroy(plan)


def test_qp_static_rejects_sizes_beyond_capacity():
    from paper_2011_01400_gb300 import gw
    s = make_system("tiny", seed=14, nk=(17, 16, 16))        # 4352 k x 4 bands > 16384 pairs
    nsig = s.sigma_hi - s.sigma_lo
    assert s.n_k * nsig > 16384
    pb = gw.Problem(s, "fp64")
    plan = gw.gw_plan_create(pb.prob)
    try:
        a0, l0 = gw.gw_device_allocations(), gw.gw_kernel_launches()
        with pytest.raises(gw.GwError) as ei:
            gw.gw_qp_static(plan, 0, s.n_k, nsig)
        assert ei.value.status == gw.GW_ERR_ARG
        assert "GW_QP_STATIC_MAX" in str(ei.value)
        assert gw.gw_device_allocations() == a0 and gw.gw_kernel_launches() == l0
    finally:
        gw.gw_plan_destroy(plan)
