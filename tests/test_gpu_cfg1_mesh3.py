"""The benchmarked call sequence (plan, gw_g0w0 over every q, gw_qp) at the band / ABF / frequency
shape of the Si-like workload (2 atoms, 78 NAO and bands, 4 occupied, 400 ABF, 32 frequencies,
Sigma_c for the 8 bands at the gap, q -> 0 head and wings on) on a 3x3x3 k mesh, so that the plain
FP64 GPU pass stays within a minute. Both split-precision paths must reproduce the FP64 GPU path's
Sigma_c, QP energies and indirect gap within 1 meV; the FP64 path itself is tied to the oracle at
this shape by tests/test_gpu_fullsize.py (q = 0 and q = 1 terms, 1e-6 meV)."""
import numpy as np
import pytest

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


def g0w0(s, prec):
    from paper_2011_01400_gb300 import gw
    nsig = s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_g0w0(plan, 0, acc)
        e, gap, nconv = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return acc.cpu().numpy(), e, gap, nconv


@pytest.fixture(scope="module")
def mesh3():
    s = make_system("cfg1", seed=1000, nk=(3, 3, 3))
    return s, g0w0(s, "fp64")


@pytest.mark.parametrize("prec", ["3xbf16", "3xtf32", "3xfp16"])
def test_split_g0w0_matches_fp64_gpu_within_1mev(mesh3, prec):
    s, (sig64, e64, gap64, nc64) = mesh3
    nsig = s.sigma_hi - s.sigma_lo
    sig, e, gap, nc = g0w0(s, prec)
    es = np.abs(sig - sig64).max() * HA_MEV
    ee = np.abs(e - e64).max() * HA_MEV
    eg = abs(gap - gap64) * HA_MEV
    print(f"cfg1 shape, 3x3x3 k, {prec} vs FP64 GPU: Sigma_c {es:.3e} meV, E_qp {ee:.3e} meV, "
          f"gap {eg:.3e} meV (gap {gap64 * HA_MEV:.1f} meV)")
    assert nc == nc64 == s.n_k * nsig
    assert np.isfinite(gap64) and 0.0 < gap64 < 1.0
    assert es <= 1.0 and ee <= 1.0 and eg <= 1.0
