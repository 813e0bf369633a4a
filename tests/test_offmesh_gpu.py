"""Sigma_c off the k mesh (gw_problem.k_offset, gw_sigma_ext, paper_2011_01400_gb300/bands.py):
W^c(q) of the ordinary plan contracted with the rows of a plan on the shifted mesh, against the
oracle's Sigma_c of the shifted system with the same W^c; and the k range of gw_sigma_ext."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system, shifted_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HA_MEV = 27211.386


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    s = make_system("cfg0", seed=41)
    t = shifted_system(s, (0.25, 0.125, -0.3), seed=42)
    om, g = O.freq_grid(s.n_freq, s.omega0)
    mu = O.mu_midgap(s)
    ref = np.zeros((s.n_k, s.sigma_hi - s.sigma_lo, s.n_freq), dtype=np.complex128)
    for q in range(s.n_k):
        _, W = O.screen(s, q, O.chi0(s, q, om), om)
        ref += O.sigma_q(t, q, W, om, g, mu)
    return s, t, mu, ref


@pytest.mark.parametrize("prec,tol_mev", [("fp64", 1e-6), ("3xfp16", 1.0), ("3xtf32", 1.0)])
def test_offmesh_sigma_matches_oracle(case, prec, tol_mev):
    from paper_2011_01400_gb300 import bands, gw
    s, t, mu, ref = case
    nsig = s.sigma_hi - s.sigma_lo
    pb, pt = gw.Problem(s, prec), gw.Problem(t, prec, mu=mu)
    accs, qps = bands.sigma_offmesh(gw, pb.prob, [pt.prob], s.n_k, nsig, s.n_freq, s.n_aux)
    sig = accs[0].cpu().numpy()
    err = np.abs(sig - ref).max() * HA_MEV
    print(f"{prec}: off-mesh Sigma_c vs oracle {err:.2e} meV")
    assert err <= tol_mev
    E, _, conv = O.qp(t, ref, O.freq_grid(s.n_freq, s.omega0)[0], mu)
    assert np.abs(qps[0] - E).max() * HA_MEV <= tol_mev


def test_k_range_touches_only_its_rows(case):
    from paper_2011_01400_gb300 import bands, gw
    s, t, mu, ref = case
    nsig = s.sigma_hi - s.sigma_lo
    pb, pt = gw.Problem(s, "fp64"), gw.Problem(t, "fp64", mu=mu)
    accs, _ = bands.sigma_offmesh(gw, pb.prob, [pt.prob], s.n_k, nsig, s.n_freq, s.n_aux, k_range=(0, 1))
    sig = accs[0].cpu().numpy()
    assert np.abs(sig[0] - ref[0]).max() * HA_MEV <= 1e-6
    assert np.abs(sig[1:]).max() == 0.0
