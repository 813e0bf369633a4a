"""Parity at the benchmark's full size: cfg1 (6x6x6 k, 78 bands, 400 ABF, 32 frequencies), the
system bench.py times (seed 1000), through the same C-ABI calls. The oracle can afford two q of
it (about a minute and a half each on the host cores): chi0 at every frequency, eps~ / W^c and the
q term of Sigma_c for every k and band of the window, at q = 1 and at q = 0 (the head and wings of
the dielectric matrix, Eq. dielectric_func_gamma)."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HA_MEV = 27211.386
Q = 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def cfg1_q1():
    s = make_system("cfg1", seed=1000)
    om, g = O.freq_grid(s.n_freq, s.omega0)
    chi = O.chi0(s, Q, om)
    _, W = O.screen(s, Q, chi, om)
    sig = O.sigma_q(s, Q, W, om, g, O.mu_midgap(s))
    return s, chi, W, sig


@pytest.fixture(scope="module")
def cfg1_q0():
    s = make_system("cfg1", seed=1000)
    assert s.head_wings == 1
    om, g = O.freq_grid(s.n_freq, s.omega0)
    chi = O.chi0(s, 0, om)
    _, W = O.screen(s, 0, chi, om)
    sig = O.sigma_q(s, 0, W, om, g, O.mu_midgap(s))
    return s, chi, W, sig


def rel_fro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("qcase", ["cfg1_q1", "cfg1_q0"])
@pytest.mark.parametrize("prec,tol_chi,tol_w,tol_sig_mev",
                         [("3xbf16", 1e-6, 1e-4, 1.0), ("3xtf32", 1e-6, 1e-4, 1.0), ("3xfp16", 1e-6, 1e-4, 1.0),
                          ("fp64", 1e-11, 1e-9, 1e-6)])
def test_cfg1_one_q_full_size(request, qcase, prec, tol_chi, tol_w, tol_sig_mev):
    """chi0 and Sigma_c hold their targets (1e-6 relative, 1 meV). W^c has none of its own: on the
    split path its screen products are FP32 (~1e-7 relative per term), and at the highest
    frequencies W^c = V^1/2 (eps~^-1 - 1) V^1/2 is a difference 1e-2..1e-3 of its terms, so its
    relative error is bounded by 1e-4 (cfg1, q = 1: 1.2e-5). On the FP64 path the bound is 1e-9:
    at q = 0 the Coulomb head eigenvalue (~40 here) enters W^c squared-root-wise on both sides and
    the same difference of terms leaves 2e-10 (q = 1: 7.6e-11)."""
    from paper_2011_01400_gb300 import gw
    s, chi_ref, W_ref, sig_ref = request.getfixturevalue(qcase)
    Q = 0 if qcase == "cfg1_q0" else 1
    N, nw, nsig = s.n_aux, s.n_freq, s.sigma_hi - s.sigma_lo
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    chi = torch.empty((nw, N, N), dtype=torch.complex128, device="cuda")
    W = torch.empty((nw, N, N), dtype=torch.complex128, device="cuda")
    acc = torch.zeros((s.n_k, nsig, nw), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_chi0(plan, 0, Q, chi)
        gw.gw_screen(plan, 0, Q, W)
        gw.gw_sigma(plan, 0, Q, acc)
    finally:
        gw.gw_plan_destroy(plan)
    chi, W, sig = chi.cpu().numpy(), W.cpu().numpy(), acc.cpu().numpy()
    ec = max(rel_fro(chi[j], chi_ref[j]) for j in range(nw))
    ew = max(rel_fro(W[j], W_ref[j]) for j in range(nw))
    es = np.abs(sig - sig_ref).max() * HA_MEV
    print(f"cfg1 q={Q} {prec}: chi0 {ec:.2e}, W^c {ew:.2e}, Sigma_c term {es:.2e} meV")
    assert ec <= tol_chi and ew <= tol_w and es <= tol_sig_mev


def test_cfg2_chi0_sampled_block():
    """cfg2 (ZnO-like: 4 atoms, 6x6x4 k, 300 bands with 36 occupied, 1600 ABF, 32 frequencies; M
    streamed per chunk of k): chi0 at q = 1 on a sampled 6 x 6 block of ABFs spread over all atoms,
    against the oracle's block form, relative Frobenius <= 1e-6 per frequency (3xBF16)."""
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg2", seed=2000)
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    mus = [0, 399, 400, 801, 1203, 1599]
    js = [0, 7, 15, 23, 31]
    ref = O.chi0_block(s, Q, om[js], mus)
    pb = gw.Problem(s, "3xbf16")
    plan = gw.gw_plan_create(pb.prob)
    chi = torch.empty((s.n_freq, s.n_aux, s.n_aux), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_chi0(plan, 0, Q, chi)
    finally:
        gw.gw_plan_destroy(plan)
    idx = torch.tensor(mus, device="cuda")
    got = chi[js][:, idx][:, :, idx].cpu().numpy()
    del chi
    err = max(rel_fro(got[j], ref[j]) for j in range(len(js)))
    print(f"cfg2 q={Q} 3xbf16: chi0 sampled block {err:.2e}")
    assert err <= 1e-6
