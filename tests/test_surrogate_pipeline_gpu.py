"""The surrogate-accelerated G0W0 pass on the GPU against the oracle, and the gain of the
trained network over the method without it."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from oracle import surrogate as S
from paper_2011_01400_gb300.synth import make_system, surrogate_init, surrogate_start

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HA_MEV = 27211.386


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_01400_gb300 import build
    build.build()


def cdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def fdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_modes_match_oracle():
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=3, n_freq=20)
    coarse, k, nb, nit = [0, 5, 10, 15], 8, 16, 30
    start = surrogate_start(s.n_aux, nb, seed=1)
    pb = gw.Problem(s, "fp64")
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_surrogate_enable(plan, None, coarse, k, nb, nit, cdev(start))
        for q in (0, 3):
            gw.gw_chi0(plan, 0, q)
            d = torch.empty((k, s.n_freq), device="cuda")
            th = torch.empty(k, dtype=torch.float64, device="cuda")
            x = torch.empty((k, len(coarse)), device="cuda")
            y = torch.empty((k, s.n_freq - len(coarse)), device="cuda")
            gw.gw_surrogate_modes(plan, 0, q, d, th, x, y)
            d_ref, th_ref = S.mode_data(s, q, start, nit, k)
            fine = [j for j in range(s.n_freq) if j not in coarse]
            x_ref, y_ref, _ = S.features(d_ref, coarse, fine)
            assert np.allclose(th.cpu().numpy(), th_ref, rtol=1e-10, atol=0)
            assert np.abs(d.cpu().numpy() - d_ref).max() <= 2e-6 * np.abs(d_ref).max()
            assert np.abs(x.cpu().numpy() - x_ref).max() <= 2e-6
            assert np.abs(y.cpu().numpy() - y_ref).max() <= 2e-6
    finally:
        gw.gw_plan_destroy(plan)


@pytest.mark.parametrize("prec,tol_mev", [("fp64", 1e-2), ("3xtf32", 1.0)])
def test_surrogate_g0w0_matches_oracle(prec, tol_mev):
    """The FP64 pass keeps the network, its inputs and the fine-frequency correction in fp32, so
    it meets the oracle to fp32 rounding of that correction (1e-2 meV on Sigma_c ~ 4e4 meV)."""
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=4, n_freq=20)
    coarse, k, nb, nit = [0, 4, 8, 12, 16], 12, 24, 10
    fine = [j for j in range(s.n_freq) if j not in coarse]
    dims = (len(coarse), 32, len(fine))
    start = surrogate_start(s.n_aux, nb, seed=2)
    # a realistic linear part from the oracle's own mode data, a random MLP with a visible output
    xs, ys = [], []
    for q in range(s.n_k):
        d, _ = S.mode_data(s, q, start, nit, k)
        x, y, _ = S.features(d, coarse, fine)
        xs.append(x)
        ys.append(y)
    L, _ = S.fit_linear(np.concatenate(xs), np.concatenate(ys), 1e-8)
    th = surrogate_init(*dims, seed=5, out_gain=1.0).astype(np.float64)
    o_L = S.n_params(*dims) - dims[0] * dims[2] - 1
    th[o_L:-1] = L.ravel()
    th[-1] = 0.02
    th = th.astype(np.float32)
    ref = S.g0w0_surrogate(s, th.astype(np.float64), dims, coarse, start, nit, k)
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    model = gw.gw_surrogate_create(*dims, fdev(th))
    nsig = s.sigma_hi - s.sigma_lo
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_surrogate_enable(plan, model, coarse, k, nb, nit, cdev(start))
        gw.gw_g0w0(plan, 0, acc)
        e, gap, nconv = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
        gw.gw_surrogate_destroy(model)
    err = np.abs(acc.cpu().numpy() - ref["sigma"]).max() * HA_MEV
    print(f"{prec}: surrogate Sigma_c vs oracle {err:.3e} meV; gap {abs(gap - ref['gap']) * HA_MEV:.3e} meV")
    assert err <= tol_mev
    assert abs(gap - ref["gap"]) * HA_MEV <= tol_mev


def gpu_mode_features(gw, s, coarse, k, nb, nit, start, prec="fp64", moments=None):
    """(x, y) training rows of one system from the plain method on the full grid (GPU); the
    frequency moments of eps~^-1 - 1 are added into `moments` when given."""
    nc, nf = len(coarse), s.n_freq - len(coarse)
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    x = torch.empty((s.n_k * k, nc), device="cuda")
    y = torch.empty((s.n_k * k, nf), device="cuda")
    try:
        gw.gw_surrogate_enable(plan, None, coarse, k, nb, nit, start)
        gw.gw_surrogate_data(plan, 0, x, y, moments)
    finally:
        gw.gw_plan_destroy(plan)
    return x, y


def test_data_pass_matches_per_q_modes():
    from paper_2011_01400_gb300 import gw
    s = make_system("cfg0", seed=8, n_freq=20)
    coarse, k, nb, nit = [0, 5, 10, 15], 6, 12, 5
    start = cdev(surrogate_start(s.n_aux, nb, seed=4))
    mom = torch.zeros((len(coarse), s.n_freq), dtype=torch.float64, device="cuda")
    x_all, y_all = gpu_mode_features(gw, s, coarse, k, nb, nit, start, moments=mom)
    fine = [j for j in range(s.n_freq) if j not in coarse]
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    mom_ref = sum(S.freq_moments(S.inverse_minus_one(O.screen(s, q, O.chi0(s, q, om), om)[0]), coarse, fine)
                  for q in range(s.n_k))
    assert np.abs(mom.cpu().numpy() - mom_ref).max() <= 1e-10 * np.abs(mom_ref).max()
    pb = gw.Problem(s, "fp64")
    plan = gw.gw_plan_create(pb.prob)
    try:
        gw.gw_surrogate_enable(plan, None, coarse, k, nb, nit, start)
        for q in range(s.n_k):
            gw.gw_chi0(plan, 0, q)
            x = torch.empty((k, 4), device="cuda")
            y = torch.empty((k, 16), device="cuda")
            gw.gw_surrogate_modes(plan, 0, q, None, None, x, y)
            assert torch.allclose(x, x_all[q * k:(q + 1) * k], rtol=0, atol=1e-6)
            assert torch.allclose(y, y_all[q * k:(q + 1) * k], rtol=0, atol=1e-6)
    finally:
        gw.gw_plan_destroy(plan)


def surrogate_qp(gw, s, model, coarse, k, nb, nit, start, prec):
    pb = gw.Problem(s, prec)
    plan = gw.gw_plan_create(pb.prob)
    nsig = s.sigma_hi - s.sigma_lo
    acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
    try:
        gw.gw_surrogate_enable(plan, model, coarse, k, nb, nit, start)
        gw.gw_g0w0(plan, 0, acc)
        e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
    finally:
        gw.gw_plan_destroy(plan)
    return e, gap


def test_trained_surrogate_gains_over_the_coarse_method():
    """Train on the plain method's data of 8 systems (GPU): L from the frequency moments of
    eps~^-1 - 1, then Adam on the MLP over the mode rows. Evaluate on a ninth system: with chi0
    on 12 of 60 frequencies, the surrogate's QP energies and gap against the full 60-point FP64
    method, next to the plain method on a 12-point grid (the same chi0 work without the
    network) and the surrogate with its MLP switched off (linear part only)."""
    from paper_2011_01400_gb300 import gw
    NW, k, nb, nit = 60, 32, 48, 8
    coarse = list(range(0, NW, 5))
    dims = (len(coarse), 256, NW - len(coarse))
    start_np = surrogate_start(96, nb, seed=9)
    start = cdev(start_np)
    mom = torch.zeros((len(coarse), NW), dtype=torch.float64, device="cuda")
    X, Y = zip(*[gpu_mode_features(gw, make_system("cfg0", seed=100 + i, n_freq=NW), coarse, k, nb, nit, start,
                                   moments=mom) for i in range(8)])
    X, Y = torch.cat(X).contiguous(), torch.cat(Y).contiguous()
    s = make_system("cfg0", seed=7, n_freq=NW)
    Xv, Yv = gpu_mode_features(gw, s, coarse, k, nb, nit, start)
    model = gw.gw_surrogate_create(*dims, fdev(surrogate_init(*dims, seed=3)))
    try:
        gw.gw_surrogate_fit_moments(model, mom, 1e-10)
        rms_lin = gw.gw_surrogate_fit_scale(model, X, Y)
        f = torch.empty_like(Yv)
        gw.gw_surrogate_forward(model, Xv, f)
        val_lin = float(torch.sqrt(torch.mean((f - Yv) ** 2)))
        hist = gw.gw_surrogate_train(model, X, Y, 200, 128, 1e-3, 17)
        gw.gw_surrogate_forward(model, Xv, f)
        val_mlp = float(torch.sqrt(torch.mean((f - Yv) ** 2)))
        e_sur, gap_sur = surrogate_qp(gw, s, model, coarse, k, nb, nit, start, "fp64")
        # the same model with its MLP output switched off (W4 = 0, b4 = 0): linear part only
        th = torch.empty(gw.gw_surrogate_param_count(*dims), device="cuda")
        gw.gw_surrogate_get_params(model, th)
        p = th.cpu().numpy()
        o_W4 = S.n_params(*dims) - dims[0] * dims[2] - 1 - dims[2] - dims[2] * dims[1]
        p[o_W4:o_W4 + dims[2] * dims[1] + dims[2]] = 0.0
        lin = gw.gw_surrogate_create(*dims, fdev(p))
        try:
            e_lin, gap_lin = surrogate_qp(gw, s, lin, coarse, k, nb, nit, start, "fp64")
        finally:
            gw.gw_surrogate_destroy(lin)
    finally:
        gw.gw_surrogate_destroy(model)
    full = O.g0w0(s)
    c12 = O.g0w0(make_system("cfg0", seed=7, n_freq=len(coarse)))
    err = lambda e, g: (np.abs(e - full["e_qp"]).max() * HA_MEV, abs(g - full["gap"]) * HA_MEV)
    es, gs = err(e_sur, gap_sur)
    el, gl = err(e_lin, gap_lin)
    ec, gc = err(c12["e_qp"], c12["gap"])
    print(f"\nmode residual rms (validation): linear {val_lin:.3e}, trained {val_mlp:.3e} (train linear {rms_lin:.3e}, "
          f"loss {hist[0]:.3e} -> {hist[-1]:.3e})")
    print(f"E_qp / gap error vs full 60-point FP64 (meV): surrogate {es:.3f} / {gs:.3f}, linear part only "
          f"{el:.3f} / {gl:.3f}, plain 12-point grid {ec:.1f} / {gc:.1f}")
    assert val_mlp < val_lin
    assert es <= 1.0 and gs <= 1.0
    assert es < 0.05 * ec and gs < 0.05 * gc
