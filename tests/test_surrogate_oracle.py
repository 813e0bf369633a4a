"""Pins of the surrogate oracle (oracle/surrogate.py) against closed forms, textbook
routines, finite differences and exact reductions to the plain method. CPU only."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from oracle import surrogate as S
from paper_2011_01400_gb300.synth import make_system


def test_bf16_round_to_nearest_even():
    e8, e7, e6 = 2.0 ** -8, 2.0 ** -7, 2.0 ** -6
    vals = np.array([1.0, 1 + e8, 1 + 3 * e8, 1 + e8 + 2.0 ** -20, -(1 + 3 * e8), 3.0, 1e-3])
    want = np.array([1.0, 1.0, 1 + e6, 1 + e7, -(1 + e6), 3.0, 0.00099945068359375])
    assert np.array_equal(S.bf16_round(vals), want)


def _rand(dims, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    th = rng.standard_normal(S.n_params(*dims)) * scale
    th[-1] = 0.7  # output scale s
    return S.pack(S.unpack(th, dims, round_bf16=True), dims)  # weights already bf16-representable


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    dims = (5, 16, 7)
    th = _rand(dims, seed)
    rng = np.random.default_rng(10 + seed)
    x = rng.standard_normal((9, dims[0]))
    y = rng.standard_normal((9, dims[2]))
    loss, g = S.loss_grad(th, dims, x, y, round_bf16=False)
    assert g[-1] == 0.0  # the output scale is not trained
    h = 1e-6
    for i in range(S.n_params(*dims) - 1):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fp = np.mean((S.forward(tp, dims, x, round_bf16=False) - y) ** 2)
        fm = np.mean((S.forward(tm, dims, x, round_bf16=False) - y) ** 2)
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-7 * max(1.0, abs(g[i]))
    assert abs(loss - np.mean((S.forward(th, dims, x, round_bf16=False) - y) ** 2)) < 1e-15


def test_gradient_of_rounded_weights():
    """With rounding on, the gradient is that of the bf16-rounded weights."""
    dims = (4, 8, 3)
    rng = np.random.default_rng(3)
    th = rng.standard_normal(S.n_params(*dims)) * 0.3
    x, y = rng.standard_normal((6, 4)), rng.standard_normal((6, 3))
    l1, g1 = S.loss_grad(th, dims, x, y, round_bf16=True)
    thr = S.pack(S.unpack(th, dims, round_bf16=True), dims)
    l2, g2 = S.loss_grad(thr, dims, x, y, round_bf16=False)
    assert l1 == l2 and np.array_equal(g1, g2)
    assert not np.array_equal(th, thr)


def test_adam_first_step_is_lr_times_sign():
    """After one step from zero moments the bias-corrected ratio m/sqrt(v) is g/|g|."""
    rng = np.random.default_rng(4)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    t1, m, v = S.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 1e-3, eps=0.0)
    assert np.allclose(t1, th - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    th, m, v = np.array([3.0, -2.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        th, m, v = S.adam_step(th, 2 * th, m, v, t, 1e-2)
    assert np.abs(th).max() < 1e-3


def test_ritz_modes_converge_to_dominant_eigenpairs():
    rng = np.random.default_rng(5)
    N, nb, k = 40, 12, 6
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    lam = np.sort(rng.uniform(0.01, 1.0, N))[::-1] * np.linspace(3, 1, N)
    A = (Q * lam) @ np.conj(Q).T
    start = rng.standard_normal((N, nb)) + 1j * rng.standard_normal((N, nb))
    th, U = S.ritz_modes(A, start, 300, k)
    assert np.allclose(th, lam[:k], rtol=1e-10)
    P_ref = Q[:, :k] @ np.conj(Q[:, :k]).T
    assert np.linalg.norm(U @ np.conj(U).T - P_ref) < 1e-8
    assert np.allclose(np.conj(U).T @ U, np.eye(k), atol=1e-12)


def test_ritz_subspace_is_span_of_powers():
    """Brute force: the Ritz vectors after n steps are those of span(A^n start), unnormalised."""
    rng = np.random.default_rng(6)
    N, nb, n = 20, 5, 3
    B = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    A = B @ np.conj(B).T / N
    start = rng.standard_normal((N, nb)) + 1j * rng.standard_normal((N, nb))
    Y = start.copy()
    for _ in range(n):
        Y = A @ Y
    G = np.conj(Y).T @ Y
    # Rayleigh-Ritz in the non-orthonormal basis Y: generalised problem H z = theta G z
    H = np.conj(Y).T @ A @ Y
    Lc = np.linalg.cholesky(G)
    Li = np.linalg.inv(Lc)
    th_ref = np.sort(np.linalg.eigvalsh(Li @ H @ np.conj(Li).T))[::-1]
    th, U = S.ritz_modes(A, start, n, nb)
    assert np.allclose(th, th_ref, rtol=1e-9)


def test_mode_diag_of_eigenbasis_is_spectrum():
    rng = np.random.default_rng(7)
    N = 10
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    lam = -rng.uniform(0, 1, N)
    X = ((Q * lam) @ np.conj(Q).T)[None]
    assert np.allclose(S.mode_diag(Q, X)[:, 0], lam, atol=1e-14)


def test_fit_linear_recovers_exact_map():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((200, 6))
    L0 = rng.standard_normal((9, 6))
    L, rms = S.fit_linear(x, x @ L0.T, 0.0)
    assert np.allclose(L, L0, atol=1e-12) and rms < 1e-12
    L1, _ = S.fit_linear(x, x @ L0.T, 1e6)
    assert np.abs(L1).max() < 1e-4  # heavy ridge shrinks to zero


def _tiny(n_freq=8, seed=0):
    return make_system("tiny", seed=seed, n_freq=n_freq)


def test_surrogate_with_all_frequencies_is_plain_method():
    s = _tiny()
    dims = (s.n_freq, 8, 1)
    th = _rand(dims, 0)
    rng = np.random.default_rng(9)
    start = rng.standard_normal((s.n_aux, 4)) + 1j * rng.standard_normal((s.n_aux, 4))
    sur = S.g0w0_surrogate(s, th, dims, list(range(s.n_freq)), start, 3, 2)
    ref = O.g0w0(s)
    assert np.abs(sur["sigma"] - ref["sigma"]).max() <= 1e-12 * np.abs(ref["sigma"]).max()
    assert abs(sur["gap"] - ref["gap"]) < 1e-12


def test_surrogate_copy_map_reassembles_plain_W():
    """g = 0 and a one-hot L (every fine frequency takes W^c of one coarse frequency):
    Sigma_c equals the plain quadrature over that piecewise-copied W^c."""
    s = _tiny(n_freq=10, seed=1)
    coarse = [0, 3, 6, 9]
    fine = [j for j in range(s.n_freq) if j not in coarse]
    src = {1: 0, 2: 1, 4: 1, 5: 2, 7: 2, 8: 3}     # fine index -> position in coarse
    dims = (len(coarse), 8, len(fine))
    p = {n: np.zeros(sh) for n, sh in S.layout(*dims)}
    p["s"] = np.ones(1)
    for i, m in enumerate(fine):
        p["L"][i, src[m]] = 1.0
    th = S.pack(p, dims)
    rng = np.random.default_rng(11)
    start = rng.standard_normal((s.n_aux, 6)) + 1j * rng.standard_normal((s.n_aux, 6))
    sur = S.g0w0_surrogate(s, th, dims, coarse, start, 4, 3)
    om, g = O.freq_grid(s.n_freq, s.omega0)
    mu = O.mu_midgap(s)
    sig = 0
    for iq in range(s.n_k):
        _, Wc = O.screen(s, iq, O.chi0(s, iq, om[coarse]), om[coarse])
        W = np.empty((s.n_freq,) + Wc.shape[1:], dtype=complex)
        W[coarse] = Wc
        for m in fine:
            W[m] = Wc[src[m]]
        sig = sig + O.sigma_q(s, iq, W, om, g, mu)
    assert np.abs(sur["sigma"] - sig).max() <= 1e-11 * np.abs(sig).max()


def test_reconstruction_mode_diagonal_is_network_output():
    """Mode diagonal of the reconstructed X at every fine frequency = sigma_l f(x_l)."""
    s = _tiny(n_freq=10, seed=2)
    coarse = [0, 2, 5, 8]
    fine = [j for j in range(s.n_freq) if j not in coarse]
    dims = (len(coarse), 8, len(fine))
    th = _rand(dims, 5, scale=0.2)
    rng = np.random.default_rng(12)
    start = rng.standard_normal((s.n_aux, 5)) + 1j * rng.standard_normal((s.n_aux, 5))
    sur = S.g0w0_surrogate(s, th, dims, coarse, start, 6, 4, keep=True)
    for iq, kq in sur["per_q"].items():
        d, U, X = kq["d"], kq["U"], kq["X"]
        sg = np.abs(d[:, 0])
        f = S.forward(th, dims, d / sg[:, None])
        got = S.mode_diag(U, X[fine])
        assert np.allclose(got, sg[:, None] * f, rtol=0, atol=1e-12 * max(1.0, np.abs(got).max()))
        assert np.allclose(S.mode_diag(U, X[coarse]), d, atol=1e-13)


def test_fit_moments_is_least_squares_over_matrix_elements():
    """Fitting L from frequency moments = least squares over the real and imaginary parts of
    every element (brute force with lstsq on the stacked elements)."""
    rng = np.random.default_rng(13)
    nw, N = 7, 5
    X = rng.standard_normal((3, nw, N, N)) + 1j * rng.standard_normal((3, nw, N, N))
    coarse, fine = [0, 3, 6], [1, 2, 4, 5]
    m = sum(S.freq_moments(Xq, coarse, fine) for Xq in X)
    L = S.fit_moments(m, 3, 0.0)
    A = np.concatenate([np.concatenate([Xq[coarse].reshape(3, -1).real, Xq[coarse].reshape(3, -1).imag], 1) for Xq in X], 1).T
    B = np.concatenate([np.concatenate([Xq[fine].reshape(4, -1).real, Xq[fine].reshape(4, -1).imag], 1) for Xq in X], 1).T
    L_ref = np.linalg.lstsq(A, B, rcond=None)[0].T
    assert np.allclose(L, L_ref, atol=1e-12)
