"""FP64 CPU oracle of the learned frequency surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import this module.
It shares no code with the CUDA path.

The paper computes chi0 and eps~^-1 at every imaginary frequency of the grid (Sec. II.A;
Eqs. chi0_matrix, symm_dielec_func). The surrogate computes them only at a coarse subset
C of the grid. It reconstructs X(w) = eps~^-1(w) - 1 at the other ("fine") frequencies F:

  X(w_m) = sum_{c in C} L_{mc} X(w_c) + U diag(sigma_l g_l(w_m)) U^H,    m in F

- U (N x n_modes): Ritz vectors of A = eps~(w_ref) - 1, w_ref = the first coarse frequency,
  after n_iter steps of subspace iteration from a given start block (ritz_modes).
- d_l(w) = u_l^H X(w) u_l: the diagonal of X in that mode basis (real, <= 0).
- sigma_l = |d_l(w_ref)|; x_l = d_l(C) / sigma_l: the network input, one row per mode.
- The network predicts d_l(F) / sigma_l as f(x) = L x + g(x), with L linear and
  g = s * MLP(x) (3 hidden layers, SiLU; s a fixed output scale, the rms residual of the
  linear fit, so that the MLP learns an O(1) target).
- Its L acts on whole matrices (the first term); g enters only on the mode diagonal.
  So the mode diagonal of the reconstruction is sigma_l f(x_l).

The MLP weight matrices W1..W4 are rounded to bfloat16 (round to nearest even) wherever
they are used; the biases and the linear map L stay fp32 (L is fitted in closed form by ridge
regression and needs more than bf16's 8 bits); arithmetic here is FP64.
"""
from __future__ import annotations

import numpy as np

from . import gw_oracle as O

# ----------------------------------------------------------------------------
# parameters: one flat fp32 vector, this order (row-major matrices [out][in])
# ----------------------------------------------------------------------------


def layout(n_in, n_hid, n_out):
    """[(name, shape)] of the flat parameter vector."""
    return [("W1", (n_hid, n_in)), ("b1", (n_hid,)),
            ("W2", (n_hid, n_hid)), ("b2", (n_hid,)),
            ("W3", (n_hid, n_hid)), ("b3", (n_hid,)),
            ("W4", (n_out, n_hid)), ("b4", (n_out,)),
            ("L", (n_out, n_in)), ("s", (1,))]


def n_params(n_in, n_hid, n_out):
    return sum(int(np.prod(s)) for _, s in layout(n_in, n_hid, n_out))


def unpack(theta, dims, round_bf16=True):
    """Flat vector -> dict of arrays (float64); MLP weight matrices rounded to bf16 if asked."""
    out, o = {}, 0
    for name, shape in layout(*dims):
        n = int(np.prod(shape))
        a = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        if round_bf16 and name[0] == "W":
            a = bf16_round(a)
        out[name] = a
        o += n
    return out


def pack(p, dims):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in layout(*dims)])


def bf16_round(a):
    """fp32 -> bfloat16 by round-to-nearest-even on the bit pattern; returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------


def forward(theta, dims, x, round_bf16=True, parts=False):
    """f(x) = L x + g(x) for a batch x [B][n_in]. With parts, also (g(x), activations)."""
    p = unpack(theta, dims, round_bf16)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(z3)
    g = p["s"][0] * (h3 @ p["W4"].T + p["b4"])
    f = g + x @ p["L"].T
    if parts:
        return f, g, dict(p=p, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)
    return f


def loss_grad(theta, dims, x, y, round_bf16=True):
    """Mean squared error over all B * n_out outputs and its gradient (flat, float64).

    Back-propagation through the same bf16-rounded weights (their rounding is treated as
    the identity when differentiating, so the gradient is the one of the rounded weights)."""
    f, _, a = forward(theta, dims, x, round_bf16, parts=True)
    p = a["p"]
    B, n_out = f.shape
    r = f - y
    loss = float(np.mean(r * r))
    df = 2.0 * r / (B * n_out)
    gr = {}
    dg = p["s"][0] * df
    gr["W4"] = dg.T @ a["h3"]
    gr["b4"] = dg.sum(axis=0)
    gr["L"] = df.T @ x
    gr["s"] = np.zeros(1)          # the output scale is fixed, not trained
    dz3 = (dg @ p["W4"]) * silu_grad(a["z3"])
    gr["W3"] = dz3.T @ a["h2"]
    gr["b3"] = dz3.sum(axis=0)
    dz2 = (dz3 @ p["W3"]) * silu_grad(a["z2"])
    gr["W2"] = dz2.T @ a["h1"]
    gr["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * silu_grad(a["z1"])
    gr["W1"] = dz1.T @ x
    gr["b1"] = dz1.sum(axis=0)
    return loss, pack(gr, dims)


def fit_linear(x, y, ridge):
    """Closed-form ridge regression of the linear map: L = argmin |x L^T - y|^2 + ridge n |L|^2
    (normal equations in FP64). Returns (L [n_out][n_in], rms of the residual y - x L^T)."""
    n, n_in = x.shape
    G = x.T @ x + ridge * n * np.eye(n_in)
    L = np.linalg.solve(G, x.T @ y).T
    r = y - x @ L.T
    return L, float(np.sqrt(np.mean(r * r)))


def freq_moments(X, coarse, fine):
    """Frequency moments of a stack X [nw][N][N]: m[a][b] = sum_e Re(conj(X_e(w_a)) X_e(w_b)),
    a over the coarse frequencies, b over the coarse then the fine ones."""
    Xf = X.reshape(X.shape[0], -1)
    cols = list(coarse) + list(fine)
    return (np.conj(Xf[list(coarse)]) @ Xf[cols].T).real


def fit_moments(m, n_in, ridge):
    """L from moments: (G + ridge tr(G)/n_in 1) L^T = R, G = m[:, :n_in], R = m[:, n_in:] (FP64)."""
    G, R = m[:, :n_in], m[:, n_in:]
    lam = ridge * np.trace(G) / n_in
    return np.linalg.solve(G + lam * np.eye(n_in), R).T


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), t counted from 1. Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------------------
# modes of eps~(w_ref)
# ----------------------------------------------------------------------------


def ritz_modes(A, start, n_iter, n_modes):
    """Subspace iteration on the Hermitian matrix A from the start block [N][n_block], then
    Rayleigh-Ritz. A = eps~(w_ref) - 1 = -V^1/2 chi0 V^1/2 is positive semidefinite, and the
    iteration converges to its dominant eigenvectors (the most strongly screened modes).
    Returns (theta [n_modes], U [N][n_modes]): the Ritz pairs of largest theta, descending.
    The subspace after n_iter steps is span(A^n_iter start), whatever orthonormalisation is
    used between the steps."""
    Q, _ = np.linalg.qr(start)
    for _ in range(n_iter):
        Q, _ = np.linalg.qr(A @ Q)
    H = np.conj(Q).T @ A @ Q
    H = 0.5 * (H + np.conj(H).T)
    th, Z = np.linalg.eigh(H)
    order = np.argsort(-th, kind="stable")[:n_modes]
    return th[order], Q @ Z[:, order]


def mode_diag(U, X):
    """d_l = u_l^H X u_l for a stack X [nw][N][N]: returns [n_modes][nw] (real part)."""
    return np.einsum("il,wij,jl->lw", np.conj(U), X, U).real


def inverse_minus_one(eps_t):
    N = eps_t.shape[-1]
    return np.array([np.linalg.inv(e) - np.eye(N) for e in eps_t])


def mode_data(sys, iq, start, n_iter, n_modes):
    """Training data from the plain method on the full grid of sys: (d [n_modes][n_freq], theta).

    eps~ and its inverse at every frequency (gw_oracle.chi0 / screen), modes of
    eps~(w_0) - 1, then the diagonal of eps~^-1 - 1 in that basis."""
    om, _ = O.freq_grid(sys.n_freq, sys.omega0)
    c = O.chi0(sys, iq, om)
    eps_t, _ = O.screen(sys, iq, c, om)
    N = sys.n_aux
    th, U = ritz_modes(eps_t[0] - np.eye(N), start, n_iter, n_modes)
    return mode_diag(U, inverse_minus_one(eps_t)), th


def features(d, coarse, fine):
    """(x, y, sigma): inputs d(C)/sigma, targets d(F)/sigma, sigma = |d(w_ref)| (w_ref = C[0])."""
    sig = np.abs(d[:, coarse[0]])
    sig = np.where(sig > 0, sig, 1.0)
    return d[:, coarse] / sig[:, None], d[:, fine] / sig[:, None], sig


# ----------------------------------------------------------------------------
# the surrogate-accelerated G0W0 pass
# ----------------------------------------------------------------------------


def g0w0_surrogate(sys, theta, dims, coarse, start, n_iter, n_modes, dxv=None, keep=False):
    """Sigma_c with chi0 / eps~ computed on the coarse frequencies only; X(w) on the other
    frequencies from the reconstruction in the module docstring; then W^c = V^1/2 X V^1/2
    and the Sigma_c quadrature on the full grid (gw_oracle.sigma_q), the QP solve and gap."""
    om, g = O.freq_grid(sys.n_freq, sys.omega0)
    mu = O.mu_midgap(sys)
    coarse = list(coarse)
    fine = [j for j in range(sys.n_freq) if j not in coarse]
    nsig = sys.sigma_hi - sys.sigma_lo
    sig_acc = np.zeros((sys.n_k, nsig, sys.n_freq), dtype=np.complex128)
    N = sys.n_aux
    kept = {}
    for iq in range(sys.n_k):
        c = O.chi0(sys, iq, om[coarse])
        eps_c, _ = O.screen(sys, iq, c, om[coarse])
        Xc = inverse_minus_one(eps_c)
        th, U = ritz_modes(eps_c[0] - np.eye(N), start, n_iter, n_modes)
        d = mode_diag(U, Xc)
        sg = np.abs(d[:, 0])
        sg = np.where(sg > 0, sg, 1.0)
        X = np.zeros((sys.n_freq, N, N), dtype=np.complex128)
        X[coarse] = Xc
        if fine:
            _, gout, a = forward(theta, dims, d / sg[:, None], parts=True)
            Lm = a["p"]["L"]
            for i, m in enumerate(fine):
                X[m] = np.einsum("c,cij->ij", Lm[i], Xc) + (U * (sg * gout[:, i])) @ np.conj(U).T
        Vh = O.hsqrt(sys.V[iq])
        W = np.array([Vh @ X[j] @ Vh for j in range(sys.n_freq)])
        sig_acc += O.sigma_q(sys, iq, W, om, g, mu)
        if keep:
            kept[iq] = dict(U=U, theta=th, d=d, X=X)
    E, gap, conv = O.qp(sys, sig_acc, om, mu, dxv)
    return dict(omega=om, g=g, mu=mu, sigma=sig_acc, e_qp=E, gap=gap, converged=conv, per_q=kept)
