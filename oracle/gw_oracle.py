"""FP64 CPU oracle of the periodic G0W0 hot path (Ren et al., arXiv:2011.01400).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this module: it is used by tests/, by __graft_entry__.smoke() and by the
cpu_baseline / reference leg of bench.py. It shares no code with the CUDA
path: it takes plain NumPy arrays (the seeded inputs) and returns plain NumPy
arrays.

Every function states the passage of the paper it follows. Steps are taken in
the paper's order with library primitives (matmul, eigh, inv, leggauss) and no
blocking or reordering. Readings of passages that are silent, ambiguous or
garbled are marked "reading:" in the docstring that uses them.

Notation (Sec. II): k, q on a Gamma-centred mesh, w_k = 1/N_k; bands m, n;
NAOs i, j; ABFs mu, nu; s = spin factor (2, doubly occupied bands).
M^mu_{ab}(k, q) == C^mu_{ab}(k+q, k): a at k+q, b at k.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# mesh helpers (index arithmetic of the Gamma-centred Monkhorst-Pack mesh)
# ----------------------------------------------------------------------------


def kpoints(nk):
    """Fractional coordinates of the Gamma-centred mesh, index (i1*n2+i2)*n3+i3."""
    n1, n2, n3 = nk
    out = []
    for i1 in range(n1):
        for i2 in range(n2):
            for i3 in range(n3):
                out.append((i1 / n1, i2 / n2, i3 / n3))
    return np.array(out)


def kfrac(sys):
    """Fractional coordinates of the system's k points: the Gamma-centred mesh, shifted by
    sys.k_offset when the system carries one (a shifted mesh k0 + i/n; the q mesh is never
    shifted, so k + q and k - q stay on the shifted mesh)."""
    return kpoints(sys.nk) + np.asarray(getattr(sys, "k_offset", np.zeros(3)), dtype=np.float64)[None, :]


def k_of(nk, ik):
    n1, n2, n3 = nk
    return ik // (n2 * n3), (ik // n3) % n2, ik % n3


def k_index(nk, a):
    n1, n2, n3 = nk
    return ((a[0] % n1) * n2 + (a[1] % n2)) * n3 + (a[2] % n3)


def k_plus(nk, ik, iq):
    a, b = k_of(nk, ik), k_of(nk, iq)
    return k_index(nk, (a[0] + b[0], a[1] + b[1], a[2] + b[2]))


def k_minus(nk, ik, iq=None):
    """-k (iq None) or k - q."""
    a = k_of(nk, ik)
    if iq is None:
        return k_index(nk, (-a[0], -a[1], -a[2]))
    b = k_of(nk, iq)
    return k_index(nk, (a[0] - b[0], a[1] - b[1], a[2] - b[2]))


# ----------------------------------------------------------------------------
# imaginary-frequency grid
# ----------------------------------------------------------------------------


def freq_grid(n, omega0=1.0):
    """Modified Gauss-Legendre grid on (0, inf).

    reading: the paper works on the imaginary axis (Sec. II.A) without naming
    its grid. Gauss-Legendre nodes x_j on (-1, 1) are mapped by
    omega = omega0 (1 + x) / (1 - x), weight g_j = 2 omega0 w_j / (1 - x_j)^2,
    so that sum_j g_j f(omega_j) ~ int_0^inf f(omega) d omega.
    """
    x, w = np.polynomial.legendre.leggauss(n)
    om = omega0 * (1.0 + x) / (1.0 - x)
    g = 2.0 * omega0 * w / (1.0 - x) ** 2
    return om, g


# ----------------------------------------------------------------------------
# step (a): LRI triple coefficients and the AO -> MO transform
# ----------------------------------------------------------------------------


def lri_ft(ctil_atom, R, kfrac):
    """Eqs. (expan_coeff_FT1/2): C~_{i(0),j(k)}^{mu(0)} = sum_R e^{i k.R} C~_{i(0),j(R)}^{mu(0)}.

    ctil_atom: [n_R, n_aux(A), n_b(A), n_basis] (mu and i on atom A, j anywhere).
    Returns D_A(k): [n_aux(A), n_b(A), n_basis] complex.
    """
    ph = np.exp(2j * np.pi * (R.astype(np.float64) @ np.asarray(kfrac, dtype=np.float64)))
    return np.tensordot(ph, ctil_atom, axes=(0, 0))


def ao_triple(sys, ik, iq):
    """Eq. (AO_triple_split2): dense C~^mu_{ij}(k+q, k), shape [n_aux, n_basis, n_basis].

    C~^mu_{ij}(k+q,k) = C~^{mu(0)}_{j(0), i(-k-q)} + C~^{mu(0)}_{i(0), j(k)}.
    reading: C~_{i(0),j(R)}^{mu(0)} is nonzero only for mu on the atom of i
    (Eq. two_center_coeff_determination), so the first term lives on
    mu in atom(j), the second on mu in atom(i); when atom(i) == atom(j) both add.
    """
    kp = kfrac(sys)
    k = kp[ik]
    kq = kp[k_plus(sys.nk, ik, iq)]
    C = np.zeros((sys.n_aux, sys.n_basis, sys.n_basis), dtype=np.complex128)
    for A in range(sys.n_atoms):
        mus = np.nonzero(sys.aux_atom == A)[0]
        ias = np.nonzero(sys.basis_atom == A)[0]
        D_k = lri_ft(sys.ctil_R[A], sys.R, k)           # [mu_A, i_A, j]
        D_mkq = lri_ft(sys.ctil_R[A], sys.R, -kq)       # [mu_A, j_A, i]
        for a, mu in enumerate(mus):
            # mu on atom(i): C~_{i(0), j(k)}
            C[mu][ias, :] += D_k[a]
            # mu on atom(j): C~_{j(0), i(-k-q)}; row index i, column index j
            C[mu][:, ias] += D_mkq[a].T
    return C


def mo_triple(sys, ik, iq, a_bands, b_bands):
    """Eq. (AO_MO_transform): C^mu_{ab}(k+q,k) = sum_ij c*_{ia}(k+q) c_{jb}(k) C~^mu_{ij}(k+q,k).

    Returns M[mu, a, b] for a in a_bands (at k+q) and b in b_bands (at k).
    """
    ikq = k_plus(sys.nk, ik, iq)
    Ct = ao_triple(sys, ik, iq)
    ca = sys.evec[ikq][:, a_bands]      # [i, a]
    cb = sys.evec[ik][:, b_bands]       # [j, b]
    return np.einsum("ia,uij,jb->uab", np.conj(ca), Ct, cb, optimize=True)


# ----------------------------------------------------------------------------
# step (b): irreducible polarizability
# ----------------------------------------------------------------------------


def chi0(sys, iq, omegas):
    """Eq. (chi0_matrix) with the occupation factors of Eq. (chi_0_realspace), Hermitised.

    chi0_{mu nu}(q, i w) = -(s / N_k) sum_k sum_{i occ(k), a unocc(k+q)}
                           M^mu_{ai}(k,q) conj(M^nu_{ai}(k,q)) 2 D / (w^2 + D^2),
    D = eps_a(k+q) - eps_i(k) > 0.
    reading: the printed matrix form drops (f_m - f_n); restoring it and
    pairing the two resonant terms (exact under time reversal) gives this
    Hermitian, negative semidefinite form, which defines chi0 here.
    """
    occ = np.arange(sys.n_occ)
    unocc = np.arange(sys.n_occ, sys.n_bands)
    out = np.zeros((len(omegas), sys.n_aux, sys.n_aux), dtype=np.complex128)
    for ik in range(sys.n_k):
        ikq = k_plus(sys.nk, ik, iq)
        M = mo_triple(sys, ik, iq, unocc, occ)            # [mu, a, i]
        D = sys.eps[ikq][unocc][:, None] - sys.eps[ik][occ][None, :]   # [a, i]
        Mf = M.reshape(sys.n_aux, -1)
        Df = D.ravel()
        for w_i, w in enumerate(omegas):
            wt = 2.0 * Df / (w * w + Df * Df)
            out[w_i] += (Mf * wt[None, :]) @ np.conj(Mf).T
    return -(sys.spin / sys.n_k) * out


def chi0_block(sys, iq, omegas, mus):
    """chi0_{mu nu}(q, i w) of Eq. (chi0_matrix) for mu, nu in the ABF subset `mus` only (the
    Hermitised form of `chi0`), from the rows C~^mu(k+q, k) of Eq. (AO_triple_split2) built one ABF
    at a time: for sampled checks of systems whose full C~ does not fit. Returns [w, len(mus), len(mus)]."""
    kp = kfrac(sys)
    occ, unocc = np.arange(sys.n_occ), np.arange(sys.n_occ, sys.n_bands)
    om = np.asarray(omegas, dtype=np.float64)
    out = np.zeros((len(om), len(mus), len(mus)), dtype=np.complex128)
    for ik in range(sys.n_k):
        ikq = k_plus(sys.nk, ik, iq)
        k, kq = kp[ik], kp[ikq]
        Ms = []
        for mu in mus:
            A = int(sys.aux_atom[mu])
            a = mu - int(np.nonzero(sys.aux_atom == A)[0][0])
            ias = np.nonzero(sys.basis_atom == A)[0]
            C = np.zeros((sys.n_basis, sys.n_basis), dtype=np.complex128)
            C[ias, :] += lri_ft(sys.ctil_R[A][:, a:a + 1], sys.R, k)[0]
            C[:, ias] += lri_ft(sys.ctil_R[A][:, a:a + 1], sys.R, -kq)[0].T
            Ms.append(np.conj(sys.evec[ikq][:, unocc]).T @ C @ sys.evec[ik][:, occ])   # [a, i]
        D = sys.eps[ikq][unocc][:, None] - sys.eps[ik][occ][None, :]
        Mf = np.array([m.ravel() for m in Ms])                                         # [mu, (a,i)]
        for j, w in enumerate(om):
            wt = (2.0 * D / (w * w + D * D)).ravel()
            out[j] += (Mf * wt[None, :]) @ np.conj(Mf).T
    return -(sys.spin / sys.n_k) * out


def chi0_literal(sys, iq, omegas):
    """Eq. (chi0_matrix) taken literally with occupations (f_m^{k+q} - f_n^k), both band orders.

    chi0 = s/N_k sum_k sum_{m,n} (f_m - f_n) C^mu_{mn}(k+q,k) C^nu_{nm}(k,k+q) / (e_m - e_n - i w),
    with C^nu_{nm}(k, k+q) = conj(C^nu_{mn}(k+q, k)) (real ABFs, Sec. II.B).
    """
    nb = np.arange(sys.n_bands)
    f = (nb < sys.n_occ).astype(np.float64)
    out = np.zeros((len(omegas), sys.n_aux, sys.n_aux), dtype=np.complex128)
    for ik in range(sys.n_k):
        ikq = k_plus(sys.nk, ik, iq)
        M = mo_triple(sys, ik, iq, nb, nb)                 # [mu, m (k+q), n (k)]
        fd = f[:, None] - f[None, :]
        de = sys.eps[ikq][:, None] - sys.eps[ik][None, :]
        Mf = M.reshape(sys.n_aux, -1)
        for w_i, w in enumerate(omegas):
            wt = (fd / (de - 1j * w)).ravel()
            out[w_i] += (Mf * wt[None, :]) @ np.conj(Mf).T
    return (sys.spin / sys.n_k) * out


# ----------------------------------------------------------------------------
# step (c): symmetrised dielectric matrix, its inverse and W
# ----------------------------------------------------------------------------


def hsqrt(V):
    """V^{1/2} of a Hermitian positive (semi)definite matrix via its eigen-decomposition."""
    lam, U = np.linalg.eigh(V)
    lam = np.clip(lam, 0.0, None)
    return (U * np.sqrt(lam)[None, :]) @ np.conj(U).T


def coulomb_eig_q0(V0):
    """Sec. III (Gamma point): eigenpairs of V^cut(q=0), lambda = 1 first (largest).

    reading: the wings of Eq. dielectric_func_gamma change sign with the lambda = 1 eigenvector.
    In the paper that vector is the G = 0 plane wave, the positive constant 1/sqrt(Omega), so
    its sign is fixed by physics; synthetic inputs have no such function, so its phase is fixed
    by convention: the largest-magnitude component (the first one on a tie) real and positive.
    """
    lam, X = np.linalg.eigh(V0)
    order = np.argsort(lam)[::-1]
    lam, X = lam[order], X[:, order].copy()
    i = int(np.argmax(np.abs(X[:, 0])))
    X[:, 0] *= np.conj(X[i, 0]) / abs(X[i, 0])
    return lam, X


def sphere_rule(n_theta=8, n_phi=16):
    """Product quadrature on the unit sphere for averages over the direction of q -> 0: Gauss-
    Legendre nodes in cos(theta) times equally spaced phi (offset by half a step). Weights sum to
    one; the point set is symmetric under q^ -> -q^, so odd moments vanish exactly.
    Returns (directions [n, 3], weights [n])."""
    u, wu = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * np.pi * (np.arange(n_phi) + 0.5) / n_phi
    dirs, wts = [], []
    for ui, wi in zip(u, wu):
        st = np.sqrt(1.0 - ui * ui)
        for p in phi:
            dirs.append((st * np.cos(p), st * np.sin(p), ui))
            wts.append(wi / 2.0 / n_phi)
    return np.array(dirs), np.array(wts)


def head_wings_q0(sys, omegas, chi0_0, qhat=None):
    """Eq. (dielectric_func_gamma) in the Coulomb eigenbasis, insulator case.

    Returns eps_X[w] (matrix in the lambda basis, lambda=1 first) and X, v.
    head:  1 - (4 pi / Omega) sum_{k,sigma} sum_{m occ < n unocc}
              2 |p_mn . q^|^2 / ([(e_m - e_n)^2 + w^2] (e_m - e_n)),  Omega = N_k Omega_cell
    wings: lambda' > 1:  -(s / N_k) sqrt(4 pi / Omega_cell) sqrt(v_l')
              sum_k sum_{i,a} (p_ia . q^) conj(Mhat^{l'}_{ai}(k)) 2 / (D^2 + w^2),
           Mhat = X^H M(k, q=0);  eps_{l' 1} = conj(eps_{1 l'}).
    body:  delta - sqrt(v_l) (X^H chi0 X)_{l l'} sqrt(v_l')  (the regular formula, l, l' > 1).
    reading: the printed wings carry garbled factors; they are taken as the
    q -> 0 limit of the regular formula under the k.p form
    <x_1, M_ai(k,q)> = q (p_ia . q^) / (e_i - e_a) (checked by a test), and the
    intraband f' term vanishes for insulators.
    """
    s = sys.spin
    NK = sys.n_k
    v, X = coulomb_eig_q0(sys.V[0])
    sv = np.sqrt(np.clip(v, 0.0, None))
    occ = np.arange(sys.n_occ)
    unocc = np.arange(sys.n_occ, sys.n_bands)
    qh = np.asarray(sys.qhat if qhat is None else qhat, dtype=np.float64)
    omega_tot = NK * sys.omega_cell
    nw = len(omegas)
    head = np.ones(nw)
    wing = np.zeros((nw, sys.n_aux), dtype=np.complex128)
    for ik in range(NK):
        e = sys.eps[ik]
        pq = np.einsum("d,dmn->mn", qh, sys.pmom[ik])[np.ix_(occ, unocc)]   # p_mn . q^, m occ, n unocc
        M = mo_triple(sys, ik, 0, unocc, occ)                    # [mu, a, i]
        Mhat = np.einsum("ul,uai->lia", np.conj(X), M)           # (X^H M)[l, i, a]
        dme = e[occ][:, None] - e[unocc][None, :]                # e_m - e_n < 0
        for w_i, w in enumerate(omegas):
            head[w_i] -= (4.0 * np.pi / omega_tot) * s * np.sum(
                2.0 * np.abs(pq) ** 2 / ((dme ** 2 + w ** 2) * dme))
            wing[w_i] += np.einsum("ia,lia->l", pq * 2.0 / (dme ** 2 + w ** 2), np.conj(Mhat))
    wing *= -(s / NK) * np.sqrt(4.0 * np.pi / sys.omega_cell) * sv[None, :]
    eps_X = np.zeros((nw, sys.n_aux, sys.n_aux), dtype=np.complex128)
    for w_i in range(nw):
        body = np.eye(sys.n_aux) - (sv[:, None] * (np.conj(X).T @ chi0_0[w_i] @ X) * sv[None, :])
        E = body.copy()
        E[0, 0] = head[w_i]
        E[0, 1:] = wing[w_i, 1:]
        E[1:, 0] = np.conj(wing[w_i, 1:])
        eps_X[w_i] = E
    return eps_X, X, v


def screen(sys, iq, chi0_q, omegas):
    """Eqs. (symm_dielec_func), (screened_W_matr); Gamma point per Sec. III.

    eps~ = 1 - V^{1/2} chi0 V^{1/2};  W^c = V^{1/2} (eps~^{-1} - 1) V^{1/2}.
    reading: the correlation part W^c = W - V is what enters Sigma_c.
    At q = 0 (head_wings set) eps~ is assembled in the Coulomb eigenbasis and
    transformed back, eps~_{mu nu} = sum X_{mu l} eps~_{l l'} X*_{nu l'},
    and W^c uses the full (truncated) V(0)^{1/2}. head_wings == 2: eps~^-1 - 1 averaged over
    the directions of q -> 0 (sphere_rule); the returned eps~ is that of sys.qhat.
    Returns (eps_tilde [w, N, N], Wc [w, N, N]).
    """
    Vh = hsqrt(sys.V[iq])
    nw = len(omegas)
    N = sys.n_aux
    eps_t = np.zeros((nw, N, N), dtype=np.complex128)
    Wc = np.zeros((nw, N, N), dtype=np.complex128)
    if iq == 0 and sys.head_wings == 2:
        # reading: for anisotropic systems the head and wings depend on the direction of q -> 0
        # (the discussion after Eq. dielectric_func_gamma); eps~^-1 - 1 is averaged over the
        # directions of sphere_rule(), each direction's eps~ assembled and inverted as for one q^.
        Xbar = np.zeros((nw, N, N), dtype=np.complex128)
        dirs, wts = sphere_rule()
        for d, wd in zip(dirs, wts):
            eps_X, X, v = head_wings_q0(sys, omegas, chi0_q, qhat=d)
            for w_i in range(nw):
                e = X @ eps_X[w_i] @ np.conj(X).T
                Xbar[w_i] += wd * (np.linalg.inv(e) - np.eye(N))
        eps_X, X, v = head_wings_q0(sys, omegas, chi0_q)
        for w_i in range(nw):
            eps_t[w_i] = X @ eps_X[w_i] @ np.conj(X).T
            Wc[w_i] = Vh @ Xbar[w_i] @ Vh
        return eps_t, Wc
    if iq == 0 and sys.head_wings:
        eps_X, X, v = head_wings_q0(sys, omegas, chi0_q)
        for w_i in range(nw):
            eps_t[w_i] = X @ eps_X[w_i] @ np.conj(X).T
    else:
        for w_i in range(nw):
            eps_t[w_i] = np.eye(N) - Vh @ chi0_q[w_i] @ Vh
    for w_i in range(nw):
        inv = np.linalg.inv(eps_t[w_i])
        Wc[w_i] = Vh @ (inv - np.eye(N)) @ Vh
    return eps_t, Wc


# ----------------------------------------------------------------------------
# step (d): correlation self-energy on the imaginary axis
# ----------------------------------------------------------------------------


def mu_midgap(sys):
    """reading: chemical potential at midgap, (max_k e_HOMO + min_k e_LUMO) / 2."""
    return 0.5 * (sys.eps[:, sys.n_occ - 1].max() + sys.eps[:, sys.n_occ].min())


def sigma_q(sys, iq, Wc_q, omegas, gweights, mu):
    """Eq. (GW_selfe_element) for one q with W^c in place of W.

    Sigma_c_n(k, i w) += -(1 / (2 pi N_q)) sum_m sum_j g_j S_nm(w'_j) 2 z / (z^2 + w'_j^2),
    S_nm(w') = sum_{mu nu} C^mu_{nm}(k, k-q) W^c_{mu nu}(q, i w') C^nu_{mn}(k-q, k),
    z = i w + mu - eps_m(k - q).
    reading: the printed formula omits w_q; taken as 1/N_q. The w' integral over
    (-inf, inf) is folded onto w' > 0 using W^c(i w') = W^c(-i w').
    Returns [N_k, n_sigma, N_w] complex.
    """
    nsig = sys.sigma_hi - sys.sigma_lo
    out = np.zeros((sys.n_k, nsig, len(omegas)), dtype=np.complex128)
    sig_b = np.arange(sys.sigma_lo, sys.sigma_hi)
    all_b = np.arange(sys.n_bands)
    for ik in range(sys.n_k):
        ikmq = k_minus(sys.nk, ik, iq)
        # C^mu_{nm}(k, k-q) = M^mu_{nm}(k-q, q): n at k = (k-q)+q, m at k-q
        M = mo_triple(sys, ikmq, iq, sig_b, all_b)        # [mu, n, m]
        em = sys.eps[ikmq]
        Mf = M.reshape(sys.n_aux, -1)
        z = 1j * np.asarray(omegas)[:, None] + mu - em[None, :]     # [w, m]
        for j, wp in enumerate(omegas):
            S = np.sum(Mf * (Wc_q[j] @ np.conj(Mf)), axis=0).real.reshape(nsig, -1)   # S_nm(w'_j)
            out[ik] += gweights[j] * np.einsum("nm,wm->nw", S, 2.0 * z / (z * z + wp * wp))
    return -out / (2.0 * np.pi * sys.n_k)


def sigma_x(sys):
    """Exchange self-energy, the bare-Coulomb part of Eq. (GW_selfe_element) (W = V + W^c):
    the frequency integral of V G over the occupied bands gives

      Sigma_x_n(k) = -(1/N_q) sum_q sum_{m occ} sum_{mu nu} C^mu_{nm}(k, k-q) V_{mu nu}(q) C^nu_{mn}(k-q, k)

    with C^nu_{mn}(k-q, k) = conj(C^nu_{nm}(k, k-q)); V(q=0) is the (truncated) Coulomb matrix
    as given. reading: w_q = 1/N_q as for Sigma_c. Returns [N_k, n_sigma] real (Ha).
    """
    nsig = sys.sigma_hi - sys.sigma_lo
    out = np.zeros((sys.n_k, nsig))
    sig_b = np.arange(sys.sigma_lo, sys.sigma_hi)
    occ = np.arange(sys.n_occ)
    for iq in range(sys.n_k):
        for ik in range(sys.n_k):
            ikmq = k_minus(sys.nk, ik, iq)
            M = mo_triple(sys, ikmq, iq, sig_b, occ)          # [mu, n, m]: n at k, m occupied at k-q
            Mf = M.reshape(sys.n_aux, -1)
            S = np.sum(Mf * (sys.V[iq] @ np.conj(Mf)), axis=0).real.reshape(nsig, -1)
            out[ik] -= S.sum(axis=1)
    return out / sys.n_k


# ----------------------------------------------------------------------------
# step (e): analytic continuation and quasiparticle equation
# ----------------------------------------------------------------------------


def two_pole_fit(z, f):
    """Two-pole model Sigma(z) = (p1 z + p0) / (z^2 + q1 z + q0) through (z_j, f_j).

    reading: the paper continues Sigma_c from the imaginary axis with the
    method of Rojas, Godby and Needs (Sec. II.A) without stating the model; a
    two-pole rational model is used. Its coefficients come from the linear
    least-squares problem of the cross-multiplied form
        f_j z_j^2 = -q1 f_j z_j - q0 f_j + p1 z_j + p0     (all N_w points),
    which stays well conditioned where a Pade interpolant through every point
    amplifies 1e-8 relative noise into 0.1 eV.
    Returns (q1, q0, p1, p0).
    """
    z = np.asarray(z, dtype=np.complex128)
    f = np.asarray(f, dtype=np.complex128)
    A = np.stack([-f * z, -f, z, np.ones_like(z)], axis=1)
    b = f * z * z
    scale = np.linalg.norm(A, axis=0)
    x, *_ = np.linalg.lstsq(A / scale[None, :], b, rcond=None)
    return x / scale


def two_pole_eval(c, x):
    q1, q0, p1, p0 = c
    return (p1 * x + p0) / (x * x + q1 * x + q0)


def two_pole_deriv(c, x):
    q1, q0, p1, p0 = c
    den = x * x + q1 * x + q0
    return (p1 * den - (p1 * x + p0) * (2.0 * x + q1)) / (den * den)


def qp_solve(eps_n, c, mu, dxv=0.0, tol=1e-10, maxit=100):
    """reading: E = eps_n + Re Sigma_c(E - mu) + dxv, Newton from E = eps_n.

    Falls back to the linearised (Z-factor) solution if Newton does not converge.
    Returns (E, converged).
    """
    E = eps_n
    for _ in range(maxit):
        s0 = two_pole_eval(c, E - mu).real
        d = two_pole_deriv(c, E - mu).real
        step = (E - eps_n - s0 - dxv) / (1.0 - d)
        E -= step
        if not np.isfinite(E):
            break
        if abs(step) < tol:
            return E, True
    s0 = two_pole_eval(c, eps_n - mu).real
    d = two_pole_deriv(c, eps_n - mu).real
    return eps_n + (s0 + dxv) / (1.0 - d), False


def qp(sys, sigma, omegas, mu, dxv=None):
    """QP energies for the sigma window and the indirect gap min_k E_LUMO - max_k E_HOMO."""
    nsig = sys.sigma_hi - sys.sigma_lo
    E = np.zeros((sys.n_k, nsig))
    conv = np.ones((sys.n_k, nsig), dtype=bool)
    zi = 1j * np.asarray(omegas)
    for ik in range(sys.n_k):
        for n in range(nsig):
            c = two_pole_fit(zi, sigma[ik, n])
            d = 0.0 if dxv is None else dxv[ik, n]
            E[ik, n], conv[ik, n] = qp_solve(sys.eps[ik, sys.sigma_lo + n], c, mu, d)
    h = sys.n_occ - 1 - sys.sigma_lo
    l = sys.n_occ - sys.sigma_lo
    gap = None
    if 0 <= h < nsig and 0 <= l < nsig:
        gap = E[:, l].min() - E[:, h].max()
    return E, gap, conv


# ----------------------------------------------------------------------------
# whole pipeline
# ----------------------------------------------------------------------------


def g0w0(sys, qs=None, keep=False, dxv=None, grid=None):
    """chi0 -> eps~ -> W^c -> Sigma_c (summed over q) -> QP energies and gap.

    grid: (frequencies, weights) of the imaginary axis; None is the modified
    Gauss-Legendre grid of scale sys.omega0."""
    if grid is None:
        om, g = freq_grid(sys.n_freq, sys.omega0)
    else:
        om, g = np.asarray(grid[0], dtype=np.float64), np.asarray(grid[1], dtype=np.float64)
    mu = mu_midgap(sys)
    qs = range(sys.n_k) if qs is None else qs
    nsig = sys.sigma_hi - sys.sigma_lo
    sig = np.zeros((sys.n_k, nsig, len(om)), dtype=np.complex128)
    kept = {}
    for iq in qs:
        c = chi0(sys, iq, om)
        e, W = screen(sys, iq, c, om)
        sig += sigma_q(sys, iq, W, om, g, mu)
        if keep:
            kept[iq] = dict(chi0=c, eps=e, Wc=W)
    E, gap, conv = qp(sys, sig, om, mu, dxv)
    return dict(omega=om, g=g, mu=mu, sigma=sig, e_qp=E, gap=gap, converged=conv, per_q=kept)
