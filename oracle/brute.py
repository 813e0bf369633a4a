"""Brute-force tier of the FP64 oracle: every loop explicit, tiny inputs only.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Independent of
gw_oracle.py in how it reaches each quantity:
  * C~(k+q, k) from the real-space LRI expansion of a Bloch product
    (Eq. realspace_expan2) summed cell by cell, not from Eq. AO_triple_split2;
  * chi0 from the literal two-term Adler-Wiser sum (Eq. chi_0_realspace /
    chi0_matrix with occupations) at +w and at -w, not from the Hermitised form;
  * V^{1/2} by the Denman-Beavers iteration, not by an eigen-decomposition;
  * Sigma_c by the unfolded w' sum over +-w'_j (Eq. GW_selfe_element), with
    W^c(-i w') computed from chi0(-i w'), not by folding.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from .gw_oracle import freq_grid, k_minus, k_of, k_plus, kpoints  # mesh/grid helpers only


def lri_coeff_realspace(sys, ik, iq, mu, i, j):
    """Coefficient of P^{q*}_mu in phi_i^{k+q*} phi_j^k from Eq. (realspace_expan2).

    phi_i^{k+q*}(r) phi_j^k(r) = sum_{Ri,Rj} e^{-i(k+q).Ri} e^{i k.Rj} phi_i(r-Ri) phi_j(r-Rj).
    Each product phi_i(r-Ri) phi_j(r-Rj) expands on ABFs of atom I at Ri with
    C~_{i(0), j(Rj-Ri)} and on ABFs of atom J at Rj with C~_{j(0), i(Ri-Rj)}.
    Collecting the terms on P_mu(r - R0 - tau_mu) for R0 = 0 gives the
    coefficient c such that the full sum is c * sum_R0 e^{-i q.R0} P_mu(r - R0).
    Returns (c at R0 = 0, c' at R0 = e_1 divided by e^{-i q.e1}) -- equal when
    the Bloch structure is right.
    """
    kp = kpoints(sys.nk)
    k = kp[ik]
    kq = kp[k_plus(sys.nk, ik, iq)]
    q = kp[iq]
    A = sys.aux_atom[mu]
    mu_loc = mu - np.nonzero(sys.aux_atom == A)[0][0]
    Rlist = [tuple(r) for r in sys.R]
    out = []
    for R0 in [(0, 0, 0), (1, 0, 0)]:
        c = 0j
        # term 1: ABF of atom I = atom(i) sitting at Ri = R0; Rj = R0 + d for stored d
        if sys.basis_atom[i] == A:
            i_loc = i - np.nonzero(sys.basis_atom == A)[0][0]
            for r_idx, d in enumerate(Rlist):
                Ri = R0
                Rj = (R0[0] + d[0], R0[1] + d[1], R0[2] + d[2])
                ph = cmath.exp(-2j * math.pi * sum(kq[x] * Ri[x] for x in range(3))) * \
                    cmath.exp(2j * math.pi * sum(k[x] * Rj[x] for x in range(3)))
                c += ph * sys.ctil_R[A][r_idx, mu_loc, i_loc, j]
        # term 2: ABF of atom J = atom(j) sitting at Rj = R0; Ri = R0 + d
        if sys.basis_atom[j] == A:
            j_loc = j - np.nonzero(sys.basis_atom == A)[0][0]
            for r_idx, d in enumerate(Rlist):
                Rj = R0
                Ri = (R0[0] + d[0], R0[1] + d[1], R0[2] + d[2])
                ph = cmath.exp(-2j * math.pi * sum(kq[x] * Ri[x] for x in range(3))) * \
                    cmath.exp(2j * math.pi * sum(k[x] * Rj[x] for x in range(3)))
                c += ph * sys.ctil_R[A][r_idx, mu_loc, j_loc, i]
        # divide out the Bloch phase of the ABF at R0
        out.append(c / cmath.exp(-2j * math.pi * sum(q[x] * R0[x] for x in range(3))))
    return out[0], out[1]


def ao_triple_brute(sys, ik, iq):
    C = np.zeros((sys.n_aux, sys.n_basis, sys.n_basis), dtype=np.complex128)
    for mu in range(sys.n_aux):
        for i in range(sys.n_basis):
            for j in range(sys.n_basis):
                C[mu, i, j] = lri_coeff_realspace(sys, ik, iq, mu, i, j)[0]
    return C


def mo_triple_brute(sys, ik, iq, Ct=None):
    """Eq. (AO_MO_transform) as an explicit quadruple loop, all bands: M[mu, m(k+q), n(k)]."""
    if Ct is None:
        Ct = ao_triple_brute(sys, ik, iq)
    ikq = k_plus(sys.nk, ik, iq)
    ca, cb = sys.evec[ikq], sys.evec[ik]
    nb = sys.n_bands
    M = np.zeros((sys.n_aux, nb, nb), dtype=np.complex128)
    for mu in range(sys.n_aux):
        for m in range(nb):
            for n in range(nb):
                acc = 0j
                for i in range(sys.n_basis):
                    for j in range(sys.n_basis):
                        acc += ca[i, m].conjugate() * cb[j, n] * Ct[mu, i, j]
                M[mu, m, n] = acc
    return M


def chi0_literal_brute(sys, iq, w, Ms):
    """Literal Adler-Wiser chi0 at one (signed) frequency w, explicit loops.

    chi0_{mu nu} = (s/N_k) sum_k sum_{m,n} (f_m - f_n) C^mu_{mn}(k+q,k) conj(C^nu_{mn}(k+q,k))
                   / (e_m(k+q) - e_n(k) - i w).
    Ms[ik] = M[mu, m, n] for this q.
    """
    N = sys.n_aux
    out = np.zeros((N, N), dtype=np.complex128)
    for ik in range(sys.n_k):
        ikq = k_plus(sys.nk, ik, iq)
        M = Ms[ik]
        for m in range(sys.n_bands):
            fm = 1.0 if m < sys.n_occ else 0.0
            for n in range(sys.n_bands):
                fn = 1.0 if n < sys.n_occ else 0.0
                if fm == fn:
                    continue
                den = sys.eps[ikq, m] - sys.eps[ik, n] - 1j * w
                for mu in range(N):
                    for nu in range(N):
                        out[mu, nu] += (fm - fn) * M[mu, m, n] * M[nu, m, n].conjugate() / den
    return (sys.spin / sys.n_k) * out


def sqrt_denman_beavers(V, iters=60):
    """Principal square root of a Hermitian positive definite matrix (Denman-Beavers)."""
    Y = V.astype(np.complex128).copy()
    Z = np.eye(V.shape[0], dtype=np.complex128)
    for _ in range(iters):
        Yi = np.linalg.inv(Y)
        Zi = np.linalg.inv(Z)
        Y, Z = 0.5 * (Y + Zi), 0.5 * (Z + Yi)
    return Y


def g0w0_brute(sys):
    """Regular (no head/wings) pipeline with every contraction as explicit loops.

    Returns dict(chi0 [q][w], Wc [q][w], sigma [k, n_sigma, w]).
    """
    om, g = freq_grid(sys.n_freq, sys.omega0)
    mu_f = 0.5 * (sys.eps[:, sys.n_occ - 1].max() + sys.eps[:, sys.n_occ].min())
    N = sys.n_aux
    Ms = {}
    for iq in range(sys.n_k):
        for ik in range(sys.n_k):
            Ms[(ik, iq)] = mo_triple_brute(sys, ik, iq)
    chi = {}
    Wc = {}
    for iq in range(sys.n_k):
        Vh = sqrt_denman_beavers(sys.V[iq])
        for sgn in (1.0, -1.0):
            for jw, w in enumerate(om):
                c = chi0_literal_brute(sys, iq, sgn * w, [Ms[(ik, iq)] for ik in range(sys.n_k)])
                eps_t = np.eye(N) - Vh @ c @ Vh
                Wc[(iq, sgn, jw)] = Vh @ (np.linalg.inv(eps_t) - np.eye(N)) @ Vh
                chi[(iq, sgn, jw)] = c
    nsig = sys.sigma_hi - sys.sigma_lo
    sig = np.zeros((sys.n_k, nsig, len(om)), dtype=np.complex128)
    for ik in range(sys.n_k):
        for iq in range(sys.n_k):
            ikmq = k_minus(sys.nk, ik, iq)
            M = Ms[(ikmq, iq)]                 # C^mu_{nm}(k, k-q) = M[mu, n, m]
            for nn in range(nsig):
                n = sys.sigma_lo + nn
                for m in range(sys.n_bands):
                    for sgn in (1.0, -1.0):
                        for jp, wp in enumerate(om):
                            W = Wc[(iq, sgn, jp)]
                            S = 0j
                            for a in range(N):
                                for b in range(N):
                                    S += M[a, n, m] * W[a, b] * M[b, n, m].conjugate()
                            for jw, w in enumerate(om):
                                den = 1j * w - 1j * sgn * wp + mu_f - sys.eps[ikmq, m]
                                sig[ik, nn, jw] += g[jp] * S / den
    sig *= -1.0 / (2.0 * math.pi * sys.n_k)
    return dict(omega=om, chi0=chi, Wc=Wc, sigma=sig, M=Ms)
