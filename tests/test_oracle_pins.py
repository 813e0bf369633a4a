"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one piece of oracle/gw_oracle.py to something other than the
oracle itself: a closed form, an exact quadrature, an invariant the equations
imply, the q -> 0 limit of the regular formula, or a brute-force evaluation
that reaches the same quantity along a different route (oracle/brute.py).
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import brute
from oracle import gw_oracle as O
from paper_2011_01400_gb300.synth import make_system

HA_MEV = 27211.386


def test_lorentzian_quadrature_exact():
    """int_0^inf 2D/(w^2+D^2) dw = pi; the mapped integrand is 2/(1+x^2) when D = omega0."""
    for n in (8, 16, 32):
        om, g = O.freq_grid(n, 1.0)
        assert abs(np.sum(g * 2.0 / (om ** 2 + 1.0)) - math.pi) < 1e-3 ** (n / 8)
    errs = []
    for n in (8, 16, 32, 64):
        om, g = O.freq_grid(n, 1.0)
        errs.append(abs(np.sum(g * 2 * 0.13 / (om ** 2 + 0.13 ** 2)) - math.pi))
    assert errs[-1] < 1e-6 and all(b < a for a, b in zip(errs, errs[1:]))
    om, g = O.freq_grid(16)
    assert np.all(om > 0) and np.all(np.diff(om) > 0) and np.all(g > 0)


def test_lri_split_matches_realspace_expansion():
    """Eq. AO_triple_split2 (oracle) equals the cell-by-cell real-space LRI sum (Eq. realspace_expan2)."""
    s = make_system("tiny", seed=3)
    for ik in range(s.n_k):
        for iq in range(s.n_k):
            C = O.ao_triple(s, ik, iq)
            for mu in range(s.n_aux):
                for i in range(s.n_basis):
                    for j in range(s.n_basis):
                        c0, c1 = brute.lri_coeff_realspace(s, ik, iq, mu, i, j)
                        assert abs(c0 - c1) < 1e-12          # Bloch structure e^{-i q.R0}
                        assert abs(C[mu, i, j] - c0) < 1e-12


def test_ao_mo_transform_conjugation(monkeypatch):
    """Eq. AO_MO_transform with C~^mu_ij = t delta_ij gives M = t c(k+q)^H c(k) (= t 1 at q = 0)."""
    s = make_system("tiny", seed=4, trs=False)
    t = 0.7 - 0.2j
    monkeypatch.setattr(O, "ao_triple",
                        lambda sys, ik, iq: np.broadcast_to(t * np.eye(sys.n_basis), (sys.n_aux, sys.n_basis, sys.n_basis)))
    bands = np.arange(s.n_bands)
    for ik in range(s.n_k):
        M0 = O.mo_triple(s, ik, 0, bands, bands)
        assert np.abs(M0 - t * np.eye(s.n_bands)[None]).max() < 1e-12
        iq = 1
        ikq = O.k_plus(s.nk, ik, iq)
        M = O.mo_triple(s, ik, iq, bands, bands)
        ref = t * np.conj(s.evec[ikq]).T @ s.evec[ik]
        assert np.abs(M - ref[None]).max() < 1e-12


def test_chi0_hermitian_nsd_and_literal():
    """chi0 Hermitian and NSD; under time reversal the Hermitised form equals the literal two-term sum."""
    s = make_system("tiny", seed=5)
    om, _ = O.freq_grid(s.n_freq)
    for iq in range(s.n_k):
        c = O.chi0(s, iq, om)
        cl = O.chi0_literal(s, iq, om)
        scale = np.abs(c).max()
        assert np.abs(c - np.conj(np.transpose(c, (0, 2, 1)))).max() < 1e-14 * scale * 10
        for x in c:
            assert np.linalg.eigvalsh(x).max() < 1e-12 * scale
        assert np.abs(c - cl).max() < 1e-12 * scale
    # without time reversal the literal form is not Hermitian, the Hermitised one is
    s2 = make_system("tiny", seed=5, trs=False)
    cl = O.chi0_literal(s2, 1, om)
    assert np.abs(cl - np.conj(np.transpose(cl, (0, 2, 1)))).max() > 1e-6 * np.abs(cl).max()


def _twoband(n_freq):
    return make_system(dict(nk=(1, 1, 1), n_atoms=2, nb_per_atom=1, naux_per_atom=3, n_bands=2,
                            n_occ=1, n_freq=n_freq, sigma=(0, 2), omega_cell=100.0),
                       seed=11, head_wings=0, v1_ratio=0.0)


def test_twoband_single_k_closed_form():
    """One occupied, one empty band, one k: rank-1 chi0, Sherman-Morrison eps~^{-1}, single-pole W^c."""
    s = _twoband(16)
    om, _ = O.freq_grid(s.n_freq)
    m = O.mo_triple(s, 0, 0, [1], [0])[:, 0, 0]
    D = s.eps[0, 1] - s.eps[0, 0]
    w = 2 * D / (om ** 2 + D ** 2)
    c = O.chi0(s, 0, om)
    ref = -s.spin * w[:, None, None] * np.outer(m, np.conj(m))[None]
    assert np.abs(c - ref).max() < 1e-14 * np.abs(ref).max() * 10
    Vh = scipy.linalg.sqrtm(s.V[0])
    u = Vh @ m
    y = Vh @ u
    Wp = math.sqrt(D * D + 2 * s.spin * D * np.vdot(u, u).real)
    _, Wc = O.screen(s, 0, c, om)
    refW = -(s.spin * D / Wp) * np.outer(y, np.conj(y))[None] * (2 * Wp / (om ** 2 + Wp ** 2))[:, None, None]
    assert np.abs(Wc - refW).max() < 1e-10 * np.abs(refW).max()


def test_single_pole_sigma_analytic():
    """Single-pole W^c gives Sigma_c_n(iw) = sum_m a_nm / (iw + mu - e_m - sgn(e_m - mu) Omega_p)."""
    errs = []
    for nf in (16, 32, 64):
        s = _twoband(nf)
        om, g = O.freq_grid(nf)
        mu = O.mu_midgap(s)
        c = O.chi0(s, 0, om)
        _, Wc = O.screen(s, 0, c, om)
        sig = O.sigma_q(s, 0, Wc, om, g, mu)
        m = O.mo_triple(s, 0, 0, [1], [0])[:, 0, 0]
        D = s.eps[0, 1] - s.eps[0, 0]
        Vh = scipy.linalg.sqrtm(s.V[0])
        y = Vh @ (Vh @ m)
        Wp = math.sqrt(D * D + 2 * s.spin * D * np.vdot(Vh @ m, Vh @ m).real)
        Mall = O.mo_triple(s, 0, 0, [0, 1], [0, 1])       # [mu, n, m]
        ref = np.zeros_like(sig)
        for n in range(2):
            for mm in range(2):
                a = (s.spin * D / Wp) * abs(np.sum(Mall[:, n, mm] * y)) ** 2
                em = s.eps[0, mm]
                ref[0, n] += a / (1j * om + mu - em - np.sign(em - mu) * Wp)
        # the convolution kernel 2z/(z^2+w'^2) peaks at w' ~ w with width |mu - e_m|; the grid
        # resolves it for w below ~1 Ha, where the quadrature must converge to the contour integral
        sel = om < 1.0
        errs.append(np.abs(sig - ref)[..., sel].max() / np.abs(ref).max())
    assert errs[2] < 1e-8 and errs[1] < errs[0]


def test_two_pole_continuation_exact_and_qp():
    """The two-pole model reproduces a two-pole Sigma exactly; the QP solution satisfies its equation."""
    om, _ = O.freq_grid(16)
    z = 1j * om
    a1, b1, a2, b2 = 0.05, -0.9, 0.08, 1.3
    f = a1 / (z - b1) + a2 / (z - b2)
    c = O.two_pole_fit(z, f)
    x = np.linspace(-0.5, 0.5, 11)
    ref = a1 / (x - b1) + a2 / (x - b2)
    assert np.abs(O.two_pole_eval(c, x) - ref).max() < 1e-11
    h = 1e-6
    num = (O.two_pole_eval(c, x + h) - O.two_pole_eval(c, x - h)) / (2 * h)
    assert np.abs(O.two_pole_deriv(c, x) - num).max() < 1e-6
    mu, e0, dxv = 0.05, 0.3, -0.01
    E, ok = O.qp_solve(e0, c, mu, dxv)
    assert ok and abs(E - e0 - (a1 / (E - mu - b1) + a2 / (E - mu - b2)) - dxv) < 1e-12


def test_head_wings_kp_limit(monkeypatch):
    """Eq. dielectric_func_gamma (head, wings, body) equals the regular eps~ at small q under the k.p model.

    V(q) = (4 pi / (Omega_cell q^2)) x1 x1^T + sum_{l>1} v_l x_l x_l^T and
    <x1, M_ai(k, q)> = q (p_ia . q^) / (e_i - e_a); the other components fixed.
    """
    s = make_system(dict(nk=(2, 1, 1), n_atoms=2, nb_per_atom=2, naux_per_atom=3, n_bands=4,
                         n_occ=2, n_freq=8, sigma=(0, 4), omega_cell=150.0), seed=21)
    rng = np.random.default_rng(0)
    N = s.n_aux
    X, _ = np.linalg.qr(rng.standard_normal((N, N)))
    v_rest = np.sort(rng.uniform(0.2, 2.0, N - 1))[::-1]
    q = 1e-3
    v1q = 4 * math.pi / (s.omega_cell * q * q)
    occ, unocc = np.arange(s.n_occ), np.arange(s.n_occ, s.n_bands)
    mhat_rest = {ik: (rng.standard_normal((N - 1, len(unocc), len(occ)))
                      + 1j * rng.standard_normal((N - 1, len(unocc), len(occ)))) * 0.05
                 for ik in range(s.n_k)}

    def M_of(ik, small_q):
        pq = np.einsum("d,dmn->mn", s.qhat, s.pmom[ik])
        e = s.eps[ik]
        head = np.zeros((len(unocc), len(occ)), dtype=complex)
        if small_q:
            for ia, a in enumerate(unocc):
                for ii, i in enumerate(occ):
                    head[ia, ii] = q * pq[i, a] / (e[i] - e[a])
        mh = np.concatenate([head[None], mhat_rest[ik]], 0)
        return np.einsum("ul,lai->uai", X, mh)

    om, _ = O.freq_grid(s.n_freq)
    # regular formula at small q (k+q taken at k: the limit)
    monkeypatch.setattr(O, "mo_triple", lambda sys, ik, iq, a, b: M_of(ik, True))
    chi_q = O.chi0(s, 0, om)
    vq = np.concatenate([[v1q], v_rest])
    reg = [np.eye(N) - (X * np.sqrt(vq)) @ X.T @ cq @ X @ (np.sqrt(vq)[:, None] * X.T) for cq in chi_q]
    # Gamma-point assembly from p (head, wings) and the body
    monkeypatch.setattr(O, "mo_triple", lambda sys, ik, iq, a, b: M_of(ik, False))
    s.V = s.V.copy()
    s.V[0] = (X * np.concatenate([[50.0], v_rest])) @ X.T
    chi_0 = O.chi0(s, 0, om)
    eps_X, Xo, v = O.head_wings_q0(s, om, chi_0)
    for w_i in range(len(om)):
        got = Xo @ eps_X[w_i] @ np.conj(Xo).T
        assert np.abs(got - reg[w_i]).max() < 1e-9 * np.abs(reg[w_i]).max()
    assert np.all(np.real([e[0, 0] for e in eps_X]) > 1.0)


def test_q0_body_is_regular_formula():
    """At q = 0 the lambda, lambda' > 1 block equals the regular eps~ in the Coulomb eigenbasis."""
    s = make_system("tiny", seed=8)
    om, _ = O.freq_grid(s.n_freq)
    c = O.chi0(s, 0, om)
    eps_X, X, v = O.head_wings_q0(s, om, c)
    Vh = O.hsqrt(s.V[0])
    for w_i in range(len(om)):
        reg = np.conj(X).T @ (np.eye(s.n_aux) - Vh @ c[w_i] @ Vh) @ X
        assert np.abs(eps_X[w_i][1:, 1:] - reg[1:, 1:]).max() < 1e-10 * np.abs(reg).max()


def test_screening_invariants():
    """eps~ >= 1 (chi0 NSD), eps~^{-1} in (0, 1], W^c negative semidefinite; also at q = 0 with head/wings."""
    s = make_system("tiny", seed=9)
    om, _ = O.freq_grid(s.n_freq)
    for iq in range(s.n_k):
        c = O.chi0(s, iq, om)
        e, W = O.screen(s, iq, c, om)
        for w_i in range(len(om)):
            ev = np.linalg.eigvalsh(0.5 * (e[w_i] + np.conj(e[w_i]).T))
            assert ev.min() > 1 - 1e-10
            assert np.linalg.eigvalsh(0.5 * (W[w_i] + np.conj(W[w_i]).T)).max() < 1e-10


def test_brute_force_pipeline_tiny():
    """Explicit-loop pipeline (real-space LRI, literal chi0 at +-w, Denman-Beavers, unfolded w') == oracle."""
    s = make_system("tiny", seed=12, head_wings=0)
    b = brute.g0w0_brute(s)
    r = O.g0w0(s, keep=True)
    om = r["omega"]
    for iq in range(s.n_k):
        ikq = None
        for jw in range(len(om)):
            c = r["per_q"][iq]["chi0"][jw]
            assert np.abs(b["chi0"][(iq, 1.0, jw)] - c).max() < 1e-12 * np.abs(c).max()
            W = r["per_q"][iq]["Wc"][jw]
            assert np.abs(b["Wc"][(iq, 1.0, jw)] - W).max() < 1e-9 * np.abs(W).max()
    assert np.abs(b["sigma"] - r["sigma"]).max() < 1e-9 * np.abs(r["sigma"]).max()
    # the dense M of the oracle equals the quadruple loop over the brute C~
    for (ik, iq), Mb in b["M"].items():
        Mo = O.mo_triple(s, ik, iq, np.arange(s.n_bands), np.arange(s.n_bands))
        assert np.abs(Mb - Mo).max() < 1e-12


def test_qp_stable_under_small_sigma_noise():
    """The continuation + QP solve moves < 0.1 meV for 1e-6 relative noise on Sigma_c (cfg0 shape)."""
    s = make_system("cfg0", seed=0)
    r = O.g0w0(s, qs=[0, 1, 3])
    rng = np.random.default_rng(1)
    sig = r["sigma"] * (1 + 1e-6 * rng.standard_normal(r["sigma"].shape))
    E, gap, conv = O.qp(s, sig, r["omega"], r["mu"])
    assert conv.all() and r["converged"].all()
    assert np.abs(E - r["e_qp"]).max() * HA_MEV < 0.1
    assert abs(gap - r["gap"]) * HA_MEV < 0.1


def test_sigma_x_closed_form_delta_lri_identity_coulomb(monkeypatch):
    """C~^mu_ij = t delta_ij for every ABF and V(q) = 1: C^mu_{nm}(k, k-q) = t <psi_nk|psi_m,k-q>,
    so Sigma_x_n(k) = -(N_aux |t|^2 / N_q) sum_q sum_{m occ} |<psi_nk|psi_m,k-q>|^2 (overlaps from c)."""
    s = make_system("tiny", seed=6, trs=False)
    t = 0.6 + 0.3j
    monkeypatch.setattr(O, "ao_triple",
                        lambda sys, ik, iq: np.broadcast_to(t * np.eye(sys.n_basis), (sys.n_aux, sys.n_basis, sys.n_basis)))
    s.V = np.broadcast_to(np.eye(s.n_aux, dtype=complex), (s.n_k, s.n_aux, s.n_aux)).copy()
    got = O.sigma_x(s)
    want = np.zeros_like(got)
    for ik in range(s.n_k):
        for iq in range(s.n_k):
            ikmq = O.k_minus(s.nk, ik, iq)
            ov = np.conj(s.evec[ik][:, s.sigma_lo:s.sigma_hi]).T @ s.evec[ikmq][:, :s.n_occ]
            want[ik] -= s.n_aux * abs(t) ** 2 * np.sum(np.abs(ov) ** 2, axis=1)
    want /= s.n_k
    assert np.allclose(got, want, rtol=1e-12, atol=0)


def test_sigma_x_negative_and_matches_loops():
    """Sigma_x <= 0 (V positive definite) and equals an explicit-loop evaluation on the brute-force
    LRI coefficients (real-space sum per cell, no half transforms)."""
    from oracle import brute as B
    s = make_system("tiny", seed=7)
    got = O.sigma_x(s)
    assert (got < 0).all()
    ref = np.zeros_like(got)
    for ik in range(s.n_k):
        for iq in range(s.n_k):
            ikmq = O.k_minus(s.nk, ik, iq)
            M = B.mo_triple_brute(s, ikmq, iq)                 # [mu, a (k-q+q = k), b (k-q)]
            for n in range(s.sigma_lo, s.sigma_hi):
                for m in range(s.n_occ):
                    a = M[:, n, m]
                    ref[ik, n - s.sigma_lo] -= (a @ s.V[iq] @ np.conj(a)).real
    ref /= s.n_k
    assert np.allclose(got, ref, rtol=1e-10, atol=0)


def test_chi0_block_is_a_block_of_chi0():
    """The ABF-subset form reproduces the matching block of the full chi0 (independent assembly of
    C~ one ABF at a time)."""
    s = make_system("cfg0", seed=9)
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    mus = [0, 17, 48, 95]
    full = O.chi0(s, 3, om[:3])
    blk = O.chi0_block(s, 3, om[:3], mus)
    assert np.abs(blk - full[:, mus][:, :, mus]).max() <= 1e-13 * np.abs(full).max()


@pytest.mark.parametrize("window", [(0, 4), (1, 3)])
def test_qp_gap_selection_hand_built(window):
    """The indirect gap takes band n_occ - 1 (HOMO) and band n_occ (LUMO) at every k, after the
    QP shift, and the window offset sigma_lo; the case (tests/qp_case.py) is built so that every
    other plausible selection gives another number."""
    import qp_case as C
    s = C.system(window)
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    E, gap, conv = O.qp(s, C.sigma_c(s, om), om, O.mu_midgap(s), C.dxv(s))
    assert conv.all()
    assert np.abs(E - C.e_expected(s)).max() < 1e-8
    assert abs(gap - C.GAP) < 1e-8


def test_mu_midgap_hand_built():
    """Midgap chemical potential of the hand-built energies: (max_k HOMO + min_k LUMO) / 2."""
    import qp_case as C
    assert abs(O.mu_midgap(C.system()) - C.MU) < 1e-15


def test_sphere_rule_moments_and_uniaxial_closed_form():
    """The direction rule of the q -> 0 average: weights sum to 1, <q_a q_b> = delta_ab / 3 and
    odd moments vanish exactly; the average of 1 / (1 + a q_z^2) is arctan(sqrt a) / sqrt a."""
    dirs, w = O.sphere_rule()
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-14)
    assert np.abs(np.einsum("n,na,nb->ab", w, dirs, dirs) - np.eye(3) / 3).max() < 1e-14
    assert np.abs(w @ dirs).max() < 1e-15
    for a in (0.1, 0.5, 1.0):
        avg = w @ (1.0 / (1.0 + a * dirs[:, 2] ** 2))
        assert abs(avg - math.atan(math.sqrt(a)) / math.sqrt(a)) < 2e-6


def test_direction_average_of_a_uniaxial_head(monkeypatch):
    """head_wings = 2 with no LRI coefficients (chi0 = 0, no wings) and a momentum matrix along z
    only: eps~(q^) is 1 except its head 1 + a q_z^2, so the averaged eps~^-1 - 1 is
    (arctan(sqrt a)/sqrt a - 1) x1 x1^H and W^c(0) = v1 times that (x1, v1 the Coulomb head pair)."""
    s = make_system("tiny", seed=8, c_scale=0.0, head_wings=2)
    s.pmom[:, 0:2] = 0.0
    s.pmom *= 0.2
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    chi = O.chi0(s, 0, om)
    assert np.abs(chi).max() == 0.0
    _, W = O.screen(s, 0, chi, om)
    v, X = O.coulomb_eig_q0(s.V[0])
    x1 = X[:, 0]
    s1 = make_system("tiny", seed=8, c_scale=0.0)
    s1.pmom[:] = s.pmom
    s1.qhat = np.array([0.0, 0.0, 1.0])
    eps_z, _, _ = O.head_wings_q0(s1, om, chi)
    for j in range(len(om)):
        a = eps_z[j][0, 0].real - 1.0
        assert 0.0 < a < 1.0
        ref = v[0] * (math.atan(math.sqrt(a)) / math.sqrt(a) - 1.0) * np.outer(x1, np.conj(x1))
        assert np.abs(W[j] - ref).max() <= 3e-6 * np.abs(ref).max()


def test_direction_average_matches_schur_form():
    """The average of eps~(q^)^-1 - 1 over the directions (direct inversions) equals its Schur-
    complement form: with G the inverse of the body block (the head row and column removed),
    y(q^) the wing column and s(q^) = head - y^H G y, eps~^-1 - 1 = (G - 1) + (1/s - 1) x1 x1^H
    - (x1 g^H + g x1^H)/s + g g^H / s, g = G y, whose average needs only <1/s>, <q^/s>, <q^ q^T/s>."""
    s = make_system("tiny", seed=9, head_wings=2)
    om, _ = O.freq_grid(s.n_freq, s.omega0)
    chi = O.chi0(s, 0, om)
    _, W = O.screen(s, 0, chi, om)
    Vh = O.hsqrt(s.V[0])
    dirs, wts = O.sphere_rule()
    N = s.n_aux
    for j in (0, len(om) - 1):
        acc = np.zeros((N, N), dtype=np.complex128)
        for d, wd in zip(dirs, wts):
            eX, X, v = O.head_wings_q0(s, om[j:j + 1], chi[j:j + 1], qhat=d)
            E = eX[0]
            G = np.zeros((N, N), dtype=np.complex128)
            G[0, 0] = 1.0
            G[1:, 1:] = np.linalg.inv(E[1:, 1:])
            y = np.zeros(N, dtype=np.complex128)
            y[1:] = E[1:, 0]
            g = G @ y
            sc = (E[0, 0] - np.conj(y) @ g).real
            e1 = np.zeros(N)
            e1[0] = 1.0
            Xl = G - np.eye(N) + (1 / sc - 1) * np.outer(e1, e1) - (np.outer(e1, np.conj(g)) + np.outer(g, e1)) / sc \
                + np.outer(g, np.conj(g)) / sc
            acc += wd * (X @ Xl @ np.conj(X).T)
        ref = Vh @ acc @ Vh
        assert np.linalg.norm(W[j] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_shifted_mesh_by_a_mesh_vector_relabels_the_points():
    """A k mesh shifted by a mesh vector is the same mesh relabelled: with the KS data carried
    along, Sigma_c at shifted point i (its rows built with the phases of k + offset, W^c from the
    unshifted q mesh) equals Sigma_c of the unshifted system at the point i + shift."""
    from paper_2011_01400_gb300.synth import shifted_system
    s = make_system("tiny", seed=10, head_wings=0)
    step = (1, 0, 0)
    perm = [O.k_index(s.nk, tuple(a + b for a, b in zip(O.k_of(s.nk, i), step))) for i in range(s.n_k)]
    t = shifted_system(s, (1.0 / s.nk[0], 0.0, 0.0), seed=11, eps=s.eps[perm], evec=s.evec[perm],
                       pmom=s.pmom[perm])
    om, g = O.freq_grid(s.n_freq, s.omega0)
    mu = O.mu_midgap(s)
    nsig = s.sigma_hi - s.sigma_lo
    sig_s = np.zeros((s.n_k, nsig, s.n_freq), dtype=np.complex128)
    sig_t = np.zeros_like(sig_s)
    for q in range(s.n_k):
        _, W = O.screen(s, q, O.chi0(s, q, om), om)
        sig_s += O.sigma_q(s, q, W, om, g, mu)
        sig_t += O.sigma_q(t, q, W, om, g, mu)
    assert np.abs(sig_t - sig_s[perm]).max() <= 1e-13 * np.abs(sig_s).max()


def _tan_midpoint(n, w0):
    """Midpoint rule on w = w0 tan(t), t in (0, pi/2): nodes and weights for an integral over (0, inf)."""
    t = (np.arange(n) + 0.5) * np.pi / (2 * n)
    return w0 * np.tan(t), w0 * (np.pi / (2 * n)) / np.cos(t) ** 2


def test_caller_grid_single_pole_sigma_analytic():
    """A caller grid (tangent-mapped midpoint rule, not the default Gauss-Legendre one) carried through
    the whole pipeline reproduces the single-pole Sigma_c of the two-band system at its own nodes:
    the mapped integrand is smooth and periodic in t, so the rule converges spectrally."""
    s = _twoband(32)
    om, g = _tan_midpoint(32, 1.0)
    r = O.g0w0(s, grid=(om, g))
    assert np.array_equal(r["omega"], om) and np.array_equal(r["g"], g)
    mu = r["mu"]
    D = s.eps[0, 1] - s.eps[0, 0]
    m = O.mo_triple(s, 0, 0, [1], [0])[:, 0, 0]
    Vh = scipy.linalg.sqrtm(s.V[0])
    y = Vh @ (Vh @ m)
    Wp = math.sqrt(D * D + 2 * s.spin * D * np.vdot(Vh @ m, Vh @ m).real)
    Mall = O.mo_triple(s, 0, 0, [0, 1], [0, 1])
    ref = np.zeros_like(r["sigma"])
    for n in range(2):
        for mm in range(2):
            a = (s.spin * D / Wp) * abs(np.sum(Mall[:, n, mm] * y)) ** 2
            em = s.eps[0, mm]
            ref[0, n] += a / (1j * om + mu - em - np.sign(em - mu) * Wp)
    sel = om < 1.0
    assert np.abs(r["sigma"] - ref)[..., sel].max() < 1e-12 * np.abs(ref).max()


def test_caller_grid_order_and_weight_scaling():
    """Reversing the nodes permutes Sigma_c and leaves the QP energies (a least-squares fit over all
    nodes) unchanged; Sigma_c is linear in the weights; the default grid passed explicitly is the
    default."""
    s = make_system("cfg0", seed=0)
    om, g = _tan_midpoint(s.n_freq, 2.0)
    r = O.g0w0(s, grid=(om, g))
    rv = O.g0w0(s, grid=(om[::-1], g[::-1]))
    assert np.abs(rv["sigma"][..., ::-1] - r["sigma"]).max() < 1e-12 * np.abs(r["sigma"]).max()
    assert np.abs(rv["e_qp"] - r["e_qp"]).max() < 1e-9
    r2 = O.g0w0(s, qs=[0, 1], grid=(om, 2.0 * g))
    r1 = O.g0w0(s, qs=[0, 1], grid=(om, g))
    assert np.abs(r2["sigma"] - 2.0 * r1["sigma"]).max() < 1e-13 * np.abs(r1["sigma"]).max()
    d = O.g0w0(s, qs=[0, 1])
    e = O.g0w0(s, qs=[0, 1], grid=O.freq_grid(s.n_freq, s.omega0))
    assert np.array_equal(d["sigma"], e["sigma"])
