"""A hand-built quasiparticle case whose indirect gap is known by construction.

Four k points (the 2x2x1 "tiny" mesh), six bands, two occupied. The KS energies, the
Sigma_x - v_xc shifts and a negligible Sigma_c (one pole of weight 1e-9 Ha) are chosen so
that every plausible wrong selection of the gap gives a different number:

    k     HOMO-1   HOMO    LUMO   LUMO+1    shift (Sigma_x - v_xc)
    0     -0.60   -0.30    0.40    0.90     HOMO-1 +0.50  -> -0.10
    1     -0.55   -0.25    0.10    0.80
    2     -0.50   -0.20    0.30    0.70     LUMO+1 -0.65  ->  0.05
    3     -0.65   -0.35    0.50    0.60     HOMO   +0.20  -> -0.15

    QP HOMO (band n_occ - 1 at every k): max over k = -0.15 (k = 3)
    QP LUMO (band n_occ at every k):     min over k =  0.10 (k = 1)
    indirect gap = 0.25 Ha.
    Wrong readings: highest occupied QP level of any band 0.20, lowest empty of any band
    0.20, smallest direct gap 0.35, shifts ignored 0.30.
    Midgap chemical potential of the KS energies: (-0.20 + 0.10) / 2 = -0.05 Ha.
"""
import numpy as np

from paper_2011_01400_gb300.synth import make_system

GAP = 0.25
MU = -0.05
EPS = np.array([[-0.60, -0.30, 0.40, 0.90, 1.50, 2.00],
                [-0.55, -0.25, 0.10, 0.80, 1.60, 2.10],
                [-0.50, -0.20, 0.30, 0.70, 1.70, 2.20],
                [-0.65, -0.35, 0.50, 0.60, 1.80, 2.30]])
SHIFT = np.zeros((4, 6))
SHIFT[0, 0] = 0.50
SHIFT[2, 3] = -0.65
SHIFT[3, 1] = 0.20
POLE_A, POLE_B = 1e-9, -1.0


def system(sigma=(0, 4)):
    s = make_system("tiny", seed=5)
    assert s.n_k == 4 and s.n_bands == 6 and s.n_occ == 2
    s.eps = EPS.copy()
    s.sigma_lo, s.sigma_hi = sigma
    return s


def sigma_c(s, omegas):
    """Sigma_c_n(k, i w) = A / (i w - B) for every (k, n) of the window: [N_k][n_sigma][n_freq]."""
    nsig = s.sigma_hi - s.sigma_lo
    f = POLE_A / (1j * np.asarray(omegas) - POLE_B)
    return np.broadcast_to(f, (s.n_k, nsig, len(omegas))).copy()


def dxv(s):
    return SHIFT[:, s.sigma_lo:s.sigma_hi].copy()


def e_expected(s):
    """QP energies to ~1e-9 Ha (Sigma_c is below 2e-9 Ha at every QP energy)."""
    return (EPS + SHIFT)[:, s.sigma_lo:s.sigma_hi]
