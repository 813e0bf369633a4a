"""Seeded synthetic inputs for the periodic G0W0 hot path.

This module only draws random inputs with the shapes and symmetries of the
method's input data (Sec. II of the paper: KS energies and eigenvectors,
two-centre LRI coefficients C~_{i(0),j(R)}^{mu(0)}, the Coulomb matrix V(q),
the momentum matrix p). It contains none of the method's arithmetic (no
Fourier transform of the LRI coefficients, no AO->MO transform, no response
function, screening or self-energy). Both the CPU oracle and the CUDA path
consume exactly the arrays produced here.

Time-reversal symmetry (the default) follows from real NAOs/ABFs (Sec. II.B):
    C~(R) real, c(-k) = c(k)*, eps(-k) = eps(k), V(-q) = V(q)*, p(-k) = -p(k)*.
Self-conjugate mesh points (k == -k mod the mesh) get real c, real V and
purely imaginary Hermitian p.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["System", "CONFIGS", "make_system", "shifted_system", "kmesh_index", "minus_k", "add_k"]


@dataclasses.dataclass
class System:
    nk: tuple               # Gamma-centred mesh (n1, n2, n3); q mesh = k mesh
    n_atoms: int
    n_basis: int
    n_bands: int
    n_occ: int
    n_aux: int
    basis_atom: np.ndarray  # int32 [n_basis], atom of each NAO (atoms contiguous)
    aux_atom: np.ndarray    # int32 [n_aux], atom of each ABF (atoms contiguous)
    R: np.ndarray           # int32 [n_R, 3] lattice vectors (lattice coordinates)
    eps: np.ndarray         # f64 [N_k, n_bands]  KS energies (Ha), sorted per k
    evec: np.ndarray        # c128 [N_k, n_basis, n_bands]  c_{i,n}(k)
    ctil_R: list            # per atom A: f64 [n_R, n_aux(A), n_b(A), n_basis] = C~_{i(0),j(R)}^{mu(0)}, mu,i on A
    V: np.ndarray           # c128 [N_q, n_aux, n_aux] Hermitian positive definite (plays V^cut)
    pmom: np.ndarray        # c128 [N_k, 3, n_bands, n_bands] momentum matrix, Hermitian in (m, n)
    omega_cell: float       # unit-cell volume (bohr^3)
    qhat: np.ndarray        # f64 [3] direction of q -> 0
    n_freq: int
    omega0: float           # scale of the modified Gauss-Legendre grid (Ha)
    sigma_lo: int           # 0-based first band of the self-energy window
    sigma_hi: int           # one past the last band of the window
    spin: float = 2.0
    head_wings: int = 1
    seed: int = 0
    trs: bool = False       # drawn with time-reversal symmetry (then the library may pair q with -q)
    k_offset: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))  # shift of the k mesh

    @property
    def n_k(self):
        return int(np.prod(self.nk))

    def ctil_flat(self):
        """All atoms' C~(R) blocks concatenated in atom order (the library layout)."""
        return np.concatenate([c.ravel() for c in self.ctil_R])


# Shapes of the paper-like workloads. "tiny" and "twoband" are test-only sizes.
CONFIGS = {
    # tiny synthetic insulator: 2x2x2 k, 2 atoms, 16 NAO + 48 ABF per atom
    "cfg0": dict(nk=(2, 2, 2), n_atoms=2, nb_per_atom=16, naux_per_atom=48, n_bands=32,
                 n_occ=4, n_freq=16, sigma=(2, 6), omega_cell=270.25),
    # Si-like 2-atom fcc cell, 6x6x6 k
    "cfg1": dict(nk=(6, 6, 6), n_atoms=2, nb_per_atom=39, naux_per_atom=200, n_bands=78,
                 n_occ=4, n_freq=32, sigma=(0, 8), omega_cell=270.25),
    # ZnO-like 4-atom wurtzite cell, 6x6x4 k
    "cfg2": dict(nk=(6, 6, 4), n_atoms=4, nb_per_atom=75, naux_per_atom=400, n_bands=300,
                 n_occ=36, n_freq=32, sigma=(32, 40), omega_cell=321.6),
    # brute-force size: every loop explicit in the test oracle
    "tiny": dict(nk=(2, 2, 1), n_atoms=2, nb_per_atom=3, naux_per_atom=5, n_bands=6,
                 n_occ=2, n_freq=8, sigma=(0, 4), omega_cell=100.0),
}


def kmesh_index(nk, i1, i2, i3):
    return ((i1 % nk[0]) * nk[1] + (i2 % nk[1])) * nk[2] + (i3 % nk[2])


def _kcoords(nk, ik):
    i3 = ik % nk[2]
    i2 = (ik // nk[2]) % nk[1]
    i1 = ik // (nk[1] * nk[2])
    return i1, i2, i3


def minus_k(nk, ik):
    i1, i2, i3 = _kcoords(nk, ik)
    return kmesh_index(nk, -i1, -i2, -i3)


def add_k(nk, ik, iq):
    a = _kcoords(nk, ik)
    b = _kcoords(nk, iq)
    return kmesh_index(nk, a[0] + b[0], a[1] + b[1], a[2] + b[2])


def _cgauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _lattice_vectors():
    R = [(0, 0, 0)]
    for d in range(3):
        for s in (1, -1):
            v = [0, 0, 0]
            v[d] = s
            R.append(tuple(v))
    return np.array(R, dtype=np.int32)


def make_system(cfg="cfg0", seed=0, *, trs=True, n_freq=None, nk=None, n_bands=None,
                n_occ=None, omega0=1.0, head_wings=1, v1_ratio=10.0, p_scale=0.5,
                c_scale=None, **over):
    """Draw one seeded synthetic system shaped like configuration `cfg`.

    Recipe: occupied energies uniform in [-0.8, -0.2] Ha, unoccupied uniform
    in [0.05, 3.0] Ha, sorted per k; c(k) = Q of the QR of a Gaussian matrix;
    C~(R) = sigma_C x Gaussian x exp(-|R|/2) on the 7 lattice vectors |R| <= 1;
    V(q) = A A^H / N_aux + 0.1 I; at q = 0 one extra rank-1 term
    v1 x x^T with v1 = v1_ratio x (largest other eigenvalue) plays the
    G = 0-like Coulomb eigenstate; p = p_scale x Hermitian Gaussian.
    sigma_C = 0.206 sqrt(N_b / (N_aux n_b(A))) puts the typical bare pair
    Coulomb integral a^H V a near 0.3 Ha, so that Sigma_c has the eV scale of
    real semiconductors (unit-variance entries give Sigma_c ~ 10^3 Ha).
    """
    p = dict(CONFIGS[cfg]) if isinstance(cfg, str) else dict(cfg)
    p.update(over)
    if nk is not None:
        p["nk"] = tuple(nk)
    if n_freq is not None:
        p["n_freq"] = n_freq
    if n_bands is not None:
        p["n_bands"] = n_bands
    if n_occ is not None:
        p["n_occ"] = n_occ
    nkm = tuple(int(x) for x in p["nk"])
    NK = int(np.prod(nkm))
    na = p["n_atoms"]
    nba = p["nb_per_atom"]
    nxa = p["naux_per_atom"]
    nb = na * nba
    nx = na * nxa
    nbands = p["n_bands"]
    nocc = p["n_occ"]
    assert nbands <= nb and 0 < nocc < nbands
    rng = np.random.default_rng(seed)

    basis_atom = np.repeat(np.arange(na, dtype=np.int32), nba)
    aux_atom = np.repeat(np.arange(na, dtype=np.int32), nxa)
    R = _lattice_vectors()
    nR = R.shape[0]

    # LRI two-centre coefficients, real (real NAOs and ABFs)
    decay = np.exp(-0.5 * np.sqrt((R.astype(np.float64) ** 2).sum(1)))
    sig_c = 0.206 * np.sqrt(nb / (nx * nba)) if c_scale is None else c_scale
    ctil = []
    for _A in range(na):
        c = sig_c * rng.standard_normal((nR, nxa, nba, nb)) * decay[:, None, None, None]
        ctil.append(np.ascontiguousarray(c))

    eps = np.zeros((NK, nbands))
    evec = np.zeros((NK, nb, nbands), dtype=np.complex128)
    pm = np.zeros((NK, 3, nbands, nbands), dtype=np.complex128)
    done = np.zeros(NK, dtype=bool)
    for ik in range(NK):
        if done[ik]:
            continue
        mk = minus_k(nkm, ik) if trs else ik
        e = np.concatenate([np.sort(rng.uniform(-0.8, -0.2, nocc)),
                            np.sort(rng.uniform(0.05, 3.0, nbands - nocc))])
        selfconj = trs and (mk == ik)
        if selfconj:
            g = rng.standard_normal((nb, nb))
        else:
            g = _cgauss(rng, (nb, nb))
        q, r = np.linalg.qr(g)
        q = q * np.sign(np.diag(r).real)[None, :] if selfconj else q
        c = q[:, :nbands]
        if selfconj:
            s = rng.standard_normal((3, nbands, nbands))
            pk = 1j * p_scale * (s - s.transpose(0, 2, 1)) / np.sqrt(2.0)
        else:
            g3 = _cgauss(rng, (3, nbands, nbands))
            pk = p_scale * (g3 + np.conj(g3.transpose(0, 2, 1))) / np.sqrt(2.0)
        eps[ik], evec[ik], pm[ik] = e, c, pk
        done[ik] = True
        if trs and mk != ik:
            eps[mk], evec[mk], pm[mk] = e, np.conj(c), -np.conj(pk)
            done[mk] = True

    V = np.zeros((NK, nx, nx), dtype=np.complex128)
    done[:] = False
    for iq in range(NK):
        if done[iq]:
            continue
        mq = minus_k(nkm, iq) if trs else iq
        selfconj = trs and (mq == iq)
        if selfconj:
            a = rng.standard_normal((nx, nx))
        else:
            a = _cgauss(rng, (nx, nx))
        v = a @ np.conj(a.T) / nx + 0.1 * np.eye(nx)
        if iq == 0 and v1_ratio > 0:
            # q = 0 plays V^cut(0): one eigenvalue standing far above the rest
            x = rng.standard_normal(nx)
            x /= np.linalg.norm(x)
            vmax = np.linalg.eigvalsh(v)[-1]
            v = v + v1_ratio * vmax * np.outer(x, x)
        v = 0.5 * (v + np.conj(v.T))
        V[iq] = v
        done[iq] = True
        if trs and mq != iq:
            V[mq] = np.conj(v)
            done[mq] = True

    lo, hi = p["sigma"]
    return System(nk=nkm, n_atoms=na, n_basis=nb, n_bands=nbands, n_occ=nocc, n_aux=nx,
                  basis_atom=basis_atom, aux_atom=aux_atom, R=R, eps=eps, evec=evec,
                  ctil_R=ctil, V=V, pmom=pm, omega_cell=float(p["omega_cell"]),
                  qhat=np.array([1.0, 0.0, 0.0]), n_freq=int(p["n_freq"]), omega0=omega0,
                  sigma_lo=int(lo), sigma_hi=int(hi), spin=2.0, head_wings=head_wings, seed=seed, trs=bool(trs))


def shifted_system(base, k_offset, seed, eps=None, evec=None, pmom=None):
    """The system `base` on the k mesh shifted by k_offset (fractional): the same atoms, basis,
    two-centre coefficients C~(R), Coulomb matrices V(q) (the q mesh is not shifted) and window,
    with KS energies, eigenvectors and momentum matrices at the shifted points k0 + i/n, drawn
    from `seed` by the recipe of make_system unless given. Sigma at an off-mesh point k0 is the
    Sigma of point 0 of this mesh (its k - q run over the shifted mesh)."""
    rng = np.random.default_rng(seed)
    NK, nb, nbands, nocc = base.n_k, base.n_basis, base.n_bands, base.n_occ
    if eps is None:
        eps = np.stack([np.concatenate([np.sort(rng.uniform(-0.8, -0.2, nocc)),
                                        np.sort(rng.uniform(0.05, 3.0, nbands - nocc))]) for _ in range(NK)])
    if evec is None:
        evec = np.stack([np.linalg.qr(_cgauss(rng, (nb, nb)))[0][:, :nbands] for _ in range(NK)])
    if pmom is None:
        g3 = _cgauss(rng, (NK, 3, nbands, nbands))
        pmom = 0.5 * (g3 + np.conj(np.swapaxes(g3, -1, -2))) / np.sqrt(2.0)
    return dataclasses.replace(base, eps=np.ascontiguousarray(eps), evec=np.ascontiguousarray(evec),
                               pmom=np.ascontiguousarray(pmom), trs=False,
                               k_offset=np.asarray(k_offset, dtype=np.float64), seed=seed)


def surrogate_init(n_in, n_hidden, n_out, seed=0, out_gain=0.01):
    """Seeded initial parameter vector of the frequency surrogate (fp32, the layout of
    gw_surrogate_create): weights N(0, 1/fan_in), the last layer scaled by out_gain so that
    the network starts close to its linear part, biases and L zero, output scale 1."""
    rng = np.random.default_rng(seed)
    H, I, O = n_hidden, n_in, n_out
    parts = [rng.standard_normal((H, I)) / np.sqrt(I), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             out_gain * rng.standard_normal((O, H)) / np.sqrt(H), np.zeros(O),
             np.zeros((O, I)), np.ones(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def surrogate_start(n_aux, n_block, seed=0):
    """Seeded complex Gaussian start block [n_aux][n_block] of the surrogate's subspace iteration."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_aux, n_block)) + 1j * rng.standard_normal((n_aux, n_block))
