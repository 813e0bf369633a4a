"""gw_plan_create and the surrogate calls reject malformed arguments with GW_ERR_ARG before touching the GPU.

Each case breaks one field of a problem that is otherwise valid up to its last check, and the
base problem also carries a decreasing aux_atom (the last check), so that no case can ever reach
a device allocation or a kernel launch with the placeholder device pointers used here, even on a
machine with a GPU. The error text names the check that fired."""
import ctypes

import pytest

from paper_2011_01400_gb300 import build as B
from paper_2011_01400_gb300 import gw

FAKE = 0x100000   # non-NULL placeholder for the device inputs; validation only tests for NULL


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gw.load()


def base():
    keep = []

    def arr(vals):
        a = (ctypes.c_int32 * len(vals))(*vals)
        keep.append(a)
        return ctypes.cast(a, ctypes.POINTER(ctypes.c_int32))

    p = gw.gw_problem()
    p.nk[:] = (2, 2, 1)
    p.n_atoms, p.n_basis, p.n_bands, p.n_occ, p.n_aux = 2, 6, 6, 2, 10
    p.basis_atom = arr([0, 0, 0, 1, 1, 1])
    p.aux_atom = arr([0, 0, 0, 0, 0, 1, 1, 1, 1, 0])      # decreasing at the end: the guard
    p.n_R = 7
    p.R = arr([0] * 21)
    p.eps = p.evec = p.ctil_R = p.V = FAKE
    p.pmom = None
    p.omega_cell, p.head_wings = 100.0, 0
    p.n_freq, p.omega0 = 8, 1.0
    p.sigma_lo, p.sigma_hi = 0, 4
    p.spin, p.mu = 2.0, float("nan")
    p.prec = gw.GW_3XBF16
    return p, keep


def create(lib, p):
    h = ctypes.c_void_p()
    st = lib.gw_plan_create(ctypes.byref(p), 1, None, ctypes.byref(h))
    assert not h.value
    return st, lib.gw_last_error().decode()


def test_guard_alone_is_rejected(lib):
    p, _keep = base()
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG and "aux_atom must be non-decreasing" in msg


CASES = [
    ("nk", lambda p: p.nk.__setitem__(2, 0), "nk out of range"),
    ("nk_big", lambda p: p.nk.__setitem__(0, 65), "nk out of range"),
    ("n_atoms", lambda p: setattr(p, "n_atoms", 0), "n_atoms out of range"),
    ("n_bands>n_basis", lambda p: setattr(p, "n_bands", 7), "bad n_basis / n_bands"),
    ("n_occ=n_bands", lambda p: setattr(p, "n_occ", 6), "n_occ must be in"),
    ("n_occ=0", lambda p: setattr(p, "n_occ", 0), "n_occ must be in"),
    ("n_aux", lambda p: setattr(p, "n_aux", 5000), "n_aux out of range"),
    ("basis_atom NULL", lambda p: setattr(p, "basis_atom", None), "basis_atom / aux_atom / R is NULL"),
    ("n_R", lambda p: setattr(p, "n_R", 0), "n_R out of range"),
    ("V NULL", lambda p: setattr(p, "V", None), "a device input pointer is NULL"),
    ("head_wings without pmom", lambda p: setattr(p, "head_wings", 1), "head_wings needs pmom"),
    ("qhat not a unit vector", lambda p: (setattr(p, "head_wings", 1), setattr(p, "pmom", FAKE),
                                          p.qhat.__setitem__(slice(0, 3), (0.5, 0.0, 0.0))), "unit vector qhat"),
    ("qhat zero", lambda p: (setattr(p, "head_wings", 1), setattr(p, "pmom", FAKE)), "unit vector qhat"),
    ("n_freq", lambda p: setattr(p, "n_freq", 0), "n_freq out of range"),
    ("omega0", lambda p: setattr(p, "omega0", 0.0), "omega0 must be > 0"),
    ("sigma window", lambda p: setattr(p, "sigma_hi", 7), "sigma window"),
    ("sigma empty", lambda p: setattr(p, "sigma_lo", 4), "sigma window"),
    ("spin", lambda p: setattr(p, "spin", 0.0), "spin must be > 0"),
    ("spin infinite", lambda p: setattr(p, "spin", float("inf")), "spin must be > 0"),
    ("omega0 infinite", lambda p: setattr(p, "omega0", float("inf")), "omega0 must be > 0"),
    ("mu infinite", lambda p: setattr(p, "mu", float("-inf")), "mu must be finite"),
    ("precision", lambda p: setattr(p, "prec", 9), "bad precision"),
]


@pytest.mark.parametrize("name,breakit,expect", CASES, ids=[c[0] for c in CASES])
def test_each_check_fires(lib, name, breakit, expect):
    p, _keep = base()
    breakit(p)
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG, (name, st, msg)
    assert expect in msg, (name, msg)


def test_atom_maps_are_checked(lib):
    p, keep = base()
    bad = (ctypes.c_int32 * 6)(0, 0, 1, 0, 1, 1)              # decreasing basis_atom
    keep.append(bad)
    p.basis_atom = ctypes.cast(bad, ctypes.POINTER(ctypes.c_int32))
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG and "basis_atom must be non-decreasing" in msg
    out = (ctypes.c_int32 * 6)(0, 0, 0, 1, 1, 2)              # atom index beyond n_atoms
    keep.append(out)
    p.basis_atom = ctypes.cast(out, ctypes.POINTER(ctypes.c_int32))
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG and "basis_atom out of range" in msg


def test_batch_count_is_checked(lib):
    p, _keep = base()
    h = ctypes.c_void_p()
    assert lib.gw_plan_create(ctypes.byref(p), 0, None, ctypes.byref(h)) == gw.GW_ERR_ARG
    assert lib.gw_plan_create(ctypes.byref(p), 5000, None, ctypes.byref(h)) == gw.GW_ERR_ARG
    assert "n_sys out of range" in lib.gw_last_error().decode()


@pytest.mark.parametrize("dims", [(12, 256, 48), (5, 40, 7), (1, 1, 1), (64, 4096, 1024)])
def test_surrogate_parameter_count_matches_the_layout(lib, dims):
    """The flat parameter vector of the network (W1 b1 W2 b2 W3 b3 W4 b4, then L and s) has the
    length the oracle's layout gives; the count needs no GPU."""
    from oracle import surrogate as S
    assert gw.gw_surrogate_param_count(*dims) == S.n_params(*dims)


@pytest.mark.parametrize("dims", [(0, 256, 48), (65, 256, 48), (12, 0, 48), (12, 4097, 48), (12, 256, 0),
                                  (12, 256, 1025)])
def test_surrogate_dims_are_checked(lib, dims):
    with pytest.raises(gw.GwError) as ei:
        gw.gw_surrogate_param_count(*dims)
    assert ei.value.status == gw.GW_ERR_ARG
    h = ctypes.c_void_p()
    d = gw.gw_surrogate_dims(*dims)
    assert lib.gw_surrogate_create(ctypes.byref(d), None, None, ctypes.byref(h)) == gw.GW_ERR_ARG
    assert not h.value


GRID_CASES = [
    ("freq without weights", [1.0, 2.0], None, "both or neither"),
    ("weights without freq", None, [1.0, 2.0], "both or neither"),
    ("zero frequency", [0.0, 2.0], [1.0, 1.0], "positive and finite"),
    ("negative weight", [1.0, 2.0], [1.0, -1.0], "positive and finite"),
    ("infinite frequency", [1.0, float("inf")], [1.0, 1.0], "positive and finite"),
    ("nan weight", [1.0, 2.0], [float("nan"), 1.0], "positive and finite"),
    ("repeated frequency", [2.0, 2.0], [1.0, 1.0], "freq must be distinct"),
]


@pytest.mark.parametrize("name,freq,wts,expect", GRID_CASES, ids=[c[0] for c in GRID_CASES])
def test_caller_grid_is_checked(lib, name, freq, wts, expect):
    p, keep = base()
    p.n_freq = 2

    def darr(vals):
        a = (ctypes.c_double * len(vals))(*vals)
        keep.append(a)
        return ctypes.cast(a, ctypes.POINTER(ctypes.c_double))

    if freq is not None:
        p.freq = darr(freq)
    if wts is not None:
        p.freq_w = darr(wts)
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG, (name, st, msg)
    assert expect in msg, (name, msg)


def test_caller_grid_replaces_omega0(lib):
    """With a grid given, omega0 is not read: a zero omega0 passes to the next check (the guard)."""
    p, keep = base()
    p.n_freq, p.omega0 = 2, 0.0
    f = (ctypes.c_double * 2)(0.5, 3.0)
    w = (ctypes.c_double * 2)(1.0, 4.0)
    keep += [f, w]
    p.freq = ctypes.cast(f, ctypes.POINTER(ctypes.c_double))
    p.freq_w = ctypes.cast(w, ctypes.POINTER(ctypes.c_double))
    st, msg = create(lib, p)
    assert st == gw.GW_ERR_ARG and "aux_atom must be non-decreasing" in msg
