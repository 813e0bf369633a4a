"""Thin Python binding of libgw (include/gw.h): argument marshalling only.

Every function here forwards to the C ABI entry of the same name. Device
memory and streams come from PyTorch; all arithmetic runs in the CUDA kernels
of libgw.so. There is no CPU path: loading fails loudly when the library is
missing.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgw.so")

GW_OK, GW_ERR_ARG, GW_ERR_NOMEM, GW_ERR_CUDA, GW_ERR_NOT_PD, GW_ERR_TIMEOUT, GW_ERR_STATE, GW_ERR_UNSUPPORTED = range(8)
GW_FP64, GW_3XTF32, GW_3XBF16, GW_3XFP16 = 0, 1, 2, 3
PREC = {"fp64": GW_FP64, "3xtf32": GW_3XTF32, "3xbf16": GW_3XBF16, "3xfp16": GW_3XFP16}

# every symbol include/gw.h declares
EXPORTS = ("gw_plan_create", "gw_plan_destroy", "gw_chi0", "gw_screen", "gw_sigma", "gw_sigma_ext", "gw_sigma_x", "gw_g0w0", "gw_g0w0_qset",
           "gw_g0w0_batch",
           "gw_plan_n_sys", "gw_qp",
           "gw_qp_static", "gw_plan_freq", "gw_plan_mu", "gw_plan_last_chi0_stats", "gw_plan_chi0_terms", "gw_kernel_launches",
           "gw_device_allocations",
           "gw_surrogate_param_count", "gw_surrogate_create", "gw_surrogate_destroy", "gw_surrogate_get_params",
           "gw_surrogate_set_params", "gw_surrogate_forward", "gw_surrogate_loss_grad", "gw_surrogate_fit_linear",
           "gw_surrogate_train", "gw_surrogate_enable", "gw_surrogate_modes", "gw_surrogate_data", "gw_surrogate_fit_moments",
           "gw_surrogate_fit_scale", "gw_problem_bytes", "gw_last_error")


class GwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gw status {status}: {msg}")
        self.status = status


class gw_surrogate_dims(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("n_out", ctypes.c_int32)]


class gw_surrogate_cfg(ctypes.Structure):
    _fields_ = [("n_coarse", ctypes.c_int32), ("coarse", ctypes.POINTER(ctypes.c_int32)),
                ("n_modes", ctypes.c_int32), ("n_block", ctypes.c_int32), ("n_iter", ctypes.c_int32),
                ("start", ctypes.c_void_p)]


class gw_problem(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int32 * 3),
        ("n_atoms", ctypes.c_int32), ("n_basis", ctypes.c_int32), ("n_bands", ctypes.c_int32),
        ("n_occ", ctypes.c_int32), ("n_aux", ctypes.c_int32),
        ("basis_atom", ctypes.POINTER(ctypes.c_int32)),
        ("aux_atom", ctypes.POINTER(ctypes.c_int32)),
        ("n_R", ctypes.c_int32),
        ("R", ctypes.POINTER(ctypes.c_int32)),
        ("eps", ctypes.c_void_p),
        ("evec", ctypes.c_void_p),
        ("ctil_R", ctypes.c_void_p),
        ("V", ctypes.c_void_p),
        ("pmom", ctypes.c_void_p),
        ("omega_cell", ctypes.c_double),
        ("qhat", ctypes.c_double * 3),
        ("head_wings", ctypes.c_int32),
        ("n_freq", ctypes.c_int32),
        ("omega0", ctypes.c_double),
        ("sigma_lo", ctypes.c_int32), ("sigma_hi", ctypes.c_int32),
        ("spin", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("prec", ctypes.c_int32),
        ("time_reversal", ctypes.c_int32),
        ("k_offset", ctypes.c_double * 3),
        ("freq", ctypes.POINTER(ctypes.c_double)),
        ("freq_w", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def load():
    """Load libgw.so (built in-tree by __graft_entry__.build()); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    lib.gw_plan_create.argtypes = [ctypes.POINTER(gw_problem), i32, vp, ctypes.POINTER(vp)]
    lib.gw_plan_destroy.argtypes = [vp]
    lib.gw_chi0.argtypes = [vp, i32, i32, vp]
    lib.gw_screen.argtypes = [vp, i32, i32, vp]
    lib.gw_sigma.argtypes = [vp, i32, i32, vp]
    lib.gw_sigma_ext.argtypes = [vp, i32, i32, vp, i32, i32, vp]
    lib.gw_g0w0.argtypes = [vp, i32, vp]
    lib.gw_g0w0_qset.argtypes = [vp, i32, ctypes.POINTER(i32), i32, vp]
    lib.gw_sigma_x.argtypes = [vp, i32, vp]
    lib.gw_g0w0_batch.argtypes = [vp, ctypes.POINTER(vp), i32]
    lib.gw_plan_n_sys.argtypes = [vp, ctypes.POINTER(i32)]
    lib.gw_qp.argtypes = [vp, i32, vp, vp, dp, dp, ctypes.POINTER(i32)]
    lib.gw_qp_static.argtypes = [vp, i32, vp, vp, dp, dp, ctypes.POINTER(i32)]
    lib.gw_plan_freq.argtypes = [vp, dp, dp]
    lib.gw_plan_mu.argtypes = [vp, dp]
    lib.gw_plan_last_chi0_stats.argtypes = [vp, dp, dp]
    lib.gw_plan_chi0_terms.argtypes = [vp, ctypes.POINTER(i32)]
    lib.gw_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.gw_device_allocations.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    i64, u64, dpp = ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)
    dimp = ctypes.POINTER(gw_surrogate_dims)
    lib.gw_surrogate_param_count.argtypes = [dimp, ctypes.POINTER(i64)]
    lib.gw_surrogate_create.argtypes = [dimp, vp, vp, ctypes.POINTER(vp)]
    lib.gw_surrogate_destroy.argtypes = [vp]
    lib.gw_surrogate_get_params.argtypes = [vp, vp]
    lib.gw_surrogate_set_params.argtypes = [vp, vp]
    lib.gw_surrogate_forward.argtypes = [vp, vp, i64, vp, vp]
    lib.gw_surrogate_loss_grad.argtypes = [vp, vp, vp, i64, dpp, vp]
    lib.gw_surrogate_fit_linear.argtypes = [vp, vp, vp, i64, ctypes.c_double, dpp]
    lib.gw_surrogate_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_double, u64, dpp]
    lib.gw_surrogate_enable.argtypes = [vp, vp, ctypes.POINTER(gw_surrogate_cfg)]
    lib.gw_surrogate_modes.argtypes = [vp, i32, i32, vp, vp, vp, vp]
    lib.gw_surrogate_data.argtypes = [vp, i32, vp, vp, vp]
    lib.gw_surrogate_fit_moments.argtypes = [vp, vp, ctypes.c_double]
    lib.gw_surrogate_fit_scale.argtypes = [vp, vp, vp, i64, dpp]
    lib.gw_last_error.argtypes = []
    lib.gw_last_error.restype = ctypes.c_char_p
    lib.gw_problem_bytes.argtypes = []
    lib.gw_problem_bytes.restype = ctypes.c_size_t
    for name in EXPORTS:
        if name not in ("gw_last_error", "gw_problem_bytes"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != GW_OK:
        raise GwError(status, load().gw_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------------------------
# ABI calls (same names as include/gw.h)
# ---------------------------------------------------------------------------------------------


def gw_plan_create(prob, n_sys=1, stream=None):
    """prob: a gw_problem, or a list of them (a batch plan with n_sys = len(list))."""
    import torch
    h = ctypes.c_void_p()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    if isinstance(prob, (list, tuple)):
        arr = (gw_problem * len(prob))(*prob)
        _check(load().gw_plan_create(arr, len(prob), ctypes.c_void_p(s), ctypes.byref(h)))
    else:
        _check(load().gw_plan_create(ctypes.byref(prob), n_sys, ctypes.c_void_p(s), ctypes.byref(h)))
    return h


def gw_g0w0_batch(plan, sigma_accs=None, n_threads=0):
    """sigma_accs: list of device tensors (or None entries) per system, or None."""
    arr = None
    if sigma_accs is not None:
        arr = (ctypes.c_void_p * len(sigma_accs))(*[None if t is None else t.data_ptr() for t in sigma_accs])
    _check(load().gw_g0w0_batch(plan, arr, int(n_threads)))


def gw_plan_n_sys(plan):
    n = ctypes.c_int32()
    _check(load().gw_plan_n_sys(plan, ctypes.byref(n)))
    return n.value


def gw_plan_destroy(plan):
    _check(load().gw_plan_destroy(plan))


def gw_chi0(plan, sys, q, chi0_out=None):
    _check(load().gw_chi0(plan, sys, q, _ptr(chi0_out)))


def gw_screen(plan, sys, q, wc_out=None):
    _check(load().gw_screen(plan, sys, q, _ptr(wc_out)))


def gw_sigma(plan, sys, q, sigma_acc=None):
    _check(load().gw_sigma(plan, sys, q, _ptr(sigma_acc)))


def gw_sigma_ext(plan, sys, q, wc, k_lo, k_hi, sigma_acc=None):
    _check(load().gw_sigma_ext(plan, sys, q, _ptr(wc), k_lo, k_hi, _ptr(sigma_acc)))


def gw_sigma_x(plan, sys, sigx):
    """sigx: device float64 tensor [N_k][n_sigma] (overwritten)."""
    _check(load().gw_sigma_x(plan, sys, _ptr(sigx)))


def gw_g0w0(plan, sys, sigma_acc=None):
    _check(load().gw_g0w0(plan, sys, _ptr(sigma_acc)))


def gw_g0w0_qset(plan, sys, q_list, sigma_acc):
    """q terms of the listed q points (host ints) accumulated into sigma_acc (device tensor)."""
    qs = np.ascontiguousarray(np.asarray(list(q_list), dtype=np.int32))
    _check(load().gw_g0w0_qset(plan, sys, qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(qs),
                               _ptr(sigma_acc)))


def gw_qp(plan, sys, n_k, n_sigma, sigma=None, dxv=None):
    e = np.zeros((n_k, n_sigma))
    gap = ctypes.c_double()
    nconv = ctypes.c_int32()
    _check(load().gw_qp(plan, sys, _ptr(sigma), _ptr(dxv),
                        e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(gap), ctypes.byref(nconv)))
    return e, gap.value, nconv.value


def gw_qp_static(plan, sys, n_k, n_sigma, sigma=None, dxv=None):
    """gw_qp with its device scratch in a fixed array of the library (no device allocation)."""
    e = np.zeros((n_k, n_sigma))
    gap = ctypes.c_double()
    nconv = ctypes.c_int32()
    _check(load().gw_qp_static(plan, sys, _ptr(sigma), _ptr(dxv),
                               e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(gap),
                               ctypes.byref(nconv)))
    return e, gap.value, nconv.value


def gw_plan_freq(plan, n_freq):
    f = np.zeros(n_freq)
    w = np.zeros(n_freq)
    _check(load().gw_plan_freq(plan, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return f, w


def gw_plan_mu(plan):
    m = ctypes.c_double()
    _check(load().gw_plan_mu(plan, ctypes.byref(m)))
    return m.value


def gw_kernel_launches():
    n = ctypes.c_uint64()
    _check(load().gw_kernel_launches(ctypes.byref(n)))
    return n.value


def gw_device_allocations():
    n = ctypes.c_uint64()
    _check(load().gw_device_allocations(ctypes.byref(n)))
    return n.value


def gw_plan_chi0_terms(plan):
    t = ctypes.c_int32()
    _check(load().gw_plan_chi0_terms(plan, ctypes.byref(t)))
    return t.value


def gw_plan_last_chi0_stats(plan):
    ms, fl = ctypes.c_double(), ctypes.c_double()
    _check(load().gw_plan_last_chi0_stats(plan, ctypes.byref(ms), ctypes.byref(fl)))
    return ms.value, fl.value


def _dims(n_in, n_hidden, n_out):
    return gw_surrogate_dims(int(n_in), int(n_hidden), int(n_out))


def gw_surrogate_param_count(n_in, n_hidden, n_out):
    c = ctypes.c_int64()
    _check(load().gw_surrogate_param_count(ctypes.byref(_dims(n_in, n_hidden, n_out)), ctypes.byref(c)))
    return c.value


def gw_surrogate_create(n_in, n_hidden, n_out, params, stream=None):
    """params: device float32 tensor [count]."""
    import torch
    h = ctypes.c_void_p()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    _check(load().gw_surrogate_create(ctypes.byref(_dims(n_in, n_hidden, n_out)), _ptr(params), ctypes.c_void_p(s),
                                      ctypes.byref(h)))
    return h


def gw_surrogate_destroy(model):
    _check(load().gw_surrogate_destroy(model))


def gw_surrogate_get_params(model, out):
    _check(load().gw_surrogate_get_params(model, _ptr(out)))
    return out


def gw_surrogate_set_params(model, params):
    _check(load().gw_surrogate_set_params(model, _ptr(params)))


def gw_surrogate_forward(model, x, f=None, g=None):
    _check(load().gw_surrogate_forward(model, _ptr(x), x.shape[0], _ptr(f), _ptr(g)))


def gw_surrogate_loss_grad(model, x, y, grad):
    loss = ctypes.c_double()
    _check(load().gw_surrogate_loss_grad(model, _ptr(x), _ptr(y), x.shape[0], ctypes.byref(loss), _ptr(grad)))
    return loss.value


def gw_surrogate_fit_linear(model, x, y, ridge):
    rms = ctypes.c_double()
    _check(load().gw_surrogate_fit_linear(model, _ptr(x), _ptr(y), x.shape[0], float(ridge), ctypes.byref(rms)))
    return rms.value


def gw_surrogate_train(model, x, y, epochs, batch, lr, seed):
    hist = np.zeros(max(int(epochs), 1))
    _check(load().gw_surrogate_train(model, _ptr(x), _ptr(y), x.shape[0], int(epochs), int(batch), float(lr),
                                     int(seed), hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return hist[:epochs]


def gw_surrogate_enable(plan, model, coarse=None, n_modes=0, n_block=0, n_iter=0, start=None):
    """coarse: host int list; start: device complex128 tensor [n_aux][n_block]. coarse None: detach."""
    if coarse is None:
        _check(load().gw_surrogate_enable(plan, model, None))
        return None
    c = np.ascontiguousarray(coarse, dtype=np.int32)
    cfg = gw_surrogate_cfg(len(c), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(n_modes), int(n_block),
                           int(n_iter), _ptr(start))
    _check(load().gw_surrogate_enable(plan, model, ctypes.byref(cfg)))
    return c


def gw_surrogate_modes(plan, sys, q, d_out=None, theta_out=None, x_out=None, y_out=None):
    _check(load().gw_surrogate_modes(plan, sys, q, _ptr(d_out), _ptr(theta_out), _ptr(x_out), _ptr(y_out)))


def gw_surrogate_data(plan, sys, x_out, y_out, moments=None):
    _check(load().gw_surrogate_data(plan, sys, _ptr(x_out), _ptr(y_out), _ptr(moments)))


def gw_surrogate_fit_moments(model, moments, ridge):
    _check(load().gw_surrogate_fit_moments(model, _ptr(moments), float(ridge)))


def gw_surrogate_fit_scale(model, x, y):
    rms = ctypes.c_double()
    _check(load().gw_surrogate_fit_scale(model, _ptr(x), _ptr(y), x.shape[0], ctypes.byref(rms)))
    return rms.value


# ---------------------------------------------------------------------------------------------
# marshalling of a seeded synthetic system into device tensors + a gw_problem
# ---------------------------------------------------------------------------------------------


class Problem:
    """Keeps the device tensors and host arrays that a gw_problem points to alive."""

    def __init__(self, system, prec="3xbf16", device="cuda", host=False, trs=None, mu=None, grid=None):
        import torch
        s = system
        self.system = s
        dev = torch.device(device)
        self.basis_atom = np.ascontiguousarray(s.basis_atom, dtype=np.int32)
        self.aux_atom = np.ascontiguousarray(s.aux_atom, dtype=np.int32)
        self.R = np.ascontiguousarray(s.R, dtype=np.int32)
        # host copies (pinned) for end-to-end timing; device copies for the ABI
        self.h = dict(eps=torch.from_numpy(np.ascontiguousarray(s.eps)),
                      evec=torch.from_numpy(np.ascontiguousarray(s.evec)),
                      ctil=torch.from_numpy(np.ascontiguousarray(s.ctil_flat())),
                      V=torch.from_numpy(np.ascontiguousarray(s.V)),
                      pmom=torch.from_numpy(np.ascontiguousarray(s.pmom)))
        if host:
            self.h = {k: v.pin_memory() for k, v in self.h.items()}
        self.d = {k: v.to(dev) for k, v in self.h.items()}
        p = gw_problem()
        p.nk[:] = list(s.nk)
        p.n_atoms, p.n_basis, p.n_bands, p.n_occ, p.n_aux = s.n_atoms, s.n_basis, s.n_bands, s.n_occ, s.n_aux
        p.basis_atom = self.basis_atom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.aux_atom = self.aux_atom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.n_R = self.R.shape[0]
        p.R = self.R.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.eps = self.d["eps"].data_ptr()
        p.evec = self.d["evec"].data_ptr()
        p.ctil_R = self.d["ctil"].data_ptr()
        p.V = self.d["V"].data_ptr()
        p.pmom = self.d["pmom"].data_ptr()
        p.omega_cell = s.omega_cell
        p.qhat[:] = list(s.qhat)
        p.head_wings = int(s.head_wings)
        p.n_freq = s.n_freq
        p.omega0 = s.omega0
        p.sigma_lo, p.sigma_hi = s.sigma_lo, s.sigma_hi
        p.spin = s.spin
        p.mu = math.nan if mu is None else float(mu)
        p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        # time-reversal symmetric inputs (the generator's default) let the q loop pair q with -q
        p.time_reversal = int(bool(getattr(s, "trs", False) if trs is None else trs))
        p.k_offset[:] = [float(x) for x in getattr(s, "k_offset", (0.0, 0.0, 0.0))]
        # a caller's imaginary-frequency grid (freq, weights); None keeps the default grid of omega0
        if grid is not None:
            self.freq = np.ascontiguousarray(grid[0], dtype=np.float64)
            self.freq_w = np.ascontiguousarray(grid[1], dtype=np.float64)
            if self.freq.shape != (s.n_freq,) or self.freq_w.shape != (s.n_freq,):
                raise ValueError("grid: freq and weights need n_freq entries each")
            p.freq = self.freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            p.freq_w = self.freq_w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.prob = p

    def upload(self):
        """Host -> device copy of every input (the end-to-end path)."""
        for k in self.d:
            self.d[k].copy_(self.h[k], non_blocking=True)

    def nbytes(self):
        return sum(v.numel() * v.element_size() for v in self.h.values())
