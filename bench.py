"""Benchmark of the periodic G0W0 hot path on one GB300 (or N independent replicas).

A step is one complete G0W0 pass over one synthetic system: plan (half-transformed
LRI coefficients, V(q)^1/2 for every q, the Coulomb head eigenvector), then for
every q: chi0 -> eps~ / W^c -> Sigma_c, then the continuation and QP solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config cfg1] [--prec 3xbf16]
  python bench.py --impl reference ...     (the FP64 CPU oracle on a bounded slice)

Prints one JSON line (rank 0). value = Sigma_c time-to-solution (s per system, whole job:
seconds per step / systems processed by all ranks), lower is better.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G0W0 Σc time-to-solution & χ0 TFLOP/s: split-prec vs FP64 on 1 GB300 @ ≤1 meV"
# DRAM bytes of one chi0 contraction launch (dram__bytes_read.sum, dram__bytes_write.sum), from an
# ncu capture of k_chi0 (3xFP16) on the cfg1 shape with a 4x4x4 k mesh (the third chi0 launch of a
# pass; its summary is kept with the other profiles). The reads stream the operand planes of every
# k and grow with the k count; the writes are the FP64 output rows, independent of it.
CHI0_DRAM_CAPTURE = dict(prec="3xfp16", n_k=64, n_aux=400, read=271.424512e6, write=39.426304e6)
WORKLOADS = {
    "cfg0": "tiny synthetic insulator: 2x2x2 k, 2 atoms, 32 NAO, 32 bands (4 occ), 96 ABF, 16 imaginary frequencies",
    "cfg1": "Si-like 2-atom fcc cell: 6x6x6 k (216 k, 216 q), 78 NAO, 78 bands (4 occ), 400 ABF, 32 imaginary "
            "frequencies, Sigma_c for the 8 bands at the gap",
    "cfg2": "ZnO-like 4-atom cell: 6x6x4 k (144 k, 144 q), 300 NAO, 300 bands (36 occ), 1600 ABF, 32 imaginary "
            "frequencies, Sigma_c for the 8 bands at the gap; M generated per chunk of k and never stored whole",
}


def q_computed(s):
    """q points whose chi0 / eps~ / W^c the pass computes: all of them, or one of each pair
    (q, -q) when the system is time-reversal symmetric (W^c(-q) = conj(W^c(q)))."""
    if not getattr(s, "trs", False):
        return s.n_k
    from paper_2011_01400_gb300.synth import minus_k
    return sum(1 for q in range(s.n_k) if minus_k(s.nk, q) >= q)


def algorithmic_flops(s):
    """Useful flops of one step (8 per complex multiply-add): chi0 Hermitian update, screen, Sigma_c."""
    NK, N, nw = s.n_k, s.n_aux, s.n_freq
    nocc, nun, nsig = s.n_occ, s.n_bands - s.n_occ, s.sigma_hi - s.sigma_lo
    nq = q_computed(s)
    chi0 = 8.0 * NK * nocc * nun * (N * (N + 1) / 2) * nw * nq
    screen = 4 * 8.0 * N ** 3 * nw * nq
    sigma = 8.0 * (NK * nsig * s.n_bands) * N * N * nw * NK
    return dict(chi0=chi0, screen=screen, sigma=sigma, total=chi0 + screen + sigma)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            bf16 = d.get("bf16_tflops_sustained") or d.get("bf16_tflops")
            hbm = d.get("hbm_gbs")
            if bf16:
                return float(bf16), float(hbm or 6800.0), "of measured"
        except Exception:
            pass
    return 1900.0, 6800.0, "of fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.idx = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(system, seconds_hint=20.0):
    """Time the FP64 oracle on bounded slices of the same workload; extrapolate by algorithmic flops.

    Slices: chi0 for q = 1 at 2 frequencies (all k); eps~/W^c for q = 1 at 2 frequencies;
    Sigma_c for q = 1 from 2 target k (all frequencies). Each slice is scaled by the ratio of
    its algorithmic flops to the full step's.
    """
    import numpy as np
    from oracle import gw_oracle as O

    s = system
    om, g = O.freq_grid(s.n_freq, s.omega0)
    mu = O.mu_midgap(s)
    fl = algorithmic_flops(s)
    iq = 1 % s.n_k
    # chi0 = M generation for every k (once per q) + one weighted product per frequency
    occ, unocc = np.arange(s.n_occ), np.arange(s.n_occ, s.n_bands)
    t0 = time.perf_counter()
    Ms = [O.mo_triple(s, ik, iq, unocc, occ).reshape(s.n_aux, -1) for ik in range(s.n_k)]
    t_m = time.perf_counter() - t0
    t0 = time.perf_counter()
    c = O.chi0(s, iq, om[:2]) if s.n_k <= 8 else None
    if c is None:
        c = np.zeros((2, s.n_aux, s.n_aux), dtype=np.complex128)
        for ik in range(s.n_k):
            ikq = O.k_plus(s.nk, ik, iq)
            D = (s.eps[ikq][unocc][:, None] - s.eps[ik][occ][None, :]).ravel()
            for w_i, w in enumerate(om[:2]):
                c[w_i] += (Ms[ik] * (2.0 * D / (w * w + D * D))[None, :]) @ np.conj(Ms[ik]).T
        c *= -(s.spin / s.n_k)
    t_h = time.perf_counter() - t0
    t_chi = t_m + t_h
    t0 = time.perf_counter()
    e, W = O.screen(s, iq, c, om[:2])
    t_scr = time.perf_counter() - t0
    # Sigma slice: two target k, all w' (needs W^c at every frequency: use the slice's W^c repeated)
    Wfull = np.repeat(W[:1], s.n_freq, axis=0)
    t0 = time.perf_counter()
    nk_s = min(2, s.n_k)
    for ik in range(nk_s):
        ikmq = O.k_minus(s.nk, ik, iq)
        M = O.mo_triple(s, ikmq, iq, np.arange(s.sigma_lo, s.sigma_hi), np.arange(s.n_bands))
        Mf = M.reshape(s.n_aux, -1)
        for j in range(s.n_freq):
            _ = np.sum(Mf * (Wfull[j] @ np.conj(Mf)), axis=0)
    t_sig = time.perf_counter() - t0
    NK, nw = s.n_k, s.n_freq
    est = NK * (t_m + t_h * nw / 2.0) + t_scr * (NK * nw / 2.0) + t_sig * (NK * NK / nk_s)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(value=est, unit="s", cores=cores, kind="oracle",
                sample=f"FP64 NumPy oracle, extrapolated: M for q=1 (all {NK} k) {t_m:.2f} s + chi0 products "
                       f"x 2 w {t_h:.2f} s, "
                       f"screen q=1 x 2 w {t_scr:.2f} s, Sigma_c q=1 x {nk_s} k x {nw} w' {t_sig:.2f} s; "
                       f"scaled to {NK} q x {nw} w and {NK} k",
                slice_seconds=t_chi + t_scr + t_sig)


def max_over_ranks(vals, world, device="cpu"):
    """Each value's maximum over the ranks of the process group (any backend: NCCL with
    device="cuda", gloo with "cpu"); the values themselves for a single process."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t = t.cpu()
    return [float(x) for x in t]


def seconds_per_system(ms_per_step_max, world, parallel="replicas"):
    """Whole-job value. Replicas: every rank processes one system per step, so the job finishes
    `world` systems in the slowest rank's step time. q-parallel: the ranks share one system per
    step, which is done when the slowest rank is."""
    return ms_per_step_max / 1e3 / (world if parallel == "replicas" else 1)


def replica_seed(config, rank, parallel="replicas"):
    """Seed of the system a rank processes: the configuration's seed, offset by the rank for
    replicas (different systems); the same system on every rank of a q-parallel run."""
    return 1000 * int(config[-1]) + (rank if parallel == "replicas" else 0)


def run_reference(args, system, world, rank):
    if rank != 0:
        return
    samples = []
    for _ in range(args.warmup):
        oracle_sample(system)
    for _ in range(args.steps):
        samples.append(oracle_sample(system))
    v = statistics.median([x["value"] for x in samples])
    cb = dict(samples[-1])
    cb["value"] = v
    line = dict(metric=METRIC, value=v, unit="s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=statistics.median([x["slice_seconds"] for x in samples]) * 1e3,
                higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=WORKLOADS[args.config], name=args.config, global_batch=1, seq_len=0,
                            parallelism="single"),
                cpu_baseline=cb, e2e=dict(value=v, unit="s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def g0w0_step(gw, plan_prob, s, torch, chi_ms, qloop="g0w0", qshard=False):
    """One complete pass: plan, the q loop (one native call, per-q calls, or this rank's part of
    the q mesh followed by the sum of Sigma_c over the ranks), QP. Returns (e_qp, gap)."""
    plan = gw.gw_plan_create(plan_prob)
    try:
        if qshard:
            from paper_2011_01400_gb300 import shard
            _, e, gap = shard.g0w0_sharded(gw, plan, 0, s)
            chi_ms.append(gw.gw_plan_last_chi0_stats(plan))
            return e, gap
        if qloop == "g0w0":
            gw.gw_g0w0(plan, 0)
            chi_ms.append(gw.gw_plan_last_chi0_stats(plan))
        else:
            tot = [0.0, 0.0]
            for q in range(s.n_k):
                gw.gw_chi0(plan, 0, q)
                ms, fl = gw.gw_plan_last_chi0_stats(plan)
                tot[0] += ms
                tot[1] += fl
                gw.gw_screen(plan, 0, q)
                gw.gw_sigma(plan, 0, q)
            chi_ms.append(tuple(tot))
        e, gap, nconv = gw.gw_qp(plan, 0, s.n_k, s.sigma_hi - s.sigma_lo)
    finally:
        gw.gw_plan_destroy(plan)
    return e, gap


def timed_pass(gw, s, prec, torch, warm=1, qs=None, sigma=False):
    """One G0W0 pass of system s at precision prec (plan, the q loop, QP), CUDA-event timed on the
    current stream after `warm` untimed passes. qs: only these q points (gw_g0w0_qset, no QP).
    Returns (seconds, e_qp, gap, (chi0 ms, chi0 flops)), and Sigma_c [N_k][n_sigma][n_freq] as a
    fifth item when sigma is set (accumulated into a caller tensor, which the QP solve then reads)."""
    pb = gw.Problem(s, prec)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    nsig = s.sigma_hi - s.sigma_lo
    out = None
    for i in range(warm + 1):
        acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda") if sigma else None
        torch.cuda.synchronize()
        ev[0].record(stream)
        plan = gw.gw_plan_create(pb.prob)
        try:
            if qs is None:
                gw.gw_g0w0(plan, 0, acc)
                e, gap, _ = gw.gw_qp(plan, 0, s.n_k, nsig, sigma=acc)
            else:
                acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
                gw.gw_g0w0_qset(plan, 0, qs, acc)
                e, gap = None, None
            chi = gw.gw_plan_last_chi0_stats(plan)
        finally:
            gw.gw_plan_destroy(plan)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out = (ev[0].elapsed_time(ev[1]) / 1e3, e, gap, chi)
    return out + (acc,) if sigma else out


def fp64_gemm_peak(torch, n=4096, reps=5):
    """Measured FP64 rate of this GPU: the best of `reps` CUDA-event-timed cuBLAS DGEMMs
    (torch.matmul, n^3, 2 n^3 flops) after one warm-up. It is the denominator of the FP64
    Cholesky-inverse's roofline fraction (that kernel runs on the same FP64 units)."""
    a = torch.randn((n, n), dtype=torch.float64, device="cuda")
    b = torch.randn((n, n), dtype=torch.float64, device="cuda")
    c = torch.matmul(a, b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        ev[0].record()
        c = torch.matmul(a, b)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        best = t if best is None else min(best, t)
    del a, b, c
    return 2.0 * n ** 3 / best / 1e12


def chi0_frac(prec, chi, s, T_rows, peak_bf16):
    """chi0 TFLOP/s (algorithmic), its fraction of the dense peak of the precision's operand type
    and the tensor-issued fraction (split products, compressed weight rows)."""
    ms, fl = chi
    a = fl / (ms * 1e-3) / 1e12
    peak = peak_bf16 * (0.5 if prec == "3xtf32" else 1.0)
    products = {"3xfp16": 3, "3xbf16": 6, "3xtf32": 3}[prec]
    return dict(chi0_tflops=a, frac=a / peak, tensor_issued_frac=a * products * T_rows / s.n_freq / peak)


def q_slice_ms(gw, s, prec, torch, q=1, reps=2):
    """Device time (ms, CUDA events) of plan creation and of chi0 -> screen -> Sigma_c for one q."""
    stream = torch.cuda.current_stream()
    pb = gw.Problem(s, prec)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    plan = gw.gw_plan_create(pb.prob)
    ev[1].record(stream)
    torch.cuda.synchronize()
    plan_ms = ev[0].elapsed_time(ev[1])
    try:
        q = q % s.n_k
        best = None
        for _ in range(reps):
            ev[0].record(stream)
            gw.gw_chi0(plan, 0, q)
            gw.gw_screen(plan, 0, q)
            gw.gw_sigma(plan, 0, q)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t = ev[0].elapsed_time(ev[1])
            best = t if best is None else min(best, t)
    finally:
        gw.gw_plan_destroy(plan)
    return plan_ms, best


def surrogate_bench(args, gw, torch):
    """Learned frequency surrogate on a 60-point grid with chi0 on 12 frequencies (every 5th,
    the lowest included): training data from the plain method on seeded systems with the
    workload's band/ABF shapes and a 2x2x2 k mesh; the linear map from the frequency moments of
    eps~^-1 - 1 (ridge), the MLP by Adam on the mode rows, all on the GPU; then the whole
    pass on the workload's k mesh against the full-grid plain pass (same precision)."""
    from paper_2011_01400_gb300.synth import make_system, surrogate_init, surrogate_start
    NW, k, nb, nit = 60, 32, 48, 8
    coarse = list(range(0, NW, 5))
    nc, nf = len(coarse), NW - len(coarse)
    dims = (nc, 256, nf)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(stream)
        out = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return out, ev[0].elapsed_time(ev[1]) / 1e3

    base = make_system(args.config, seed=0, n_freq=NW, nk=(2, 2, 2))
    start = torch.from_numpy(surrogate_start(base.n_aux, nb, seed=9)).cuda()

    mom = torch.zeros((nc, NW), dtype=torch.float64, device="cuda")

    def features(sysm):
        pb = gw.Problem(sysm, args.prec)
        plan = gw.gw_plan_create(pb.prob)
        x = torch.empty((sysm.n_k * k, nc), device="cuda")
        y = torch.empty((sysm.n_k * k, nf), device="cuda")
        try:
            gw.gw_surrogate_enable(plan, None, coarse, k, nb, nit, start)
            gw.gw_surrogate_data(plan, 0, x, y, mom)
        finally:
            gw.gw_plan_destroy(plan)
        return x, y

    def data():
        X, Y = zip(*[features(make_system(args.config, seed=50000 + i, n_freq=NW, nk=(2, 2, 2)))
                     for i in range(args.sur_systems)])
        return torch.cat(X).contiguous(), torch.cat(Y).contiguous()

    (X, Y), t_data = timed(data)
    model = gw.gw_surrogate_create(*dims, torch.from_numpy(surrogate_init(*dims, seed=3)).cuda())
    try:
        def train():
            gw.gw_surrogate_fit_moments(model, mom, 1e-10)
            r = gw.gw_surrogate_fit_scale(model, X, Y)
            h = gw.gw_surrogate_train(model, X, Y, args.sur_epochs, 256, 1e-3, 17)
            return r, h
        (rms, hist), t_train = timed(train)
        ev_sys = make_system(args.config, seed=1000 * int(args.config[-1]) + 1, n_freq=NW)
        pb = gw.Problem(ev_sys, args.prec)
        nsig = ev_sys.sigma_hi - ev_sys.sigma_lo

        def full_pass():
            plan = gw.gw_plan_create(pb.prob)
            try:
                gw.gw_g0w0(plan, 0)
                return gw.gw_qp(plan, 0, ev_sys.n_k, nsig)
            finally:
                gw.gw_plan_destroy(plan)

        def sur_pass():
            plan = gw.gw_plan_create(pb.prob)
            try:
                gw.gw_surrogate_enable(plan, model, coarse, k, nb, nit, start)
                gw.gw_g0w0(plan, 0)
                return gw.gw_qp(plan, 0, ev_sys.n_k, nsig)
            finally:
                gw.gw_plan_destroy(plan)

        sur_pass()  # warm-up (group buffers, module loading)
        (e_s, gap_s, _), t_sur = timed(sur_pass)
        (e_f, gap_f, _), t_full = timed(full_pass)
        # the linear map alone: the network's output scale s (the last parameter) set to 0
        nparam = gw.gw_surrogate_param_count(*dims)
        theta = gw.gw_surrogate_get_params(model, torch.empty(nparam, device="cuda"))
        th0 = theta.clone()
        th0[-1] = 0.0
        gw.gw_surrogate_set_params(model, th0)
        e_l, gap_l, _ = sur_pass()
        gw.gw_surrogate_set_params(model, theta)
        # the plain method on the 12 coarse points alone (their own Gauss-Legendre grid: the
        # chi0 / eps~ work of the surrogate pass without the reconstruction)
        sys12 = make_system(args.config, seed=1000 * int(args.config[-1]) + 1, n_freq=nc)
        pb12 = gw.Problem(sys12, args.prec)
        plan12 = gw.gw_plan_create(pb12.prob)
        try:
            gw.gw_g0w0(plan12, 0)
            e_12, gap_12, _ = gw.gw_qp(plan12, 0, sys12.n_k, nsig)
        finally:
            gw.gw_plan_destroy(plan12)
    finally:
        gw.gw_surrogate_destroy(model)
    ha = 27211.386
    return dict(workload=f"{WORKLOADS[args.config]}, on a 60-point grid; chi0 / eps~ on 12 of them",
                precision=args.prec, train_systems=args.sur_systems, train_rows=int(X.shape[0]),
                train_data_s=t_data, train_s=t_train, epochs=args.sur_epochs,
                linear_rms=rms, loss_first=float(hist[0]) if len(hist) else None,
                loss_last=float(hist[-1]) if len(hist) else None,
                surrogate_step_s=t_sur, full_grid_step_s=t_full, speedup=t_full / t_sur,
                max_abs_dE_qp_meV=float(abs(e_s - e_f).max() * ha), abs_dgap_meV=float(abs(gap_s - gap_f) * ha),
                linear_only=dict(max_abs_dE_qp_meV=float(abs(e_l - e_f).max() * ha),
                                 abs_dgap_meV=float(abs(gap_l - gap_f) * ha)),
                plain_12_point_grid=dict(max_abs_dE_qp_meV=float(abs(e_12 - e_f).max() * ha),
                                         abs_dgap_meV=float(abs(gap_12 - gap_f) * ha)),
                error_reference="the plain method on the full 60-point grid, same precision, same system")


def batch_systems(n, seed0=30000):
    """Seeded systems of uneven size for the batch measurement: 2 atoms, bands 20-80 (n_occ 4-8),
    ABFs 60-200 per atom, k mesh 2x2x2 / 3x3x3 / 4x4x4, 16-32 frequencies, Sigma_c for the
    4 bands at the gap."""
    import numpy as np
    from paper_2011_01400_gb300.synth import make_system
    out = []
    for i in range(n):
        r = np.random.default_rng(seed0 + i)
        nb = int(r.integers(10, 41)) * 2
        nocc = int(r.integers(4, 9))
        nx = int(r.integers(60, 201))
        nkm = [(2, 2, 2), (3, 3, 3), (4, 4, 4)][int(r.integers(0, 3))]
        nw = int(r.integers(16, 33))
        cfg = dict(nk=nkm, n_atoms=2, nb_per_atom=nb // 2, naux_per_atom=nx, n_bands=nb, n_occ=nocc,
                   n_freq=nw, sigma=(nocc - 2, nocc + 2), omega_cell=270.25)
        out.append(make_system(cfg, seed=seed0 + i))
    return out


def batch_bench(args, gw, torch):
    """Many independent systems of uneven size in one batch plan: gw_g0w0_batch with the q loops
    of the systems running concurrently, against the same systems one after another, and the
    split-precision QP gaps against the FP64 GPU path on the 4 smallest systems."""
    ss = batch_systems(args.batch)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def run(prec, systems, threads):
        pbs = [gw.Problem(s, prec) for s in systems]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = gw.gw_plan_create([pb.prob for pb in pbs])
        torch.cuda.synchronize()
        t_plan = time.perf_counter() - t0
        try:
            gw.gw_g0w0_batch(plan, None, threads)   # warm-up (group buffers)
            torch.cuda.synchronize()
            ev[0].record(stream)
            gw.gw_g0w0_batch(plan, None, threads)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t = ev[0].elapsed_time(ev[1]) / 1e3
            gaps = [gw.gw_qp(plan, i, s.n_k, s.sigma_hi - s.sigma_lo)[1] for i, s in enumerate(systems)]
        finally:
            gw.gw_plan_destroy(plan)
        return t, t_plan, gaps

    t_conc, t_plan, gaps = run(args.prec, ss, 8)
    t_seq, _, _ = run(args.prec, ss, 1)
    sub = sorted(ss, key=lambda x: algorithmic_flops(x)["total"])[:4]   # the FP64 path is slow: smallest 4
    _, _, gaps64 = run("fp64", sub, 8)
    _, _, gaps_sub = run(args.prec, sub, 8)
    fl = sum(algorithmic_flops(s)["total"] for s in ss)
    ha = 27211.386
    dg = [abs(a - b) * ha for a, b in zip(gaps_sub, gaps64) if a == a and b == b]
    return dict(workload=f"{len(ss)} seeded systems: 2 atoms, 20-80 bands (4-8 occupied), 120-400 ABF, "
                         f"k mesh 2^3/3^3/4^3, 16-32 frequencies",
                precision=args.prec, systems=len(ss), plan_create_s=t_plan,
                concurrent_s=t_conc, sequential_s=t_seq, concurrency_speedup=t_seq / t_conc,
                aggregate_useful_tflops=fl / t_conc / 1e12, threads=8,
                max_abs_dgap_vs_fp64_meV=max(dg) if dg else None, fp64_checked_systems=len(sub),
                note="q loops of the systems run concurrently on their own streams (host thread pool); "
                     "the time covers the whole G0W0 pass of every system, plans built beforehand")


def run_slice(args, gw, torch, s, world, rank):
    """Large workloads (cfg2): a whole pass takes tens of minutes, so a step is a labelled bounded
    slice: plan creation plus the complete q loop (chi0 over all k and frequencies, eps~ / W^c,
    Sigma_c) of `--qslice` q points through gw_g0w0_qset. value extrapolates the pass as plan +
    N_q x (slice time per q); the slice itself is reported as measured."""
    qs = list(range(1, 1 + args.qslice))
    pb = gw.Problem(s, args.prec)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    nsig = s.sigma_hi - s.sigma_lo
    res = []
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    l0 = None
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            clocks.start()
            l0 = gw.gw_kernel_launches()
        torch.cuda.synchronize()
        ev[0].record(stream)
        plan = gw.gw_plan_create(pb.prob)
        ev[1].record(stream)
        try:
            acc = torch.zeros((s.n_k, nsig, s.n_freq), dtype=torch.complex128, device="cuda")
            ev[2].record(stream)
            gw.gw_g0w0_qset(plan, 0, qs, acc)
            ev[3].record(stream)
            chi = gw.gw_plan_last_chi0_stats(plan)
            T_rows = gw.gw_plan_chi0_terms(plan) or s.n_freq
        finally:
            gw.gw_plan_destroy(plan)
        torch.cuda.synchronize()
        if i >= args.warmup:
            res.append((ev[0].elapsed_time(ev[1]) / 1e3, ev[2].elapsed_time(ev[3]) / 1e3, chi))
    ck = clocks.stop()
    launches = gw.gw_kernel_launches() - l0
    if rank != 0:
        return
    plan_s = statistics.median(r[0] for r in res)
    slice_s = statistics.median(r[1] for r in res)
    chi = res[-1][2]
    peak_bf16, _, peak_kind = load_peaks()
    fr = chi0_frac(args.prec, chi, s, T_rows, peak_bf16)
    peak = peak_bf16 * (0.5 if args.prec == "3xtf32" else 1.0)
    est = plan_s + s.n_k * slice_s / len(qs)
    line = dict(metric=METRIC, value=est, unit="s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=(plan_s + slice_s) * 1e3, higher_is_better=False, scaling="weak", vs_baseline=None,
                dtype={"3xfp16": "fp16x2-split/f32-acc/f64", "3xbf16": "bf16x3-split/f32-acc/f64",
                       "3xtf32": "tf32x2-split/f32-acc/f64", "fp64": "f64"}[args.prec],
                data="synthetic",
                config=dict(workload=WORKLOADS[args.config], name=args.config, precision=args.prec,
                            slice=f"plan + the q loop of q = {qs} (all k, all {s.n_freq} frequencies); value = "
                                  f"plan + {s.n_k} x slice per q (extrapolated, labelled)",
                            global_batch=1, seq_len=0, parallelism="single",
                            l2="inputs larger than L2 (chi0 operand plane 7 GB per q)"),
                value_kind="extrapolated from the measured slice", plan_s=plan_s, slice_s=slice_s,
                slice_q=len(qs), chi0_tflops=fr["chi0_tflops"],
                roofline=dict(bound="tensor", achieved=fr["chi0_tflops"], peak=peak, unit="TFLOP/s",
                              frac=fr["frac"], traffic=None, kernel="k_chi0",
                              tensor_issued_frac=fr["tensor_issued_frac"], chi0_weight_rows=T_rows,
                              peak_note=f"dense peak of the operand type, {peak_kind}"),
                e2e=None, gpu_launches=launches, clocks=ck)
    print(json.dumps(line), flush=True)


def run_device(args, system, world, rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as ge
    ge.build()
    from paper_2011_01400_gb300 import gw

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    s = system
    if args.config == "cfg2":
        return run_slice(args, gw, torch, s, world, rank)
    pb = gw.Problem(s, args.prec, host=True)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    qshard = world > 1 and args.parallel == "qshard"
    mode = "qshard" if qshard else "replicas"
    chi_ms = []
    for _ in range(args.warmup):
        g0w0_step(gw, pb.prob, s, torch, chi_ms, args.qloop, qshard)
    torch.cuda.synchronize()
    # device-resident timed region
    chi_ms.clear()
    clocks = Clocks(dev)
    l0 = gw.gw_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        e, gap = g0w0_step(gw, pb.prob, s, torch, chi_ms, args.qloop, qshard)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    launches = gw.gw_kernel_launches() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    # end to end: host inputs copied in every step, QP energies read back
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    chi_e2e = []
    ms_e2e = float("nan")
    if not args.no_e2e:
        e0.record(stream)
        for _ in range(args.steps):
            pb.upload()
            e_qp, gap = g0w0_step(gw, pb.prob, s, torch, chi_e2e, args.qloop, qshard)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = e0.elapsed_time(e1) / args.steps
    # matched-accuracy comparison with the plain FP64 method on the GPU: one q slice each
    fp64 = None
    if not args.no_fp64_slice:
        p64, q64 = q_slice_ms(gw, s, "fp64", torch)
        psp, qsp = q_slice_ms(gw, s, args.prec, torch)
        fp64 = dict(q_slice="q = 1: chi0 -> eps~/W^c -> Sigma_c through the per-q C ABI calls (best of 2)",
                    fp64_plan_ms=p64, fp64_q_ms=q64, split_plan_ms=psp, split_q_ms=qsp,
                    speedup_q=q64 / qsp,
                    fp64_step_s_extrapolated=(p64 + s.n_k * q64) / 1e3,
                    speedup_step_extrapolated=(p64 + s.n_k * q64) / ms)
    ms, ms_e2e = max_over_ranks([ms, ms_e2e], world, "cuda")
    if rank != 0:
        return
    fl = algorithmic_flops(s)
    chi_avg_ms = sum(x[0] for x in chi_ms) / len(chi_ms)       # chi0 launches of one step (all q)
    chi_flops = chi_ms[0][1]
    plan_t = gw.gw_plan_create(pb.prob)     # weight rows of the compressed chi0 (same for every q here)
    try:
        gw.gw_chi0(plan_t, 0, 1 % s.n_k)
        T_rows = gw.gw_plan_chi0_terms(plan_t) or s.n_freq
    finally:
        gw.gw_plan_destroy(plan_t)
    peak_bf16, peak_hbm, peak_kind = load_peaks()
    tf32 = args.prec == "3xtf32"
    peak = peak_bf16 * (0.5 if tf32 else 1.0) if args.prec != "fp64" else 1.25
    achieved = chi_flops / (chi_avg_ms * 1e-3) / 1e12
    products = {"3xfp16": 3, "3xbf16": 6, "3xtf32": 3, "fp64": 1}[args.prec]
    cap = CHI0_DRAM_CAPTURE
    traffic = None
    if cap is not None and args.prec == cap["prec"] and s.n_aux == cap["n_aux"]:
        traffic = cap["read"] * s.n_k / cap["n_k"] + cap["write"]
    line = dict(
        metric=METRIC,
        value=seconds_per_system(ms, world, mode),
        unit="s",
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=False, scaling="strong" if qshard else "weak", vs_baseline=None,
        dtype={"3xfp16": "fp16x2-split/f32-acc/f64", "3xbf16": "bf16x3-split/f32-acc/f64",
               "3xtf32": "tf32x2-split/f32-acc/f64", "fp64": "f64"}[args.prec],
        data="synthetic",
        config=dict(workload=WORKLOADS[args.config] + (f" (k mesh overridden to {args.nk})" if args.nk else ""),
                    name=args.config, precision=args.prec, systems_per_step=1 if qshard else world,
                    q_loop="q-parallel (gw_g0w0_qset, pairs {q, -q} kept on one rank, + Sigma_c sum over ranks)" if qshard else args.qloop,
                    global_batch=1 if qshard else world, seq_len=0, parallelism=mode if world > 1 else "single",
                    time_reversal=bool(getattr(s, "trs", False)),
                    q0={0: "regular formula", 1: "head and wings along x", 2: "head and wings averaged over the "
                        "direction of q -> 0 (128-point sphere rule)"}[s.head_wings],
                    q_chi0_computed=f"{q_computed(s)} of {s.n_k} (W^c(-q) = conj(W^c(q)) for the pairs)"
                    if getattr(s, "trs", False) else f"{s.n_k} of {s.n_k}",
                    l2="inputs larger than L2 (chi0 operand planes 0.4-0.6 GB per q, by split)"),
        chi0_tflops=achieved,
        step_useful_tflops=fl["total"] / (ms * 1e-3) / 1e12,
        roofline=dict(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                      traffic=traffic, kernel="k_chi0 (tcgen05 weighted Hermitian update, Re/Im rows stacked on M)",
                      traffic_note=None if traffic is None else
                      f"DRAM bytes per launch (one q), scaled from an ncu capture on {cap['n_k']} k: "
                      f"reads x {s.n_k}/{cap['n_k']}, writes as captured",
                      peak_note=f"{'TF32' if tf32 else ('FP16' if args.prec == '3xfp16' else 'BF16')} dense "
                                f"{peak_kind} (FP16 and BF16 share the rate); achieved counts algorithmic "
                                f"flops (8 per complex MAC, lower triangle, all {s.n_freq} frequencies); the "
                                f"kernel runs {T_rows} compressed weight rows instead of {s.n_freq} frequencies and "
                                f"x{products} split products: tensor-issued = achieved x {products} x "
                                f"{T_rows}/{s.n_freq}",
                      chi0_weight_rows=T_rows,
                      tensor_issued_frac=achieved * products * T_rows / s.n_freq / peak),
        e2e=None if args.no_e2e else dict(value=seconds_per_system(ms_e2e, world, mode), unit="s", h2d_bytes_per_step=pb.nbytes(),
                                          d2h_bytes_per_step=s.n_k * (s.sigma_hi - s.sigma_lo) * 8 + 8),
        gpu_launches=launches,
        clocks=ck,
        fp64_gpu=fp64,
        gap_ha=gap,
    )
    ha = 27211.386
    if world == 1 and not args.no_extras and args.prec != "fp64":
        # the other split precisions on the same system: one timed pass each after one warm-up
        others = {}
        for p in ("3xfp16", "3xbf16", "3xtf32"):
            if p == args.prec:
                continue
            t, e_p, gap_p, chi = timed_pass(gw, s, p, torch)
            others[p] = dict(step_s=t, **chi0_frac(p, chi, s, T_rows, peak_bf16),
                             max_abs_dE_qp_meV_vs_main=float(abs(e_p - e).max() * ha),
                             abs_dgap_meV_vs_main=float(abs(gap_p - gap) * ha))
        line["other_precisions"] = others
        # like for like at matched accuracy: the whole pass in FP64 and split precision on the
        # workload's band / ABF / frequency shape with a 3x3x3 k mesh
        from paper_2011_01400_gb300.synth import make_system
        s3 = make_system(args.config, seed=replica_seed(args.config, 0), nk=(3, 3, 3), head_wings=args.head_wings)
        t64, e64, g64, _, sig64 = timed_pass(gw, s3, "fp64", torch, warm=0, sigma=True)
        fp64_pass = dict(system=f"{args.config} shape on a 3x3x3 k mesh (27 k, 27 q), seed "
                                f"{replica_seed(args.config, 0)}; plan + gw_g0w0 + gw_qp, CUDA events",
                         fp64_s=t64)
        for p in ("3xfp16", "3xbf16", "3xtf32"):
            tp, ep, gp, _, sigp = timed_pass(gw, s3, p, torch, sigma=True)
            de = abs(ep - e64)
            kn = np.unravel_index(int(de.argmax()), de.shape)
            fp64_pass[p] = dict(step_s=tp, speedup=t64 / tp, max_abs_dE_qp_meV=float(de.max() * ha),
                                abs_dgap_meV=float(abs(gp - g64) * ha),
                                max_abs_dsigma_c_meV=float((sigp - sig64).abs().max()) * ha,
                                dE_qp_argmax_k_band=[int(kn[0]), int(kn[1]) + s3.sigma_lo])
        line["fp64_pass"] = fp64_pass
    if world == 1 and not args.no_extras:
        # the FP64 Cholesky-inverse of eps~: its share of the step and its FP64 rate against a
        # measured FP64 GEMM (4 N^3 flops per (q, w) matrix: N^3 / 2 complex multiply-adds)
        peak64 = fp64_gemm_peak(torch)
        nq = q_computed(s)
        chol_flops = 4.0 * s.n_aux ** 3 * s.n_freq * nq
        line["fp64_peak"] = dict(dgemm_tflops=peak64, method="cuBLAS DGEMM via torch.matmul, 4096^3, best of 5, "
                                                           "CUDA events", cholesky_flops_per_step=chol_flops)
    # the learned surrogate and the batch of uneven systems: part of the default N = 1 line
    if args.surrogate or (world == 1 and not args.no_extras):
        line["surrogate"] = surrogate_bench(args, gw, torch)
    if args.batch or (world == 1 and not args.no_extras):
        if not args.batch:
            args.batch = 64
        line["batch"] = batch_bench(args, gw, torch)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(s)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="cfg1", choices=list(WORKLOADS))
    ap.add_argument("--prec", default="3xfp16", choices=["3xfp16", "3xbf16", "3xtf32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-slice", action="store_true")
    ap.add_argument("--qslice", type=int, default=2, help="cfg2: q points of the timed slice")
    ap.add_argument("--head-wings", type=int, default=2, choices=[0, 1, 2],
                    help="q -> 0: 2 = head and wings averaged over the direction of q (default), 1 = along x, "
                         "0 = regular formula")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other split precisions, the FP64 pass on the 3x3x3 mesh, the surrogate "
                         "and the batch (the last two can be asked for again with --surrogate / --batch)")
    ap.add_argument("--qloop", default="g0w0", choices=["g0w0", "perq"],
                    help="q loop in one gw_g0w0 call (default) or as per-q gw_chi0/gw_screen/gw_sigma calls")
    ap.add_argument("--nk", default=None, help="override the k mesh, e.g. 4,4,4 (profiling captures)")
    ap.add_argument("--surrogate", action="store_true",
                    help="train the frequency surrogate and time it against the full 60-point grid (part of the "
                         "default N = 1 line; this flag asks for it with --no-extras too)")
    ap.add_argument("--sur-systems", type=int, default=64, help="training systems of the surrogate")
    ap.add_argument("--sur-epochs", type=int, default=40, help="training epochs of the surrogate")
    ap.add_argument("--parallel", default="qshard", choices=["qshard", "replicas"],
                    help="N > 1: split the q mesh of one system over the ranks and sum Sigma_c (default), or "
                         "run one independent system per rank")
    ap.add_argument("--batch", type=int, default=0,
                    help="run a batch of this many seeded systems of uneven size (64 in the default N = 1 line)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "native":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2011_01400_gb300.synth import make_system
    over = {}
    if args.nk:
        over["nk"] = tuple(int(x) for x in args.nk.split(","))
    over["head_wings"] = args.head_wings
    system = make_system(args.config, seed=replica_seed(args.config, rank, args.parallel), **over)
    if args.impl == "reference":
        run_reference(args, system, world, rank)
    else:
        run_device(args, system, world, rank)
    if world > 1 and args.impl == "native":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
