#!/usr/bin/env python
"""Benchmark of one NQS-VMC SR step on the 8x8 Heisenberg workload.

Workload (synthetic): 2D Heisenberg antiferromagnet 8x8, periodic, complex RBM alpha = 2
(M = 128, P = 8384), Marshall phase in a_i, parameters N(0, 0.01^2) from a seed; 8192
Markov chains with exchange moves in the Sz = 0 sector, one sample per chain per SR step
(one sweep apart), Ns = 8192; dense S (8384^2) and the regularised solve; Euler update.

One "step" is vmc_sr_step: sampling with fused E_loc and tanh(theta), energy statistics,
<O> and F, the centred log-derivative matrix, the S contraction, the shifted solve and
the parameter update.  Inputs (parameters, chains) are resident in HBM when the timed
region starts; the e2e figure instead copies the parameters in from pinned host memory
and the updated parameters and statistics out, every step, through the same C ABI.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("effective MC samples/s incl. E_loc+O_k and SR steps/s vs plain FP32 path at "
          "|dE/N|<=1e-4")

DT = 0.02

# workloads: (model, Lx, Ly, J, h, alpha, chains, samples per chain, shift, solver)
WORKLOADS = {
    "heis2d_8x8_alpha2_c8192": dict(model=1, Lx=8, Ly=8, J=1.0, h=0.0, alpha=2, chains=8192,
                                    spc=1, shift=1e-3, solver="tc", marshall=True),
    "heis2d_16x16_alpha2_c65536": dict(model=1, Lx=16, Ly=16, J=1.0, h=0.0, alpha=2,
                                       chains=65536, spc=1, shift=1e-3, solver="cg",
                                       marshall=True),
    "tfim1d_N10_alpha1_c256": dict(model=0, Lx=10, Ly=1, J=1.0, h=1.0, alpha=1, chains=256,
                                   spc=200, shift=1e-4, solver="mixed", marshall=False,
                                   precision="fp32"),
}
# batched sampling of many independent lattices (one sweep + a record per chain per step)
BATCHED = {"tfim2d_batched48_alpha2_c1024": dict(sizes=[4] * 16 + [6] * 16 + [8] * 16, alpha=2,
                                                 chains=1024, h_lo=2.0, h_hi=4.0, h_seed=7)}
# learned independent proposal against single-flip moves on a near-critical TFIM
LEARNED = {"tfim2d_12x12_h3.04_alpha2_c16384_made256": dict(L=12, h=3.04, alpha=2, chains=16384,
                                                            hidden=256, sr_steps=200,
                                                            train_records=16, epochs=10,
                                                            lr=1e-3, tau_rounds=200)}
# real-time TDVP (pseudo-inverse + SNR regularisation, adaptive Heun) of the 1D chain
TDVP = {"tfim1d_N10_alpha1_c256_tdvp": dict(N=10, alpha=1, chains=256, spc=200, J=1.0, h=1.0,
                                             eps_pinv=1e-8, eps_snr=2.0, eps_step=1e-6,
                                             tau0=1e-3)}
# the other ansatz families and the excited-state search (section 8(f) workloads, 1D chain)
FAMILIES = {
    "tfim1d_N10_made32_c51200_ar": dict(kind="ar", N=10, H=32, chains=256, spc=200, h=1.0, dt=0.05),
    "tfim1d_L10_g0.7_cnn2_c200x200": dict(kind="cnn", N=10, alpha=2, chains=200, spc=200, h=0.7,
                                          dt=1e-2),
    "tfim1d_N10_alpha1_c256_excited": dict(kind="excited", N=10, alpha=1, chains=256, spc=200,
                                           h=1.0, dt=0.05),
}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one S-Gram launch (one FP16
# product) of the default workload, from an ncu capture of the same command (2.207 GB read,
# 0.273 GB written); None once the kernel changes until it is taken again
GRAM_F16_TRAFFIC = 2.479496e9
DEFAULT_WORKLOAD = "heis2d_8x8_alpha2_c8192"
W = WORKLOADS[DEFAULT_WORKLOAD]
LX, LY, ALPHA, CHAINS, SHIFT = W["Lx"], W["Ly"], W["alpha"], W["chains"], W["shift"]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons during the timed region: NVML polled
    every 20 ms when the Python binding is importable, else nvidia-smi every 100 ms.  One
    reading is taken on entry and one on exit, so that even a short region has samples.
    Reads only; changes no setting."""
    BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
            "sw_power_cap": 0x4}
    SMI_Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []          # (sm MHz, max sm MHz, set of active reasons)
        self.stop = threading.Event()
        self.err = None
        self.mode = None

    # ---- NVML ----
    def _nvml_handle(self):
        import pynvml
        pynvml.nvmlInit()
        import torch
        pr = torch.cuda.get_device_properties(self.index)
        try:
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            return pynvml.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            if pynvml.nvmlDeviceGetCount() == 1:
                return pynvml.nvmlDeviceGetHandleByIndex(0)
            raise

    def _nvml_sample(self):
        import pynvml
        sm = pynvml.nvmlDeviceGetClockInfo(self.h, pynvml.NVML_CLOCK_SM)
        mx = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
        r = int(pynvml.nvmlDeviceGetCurrentClocksEventReasons(self.h))
        self.rows.append((float(sm), float(mx), {k for k, bit in self.BITS.items() if r & bit}))

    # ---- nvidia-smi ----
    def _smi_target(self):
        import torch
        pr = torch.cuda.get_device_properties(self.index)
        return f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"

    def _smi_parse(self, line):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 6:
            return
        try:
            sm, mx = float(parts[0]), float(parts[1])
        except ValueError:
            return
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        act = {names[k] for k in range(4) if parts[2 + k].lower().startswith("active")}
        self.rows.append((sm, mx, act))

    def _smi_once(self):
        out = subprocess.run(["nvidia-smi", "-i", self.target, f"--query-gpu={self.SMI_Q}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10)
        for line in out.stdout.splitlines():
            self._smi_parse(line)

    def _smi_read(self):
        for line in self.proc.stdout:
            self._smi_parse(line)

    def __enter__(self):
        try:
            self.h = self._nvml_handle()
            self._nvml_sample()
            self.mode = "NVML, 20 ms"
            self.t = threading.Thread(target=self._loop, daemon=True)
            self.t.start()
            return self
        except Exception as e:
            self.err = f"NVML: {type(e).__name__}: {e}"
        try:
            self.target = self._smi_target()
            self._smi_once()
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.target, f"--query-gpu={self.SMI_Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._smi_read, daemon=True)
            self.t.start()
            self.mode = "nvidia-smi, 100 ms"
        except Exception as e:
            self.err = (self.err or "") + f"; nvidia-smi: {type(e).__name__}: {e}"
        return self

    def _loop(self):
        while not self.stop.wait(0.02):
            try:
                self._nvml_sample()
            except Exception:
                return

    def __exit__(self, *a):
        if self.mode and self.mode.startswith("NVML"):
            self.stop.set()
            self.t.join(timeout=1)
            try:
                self._nvml_sample()
            except Exception:
                pass
        elif self.mode:
            try:
                self._smi_once()
            except Exception:
                pass
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"],
                    "error": self.err}
        reasons = sorted(set().union(*(r[2] for r in self.rows)))
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": max(r[1] for r in self.rows), "reasons": reasons,
                "samples": len(self.rows), "source": self.mode}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws, device="cuda"):
    """Each entry's largest value over the ranks (a timed region lasts as long as its slowest
    replica); every rank gets the result.  One rank: the values as they are."""
    vals = [float(v) for v in values]
    if ws <= 1:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_rate(ws, units_per_rank, ms):
    """Whole-job throughput of ws replicas that each processed units_per_rank units in a
    region of ms milliseconds (the max over the ranks)."""
    return ws * units_per_rank / (ms / 1e3)


# ----------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------------------
def cpu_baseline(budget_s: float = 20.0):
    """The oracle on a bounded sample of the default workload's step, extrapolated to the
    full step (the oracle's plain loops would take an hour per full step here)."""
    import oracle
    from paper_2108_03409_b300 import inputs
    N, M = LX * LY, ALPHA * LX * LY
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.01, seed=1234, marshall=(LX, LY))
    cores = oracle.num_threads()
    t_all = time.perf_counter()
    # (a) sampling + E_loc + O_k on c chains (one sweep, one sample each)
    c = 512
    s0 = inputs.random_sz0_spins(c, N, seed=99)
    t0 = time.perf_counter()
    s, _, _, _ = oracle.metropolis(1, LX, LY, M, p, s0, seed=1, n_sweeps=1)
    E = oracle.eloc(1, LX, LY, 1.0, 0.0, M, p, s)
    O = oracle.ok(N, M, p, s)
    m_samp = time.perf_counter() - t0
    t_samp = m_samp * (CHAINS / c)
    # (b) S rows: r rows of the 8384 x 8384 matrix from c samples, scaled to Ns x P rows
    r = 128
    kk = np.repeat(np.arange(r), P)
    ll = np.tile(np.arange(P), r)
    t0 = time.perf_counter()
    oracle.sr_entries(O, E, kk, ll, np.arange(P))
    m_S = time.perf_counter() - t0
    t_S = m_S * (P / r) * (CHAINS / c)
    # (c) FP64 Cholesky at n = 2048, scaled by (P/n)^3
    n = 2048
    A = np.random.default_rng(0).normal(size=(n, n)) + 0j
    A = A @ A.conj().T / n + np.eye(n)
    F = np.ones(n, np.complex128)
    t0 = time.perf_counter()
    oracle.cholesky_solve(A, F)
    m_chol = time.perf_counter() - t0
    t_chol = m_chol * (P / n) ** 3
    t_step = t_samp + t_S + t_chol
    measured = time.perf_counter() - t_all
    return {"value": 1.0 / t_step, "unit": "SR steps/s", "cores": cores, "kind": "oracle",
            "extrapolated": True,
            "measured_s": measured,
            "measured_fraction": {"chains": c / CHAINS, "S_rows": r / P,
                                  "cholesky_flops": (n / P) ** 3},
            "sample": (f"FP64 oracle, {cores} threads, EXTRAPOLATED from a measured {measured:.1f} s "
                       f"bounded sample: Metropolis sweep + E_loc + O_k of {c} of "
                       f"{CHAINS} chains (x{CHAINS // c}), {r} of {P} rows of S (x{P // r} rows, "
                       f"x{CHAINS // c} samples), Cholesky solve at n={n} (x(P/n)^3); "
                       f"estimated step {t_step:.1f} s = sample {t_samp:.1f} + S {t_S:.1f} + "
                       f"solve {t_chol:.1f}")}


def cpu_oracle_sr_step_1d():
    """One FULL oracle SR step, measured (not extrapolated), on the 1D TFIM workload
    (N = 10, alpha = 1, P = 120, 256 chains x 200 samples = 51 200 samples, 20
    thermalisation sweeps, dt 0.02, shift 1e-4): Metropolis, E_loc, O_k, S and F,
    shifted Cholesky solve, Euler update, all in the FP64 oracle."""
    import oracle
    from paper_2108_03409_b300 import inputs
    N, M, C, R = 10, 10, 256, 200
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    s = inputs.random_spins(C, N, seed=99)
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    s, _, _, _ = oracle.metropolis(0, N, 1, M, p, s, seed=1, n_sweeps=20)
    _, rec, _, _ = oracle.metropolis(0, N, 1, M, p, s, seed=1, sweep0=20, n_sweeps=R, record=True)
    smp = rec.reshape(-1, N)
    E = oracle.eloc(0, N, 1, 1.0, 1.0, M, p, smp)
    O = oracle.ok(N, M, p, smp)
    S, F, _ = oracle.sr_matrices(O, E)
    x = oracle.cholesky_solve(oracle.shift(S, 1e-4, 0), F)
    oracle.update(p, x, DT)
    t = time.perf_counter() - t0
    return {"value": 1.0 / t, "unit": "SR steps/s", "cores": cores, "kind": "oracle",
            "extrapolated": False, "workload": "tfim1d_N10_alpha1_c256",
            "sample": (f"one full FP64 oracle SR step of the 1D TFIM workload (N=10, P=120, "
                       f"{C}x{R} = {C * R} samples, 20 thermalisation sweeps), {cores} threads, "
                       f"{t:.2f} s")}


def run_reference(args):
    """The oracle as it stands, on the host cores: W + K steps, each one bounded sample of the
    default workload's SR step (see cpu_baseline); ms_per_step is the measured wall time of
    one such sample step, value the full step's rate extrapolated from it."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline()
    t0 = time.perf_counter()
    runs = [cpu_baseline() for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    value = statistics.median(r["value"] for r in runs)
    cb = dict(runs[-1])
    cb["value"] = value
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "SR steps/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "extrapolated": True,
           "note": ("each step is a bounded sample of the full step (ms_per_step is its measured "
                    "wall time); value is the full step's rate extrapolated from it"),
           "config": {"workload": "heis2d_8x8_alpha2_c8192", "N": 64, "M": 128, "P": 8384,
                      "chains": CHAINS, "Ns": CHAINS, "shift": SHIFT},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "SR steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def _energy_estimate(ctx, vmc, vstats, torch, C, N, R=16):
    """<E>/N at the context's current parameters from R recorded sweeps of every chain, with
    the error bar sqrt(var / n * 2 tau_int(E))."""
    el = torch.zeros((R * C, 2), dtype=torch.float32, device="cuda")
    vmc.vmc_sample(ctx, 0, 0, R, None, None, el)
    e = el[:, 0].double().reshape(R, C).cpu().numpy()
    del el
    tau = vstats.integrated_autocorr_time(e[:, :4096])
    return float(e.mean()) / N, float(np.sqrt(e.var() / e.size * 2 * tau)) / N, tau


def _paired_energy_difference(vctx, pctx, vmc, vstats, torch, C, N, R=32):
    """<E>(theta_p) - <E>(theta_v) from one sample set drawn from |psi_v|^2 (R recorded sweeps
    of every chain of the variant's context), reweighted by |psi_p / psi_v|^2 for the plain
    parameters: the two estimates share their samples, so the difference has a far smaller
    statistical error than two independent estimates.  Error bar from the linearised
    per-sample difference d_s with its integrated autocorrelation time."""
    n = R * C
    sp = torch.zeros((n, N), dtype=torch.int8, device="cuda")
    lv = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ev = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    vmc.vmc_sample(vctx, 0, 0, R, sp, lv, ev)
    lp = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ep = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    vmc.vmc_logpsi(pctx, 0, sp, lp)
    vmc.vmc_local_energy(pctx, 0, sp, ep)
    Ev = ev[:, 0].double().cpu().numpy()
    Ep = ep[:, 0].double().cpu().numpy()
    dl = 2.0 * (lp[:, 0].double() - lv[:, 0].double()).cpu().numpy()
    w = np.exp(dl - dl.max())
    w /= w.mean()
    ep_est = float(np.sum(w * Ep) / np.sum(w))
    ev_est = float(Ev.mean())
    d = w * (Ep - ep_est) - (Ev - ev_est)
    tau = vstats.integrated_autocorr_time(d.reshape(R, C)[:, :4096])
    err = float(np.sqrt(d.var() / n * 2 * tau))
    return (ep_est - ev_est) / N, err / N, ev_est / N, ep_est / N


def _sr_arm(wl, prec, solver, steps, warmup, rank, stream, clk_index, vmc, inputs, barrier,
            torch, clocks=True):
    """One arm of the SR-step benchmark: a fresh context from the seeded parameters and
    chains, `warmup` untimed steps, then `steps` steps timed with CUDA events on the
    context's stream.  Returns the context (still alive) and the measurements."""
    N, M = LX * LY, ALPHA * LX * LY
    cg = solver == vmc.SOLVER_CG
    cfg = vmc.make_config(seed=1 + rank, n_chains=CHAINS, therm_sweeps=20, sweeps_per_sample=1,
                          samples_per_chain=wl["spc"], precision=prec, solver=solver, shift=SHIFT,
                          cg_tol=1e-6, cg_maxit=1000 if cg else 50)
    lat = vmc.make_lattice(wl["model"], LX, LY, wl["J"], wl["h"], ALPHA)
    ctx = vmc.vmc_init(cfg, [lat], stream.cuda_stream)
    p0 = inputs.rbm_params(N, M, 0.01, seed=1234, marshall=(LX, LY) if wl["marshall"] else None)
    vmc.vmc_set_params(ctx, 0, p0)
    vmc.vmc_set_chains(ctx, 0, inputs.initial_spins(wl["model"], CHAINS, N, seed=99 + rank))
    unconverged = [0]

    def step():
        try:
            return vmc.vmc_sr_step(ctx, 0, DT)
        except vmc.VmcError as e:          # a CG that stopped above cg_tol: reported, not hidden
            if e.status != vmc.VMC_ERR_NUMERIC or getattr(e, "stats", None) is None:
                raise
            unconverged[0] += 1
            return e.stats

    warm = [step() for _ in range(warmup)]
    barrier()
    launches0 = vmc.vmc_kernel_launches(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st_list = []
    clk = ClockSampler(clk_index) if clocks else None
    if clk:
        clk.__enter__()
    ev0.record(stream)
    for _ in range(steps):
        st_list.append(step())
    ev1.record(stream)
    barrier()
    if clk:
        clk.__exit__(None, None, None)
    ms = ev0.elapsed_time(ev1)
    return {"ctx": ctx, "ms": ms, "st": st_list, "warm": warm, "clk": clk,
            "launches": vmc.vmc_kernel_launches(ctx) - launches0, "unconverged": unconverged[0]}


def run_ours(args):
    global LX, LY, ALPHA, CHAINS, SHIFT
    wl = WORKLOADS[args.workload]
    LX, LY, ALPHA, CHAINS, SHIFT = wl["Lx"], wl["Ly"], wl["alpha"], wl["chains"], wl["shift"]
    import torch
    from paper_2108_03409_b300 import build as vbuild
    from paper_2108_03409_b300 import inputs, stats as vstats, vmc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    prec_name = args.precision or wl.get("precision", "bf16split")
    prec = {"fp32": vmc.PREC_FP32, "bf16split": vmc.PREC_BF16SPLIT}[prec_name]
    solver_name = args.solver or wl["solver"]
    solvers = {"fp64": vmc.SOLVER_CHOLESKY_FP64, "mixed": vmc.SOLVER_CHOLESKY_MIXED,
               "tc": vmc.SOLVER_CHOLESKY_TC, "cg": vmc.SOLVER_CG}
    solver = solvers[solver_name]
    N, M = LX * LY, ALPHA * LX * LY
    P = N + M + N * M
    stream = torch.cuda.current_stream()
    Ns = CHAINS * wl["spc"]
    cg = solver == vmc.SOLVER_CG

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    arm = _sr_arm(wl, prec, solver, args.steps, args.warmup, rank, stream, local, vmc, inputs,
                  barrier, torch)
    ctx, st_list, clk, launches = arm["ctx"], arm["st"], arm["clk"], arm["launches"]
    ms = max_over_ranks([arm["ms"]], ws)[0]
    ms_step = ms / args.steps
    value = replica_rate(ws, args.steps, ms)

    # e2e: parameters in from pinned host memory, parameters + statistics out, every step
    host_p = torch.from_numpy(vmc.vmc_get_params(ctx, 0).view(np.float64).copy()).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        vmc.load().vmc_set_params(ctx, 0, host_p.data_ptr())
        try:
            vmc.vmc_sr_step(ctx, 0, DT)
        except vmc.VmcError as e:
            if e.status != vmc.VMC_ERR_NUMERIC:
                raise
        vmc.load().vmc_get_params(ctx, 0, host_p.data_ptr())
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = ws / e2e_s

    # integrated autocorrelation time of E_loc at the final parameters (sampler only)
    T = 200
    cs = min(CHAINS, 2048)
    el = torch.zeros((T * CHAINS, 2), dtype=torch.float32, device="cuda")
    vmc.vmc_sample(ctx, 0, 0, T, None, None, el)
    e_series = el[:, 0].reshape(T, CHAINS)[:, :cs].double().cpu().numpy()
    del el
    tau = vstats.integrated_autocorr_time(e_series)

    ms_samp = statistics.mean(s.ms_sample + s.ms_grad for s in st_list)
    ms_gram = statistics.mean(s.ms_gram for s in st_list)
    eff = Ns / (ms_samp / 1e3) / (2 * tau)
    pk, pk_kind = peaks()
    # dominant kernel: the S contraction.  Algorithmic work as the hot-path table counts it:
    # 8 P^2 Ns flops for the full real Gram of [Re Obar | Im Obar], half of it for the
    # symmetric (lower) tiles, times 3 for the BF16 hi/lo split = 12 P^2 Ns on the tensor
    # pipe (4 P^2 Ns "plain-equivalent" flops of one FP32 product).
    # The SR step's tensor-core S only feeds the factor that preconditions CG on the exact
    # FP32 operator: one FP16 product, 4 P^2 Ns flops, against the FP16 dense peak (the
    # measured BF16 peak x the nominal FP16 : BF16 ratio of 1).
    fused_f16 = prec == vmc.PREC_BF16SPLIT and solver_name in ("tc", "mixed")
    if fused_f16:
        alg_flops, alg_text = 4.0 * P * P * Ns, "4*P^2*Ns flops (Hermitian half of the real Gram, one FP16 product)"
        roof = {"bound": "tensor", "peak": pk.get("bf16_tflops", 1766.8),
                "peak_kind": f"fp16 dense burst = bf16 dense burst ({pk_kind}) x 1 (nominal ratio); "
                             "the step keeps the SM clock at max"}
    elif prec == vmc.PREC_BF16SPLIT:
        alg_flops, alg_text = 12.0 * P * P * Ns, "12*P^2*Ns flops (Hermitian half of the real Gram, x3 BF16 split)"
        roof = {"bound": "tensor", "peak": pk.get("bf16_tflops", 1766.8),
                "peak_kind": f"bf16 dense burst ({pk_kind}); the step keeps the SM clock at max"}
    else:
        alg_flops, alg_text = 4.0 * P * P * Ns, "4*P^2*Ns flops (Hermitian half of the real Gram)"
        fp32_peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        roof = {"bound": "alu", "peak": fp32_peak,
                "peak_kind": "FP32 FMA: 148 SMs x 128 lanes x 2 flop x max SM clock"}
    achieved = alg_flops / (ms_gram / 1e3) / 1e12
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one S-Gram launch of
    # this kernel on this workload, from an ncu capture of the same command
    traffic = GRAM_F16_TRAFFIC if (fused_f16 and args.workload == DEFAULT_WORKLOAD) else None
    roofline = {"bound": roof["bound"], "achieved": achieved, "peak": roof["peak"],
                "unit": "TFLOP/s", "frac": achieved / roof["peak"], "traffic": traffic,
                "kernel": "gram_tc" if prec == vmc.PREC_BF16SPLIT else "gram_f32",
                "peak_source": roof["peak_kind"], "algorithmic": alg_text,
                "ms_per_launch": ms_gram}
    if prec == vmc.PREC_BF16SPLIT:
        if not fused_f16:
            roofline["plain_equivalent_frac"] = achieved / 3.0 / roof["peak"]
        roofline["frac_of_sustained"] = achieved / pk.get("bf16_tflops_sustained", 1387.8)
    # bytes the step streams (each larger than the 126 MB L2, so no flush between steps)
    if solver_name == "cg":
        l2_note = (f"working set (t {Ns * M * 8 / 1e6:.0f} MB read twice per CG iteration, "
                   f"spins {Ns * N * 2 / 1e6:.0f} MB as BF16) larger than L2; no flush")
    else:
        ws_bytes = P * P * 16 + 2 * P * Ns * 4
        l2_note = (f"working set (S {P * P * 16 / 1e9:.2f} GB, X {2 * P * Ns * 4 / 1e9:.2f} GB) "
                   + ("larger than L2; no flush" if ws_bytes > 126e6 else
                      "fits in L2 (a small parity-size workload); not flushed"))
    out = {"metric": METRIC, "value": value, "unit": "SR steps/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": ("f32" if prec == vmc.PREC_FP32 else
                     "f16 S for the CG preconditioner / f32 CG operator and accumulation" if fused_f16
                     else "bf16x3-split/f32-accum"),
           "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "M": M, "P": P,
                      "chains": CHAINS, "Ns": Ns, "shift": SHIFT, "dt": DT,
                      "precision": prec_name, "solver": solver_name,
                      "solver_tol": 1e-6, "l2": l2_note,
                      "parallelism": f"replicas x{ws}"},
           "eff_samples_per_s": {"value": eff * ws, "unit": "samples/s", "tau_int_E": tau,
                                 "ms_sample_eloc_ok": ms_samp},
           "phases_ms": {k: statistics.mean(getattr(s, k) for s in st_list)
                         for k in ("ms_sample", "ms_grad", "ms_qfm", "ms_solve", "ms_update",
                                   "ms_gram")},
           "energy_per_site": st_list[-1].e_mean_re / N,
           "solver_iters": st_list[-1].solver_iters, "solver_relres": st_list[-1].solver_relres,
           "solver_relres_explicit": st_list[-1].solver_relres_explicit,
           "solver_converged": all(s.solver_converged for s in st_list),
           "unconverged_steps": arm["unconverged"],
           "roofline": roofline,
           "e2e": {"value": e2e_value, "unit": "SR steps/s", "h2d_bytes_per_step": P * 16,
                   "d2h_bytes_per_step": P * 16 + 4 * 8 * 0 + 64},
           "gpu_launches": launches,
           "clocks": clk.summary()}
    if cg:
        out["roofline"] = None
        out["note"] = "CG workload: per-iteration kernels reported in phases_ms; no dense S"

    # The metric's own comparison: the plain FP32 path (SIMT FP32 Gram, FP32 SIMT factor +
    # refinement) from the same seeded parameters and chains, timed the same way, and the
    # equal-accuracy gate on the same theta: from one identical state (parameters and chains
    # of the plain arm after its steps) each arm takes one SR step, and <E> at the two
    # updated parameter sets must agree to |dE|/N <= 1e-4 with three standard errors of the
    # difference included (a paired estimate: one sample set, reweighted).
    if (args.workload == DEFAULT_WORKLOAD and not args.no_plain and prec != vmc.PREC_FP32):
        e_traj_var = _energy_estimate(ctx, vmc, vstats, torch, CHAINS, N)[0]
        plain_steps = max(2, min(args.steps, 5))
        pa = _sr_arm(wl, vmc.PREC_FP32, vmc.SOLVER_CHOLESKY_MIXED, plain_steps, args.warmup, rank,
                     stream, local, vmc, inputs, barrier, torch, clocks=False)
        pctx = pa["ctx"]
        # the variant ran warmup + steps + e2e steps; bring the plain arm to the same count
        for _ in range(max(0, args.steps + e2e_steps - plain_steps)):
            vmc.vmc_sr_step(pctx, 0, DT)
        e_traj_pl = _energy_estimate(pctx, vmc, vstats, torch, CHAINS, N)[0]
        ms_pl = pa["ms"] / plain_steps
        ms_samp_pl = statistics.mean(s.ms_sample + s.ms_grad for s in pa["st"])
        eff_pl = Ns / (ms_samp_pl / 1e3) / (2 * tau)
        theta0 = vmc.vmc_get_params(pctx, 0)
        chains0 = vmc.vmc_get_chains(pctx, 0, CHAINS, N)
        for c in (ctx, pctx):
            vmc.vmc_set_params(c, 0, theta0)
            vmc.vmc_set_chains(c, 0, chains0)
        # one sample set (the plain arm's sampler from the shared state) for both arms' steps,
        # so that the difference is the arithmetic's and not the Monte Carlo noise of two
        # sample sets (the arms' theta differ in their last bits, which can flip a
        # near-threshold Metropolis decision)
        spc = wl["spc"]
        ss = torch.zeros((CHAINS * spc, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(pctx, 0, 0, spc, ss)
        vmc.vmc_set_chains(pctx, 0, chains0)
        e_before = None
        for c in (ctx, pctx):
            e_before = vmc.vmc_sr_step_on(c, 0, ss, DT).e_mean_re / N
        dE, err, e_v, e_p = _paired_energy_difference(ctx, pctx, vmc, vstats, torch, CHAINS, N)
        vmc.vmc_destroy(pctx)
        out["plain_fp32"] = {"sr_steps_per_s": ws * 1e3 / ms_pl, "ms_per_step": ms_pl,
                             "eff_samples_per_s": eff_pl * ws, "steps": plain_steps,
                             "precision": "fp32", "solver": "mixed",
                             "phases_ms": {k: statistics.mean(getattr(s, k) for s in pa["st"])
                                           for k in ("ms_sample", "ms_grad", "ms_qfm",
                                                     "ms_solve", "ms_update", "ms_gram")}}
        out["vs_plain_fp32"] = {"sr_steps_per_s": value / (ws * 1e3 / ms_pl),
                                "eff_samples_per_s": (eff * ws) / (eff_pl * ws)}
        out["equal_accuracy"] = {
            "how": ("one SR step of each arm from the same theta on one sample set (drawn by the "
                    "plain arm's sampler from the shared chains); <E>/N at the two "
                    "updated parameter sets from one set of 32 sweeps x all chains drawn at the "
                    "variant's parameters, the plain one reweighted by |psi_plain/psi_variant|^2; "
                    "ok = |dE|/N + 3 sigma <= 1e-4"),
            "e_before_per_site": e_before,
            "e_per_site_variant": e_v, "e_per_site_plain": e_p,
            "dE_per_site": dE, "err_dE_per_site": err,
            "ok": bool(abs(dE) + 3 * err <= 1e-4),
            "trajectory_dE_per_site": {
                "sr_steps_each": args.warmup + args.steps + e2e_steps,
                "variant": e_traj_var, "plain": e_traj_pl,
                "note": "independent trajectories: once the parameters differ in their last "
                        "bits the chains take other Metropolis decisions, so each arm's later "
                        "steps see other samples; the difference is Monte Carlo noise of the "
                        "SR trajectory while E still falls quickly; informational, not the gate"}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == DEFAULT_WORKLOAD:
        out["cpu_baseline"] = cpu_baseline()
        out["cpu_baseline_measured"] = cpu_oracle_sr_step_1d()
    if ctx is not None:
        vmc.vmc_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batched(args):
    """48 TFIM lattices of uneven size: one persistent launch (autotuned, CUDA graph) per
    step against 48 per-lattice launches of the same sweeps.  A step is one sweep of every
    chain of every lattice plus the record (spins and fused E_loc) of each chain."""
    import torch
    from paper_2108_03409_b300 import build as vbuild
    from paper_2108_03409_b300 import inputs, vmc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    wl = BATCHED[args.workload]
    C, alpha = wl["chains"], wl["alpha"]
    hs = inputs.uniform_fields(len(wl["sizes"]), wl["h_lo"], wl["h_hi"], wl["h_seed"])
    lats = [vmc.make_lattice(vmc.MODEL_TFIM, L, L, 1.0, float(h), alpha)
            for L, h in zip(wl["sizes"], hs)]
    Ns_ = [L * L for L in wl["sizes"]]
    stream = torch.cuda.current_stream()
    cfg = vmc.make_config(seed=1 + rank, n_chains=C, solver=vmc.SOLVER_CG)
    ctx = vmc.vmc_init(cfg, lats, stream.cuda_stream)
    for l, N in enumerate(Ns_):
        vmc.vmc_set_params(ctx, l, inputs.rbm_params(N, alpha * N, 0.01, seed=1234 + l))
        vmc.vmc_set_chains(ctx, l, inputs.random_spins(C, N, seed=99 + 1000 * rank + l))
    n_lat, tot = len(Ns_), sum(Ns_)
    spins = torch.zeros(C * tot, dtype=torch.int8, device="cuda")
    eloc = torch.zeros((n_lat * C, 2), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    outs = []
    off = 0
    for N in Ns_:
        outs.append(spins[off:off + C * N].view(C, N))
        off += C * N

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    vmc.vmc_sample_all(ctx, 20, 0, None, None, False)       # thermalise (and autotune)
    for _ in range(args.warmup):
        vmc.vmc_sample_all(ctx, 0, 1, spins, eloc, True)
        for l in range(n_lat):
            vmc.vmc_sample(ctx, l, 0, 1, outs[l], None, eloc[l * C:(l + 1) * C])
    barrier()

    def timed(fn):
        evs = []
        for _ in range(args.steps):
            flush.zero_()               # L2 flushed between timed iterations
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        barrier()
        return sum(a.elapsed_time(b) for a, b in evs)

    launches0 = vmc.vmc_kernel_launches(ctx)
    with ClockSampler(local) as clk:
        ms_b = timed(lambda: vmc.vmc_sample_all(ctx, 0, 1, spins, eloc, True))
    launches = vmc.vmc_kernel_launches(ctx) - launches0

    def per_lattice():
        for l in range(n_lat):
            vmc.vmc_sample(ctx, l, 0, 1, outs[l], None, eloc[l * C:(l + 1) * C])
    ms_p = timed(per_lattice)
    ms_ng = timed(lambda: vmc.vmc_sample_all(ctx, 0, 1, spins, eloc, False))
    ms_b, ms_p, ms_ng = max_over_ranks([ms_b, ms_p, ms_ng], ws)
    samples = n_lat * C
    value = ws * samples * args.steps / (ms_b / 1e3)

    # e2e: the chains in from pinned host memory and the records out, every step
    host_in = [torch.from_numpy(vmc.vmc_get_chains(ctx, l, C, N)).pin_memory()
               for l, N in enumerate(Ns_)]
    host_s = torch.empty(C * tot, dtype=torch.int8).pin_memory()
    host_e = torch.empty((n_lat * C, 2), dtype=torch.float32).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for l in range(n_lat):
            vmc.load().vmc_set_chains(ctx, l, host_in[l].data_ptr())
        vmc.vmc_sample_all(ctx, 0, 1, spins, eloc, True)
        host_s.copy_(spins)
        host_e.copy_(eloc)
    barrier()
    e2e = ws * samples * args.steps / (time.perf_counter() - t0)

    # ALU roofline of the persistent sweep kernel: per proposed flip and hidden unit the
    # ratio cosh(theta - d)/cosh(theta) = cosh d - tanh(theta) sinh d and its squared
    # modulus take 22 FP32 operations (18 arithmetic, 4 elementary functions counted once);
    # the record's local energy evaluates the same ratio, without the modulus (19), for each
    # of the N flips.  One step (one sweep of N proposals and one record per chain) does
    # (22 + 19) * sum_l C * N_l * M_l flops.
    flops = (22.0 + 19.0) * sum(C * N * alpha * N for N in Ns_)
    pk, pk_kind = peaks()
    fp32_peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    achieved = flops / (ms_b / args.steps / 1e3) / 1e12
    out = {"metric": METRIC, "value": value, "unit": "samples/s (incl. E_loc)", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": args.workload, "lattices": "16 x 4x4, 16 x 6x6, 16 x 8x8 TFIM",
                      "alpha": alpha, "chains_per_lattice": C, "h": "U[2,4] seed 7",
                      "l2": "flushed (256 MB write) before every timed step",
                      "parallelism": f"replicas x{ws}"},
           "per_lattice_launches": {"value": ws * samples * args.steps / (ms_p / 1e3),
                                    "ms_per_step": ms_p / args.steps},
           "batched_no_graph": {"value": ws * samples * args.steps / (ms_ng / 1e3),
                                "ms_per_step": ms_ng / args.steps},
           "speedup_vs_per_lattice": ms_p / ms_b,
           "autotuned_warps_per_block": vmc.vmc_autotuned_warps_per_block(ctx),
           "autotuned_slots_per_lane": vmc.vmc_autotuned_slots_per_lane(ctx),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                        "kernel": "sample_batched",
                        "peak_source": "FP32 FMA: 148 SMs x 128 lanes x 2 flop x max SM clock",
                        "algorithmic": "22 flops per proposed flip and 19 per local-energy flip ratio, per hidden unit"},
           "e2e": {"value": e2e, "unit": "samples/s (incl. E_loc)",
                   "h2d_bytes_per_step": C * tot, "d2h_bytes_per_step": C * tot + n_lat * C * 8},
           "gpu_launches": launches,
           "clocks": clk.summary()}
    vmc.vmc_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_learned(args):
    """Learned proposal: the RBM is first optimised by plain SR steps (matrix-free CG), the
    MADE proposal is trained on 2^18 samples of the local chains, then both samplers run from
    the same state.  A step is one round on every chain (a learned proposal + accept, or one
    single-flip sweep) with the E_loc record; tau_int(E) comes from a longer run of each."""
    import torch
    from paper_2108_03409_b300 import build as vbuild
    from paper_2108_03409_b300 import inputs, stats as vstats, vmc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    wl = LEARNED[args.workload]
    L, C, H = wl["L"], wl["chains"], wl["hidden"]
    N, M = L * L, wl["alpha"] * L * L
    stream = torch.cuda.current_stream()
    lat = [vmc.make_lattice(vmc.MODEL_TFIM, L, L, 1.0, wl["h"], wl["alpha"])]
    # the checkpoint: plain SR steps by matrix-free CG with the operator on the tensor cores
    # and a diagonal shift of 1e-2 (with 1e-3 near this critical point the CG needs 700-1000
    # iterations and more per step and stalls: the FP32 SIMT operator at its 1e-6 rounding
    # floor, the BF16-split one above it); a step whose CG stops above cg_tol is counted and
    # not applied
    pcfg = vmc.make_config(seed=1 + rank, n_chains=C, therm_sweeps=20, solver=vmc.SOLVER_CG,
                           precision=vmc.PREC_BF16SPLIT, shift=1e-2, cg_maxit=1000, cg_tol=1e-6)
    pctx = vmc.vmc_init(pcfg, lat, stream.cuda_stream)
    vmc.vmc_set_params(pctx, 0, inputs.rbm_params(N, M, 0.01, seed=1234))
    vmc.vmc_set_chains(pctx, 0, inputs.random_spins(C, N, seed=99 + rank))
    t0 = time.perf_counter()
    unconverged, sr_iters = 0, []
    for _ in range(wl["sr_steps"]):
        try:
            st = vmc.vmc_sr_step(pctx, 0, DT)
        except vmc.VmcError as e:
            if e.status != vmc.VMC_ERR_NUMERIC or getattr(e, "stats", None) is None:
                raise
            st = e.stats
            unconverged += 1
        sr_iters.append(st.solver_iters)
    t_sr = time.perf_counter() - t0
    e_sr = st.e_mean_re / N
    theta_ck, chains_ck = vmc.vmc_get_params(pctx, 0), vmc.vmc_get_chains(pctx, 0, C, N)
    vmc.vmc_destroy(pctx)
    # both samplers run in FP32 from the checkpoint
    cfg = vmc.make_config(seed=1 + rank, n_chains=C, therm_sweeps=20, solver=vmc.SOLVER_CG,
                          shift=1e-3, cg_maxit=1000, cg_tol=1e-6, made_hidden=H, made_batch=4096)
    ctx = vmc.vmc_init(cfg, lat, stream.cuda_stream)
    vmc.vmc_set_params(ctx, 0, theta_ck)
    vmc.vmc_set_chains(ctx, 0, chains_ck)
    # training set: 2^18 samples of the local chains (one sweep apart)
    R = wl["train_records"]
    train = torch.zeros((R * C, N), dtype=torch.int8, device="cuda")
    vmc.vmc_sample(ctx, 0, 0, R, train)
    vmc.vmc_made_set_params(ctx, 0, inputs.made_params(N, H, seed=5))
    t0 = time.perf_counter()
    loss = vmc.vmc_proposal_train(ctx, 0, train, epochs=wl["epochs"], lr=wl["lr"])
    t_train = time.perf_counter() - t0
    del train
    chains0 = vmc.vmc_get_chains(ctx, 0, C, N)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    el1 = torch.zeros((C, 2), dtype=torch.float32, device="cuda")

    def timed(fn, steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        barrier()
        return a.elapsed_time(b)

    local_round = lambda: vmc.vmc_sample(ctx, 0, 0, 1, None, None, el1)
    learned_round = lambda: vmc.vmc_sample_learned(ctx, 0, 1, None, el1)
    for _ in range(args.warmup):
        local_round()
        learned_round()
    barrier()
    launches0 = vmc.vmc_kernel_launches(ctx)
    with ClockSampler(local) as clk:
        ms_lrn = timed(learned_round, args.steps)
    launches = vmc.vmc_kernel_launches(ctx) - launches0
    ms_loc = timed(local_round, args.steps)

    # tau_int(E), <E> +- err and acceptance of both samplers from the same start
    T = wl["tau_rounds"]
    res = {}
    for name in ("local", "learned"):
        vmc.vmc_set_chains(ctx, 0, chains0)
        el = torch.zeros((T * C, 2), dtype=torch.float32, device="cuda")
        if name == "local":
            vmc.vmc_sample(ctx, 0, 0, T, None, None, el)
            acc = None
        else:
            acc = vmc.vmc_sample_learned(ctx, 0, T, None, el)
        e = el[:, 0].double().reshape(T, C).cpu().numpy()
        del el
        tau = vstats.integrated_autocorr_time(e[:, :4096])
        err = float(np.sqrt(e.var() / e.size * 2 * tau))
        res[name] = {"tau_int_E": tau, "e_per_site": float(e.mean()) / N, "err_per_site": err / N,
                     "acceptance": acc}
    t_loc = ms_loc / args.steps / 1e3
    t_lrn = ms_lrn / args.steps / 1e3
    eff_loc = ws * C / t_loc / (2 * res["local"]["tau_int_E"])
    eff_lrn = ws * C / t_lrn / (2 * res["learned"]["tau_int_E"])
    res["local"].update({"samples_per_s": ws * C / t_loc, "eff_samples_per_s": eff_loc,
                         "ms_per_round": t_loc * 1e3})
    res["learned"].update({"samples_per_s": ws * C / t_lrn, "eff_samples_per_s": eff_lrn,
                           "ms_per_round": t_lrn * 1e3})
    dE = abs(res["learned"]["e_per_site"] - res["local"]["e_per_site"])
    comb = float(np.hypot(res["learned"]["err_per_site"], res["local"]["err_per_site"]))
    out = {"metric": METRIC, "value": eff_lrn, "unit": "effective samples/s (incl. E_loc)",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_lrn * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (MADE f32 weights)", "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "M": M, "h": wl["h"], "chains": C,
                      "made_hidden": H, "sr_steps_checkpoint": wl["sr_steps"],
                      "train_samples": R * C, "epochs": wl["epochs"],
                      "l2": "chains + weights fit L2; no flush (sampler rounds)",
                      "parallelism": f"replicas x{ws}"},
           "samplers": res, "speedup_eff_vs_local": eff_lrn / eff_loc,
           "equal_accuracy": {"dE_per_site": dE, "combined_err_per_site": comb,
                              "ok": bool(dE <= 1e-4 and dE <= 3 * comb)},
           # the learned part is accepted only if <E> agrees within error bars AND the
           # integrated autocorrelation time of E drops (and, for the >= 3x target, the
           # effective samples/s are at least 3x those of the local moves)
           "learned_proposal_verdict": {
               "energy_agrees": bool(dE <= 1e-4 and dE <= 3 * comb),
               "tau_int_drops": bool(res["learned"]["tau_int_E"] < res["local"]["tau_int_E"]),
               "eff_speedup": eff_lrn / eff_loc,
               "meets_3x": bool(eff_lrn >= 3 * eff_loc),
               "verdict": ("accepted" if (dE <= 1e-4 and dE <= 3 * comb and
                                          res["learned"]["tau_int_E"] < res["local"]["tau_int_E"])
                           else "rejected")},
           "checkpoint": {"e_per_site": e_sr, "s": t_sr, "cg_iters_max": max(sr_iters),
                          "cg_iters_mean": float(np.mean(sr_iters)),
                          "unconverged_steps": unconverged,
                          "solver": "CG, BF16-split operator, shift 1e-2, relative residual 1e-6"},
           "train": {"loss": loss, "s": t_train},
           "roofline": None,
           "note": "sampler comparison; rooflines of the sweep and Gram kernels are in the "
                   "default workload's line",
           "gpu_launches": launches, "clocks": clk.summary()}
    vmc.vmc_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_tdvp(args):
    """Real-time TDVP of the 1D TFIM chain (N = 10, alpha = 1, P = 120): a quench from the
    near-uniform seeded state under J = h = 1, Monte Carlo right-hand sides (256 chains x 200
    samples per evaluation), the paper's regularisation (eps_pinv = 1e-8 soft, eps_SNR = 2)
    and integrator tolerance (1e-6).  A step is one accepted adaptive Heun step (1 + 4 x
    attempts right-hand sides, each: sampling with fused E_loc, FP64 moments and Grams,
    Jacobi eigen-decomposition, damped solve)."""
    import torch
    from paper_2108_03409_b300 import build as vbuild
    from paper_2108_03409_b300 import inputs, vmc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    wl = TDVP[args.workload]
    N, M = wl["N"], wl["alpha"] * wl["N"]
    P = N + M + N * M
    C, spc = wl["chains"], wl["spc"]
    stream = torch.cuda.current_stream()
    cfg = vmc.make_config(seed=1 + rank, n_chains=C, samples_per_chain=spc, therm_sweeps=20,
                          solver=vmc.SOLVER_CG, tdvp=1)
    ctx = vmc.vmc_init(cfg, [vmc.make_lattice(vmc.MODEL_TFIM, N, 1, wl["J"], wl["h"], wl["alpha"])],
                       stream.cuda_stream)
    vmc.vmc_set_params(ctx, 0, inputs.rbm_params(N, M, 0.01, seed=1234))
    vmc.vmc_set_chains(ctx, 0, inputs.random_spins(C, N, seed=99 + rank))
    opts = vmc.make_tdvp_opts(gamma=1j, eps_pinv=wl["eps_pinv"], pinv_soft=1,
                              eps_snr=wl["eps_snr"], eps_step=wl["eps_step"], tau_max=0.05)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    t, tau = 0.0, wl["tau0"]
    for _ in range(args.warmup):
        t, tau, _ = vmc.vmc_tdvp_step(ctx, 0, opts, t, tau)
    barrier()
    launches0 = vmc.vmc_kernel_launches(ctx)
    sts = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            t, tau, st = vmc.vmc_tdvp_step(ctx, 0, opts, t, tau)
            sts.append(st)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = vmc.vmc_kernel_launches(ctx) - launches0
    ms = max_over_ranks([ms], ws)[0]
    evals = sum(s.rhs_evals for s in sts)
    value = ws * args.steps / (ms / 1e3)
    # e2e: the parameters in from pinned host memory and out again around every step
    host_p = torch.from_numpy(vmc.vmc_get_params(ctx, 0).view(np.float64).copy()).pin_memory()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        vmc.load().vmc_set_params(ctx, 0, host_p.data_ptr())
        t, tau, _ = vmc.vmc_tdvp_step(ctx, 0, opts, t, tau)
        vmc.load().vmc_get_params(ctx, 0, host_p.data_ptr())
    barrier()
    e2e = ws * e2e_steps / (time.perf_counter() - t0)
    # dominant kernel: the FP64 S/Q Gram of one evaluation.  Algorithmic work: for every
    # entry of the lower triangle of S (P(P+1)/2) and every sample, one complex product
    # conj(Obar_k) Obar_l (6 flops) accumulated into S and into Q with real weights (4 flops
    # each): 14 FP64 flops per entry and sample.
    Ns = C * spc
    ms_gram = statistics.mean(s.ms_gram for s in sts)
    flops = 14.0 * P * (P + 1) / 2 * Ns
    fp64_peak = 1.25
    achieved = flops / (ms_gram / 1e3) / 1e12
    out = {"metric": METRIC, "value": value, "unit": "TDVP steps/s (adaptive Heun, real time)",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (FP32 sampler and E_loc)", "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "M": M, "P": P, "chains": C,
                      "samples_per_eval": Ns, "eps_pinv": wl["eps_pinv"], "eps_snr": wl["eps_snr"],
                      "eps_step": wl["eps_step"], "l2": "working set below L2 (P = 120); not flushed",
                      "parallelism": f"replicas x{ws}"},
           "rhs_evals_per_s": ws * evals / (ms / 1e3),
           "t_reached": t, "tau_last": sts[-1].tau_used, "retries": sum(s.retries for s in sts),
           "per_eval_ms": {"gram": ms_gram, "eig": statistics.mean(s.ms_eig for s in sts),
                           "jacobi_sweeps": statistics.mean(s.jacobi_sweeps for s in sts)},
           "energy": {"start_or_last": sts[-1].e_mean_re, "stderr": sts[-1].e_stderr},
           "kept_components": sts[-1].kept, "snr_min": sts[-1].snr_min,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp64_peak, "traffic": None, "kernel": "tdvp_gram",
                        "peak_source": "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)",
                        "algorithmic": "14 FP64 flops per lower-triangle entry of S and sample"},
           "e2e": {"value": e2e, "unit": "TDVP steps/s", "h2d_bytes_per_step": P * 16,
                   "d2h_bytes_per_step": P * 16},
           "gpu_launches": launches, "clocks": clk.summary()}
    vmc.vmc_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_family(args):
    """One step of another ansatz family (autoregressive network, CNN-ELU) or of the
    excited-state search on the 1D chain, timed like the SR step: W untimed steps, K timed
    with CUDA events; the dominant kernel's roofline from its own event timing."""
    import torch
    from paper_2108_03409_b300 import build as vbuild
    from paper_2108_03409_b300 import inputs, vmc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    wl = FAMILIES[args.workload]
    kind, N, C, spc = wl["kind"], wl["N"], wl["chains"], wl["spc"]
    Ns = C * spc
    stream = torch.cuda.current_stream()
    pk, pk_kind = peaks()
    fp32_peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    lat = vmc.make_lattice(vmc.MODEL_TFIM, N, 1, 1.0, wl["h"], wl.get("alpha", 1))
    if kind == "ar":
        H = wl["H"]
        P = inputs.made_params(N, H, seed=5).size
        cfg = vmc.make_config(seed=1 + rank, n_chains=C, samples_per_chain=spc,
                              solver=vmc.SOLVER_CHOLESKY_MIXED, shift=1e-3, shift_mode=1,
                              made_hidden=H, ar_ansatz=1, cg_tol=1e-10, cg_maxit=50)
        ctx = vmc.vmc_init(cfg, [lat], stream.cuda_stream)
        vmc.vmc_ar_set_params(ctx, 0, inputs.made_params(N, H, seed=5).astype(np.float64))
        step = lambda: vmc.vmc_ar_sr_step(ctx, 0, wl["dt"])
        unit = "SR steps/s (autoregressive ansatz, direct sampling)"
    elif kind == "cnn":
        alpha = wl["alpha"]
        P = alpha * (N + 1)
        cfg = vmc.make_config(seed=1 + rank, n_chains=C, samples_per_chain=spc, therm_sweeps=20,
                              solver=vmc.SOLVER_CG, tdvp=1, cnn_ansatz=1)
        ctx = vmc.vmc_init(cfg, [lat], stream.cuda_stream)
        vmc.vmc_cnn_set_params(ctx, 0, np.random.default_rng(1).normal(0, 0.1, P))
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(C, N, seed=9 + rank))
        counter = [0]

        def step():
            opts = vmc.make_tdvp_opts(gamma=1.0, shift=10.0 * 0.95 ** counter[0], eps_pinv=1e-8)
            counter[0] += 1
            return vmc.vmc_cnn_sr_step(ctx, 0, wl["dt"], opts)
        unit = "SR steps/s (CNN-ELU ansatz, shift + pseudo-inverse recipe)"
    else:
        M = wl["alpha"] * N
        P = N + M + N * M
        cfg = vmc.make_config(seed=1 + rank, n_chains=C, samples_per_chain=spc, therm_sweeps=20,
                              solver=vmc.SOLVER_CG, tdvp=1)
        ctx = vmc.vmc_init(cfg, [lat, lat], stream.cuda_stream)
        vmc.vmc_set_params(ctx, 0, inputs.rbm_params(N, M, 0.1, seed=77))
        vmc.vmc_set_params(ctx, 1, inputs.rbm_params(N, M, 0.01, seed=1234))
        for l in (0, 1):
            vmc.vmc_set_chains(ctx, l, inputs.random_spins(C, N, seed=8 + l + 10 * rank))
        opts = vmc.make_tdvp_opts(gamma=1.0, shift=1e-3)
        step = lambda: vmc.vmc_excited_step(ctx, 0, 1, wl["dt"], opts)
        unit = "excited-state search steps/s"

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    launches0 = vmc.vmc_kernel_launches(ctx)
    sts = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            sts.append(step())
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = vmc.vmc_kernel_launches(ctx) - launches0
    ms = max_over_ranks([ms], ws)[0]
    value = ws * args.steps / (ms / 1e3)
    if kind == "ar":
        ms_k = statistics.mean(s.ms_gram for s in sts)
        flops = 1.0 * P * P * Ns     # the lower half of the real P x P Gram: P(P+1)/2 x Ns x 2
        roof = {"bound": "alu", "kernel": "gram_f32", "peak": fp32_peak, "algorithmic":
                "P^2 Ns FP32 flops (lower half of the real Gram: P(P+1)/2 entries x Ns x 2)",
                "peak_source": "FP32 FMA: 148 SMs x 128 lanes x 2 flop x max SM clock"}
        extra = {"energy_per_site": sts[-1].e_mean_re / N, "phases_ms": {
            k: statistics.mean(getattr(s, k) for s in sts) for k in ("ms_sample", "ms_grad",
                                                                     "ms_qfm", "ms_solve")}}
    else:
        td = [s.tdvp if kind == "excited" else s for s in sts]
        ms_k = statistics.mean(t.ms_gram for t in td)
        flops = 14.0 * P * (P + 1) / 2 * Ns
        roof = {"bound": "alu", "kernel": "tdvp_gram", "peak": 1.25, "algorithmic":
                "14 FP64 flops per lower-triangle entry of S and sample",
                "peak_source": "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"}
        extra = {"energy_per_site": td[-1].e_mean_re / N,
                 "per_step_ms": {"gram": ms_k, "eig": statistics.mean(t.ms_eig for t in td)}}
        if kind == "excited":
            extra["ess_fraction"] = sts[-1].ess / Ns
    achieved = flops / (ms_k / 1e3) / 1e12
    roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"],
                 "traffic": None, "ms_per_launch": ms_k})
    out = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 sampling, f32/f64 reductions",
           "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "P": P, "samples_per_step": Ns,
                      "l2": "working set below L2 except the sample buffers; not flushed",
                      "parallelism": f"replicas x{ws}"},
           "roofline": roof, "gpu_launches": launches, "clocks": clk.summary(),
           "e2e": None, **extra}
    vmc.vmc_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16split"],
                    help="default: the workload's (bf16split, fp32 for the 1D chain)")
    ap.add_argument("--solver", default=None, choices=["mixed", "tc", "fp64", "cg"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(BATCHED) + sorted(LEARNED) + sorted(TDVP)
                    + sorted(FAMILIES))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain FP32 comparison arm of the default workload")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in BATCHED:
        run_batched(args)
    elif args.workload in LEARNED:
        run_learned(args)
    elif args.workload in TDVP:
        run_tdvp(args)
    elif args.workload in FAMILIES:
        run_family(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
