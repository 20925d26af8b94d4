"""Throughput benchmark of the Lanczos GW hot path on GB300.

One step = one lgw_sigma_c call on the mid-size system (N_v=128, N_c=1024,
N_vc=131072, N_aux=2048, k=200 Lanczos steps with full classical
Gram-Schmidt reorthogonalisation against every stored basis vector -- a
second pass where the norm criterion asks for it -- and 1000 frequencies) for a batch of target states, each
summed over 256 orbitals: start vectors, every Lanczos step, spectral map,
continued fractions on the grid and the QP solve.  Metric: QP states per
second (higher is better), whole job over all ranks.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QP states/sec & Lanczos GEMM TFLOP/s, mixed vs FP64 plain path at 1 meV"
M_PER_TARGET = 256


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), \
            d.get("bf16_tflops_sustained", 1700.0), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                s, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            sm.append(s)
            smax.append(mx)
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = sorted(sm)[len(sm) // 4:] or sm   # drop the idle quarter
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (reported baseline)
# ---------------------------------------------------------------------------
def _oracle_worker(conn, n_vec, k, offset):
    """One oracle process: builds the mid-size system once (untimed), then runs
    the oracle's Lanczos, pole sums and QP solve on its n_vec start vectors
    (summed orbitals offset .. offset + n_vec - 1 of the first target) each
    time the parent sends "run", and returns the monotonic start and end."""
    import gw_inputs
    import oracle as O
    wl = gw_inputs.mid(n_targets=1, k=k)
    wl.M = np.ascontiguousarray(wl.M[:, offset:offset + n_vec])
    wl.m_idx = wl.m_idx[offset:offset + n_vec]
    conn.send("ready")
    while conn.recv() == "run":
        t0 = time.monotonic()
        _, poles, _ = O.sigma_lanczos(wl, k=k)
        O.solve_all_qp(wl, poles)
        conn.send((t0, time.monotonic()))
    conn.close()


def _host_memory_available():
    """Bytes this process may still allocate: MemAvailable, capped by a cgroup
    memory limit if one is set."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    avail = int(ln.split()[1]) * 1024
    except OSError:
        pass
    for lim, use in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                     ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                      "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(lim) as f:
                t = f.read().strip()
            if t == "max":
                continue
            with open(use) as f:
                free = int(t) - int(f.read().strip())
            avail = free if avail is None else min(avail, free)
        except (OSError, ValueError):
            continue
    return avail


class OraclePool:
    """The CPU oracle spread over the host cores: ``procs`` spawned processes,
    each with its own copy of the system and cores // procs BLAS threads,
    each running ``n_vec`` start vectors per step.  A step's time is from the
    first process's start to the last one's end."""

    WORKER_BYTES = 3.5e9     # L (2.1 GB FP64), basis (0.4 GB), temporaries

    def __init__(self, n_vec=1, k=200, procs=0):
        import multiprocessing as mp
        try:
            cores = len(os.sched_getaffinity(0))
        except Exception:
            cores = os.cpu_count() or 1
        if procs <= 0:
            avail = _host_memory_available()
            by_mem = int(0.5 * avail / self.WORKER_BYTES) if avail else 1
            procs = max(1, min(8, cores // 2, by_mem))
        self.procs, self.n_vec, self.k = procs, n_vec, k
        self.threads = max(1, cores // procs)
        self.cores = self.threads * procs
        ctx = mp.get_context("spawn")
        saved = {v: os.environ.get(v) for v in
                 ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = str(self.threads)
        self.conns, self.procs_ = [], []
        try:
            for i in range(procs):
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_oracle_worker, args=(b, n_vec, k, i * n_vec),
                                 daemon=True)
                pr.start()
                self.conns.append(a)
                self.procs_.append(pr)
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        for c in self.conns:
            if not c.poll(900) or c.recv() != "ready":
                self.close()
                raise RuntimeError("oracle worker did not start")

    def step(self):
        """Seconds of one step (every process runs its vectors once)."""
        for c in self.conns:
            c.send("run")
        t = [c.recv() for c in self.conns]
        return max(e for _, e in t) - min(s for s, _ in t)

    def states_per_s(self, seconds):
        return self.procs * self.n_vec / seconds / M_PER_TARGET

    def sample(self, seconds):
        return (f"{self.procs} processes x {self.n_vec} start vectors (summed orbitals "
                f"0..{self.procs * self.n_vec - 1} of one QP state's 256) of the N_vc=131072, "
                f"N_aux=2048 system, k={self.k} CGS2 Lanczos + pole sums + QP, numpy FP64, "
                f"{self.threads} BLAS threads each ({seconds:.1f} s per step); "
                f"states/s = vectors/s / 256")

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except Exception:
                pass
        for pr in self.procs_:
            pr.join(30)
            if pr.is_alive():
                pr.terminate()


def cpu_baseline_leg(args):
    """The oracle on the host cores, one step of the pool (by default half the
    cores' worth of processes, at most 8, one start vector each: about 45 s
    on 16 Grace cores, where host memory bandwidth bounds the scaling)."""
    pool = OraclePool(n_vec=args.ref_vectors, k=args.k, procs=args.ref_procs)
    try:
        dt = pool.step()
    finally:
        pool.close()
    return {"value": pool.states_per_s(dt), "unit": "QP states/s", "cores": pool.cores,
            "kind": "oracle", "sample": pool.sample(dt)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # every step is a bounded sample: two processes of one start vector each
    # (unless --ref-procs says otherwise), so that warm-up plus timed steps
    # end within a few minutes
    pool = OraclePool(n_vec=args.ref_vectors, k=args.k, procs=args.ref_procs or 2)
    try:
        times = []
        for i in range(args.warmup + args.steps):
            dt = pool.step()
            if i >= args.warmup:
                times.append(dt)
    finally:
        pool.close()
    per_step = statistics.mean(times)
    value = pool.states_per_s(per_step)
    line = {
        "metric": METRIC, "value": value, "unit": "QP states/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": _config(args), "gpu_launches": 0,
        "cpu_baseline": {"value": value, "unit": "QP states/s", "cores": pool.cores,
                         "kind": "oracle", "sample": pool.sample(per_step)},
        "e2e": {"value": value, "unit": "QP states/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


GS_SCHEDULE = {
    "dcgs": "delayed classical Gram-Schmidt: one pass over the stored basis per step "
            "(projection of w_j and the delayed update of q_j in the same sweep), second "
            "pass where the norm drops below 1/sqrt(2)",
    "cgs1k": "classical Gram-Schmidt, two passes over the basis per step (dots, update), "
             "second projection where the norm drops below 1/sqrt(2)",
    "cgs2": "classical Gram-Schmidt, always two projections (four passes over the basis)",
    "none": "three-term recurrence only",
}


def _reorth_arith(args):
    if args.precision == "fp64" and args.reorth_arith == "auto":
        a = "fp64"
    else:
        a = {"auto": "split", "split": "split"}.get(args.reorth_arith, args.reorth_arith)
    return {"split": "split48: basis stored as float pairs hi+lo (48 significant bits), "
                     "double-float dot products on the FP32 pipe, FP64 recurrence",
            "split32": "split32: float-only basis, double-float dot products, FP64 recurrence",
            "fp64": "fp64: basis, dots and updates in FP64"}[a]


def _config(args):
    return {"workload": (f"Lanczos GW Sigma_c + QP, N_v=128 N_c=1024 (N_vc=131072) "
                         f"N_aux=2048, k={args.k} {args.reorth.upper()}, {args.tps} targets x "
                         f"256 summed orbitals per step, 1000 frequencies"),
            "n_vc": 131072, "n_aux": 2048, "k": args.k, "targets_per_step": args.tps,
            "start_vectors_per_step": args.tps * M_PER_TARGET, "n_freq": 1000,
            "reorth": args.reorth, "gram_schmidt": GS_SCHEDULE[args.reorth],
            "reorth_arith": _reorth_arith(args), "precision": args.precision,
            "l2": "inputs larger than L2 (Krylov basis ~107 GB, bf16 L 2x0.54 GB)",
            "parallelism": f"replicas x{args.gpus}"}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def _guarded(fn, *a, **kw):
    """Run one comparison leg; a failure is recorded in its place instead of
    ending the benchmark (the headline line is still printed)."""
    try:
        return fn(*a, **kw)
    except Exception as ex:   # noqa: BLE001 - any failure of a side leg
        return {"error": f"{type(ex).__name__}: {ex}"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import gw_inputs
    from paper_2310_20103_gb300 import lgw as L
    from paper_2310_20103_gb300 import replicas as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    solo = rank == 0 and world == 1     # the comparison legs run on one replica only

    wl = gw_inputs.mid(n_targets=32, k=args.k)
    n_t_all = wl.n_t
    stream = torch.cuda.current_stream(dev)
    h = L.lgw_create(local, stream)
    eps_d = torch.from_numpy(wl.eps).to(dev)
    L_d = torch.from_numpy(wl.L).to(dev)
    M_all = torch.from_numpy(wl.M).to(dev)
    omega_d = torch.from_numpy(wl.omega).to(dev)
    m_idx_d = torch.from_numpy(wl.m_idx).to(dev)
    tgt_all = torch.from_numpy(wl.targets).to(dev)
    sysd = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, eps_d, L_d, wl.kernel_factor)
    tps = args.tps
    B_step = tps * M_PER_TARGET

    def options(**kw):
        base = dict(k=args.k, precision=args.precision, reorth=args.reorth, b_sub=B_step,
                    reorth_arith=args.reorth_arith)
        base.update(kw)
        return L.Options(**base)

    opts = options()
    sig = torch.empty(tps, wl.omega.size, 2, dtype=torch.float64, device=dev)
    e = torch.empty(tps, dtype=torch.float64, device=dev)
    z = torch.empty(tps, dtype=torch.float64, device=dev)

    def batch(i):
        ts = torch.tensor(R.targets_for_step(i, rank, world, tps, n_t_all), device=dev)
        return L.Problem(targets=tgt_all[ts].contiguous(), m_idx=m_idx_d, omega=omega_d,
                         delta=wl.delta, M=M_all[ts].contiguous())

    def barrier():
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        L.lgw_sigma_c(h, sysd, batch(i), opts, sig, e, z)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for i in range(args.steps):
        reps.append(L.lgw_sigma_c(h, sysd, batch(args.warmup + i), opts, sig, e, z,
                                  report=True))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = R.max_over_ranks(ms, dev) if world > 1 else ms
    states = tps * args.steps * world
    value = states / (ms_max / 1e3)

    # The comparison legs all run on one batch (the first timed one, 2
    # targets x 256 summed orbitals): the headline result on that batch is
    # the reference for their QP differences.
    cmp_batch = batch(args.warmup)
    cmp_targets = [int(t) for t in wl.targets[R.targets_for_step(args.warmup, rank, world, tps,
                                                                  n_t_all)]]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed_step(hh, ss, o, poly=None):
        """One untimed call (workspace, E4M3 copies, tile tuning), then one
        call timed with CUDA events on the stream; returns (ms, E, Sigma, report)."""
        for rep_i in range(2):
            if rep_i == 1:
                e0.record(stream)
            if poly is None:
                r = L.lgw_sigma_c(hh, ss, cmp_batch, o, sig, e, z, report=rep_i == 1)
            else:
                r = L.lgw_sigma_c_poly(hh, ss, cmp_batch, o, poly[0], poly[1], poly[2], sig, e,
                                       report=rep_i == 1)
            if rep_i == 1:
                e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1), e.cpu().numpy().copy(), sig.cpu().numpy().copy(), r

    legs = {}
    e_head = sig_head = None
    if solo:
        ms_head, e_head, sig_head, _ = timed_step(h, sysd, opts)

        def leg(name, o, note):
            lms, le, lsig, lr = timed_step(h, sysd, o)
            g8 = lr["ms_gemm1"] + lr["ms_gemm2"]
            legs[name] = {"value": tps / (lms / 1e3), "unit": "QP states/s", "ms_per_step": lms,
                          "steps": 1, "what": note,
                          "gemm_tflops": lr["gemm_flops"] / (g8 * 1e-3) / 1e12 if g8 else None,
                          "qp_diff_mev_vs_headline": float(np.abs(le - e_head).max() * 1e3),
                          "sigma_max_diff_mev_vs_headline":
                              float(np.abs(lsig - sig_head).max() * 1e3)}
        if not args.no_variants:
            for name, o, note in [
                    ("cgs1k_two_pass_step", options(reorth="cgs1k"),
                     "two-pass CGS1K (dots, then update) on the same float-pair basis"),
                    ("cgs2_step", options(reorth="cgs2"),
                     "CGS2 (always two passes) on the same float-pair basis"),
                    ("float_basis_step", options(reorth_arith="split32"),
                     "delayed single sweep against a float-only basis (split32)")] + (
                    [("fp8_step", options(precision="fp8"),
                      "E4M3 contractions (kind::f8f6f4) with power-of-two scales"),
                     ("fp8_deq_step", options(precision="fp8_deq"),
                      "E4M3 L widened to FP16 in shared memory, FP16 operands (kind::f16)")]
                    if args.precision == "bf16" else []):
                err = _guarded(leg, name, o, note)
                if err is not None:
                    legs[name] = err
        # the paper's polynomial form (Lanczos on p_g(C) ~ C^1/2, no
        # reorthogonalisation) on the same batch, against the primary result;
        # the library fits p_g on its own estimate of C's spectral interval
        # (x_lo = x_hi = 0)
        if not args.no_poly:
            def poly_leg():
                x_lo, x_hi = L.lgw_spectral_interval(h, sysd, 32)
                poly = {"interval": [x_lo, x_hi], "interval_source":
                        "lgw_spectral_interval: min Delta^2, largest Ritz value of 32 "
                        "FP64 Lanczos steps + its residual", "reorth": "none", "runs": []}
                for g, kp in ((8, 8), (16, 16)):
                    pms, pe, _, rp = timed_step(h, sysd, options(k=kp, reorth="none"),
                                                poly=(g, 0.0, 0.0))
                    poly["runs"].append({"g": g, "k": kp, "value": tps / (pms / 1e3),
                                         "unit": "QP states/s", "ms_per_step": pms,
                                         "gemm_ms": rp["ms_gemm1"] + rp["ms_gemm2"],
                                         "qp_diff_mev_vs_primary": float(
                                             np.abs(pe - e_head).max() * 1e3)})
                return poly
            legs["poly_variant"] = _guarded(poly_leg)

    # --- end to end through the public API with pinned host buffers ---
    eps_h = torch.from_numpy(wl.eps).pin_memory()
    L_h = torch.from_numpy(wl.L).pin_memory()
    M_h = torch.from_numpy(wl.M).pin_memory()
    om_h = torch.from_numpy(wl.omega).pin_memory()
    mi_h = torch.from_numpy(wl.m_idx).pin_memory()
    tg_h = torch.from_numpy(wl.targets).pin_memory()
    sig_h = torch.empty(tps, wl.omega.size, 2, dtype=torch.float64).pin_memory()
    e_h = torch.empty(tps, dtype=torch.float64).pin_memory()
    z_h = torch.empty(tps, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    h2d = d2h = 0
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ts = R.targets_for_step(i, rank, world, tps, n_t_all)
        Mb = M_h[ts].contiguous().pin_memory()
        tb = tg_h[ts].contiguous().pin_memory()
        s2 = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, eps_h, L_h, wl.kernel_factor)
        prob = L.Problem(targets=tb, m_idx=mi_h, omega=om_h, delta=wl.delta, M=Mb)
        L.lgw_sigma_c(h, s2, prob, opts, sig_h, e_h, z_h)
        L.lgw_release_system(s2)
        h2d = (eps_h.numel() + L_h.numel() + Mb.numel() + om_h.numel()) * 8 + \
            (tb.numel() + mi_h.numel()) * 4
        d2h = (sig_h.numel() + e_h.numel() + z_h.numel()) * 8
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_max = R.max_over_ranks(e2e_s, dev) if world > 1 else e2e_s
    e2e_value = tps * e2e_steps * world / e2e_max

    # --- per-kernel breakdown from the timed steps (CUDA events on the stream) ---
    agg = {k: sum(r[k] for r in reps) for k in reps[0] if k.startswith("ms_") or k in (
        "gemm_flops", "reorth_elems", "gpu_launches", "n_second_pass")}
    r0 = reps[0]
    nvc = wl.n_vc
    B = r0["n_vectors"] * args.steps
    kk = args.k
    launches_per_cat = r0["n_sub_batches"] * kk * args.steps
    hbm, bf16_burst, bf16_sus, peak_src = _peaks()
    bytes_, ms_k, kname, tkey, rows_t = _roofline_kernel(args, agg, nvc, B, kk)
    achieved = bytes_ / (ms_k / 1e3) / 1e9
    traffic = _dram_traffic(tkey, rows_t, nvc * B * kk, launches_per_cat)
    gemm_ms = agg["ms_gemm1"] + agg["ms_gemm2"]
    gemm_tflops = agg["gemm_flops"] / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": "QP states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 contractions, f64 recurrence/reorth/CF" if args.precision == "bf16" else "f64",
        "data": "synthetic (seeded stand-in for the Si-cluster workloads)",
        "config": _config(args),
        "gpu_launches": int(agg["gpu_launches"]),
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "QP states/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_src,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram bytes of the same kernel on a 64-vector case, "
                                        "scaled per processed element (profiles/)")
                     if traffic else "no ncu capture of this kernel version",
                     "algorithmic_bytes_per_launch": bytes_ / launches_per_cat,
                     "launches": launches_per_cat,
                     "avg_launch_ms": ms_k / launches_per_cat},
        "gemm": {"tflops": gemm_tflops, "peak_bf16_tflops": bf16_sus,
                 "frac": (gemm_tflops / bf16_sus) if gemm_tflops else None,
                 "ms_gemm1": agg["ms_gemm1"], "ms_gemm2": agg["ms_gemm2"],
                 "splits": r0["gemm1_splits"]},
        "breakdown_ms": {k: agg[k] for k in agg if k.startswith("ms_")},
        "n_second_pass": int(agg["n_second_pass"]),
    }
    line.update(legs)
    if solo:
        line["comparison_batch"] = {"targets": cmp_targets, "summed_orbitals": M_PER_TARGET,
                                    "start_vectors": B_step}
    L.lgw_release_system(sysd)
    L.lgw_destroy(h)
    if solo and not args.no_fp64_compare:
        fl = _guarded(fp64_legs, args, L, wl, eps_d, L_d, cmp_batch, e_head, sig_head, value,
                      dev, stream)
        line.update(fl if "error" not in fl else {"fp64_path": fl})
    del L_d, M_all
    torch.cuda.empty_cache()
    if solo and not args.no_adjoint:
        ha = L.lgw_create(local, stream)
        line["adjoint"] = _guarded(adjoint_leg, L, ha, dev)
        L.lgw_destroy(ha)
    if solo and not args.no_batched:
        hb = L.lgw_create(local, stream)
        line["batched"] = _guarded(batched_leg, L, hb, dev, max_targets=args.batched_targets,
                                   reorth=args.reorth)
        L.lgw_destroy(hb)
    torch.cuda.empty_cache()
    if solo and not args.no_large:
        line["large"] = _guarded(large_leg, L, dev, n_targets=args.large_targets)
    if solo and not args.no_cpu_baseline:
        line["cpu_baseline"] = _guarded(cpu_baseline_leg, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _roofline_kernel(args, agg, nvc, B, k):
    """Algorithmic bytes, CUDA-event time and name of the dominant kernel of
    the timed steps, with the key of its ncu traffic coefficients.  Basis
    row-elements: reorth_elems counts N_vc * sum_j (j+1) per vector (rows
    0..j at step j); the delayed sweep of step j reads rows 0..j-1, one
    fewer per step (every vector runs all k steps here)."""
    rows = agg["reorth_elems"]
    es = float(nvc) * B * k            # element-steps
    split = args.precision != "fp64" and args.reorth_arith in ("auto", "split", "split32")
    lo = args.reorth_arith != "split32"
    if args.reorth == "dcgs" and split:
        rows_d = rows - es
        per_row = 8.0 if lo else 4.0
        # reads: carried vector (8), c_K Delta^1/2 L y (4); writes: basis
        # row j (8 or 4), carried vector (8), bf16 operand (2)
        per_es = 8.0 + 4.0 + per_row + 8.0 + 2.0
        return (per_row * rows_d + per_es * es, agg["ms_dots"],
                "k_sweep_dcgs (delayed single-sweep Gram-Schmidt: double-float Q^T v, "
                "delayed q_j update, w_j)", "k_sweep_dcgs", rows_d)
    if split:   # float-pair basis: hi+lo read by the dots, hi by the update
        by = {
            "update": (4.0 * rows + 16.0 * es, agg["ms_update"],
                       "k_update_split<1> (w -= Q h in FP32 from the hi basis)", None),
            "dots": (8.0 * rows + 28.0 * es, agg["ms_dots"],
                     "k_dots_split<1> (w assembly, alpha axpy, double-float Q^T w)",
                     "k_dots_split"),
        }
    else:
        by = {
            "update": (8.0 * rows + 16.0 * es, agg["ms_update"],
                       "k_update (first Gram-Schmidt update w -= Q h)", None),
            "dots": (8.0 * rows + 24.0 * es, agg["ms_dots"],
                     "k_alpha_axpy (alpha, axpy, first-pass Q^T w)", None),
        }
    dom = max(by, key=lambda x: by[x][1])
    return by[dom] + (rows,)


def _dram_traffic(key, rows, elem_steps, launches):
    """DRAM bytes per launch of the dominant kernel from the ncu coefficients in
    profiles/<key>_traffic.txt (bytes per basis-row element and per
    element-step, fitted on a small case of the same kernel), or None when
    no capture of this kernel exists."""
    if key is None or rows is None:
        return None
    try:
        vals = {}
        with open(os.path.join(ROOT, "profiles", f"{key}_traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 2:
                    vals[parts[0]] = parts[1]
        per_row = float(vals["bytes_per_row_element"])
        per_step = float(vals["bytes_per_element_step"])
    except Exception:
        return None
    return (per_row * rows + per_step * elem_steps) / launches


def fp64_legs(args, L, wl, eps_d, L_d, prob, e_head, sig_head, value_head, dev, stream):
    """On the comparison batch (the same 512 start vectors, k, frequencies),
    in a fresh handle so that no other Krylov basis shares the device:
      cgs2_fp64_basis_step  BF16 contractions, CGS2 against an FP64 basis
                            (every product and sum on the FP64 pipe);
      fp64_path             the plain FP64 GPU path: FP64 CUDA-core
                            contractions, FP64 basis, CGS1K; its QP energies
                            against the headline's (the 1 meV criterion).
    mixed_over_fp64 = headline states/s over the FP64 path's states/s."""
    import torch
    tps = args.tps
    h = L.lgw_create(dev.index if dev.index is not None else 0, stream)
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, eps_d, L_d, wl.kernel_factor)
    sig = torch.empty(tps, wl.omega.size, 2, dtype=torch.float64, device=dev)
    e = torch.empty(tps, dtype=torch.float64, device=dev)
    out = {}
    runs = [("cgs2_fp64_basis_step", "bf16", "cgs2", args.k, 1,
             "BF16 contractions, CGS2 against an FP64 Krylov basis (FP64 dots and updates)"),
            ("fp64_path", "fp64", "cgs1k", args.fp64_k, 0,
             "plain FP64 path: FP64 CUDA-core contractions, FP64 basis, CGS1K")]
    for name, prec, reorth, kk, warm, note in runs:
        o = L.Options(k=kk, precision=prec, reorth=reorth, b_sub=tps * M_PER_TARGET,
                      reorth_arith="fp64")
        if warm:
            L.lgw_sigma_c(h, s, prob, o, sig, e)
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = L.lgw_sigma_c(h, s, prob, o, sig, e, report=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        gms = rep["ms_gemm1"] + rep["ms_gemm2"]
        d = {"value": tps / dt, "unit": "QP states/s", "seconds": dt, "k": kk, "what": note,
             "gemm_tflops": rep["gemm_flops"] / (gms * 1e-3) / 1e12 if gms else None,
             "breakdown_ms": {x: round(v, 1) for x, v in rep.items() if x.startswith("ms_")}}
        if kk == args.k:
            d["qp_diff_mev_vs_headline"] = float(np.abs(e.cpu().numpy() - e_head).max() * 1e3)
            d["sigma_max_diff_mev_vs_headline"] = float(
                np.abs(sig.cpu().numpy() - sig_head).max() * 1e3)
        out[name] = d
    fp = out["fp64_path"]
    fp["sample"] = (f"the headline's comparison batch: {tps} targets x 256 summed orbitals "
                    f"({tps * M_PER_TARGET} start vectors), k {fp['k']}, one call")
    if fp["k"] == args.k:
        fp["mixed_over_fp64"] = value_head / fp["value"]
    L.lgw_release_system(s)
    L.lgw_destroy(h)
    return out


def adjoint_leg(L, h, dev, n_targets=8, compare=True):
    """Differentiation workload (N_v 64, N_c 512, N_aux 1024, 8 targets x 128
    summed orbitals, k 120): time of the BF16 forward and of the backward
    (dE/dL, dE/deps), and on one target x 128 orbitals the BF16 gradient
    against the FP64 gradient (relative to the largest entry)."""
    import torch
    import gw_inputs as gi

    def tt(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    def one(wl, prec, reps):
        s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, tt(wl.eps), tt(wl.L))
        prob = L.Problem(targets=tt(wl.targets), m_idx=tt(wl.m_idx), omega=tt(wl.omega),
                         delta=wl.delta, M=tt(wl.M))
        o = L.Options(k=wl.k, precision=prec, reorth="cgs2")
        sg = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=dev)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=dev)
        dL = torch.empty(wl.n_vc, wl.n_aux, dtype=torch.float64, device=dev)
        de = torch.empty(wl.n_v + wl.n_c, dtype=torch.float64, device=dev)
        dE = tt(np.linspace(-1.0, 1.0, wl.n_t))
        tf, tb = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.lgw_sigma_c(h, s, prob, o, sg, e)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            L.lgw_sigma_c_backward(h, s, prob, o, dE, dL, de)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            tf.append(t1 - t0)
            tb.append(t2 - t1)
        L.lgw_release_system(s)
        return min(tf), min(tb), dL.cpu().numpy(), de.cpu().numpy()

    wl = gi.differentiation(n_targets=n_targets)
    f16, b16, _, _ = one(wl, "bf16", 2)
    out = {"workload": f"differentiation: N_v 64, N_c 512 (N_vc 32768), N_aux 1024, "
                       f"{n_targets} targets x 128 summed orbitals (B {128 * n_targets}), "
                       f"k 120, CGS2, BF16",
           "forward_s": f16, "backward_s": b16, "backward_over_forward": b16 / f16}
    if not compare:
        return out
    out["exact_short_k"] = _guarded(exact_adjoint_leg, L, h, dev)
    sub = gi.differentiation(n_targets=1, n_m=128)
    _, bs16, dl16, de16 = one(sub, "bf16", 1)
    f64, b64, dl64, de64 = one(sub, "fp64", 1)
    out["gradient_vs_fp64"] = {
                "sample": "1 target x 128 summed orbitals",
                "dL_rel": float(np.abs(dl16 - dl64).max() / np.abs(dl64).max()),
                "deps_rel": float(np.abs(de16 - de64).max() / np.abs(de64).max()),
                "fp64_forward_s": f64, "fp64_backward_s": b64, "bf16_backward_s": bs16}
    return out


def exact_adjoint_leg(L, h, dev, n_m=128):
    """Exact k-step adjoint (FP64, no reorthogonalisation, reverse mode with
    Krylov checkpoints) at the paper's short depths on the differentiation
    shapes, 1 target x n_m summed orbitals: the plain recurrence at k 8 and
    the polynomial form at g 8, k 8 (interval from lgw_spectral_interval),
    forward and backward seconds (best of 2)."""
    import torch
    import gw_inputs as gi

    def tt(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    wl = gi.differentiation(n_targets=1, n_m=n_m, k=8)
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, tt(wl.eps), tt(wl.L))
    try:
        prob = L.Problem(targets=tt(wl.targets), m_idx=tt(wl.m_idx), omega=tt(wl.omega),
                         delta=wl.delta, M=tt(wl.M))
        o = L.Options(k=8, precision="fp64", reorth="none")
        lo, hi = L.lgw_spectral_interval(h, s, 32)
        sg = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=dev)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=dev)
        dL = torch.empty(wl.n_vc, wl.n_aux, dtype=torch.float64, device=dev)
        de = torch.empty(wl.n_v + wl.n_c, dtype=torch.float64, device=dev)
        dE = tt(np.ones(wl.n_t))

        def timed(fn):
            best = 1e30
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            return best

        out = {"workload": f"N_vc 32768, N_aux 1024, 1 target x {n_m} summed orbitals, k 8, "
                           f"FP64, no reorthogonalisation, checkpoints every 16 steps"}
        f = timed(lambda: L.lgw_sigma_c(h, s, prob, o, sg, e))
        b = timed(lambda: L.lgw_sigma_c_backward(h, s, prob, o, dE, dL, de))
        out["plain"] = {"forward_s": f, "backward_s": b, "backward_over_forward": b / f}
        f = timed(lambda: L.lgw_sigma_c_poly(h, s, prob, o, 8, lo, hi, sg, e))
        b = timed(lambda: L.lgw_sigma_c_poly_backward(h, s, prob, o, 8, lo, hi, dE, dL, de))
        out["poly_g8"] = {"forward_s": f, "backward_s": b, "backward_over_forward": b / f}
        return out
    finally:
        L.lgw_release_system(s)


def batched_leg(L, h, dev, max_targets=64, k=150, reorth="dcgs", reps=1):
    """Batched-uneven workload: the 16 systems (N_vc 4975..62392, N_aux
    512..2048, seed 100+i), min(drawn, max_targets) targets each (the drawn
    8..64 by default) x up to 256 summed orbitals, k 150, BF16, one
    lgw_sigma_c_batched call per step; eager launches vs CUDA-graph replay
    (graphs captured in the untimed call).  QP states/s = targets of all
    systems / wall time of a call."""
    import torch
    import gw_inputs as gi

    def tt(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    wls = [gi.batched_uneven(i, k=k, max_targets=max_targets) for i in range(16)]
    systems = [L.lgw_prepare_system(h, w.n_v, w.n_c, w.n_aux, tt(w.eps), tt(w.L)) for w in wls]
    probs = [L.Problem(targets=tt(w.targets), m_idx=tt(w.m_idx), omega=tt(w.omega),
                       delta=w.delta, M=tt(w.M)) for w in wls]
    sig = [torch.empty(w.n_t, w.omega.size, 2, dtype=torch.float64, device=dev) for w in wls]
    e = [torch.empty(w.n_t, dtype=torch.float64, device=dev) for w in wls]
    n_t = sum(w.n_t for w in wls)
    out = {"workload": f"batched-uneven: 16 systems, N_vc {min(w.n_vc for w in wls)}.."
                       f"{max(w.n_vc for w in wls)}, N_aux {min(w.n_aux for w in wls)}.."
                       f"{max(w.n_aux for w in wls)}, {n_t} targets, "
                       f"{sum(w.n_t * w.n_m for w in wls)} start vectors, k {k}, BF16, "
                       f"{reorth.upper()}",
           "unit": "QP states/s"}
    res = {}
    for g in (0, 1):
        o = L.Options(k=k, precision="bf16", reorth=reorth, use_graph=g)
        L.lgw_sigma_c_batched(h, systems, probs, o, sig, e)
        torch.cuda.synchronize()
        ts = []
        launches = 0
        for _ in range(reps):
            t0 = time.perf_counter()
            rep = L.lgw_sigma_c_batched(h, systems, probs, o, sig, e, report=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            launches = rep["gpu_launches"]
        res[g] = (min(ts), [x.cpu().numpy() for x in e], launches)
    for s in systems:
        L.lgw_release_system(s)
    out["eager"] = {"value": n_t / res[0][0], "seconds": res[0][0], "gpu_launches": res[0][2]}
    out["graph"] = {"value": n_t / res[1][0], "seconds": res[1][0], "gpu_launches": res[1][2]}
    out["graph_over_eager"] = res[0][0] / res[1][0]
    out["graph_equals_eager"] = all(np.array_equal(a, b) for a, b in zip(res[0][1], res[1][1]))
    return out


def large_leg(L, dev, n_targets=2, k=300):
    """Large cluster-sized system (N_vc 1.6M, N_aux 8192), n_targets x 1024
    summed orbitals in one sub-batch, k 300 without reorthogonalisation,
    2000 frequencies: QP states/s with E4M3 contractions, with E4M3 L widened
    to FP16 in shared memory and with BF16 contractions, and the differences
    of E_qp and Sigma from the BF16 run in meV.  L (105 GB FP64)
    is drawn on the device; the system keeps the BF16 and E4M3 copies only
    (LGW_SYS_NO_FP64), so the FP64 copy is freed before the runs."""
    import torch
    import gw_inputs as gi

    def tt(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    wl, sigma_L = gi.large_cluster(n_targets=n_targets, k=k)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    Ld = torch.randn(wl.n_v * wl.n_c, wl.n_aux, dtype=torch.float64, device=dev, generator=g)
    Ld.mul_(sigma_L)
    h = L.lgw_create(0)
    t0 = time.perf_counter()
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, tt(wl.eps), Ld,
                             flags=L.SYS_NO_FP64 | L.SYS_FP8)
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    del Ld
    torch.cuda.empty_cache()
    prob = L.Problem(targets=tt(wl.targets), m_idx=tt(wl.m_idx), omega=tt(wl.omega),
                     delta=wl.delta, M=tt(wl.M))
    B = wl.n_t * wl.n_m
    out = {"workload": f"large cluster: N_v 400, N_c 4000 (N_vc 1.6M), N_aux 8192, "
                       f"{wl.n_t} targets x {wl.n_m} summed orbitals (B {B}, one sub-batch), "
                       f"k {k}, no reorthogonalisation, 2000 frequencies",
           "data": "L drawn on the device (torch Philox, seed 5), eps and M numpy seed 5",
           "prepare_s": t_prep, "unit": "QP states/s"}
    res = {}
    for prec in ("fp8", "fp8_deq", "bf16"):
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=dev)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=dev)
        warm = L.Options(k=2, precision=prec, reorth="none", b_sub=B)
        L.lgw_sigma_c(h, s, prob, warm, sig, e)
        torch.cuda.synchronize()
        o = L.Options(k=k, precision=prec, reorth="none", b_sub=B)
        t0 = time.perf_counter()
        rep = L.lgw_sigma_c(h, s, prob, o, sig, e, report=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        gms = rep["ms_gemm1"] + rep["ms_gemm2"]
        res[prec] = (sig.cpu().numpy(), e.cpu().numpy())
        out[prec] = {"value": wl.n_t / dt, "seconds": dt,
                     "gemm_tflops": rep["gemm_flops"] / (gms * 1e-3) / 1e12 if gms else None,
                     "ms_gemm1": rep["ms_gemm1"], "ms_gemm2": rep["ms_gemm2"],
                     "ms_total": rep["ms_total"], "k_min": rep["k_min"],
                     "breakdown_ms": {kk: round(v, 1) for kk, v in rep.items()
                                      if kk.startswith("ms_")}}
    out["qp_diff_mev_fp8_vs_bf16"] = float(np.abs(res["fp8"][1] - res["bf16"][1]).max() * 1e3)
    out["sigma_max_diff_mev_fp8_vs_bf16"] = float(np.abs(res["fp8"][0] - res["bf16"][0]).max()
                                                  * 1e3)
    out["qp_diff_mev_fp8_deq_vs_bf16"] = float(np.abs(res["fp8_deq"][1] - res["bf16"][1]).max()
                                               * 1e3)
    out["sigma_max_diff_mev_fp8_deq_vs_bf16"] = float(
        np.abs(res["fp8_deq"][0] - res["bf16"][0]).max() * 1e3)
    out["sigma_scale_mev"] = float(np.abs(res["bf16"][0]).max() * 1e3)
    L.lgw_release_system(s)
    L.lgw_destroy(h)
    return out


def profile_case(prec="bf16", reorth="dcgs", n_vec=64, k=48):
    """The small case the kernel profiles are taken on: the mid-size system
    (N_vc 131072, N_aux 2048), n_vec start vectors (HOMO-15 and on, 256
    summed orbitals each; 64 by default), k steps (48 by default), one
    lgw_sigma_c call with a report.  The default Krylov basis is about 3 GB,
    larger than L2; n_vec 512 with k 4 gives the benchmark's contraction
    shapes on a 2.7 GB basis."""
    import torch
    sys.path.insert(0, ROOT)
    import gw_inputs as gi
    from paper_2310_20103_gb300 import lgw as L

    def tt(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")

    n_t = max(1, (n_vec + 255) // 256)
    n_m = min(256, n_vec)
    wl = gi.mid(n_targets=n_t, k=k)
    h = L.lgw_create(0)
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, tt(wl.eps), tt(wl.L))
    prob = L.Problem(targets=tt(wl.targets), m_idx=tt(wl.m_idx[:n_m]), omega=tt(wl.omega),
                     delta=wl.delta, M=tt(wl.M[:, :n_m]))
    sig = torch.empty(n_t, wl.omega.size, 2, dtype=torch.float64, device="cuda:0")
    e = torch.empty(n_t, dtype=torch.float64, device="cuda:0")
    opts = L.Options(k=k, precision=prec, reorth=reorth, b_sub=n_t * n_m)
    # the first call makes the workspace and tunes the contraction tiles; the
    # second, inside the NVTX range "lgw_profile", is the one to capture
    # (ncu --nvtx --nvtx-include "lgw_profile/")
    L.lgw_sigma_c(h, s, prob, opts, sig, e)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("lgw_profile")
    rep = L.lgw_sigma_c(h, s, prob, opts, sig, e, report=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({kk: (round(v, 3) if isinstance(v, float) else v) for kk, v in rep.items()}),
          flush=True)
    L.lgw_release_system(s)
    L.lgw_destroy(h)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lgw", choices=["lgw", "reference"])
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--tps", type=int, default=2, help="target states per step")
    ap.add_argument("--reorth", default="dcgs", choices=["dcgs", "cgs2", "cgs1k", "none"])
    ap.add_argument("--reorth-arith", default="auto",
                    choices=["auto", "split", "split32", "fp64"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp64-k", type=int, default=200,
                    help="Lanczos steps of the FP64-path leg (the headline's k for a "
                         "like-for-like ratio)")
    ap.add_argument("--ref-vectors", type=int, default=1,
                    help="start vectors per oracle process and step")
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="oracle processes (0: cpu_baseline half the cores, at most 8, "
                         "within memory; the reference arm 2)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the one-step variant legs (CGS1K, CGS2, float basis, E4M3)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-poly", action="store_true")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint leg (differentiation workload) and print it")
    ap.add_argument("--adjoint-targets", type=int, default=8)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched-uneven leg and print it")
    ap.add_argument("--batched-targets", type=int, default=64)
    ap.add_argument("--large-only", action="store_true",
                    help="run only the large cluster-sized leg (about 2 minutes, ~240 GB)")
    ap.add_argument("--large-targets", type=int, default=2)
    ap.add_argument("--profile-case", action="store_true",
                    help="one small call for kernel profiles (mid-size system, 64 start "
                         "vectors, k 48, CGS1K; about 3 GB on the device) and its report")
    ap.add_argument("--profile-precision", default="bf16",
                    choices=["bf16", "fp8", "fp8_deq", "fp64"])
    ap.add_argument("--profile-reorth", default="dcgs", choices=["dcgs", "cgs1k", "cgs2", "none"])
    ap.add_argument("--profile-vectors", type=int, default=64)
    ap.add_argument("--profile-k", type=int, default=48)
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_precision, args.profile_reorth, args.profile_vectors,
                     args.profile_k)
        return
    if args.adjoint_only:
        import torch
        sys.path.insert(0, ROOT)
        from paper_2310_20103_gb300 import lgw as L
        h = L.lgw_create(0)
        out = adjoint_leg(L, h, "cuda:0", n_targets=args.adjoint_targets,
                          compare=args.adjoint_targets == 8)
        L.lgw_destroy(h)
        print(json.dumps({"adjoint": out}), flush=True)
        return
    if args.large_only:
        import torch
        sys.path.insert(0, ROOT)
        from paper_2310_20103_gb300 import lgw as L
        print(json.dumps({"large": large_leg(L, "cuda:0", n_targets=args.large_targets)}),
              flush=True)
        return
    if args.batched_only:
        import torch
        sys.path.insert(0, ROOT)
        from paper_2310_20103_gb300 import lgw as L
        h = L.lgw_create(0)
        out = batched_leg(L, h, "cuda:0", max_targets=args.batched_targets, reorth=args.reorth)
        L.lgw_destroy(h)
        print(json.dumps({"batched": out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
