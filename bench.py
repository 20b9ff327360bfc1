"""Benchmark of the QR-CTMRG hot path on B300: iterations per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision split|fp64]
                    [--workload d2_D6_chi144] [--impl ours|reference]

One step is one QR-CTMRG iteration of the library (reduced corner C T, QR,
T' = Q^T (T a) Q, corner update from (T', R, Q), symmetrise/normalise; the
corner-spectrum convergence test runs every ``check_every`` steps and its
8-byte result is read back each time).  The timed steps run on resident
device buffers after W warm-up steps; the energy per site and the
energy-gradient time are measured after the timed region and reported beside
the iteration rate.  With --gpus N > 1 (torchrun) every rank runs an
independent replica of the same workload (no data-path collective) and the
value is the sum of the replicas' iteration rates (weak scaling).

``--impl reference`` times the plain FP64 CPU oracle (the checker the GPU
path is compared against) on the host cores, one oracle QR-CTMRG iteration
per step, on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qrctm_inputs as qi  # noqa: E402

METRIC = "QR-CTMRG iterations/s (d=2, D=6, chi=144)"
UNIT = "iter/s"


def algorithmic_flops(d, D, chi):
    """Per-phase algorithmic flops of one QR-CTMRG iteration (split layers).

    ct = C T: 2 chi^3 D^2; QR of the (chi D^2) x chi corner: factorisation
    plus explicit Q, 2 (2 m n^2 - 2 n^3 / 3); X1 = Q^T T: 2 chi^3 D^4; ket and
    bra absorption: 2 x 2 chi^2 d D^6; T' = X2 Q: 2 chi^3 D^4; corner update:
    4 chi^3 D^2."""
    D2 = D * D
    m, n = chi * D2, chi
    return {
        "ct": 2.0 * chi ** 3 * D2,
        "qr": 2.0 * (2.0 * m * n * n - 2.0 * n ** 3 / 3.0),
        "x1": 2.0 * chi ** 3 * D2 * D2,
        "absorb": 4.0 * chi ** 2 * d * D2 ** 3,
        "project": 2.0 * chi ** 3 * D2 * D2,
        "corner": 4.0 * chi ** 3 * D2,
    }


FP64_PEAK_TFLOPS = 1.25


def fp32_simt_peak():
    return 148 * 128 * 2 * 2.032e9 / 1e12


def tf32_peak_sustained(peaks):
    """Dense TF32 peak for a kernel inside a long step: the measured
    sustained BF16 rate scaled by the nominal TF32/BF16 ratio 1.1/2.25."""
    if "bf16_tflops_sustained" in peaks:
        return (peaks["bf16_tflops_sustained"] * 1.1 / 2.25,
                "tf32 = measured sustained bf16 x 1.1/2.25")
    return 1400.0 * 1.1 / 2.25, "tf32 = fallback sustained bf16 1.4 PFLOP/s x 1.1/2.25"


def panel_flops(d, D, chi, m=None):
    """Average flops of one FP64 panel launch: Householder factorisation of
    an mr x nb block, 2 mr nb^2 - 2 nb^3 / 3, over the panels of the
    m x chi reduced corner (m = chi D^2 unless given; nb = 32)."""
    m, n = (chi * D * D if m is None else m), chi
    tot, cnt = 0.0, 0
    for j0 in range(0, n, 32):
        nb = min(32, n - j0)
        mr = m - j0
        tot += 2.0 * mr * nb * nb - 2.0 * nb ** 3 / 3.0
        cnt += 1
    return tot / cnt


def load_traffic(precision, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu capture summary of this precision and workload,
    keyed by step phase (first column), with the name of the kernel the
    capture measured (the rest of the line); empty when there is none."""
    out = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", f"traffic_{precision}_{workload}.txt")):
            parts = line.split()
            if len(parts) >= 2 and not line.startswith("#"):
                out[parts[0]] = (float(parts[1]), " ".join(parts[2:]))
    except OSError:
        pass
    return out


def traffic_of(traffic, phase, kernel):
    """Captured bytes of a phase, or None when the capture measured another
    kernel than the one the row names (a capture older than the kernel)."""
    t = traffic.get(phase)
    if t is None:
        return None
    nbytes, name = t
    return nbytes if name.startswith(kernel.split(" (")[0]) else None


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=self.out,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.out.close()
        except Exception:
            pass

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_sample(w, n_steps):
    """Oracle QR-CTMRG iterations on the host (bounded sample).  The per-step
    cost does not depend on the values, so a symmetric random environment of
    the workload's shape stands in for the converged one."""
    from oracle import qrctm_oracle as o
    d, D, chi = w["d"], w["D"], w["chi"]
    A = o.normalized_input(qi.raw_tensor(d, D, w["seed"], w["decay"], w["bias"]))
    rng = np.random.default_rng(1)
    C, T = o.sym_norm(rng.standard_normal((chi, chi)), rng.standard_normal((chi, D * D, chi)))
    layers = "split" if 2 * d < D * D else "double"
    times = []
    for _ in range(n_steps):
        t0 = time.perf_counter()
        C, T = o.qr_step(C, T, A, layers)
        times.append(time.perf_counter() - t0)
    return times, layers


def oracle_sample_threads(workload, n_steps, threads):
    """oracle_sample in a child process whose BLAS pools have `threads`
    threads; returns {value, unit, cores} or {unavailable}."""
    import subprocess
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample-only",
                            "--workload", workload, "--cpu-sample", str(n_steps)],
                           env=env, capture_output=True, text=True, timeout=600)
        out = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": out["value"], "unit": UNIT, "cores": out["cores"]}
    except Exception as exc:
        return {"unavailable": str(exc)[:160]}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (the job's time) when running under
    torch.distributed, else ms."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps, world, ms):
    """Whole-job iterations/s: every rank runs `steps` iterations of its own
    replica (weak scaling), timed by the slowest rank."""
    return world * steps / (ms / 1e3)


def converge(ctx, tol, max_iter, floor=False, window=100):
    """Iterate until the spectrum change is below tol; with floor, also stop
    once it has not decreased by 2% over 3 windows (the precision floor).
    Returns (iterations, last change, stopped at the floor)."""
    its, best, best_at = 0, float("inf"), 0
    dl = float("inf")
    while its < max_iter:
        n, dl = ctx.run_to_convergence(tol=tol, max_iter=min(window, max_iter - its))
        its += n
        if dl < tol:
            return its, dl, False
        if dl < 0.98 * best:
            best, best_at = dl, its
        elif floor and its - best_at >= 3 * window:
            return its, dl, True
    return its, dl, False


def timed_region(q, one_step, steps, dist, local):
    """Exactly `steps` calls of one_step between CUDA events on the current
    stream, with a barrier and a device synchronisation on both sides, clocks
    sampled meanwhile.  Returns (ms of the slowest rank, kernels launched,
    clock summary)."""
    import torch
    stream = torch.cuda.current_stream()
    launches0 = q.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = local
    with ClockSampler(gpu_id) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for i in range(steps):
            one_step(i)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if dist is not None:
            dist.barrier()
    launches = q.kernel_launches() - launches0
    return max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda"), launches, clk.summary()


def phase_profile(ctx, one_step, steps):
    """Per-phase device times from CUDA events around each phase, on a pass
    after the timed one (the events are not part of the timed region).
    Returns ({phase: (ms, count)}, ms of the pass)."""
    import torch
    stream = torch.cuda.current_stream()
    ctx.set_profiling(True)
    ctx.phase_times()                                 # reset accumulators
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for i in range(steps):
        one_step(i)
    pe1.record(stream)
    torch.cuda.synchronize()
    prof_ms = pe0.elapsed_time(pe1)
    phases = ctx.phase_times()
    ctx.set_profiling(False)
    return phases, prof_ms


def tc_kernel_name(N, K, pre=0, M=0):
    """Name of the tensor-core kernel instance the engine launches for an
    M x N, K-deep product (the tile choice of gemm_tc); pre = 1 when B
    comes pre-split, 2 when both operands do."""
    if pre == 2 and N > 192 and K < 512 and ((M + 127) // 128) * ((N + 127) // 128) >= 296:
        return "tc_tf32x3_kernel<128, 2, 2>"
    if N <= 32:
        bn = (32, 2)
    elif N <= 64:
        bn = (64, 2)
    elif N <= 96:
        bn = (96, 2)
    elif N <= 128:
        bn = (64, 2)
    elif N <= 144:
        bn = (144, 1)
    elif N <= 192 or K >= 512:
        bn = (192, 1)
    else:
        bn = (96, 2)
    return f"tc_tf32x3_kernel<{bn[0]}, {bn[1]}, {pre}>"


def roofline_rows(kernels, phases, prof_ms, traffic):
    """One roofline entry per (phase -> single kernel): algorithmic flops per
    launch over its average CUDA-event duration."""
    rows = {}
    for ph, (kname, flops, bound_k, peak_k, note_k) in kernels.items():
        ms_k, n_k = phases[ph]
        if n_k == 0:
            continue
        avg = ms_k / n_k / 1e3
        ach = flops / avg / 1e12
        rows[ph] = {"kernel": kname, "bound": bound_k, "achieved": ach, "peak": peak_k,
                    "unit": "TFLOP/s", "frac": ach / peak_k, "avg_launch_ms": avg * 1e3,
                    "launches": n_k, "share_of_step": ms_k / prof_ms,
                    "algorithmic_flops_per_launch": flops, "peak_source": note_k,
                    "traffic": traffic_of(traffic, ph, kname)}
    return rows


def onsager_ln_kappa(beta, n=2048):
    """Exact -beta f of the square-lattice Ising model (Onsager), midpoint
    rule on the periodic square; reported beside the Ising workload."""
    t = 2 * np.pi * (np.arange(n) + 0.5) / n
    c = np.cos(t)
    arg = np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c[:, None] + c[None, :])
    return float(np.log(2.0) + 0.5 * np.mean(np.log(arg)))


def oracle_network_sample(w, n_steps):
    """Oracle QR-CTMRG iterations on a classical network (bounded sample) from
    a random symmetric environment of the workload's shape."""
    from oracle import qrctm_oracle as o
    a, _, _ = qi.network_input(w["model"], w["q"], w["beta"])
    chi, b = w["chi"], w["q"]
    rng = np.random.default_rng(1)
    C, T = o.sym_norm(rng.standard_normal((chi, chi)), rng.standard_normal((chi, b, chi)))
    times = []
    for _ in range(n_steps):
        t0 = time.perf_counter()
        C, T = o.qr_step(C, T, a, "network")
        times.append(time.perf_counter() - t0)
    return times


def bench_network(args, w, q, dist, world, rank, local):
    """Classical network fed directly (Discussion: classical partition
    functions): QR-CTMRG (or the standard step) iterations/s, FP64."""
    import torch
    chi, b = w["chi"], w["q"]
    a_h, aobs_h, v_h = qi.network_input(w["model"], w["q"], w["beta"])
    a = torch.tensor(a_h, dtype=torch.float64, device="cuda")
    a_obs = torch.tensor(aobs_h, dtype=torch.float64, device="cuda")
    v = torch.tensor(v_h, dtype=torch.float64, device="cuda") if w["fixed"] else None
    ce = args.check_every
    ctx = q.QRCTM(1, b, chi, layers="network", check_every=ce, method=args.method)
    ctx.init_env_network(a, v)

    def one_step(i):
        ctx.step(1, want_delta=(i % ce == ce - 1))

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    ms, launches, clocks = timed_region(q, one_step, args.steps, dist, local)
    value = job_rate(args.steps, world, ms)
    phases, prof_ms = phase_profile(ctx, one_step, max(ce, min(args.steps, 10 * ce)))
    m = chi * b
    fp64_note = "fp64 nominal 1.25 TFLOP/s (CUDA-core FP64 pipe)"
    kernels = {
        "qr_panel": ("qr_panel_kernel", panel_flops(1, 1, chi, m), "alu", FP64_PEAK_TFLOPS,
                     fp64_note),
        "x1": ("gemm_f64_kernel", 2.0 * chi ** 3 * b * b, "alu", FP64_PEAK_TFLOPS, fp64_note),
        "absorb": ("gemm_f64_kernel", 2.0 * chi ** 2 * b ** 4, "alu", FP64_PEAK_TFLOPS, fp64_note),
        "project": ("gemm_f64_kernel", 2.0 * chi ** 3 * b * b, "alu", FP64_PEAK_TFLOPS,
                    fp64_note),
    }
    if args.method == "eigen":
        kernels.pop("qr_panel")
    rows = roofline_rows(kernels, phases, prof_ms, {})
    dom = max(rows, key=lambda k: rows[k]["share_of_step"])
    share = {k: round(phases[k][0] / prof_ms, 4) for k in ("ct", "qr", "x1", "absorb", "project",
                                                      "corner", "symnorm", "spectrum",
                                                      "qr_panel")}
    # e2e through the public API from pinned host buffers: per step (a, C, T)
    # in, re-initialise from them, one iteration with its convergence test,
    # (C, T) out
    C_d, T_d, _ = ctx.get_env(spectrum=False)
    ha, hC, hT = a.cpu().pin_memory(), C_d.cpu().pin_memory(), T_d.cpu().pin_memory()
    da, dC, dT = torch.empty_like(a), torch.empty_like(C_d), torch.empty_like(T_d)
    oC, oT = torch.empty_like(hC).pin_memory(), torch.empty_like(hT).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        da.copy_(ha, non_blocking=True)
        dC.copy_(hC, non_blocking=True)
        dT.copy_(hT, non_blocking=True)
        ctx.init_env_network(da, None, dC, dT)
        ctx.step(1, want_delta=True)
        Cn, Tn, _ = ctx.get_env(spectrum=False)
        oC.copy_(Cn, non_blocking=True)
        oT.copy_(Tn, non_blocking=True)
        torch.cuda.synchronize()
        # the result becomes the next step's pinned input: swap the buffers
        hC, oC = oC, hC
        hT, oT = oT, hT
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    h2d = (ha.numel() + hC.numel() + hT.numel()) * 8
    d2h = (oC.numel() + oT.numel()) * 8 + 8
    extras = {}
    if not args.no_extras:
        cctx = q.QRCTM(1, b, chi, layers="network", check_every=ce, method=args.method)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cctx.init_env_network(a, v)
        its, dl, _ = converge(cctx, args.conv_tol or 1e-10, 4000)
        torch.cuda.synchronize()
        extras["time_to_converged_s"] = time.perf_counter() - t0
        extras["converged_iterations"] = its
        extras["converged_delta"] = dl
        t0 = time.perf_counter()
        lk, mo = cctx.network_observables(a_obs)
        extras["observables_ms"] = 1e3 * (time.perf_counter() - t0)
        extras["ln_kappa"] = lk
        extras["observable"] = mo
        if w["model"] == "ising":
            extras["ln_kappa_minus_onsager"] = lk - onsager_ln_kappa(w["beta"])
        cctx.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times = oracle_network_sample(w, args.cpu_sample)
        cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": cpu_threads(),
               "kind": "oracle",
               "sample": f"{len(times)} oracle QR-CTMRG iterations on the network tensor "
                         f"(NumPy FP64, bond {b}, chi={chi}) from a random symmetric environment"}
    if rank == 0:
        name = "QR-CTMRG" if args.method == "qr" else "standard C4v CTMRG (eigendecomposition)"
        line = {
            "metric": f"{name} iterations/s ({args.workload}, classical network)",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "model": w["model"], "q": w["q"],
                       "beta": w["beta"], "chi": chi, "bond": b, "method": args.method,
                       "layers": "network", "check_every": ce,
                       "parallelism": f"replicas{world}",
                       "l2": "per-step intermediates "
                             f"{(chi * b) ** 2 * 8 / 1e6:.1f} MB (X1); L2 not flushed"},
            "roofline": rows[dom],
            "roofline_kernels": rows,
            "phase_share": share,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "convergence": extras,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


# k of the tracked steps per D in the paper's timing of optimisation steps
# (Fig. 3(b): chi = 5 D^2, k = 10, 12, 14, 16, 20, 24 for D = 2..7)
PAPER_K = {2: 10, 3: 12, 4: 14, 5: 16, 6: 20, 7: 24}


def opt_step_rate(q, ctx, A, C, T, k, J2, steps, warmup, dist, local, grad):
    """Optimisation steps/s: one step = the environment of the previous point
    handed back in, two untracked QR-CTMRG steps, then the energy and its
    gradient through k tracked steps (the unit of Fig. 3(b))."""
    import torch

    def one_step(i):
        ctx.init_env(A, C, T)
        ctx.step(2, want_delta=False)
        ctx.energy_grad(1.0, J2, mode="unroll", k_unroll=k, grad=grad)

    for i in range(warmup):
        one_step(i)
    torch.cuda.synchronize()
    return timed_region(q, one_step, steps, dist, local)


def bench_opt(args, q, dist, world, rank, local):
    """Time per variational optimisation step (Automatic differentiation
    paragraph, Fig. 3(b)): the paper's unit through the public API, and the
    L-BFGS loop (qrctm_optimize) per accepted step."""
    import torch
    J2 = args.j2
    if args.mode == "opt":
        w = qi.WORKLOADS[args.workload]
        cases = [(w["D"], w["chi"], PAPER_K.get(w["D"], 20), w)]
    else:
        cases = [(D, 5 * D * D, PAPER_K[D], dict(d=2, D=D, chi=5 * D * D, seed=0, decay=True,
                                                 bias=0.0)) for D in range(2, 8)]
    rows = []
    for D, chi, k, w in cases:
        d = w["d"]
        X = torch.tensor(qi.raw_tensor(d, D, w["seed"], w["decay"], w["bias"]),
                         dtype=torch.float64, device="cuda")
        A = q.c4v_symmetrize(X, normalize=True)
        ctx = q.QRCTM(d, D, chi, precision=args.precision, check_every=args.check_every,
                      with_grad=True, with_nnn=J2 != 0, opt_history=10)
        ctx.init_env(A)
        converge(ctx, 1e-8, 2000, floor=args.precision == "split")
        C, T, _ = ctx.get_env(spectrum=False)
        grad = torch.empty_like(A)
        steps = args.steps
        ms, launches, clocks = opt_step_rate(q, ctx, A, C, T, k, J2, steps, args.warmup
                                             if args.mode == "opt" else 1, dist, local, grad)
        row = {"D": D, "chi": chi, "k": k, "ms_per_step": ms / steps,
               "steps_per_s": job_rate(steps, world, ms), "gpu_launches": int(launches),
               "clocks": clocks}
        if args.mode == "opt" and not args.no_extras:
            # the L-BFGS loop itself: accepted steps, evaluations, wall time
            A2 = A.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            en, evals, failed = ctx.optimize(A2, args.opt_steps, J2=J2, k_unroll=k,
                                             env_tol=1e-8 if args.precision == "fp64" else 1e-6)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            row["lbfgs"] = {"accepted_steps": len(en) - 1, "evaluations": evals,
                            "wall_s": wall, "energies": [float(x) for x in en],
                            "line_search_failed": bool(failed)}
        rows.append(row)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    head = rows[-1] if args.mode == "opt" else next(r for r in rows if r["D"] == 6)
    if rank == 0:
        line = {
            "metric": (f"optimisation steps/s ({args.workload}, 2 untracked + k={head['k']} "
                       "tracked QR-CTMRG steps, energy, gradient)" if args.mode == "opt" else
                       "optimisation steps/s (d=2, D=6, chi=180, k=20; sweep D=2..7, chi=5D^2)"),
            "value": head["steps_per_s"], "unit": "opt-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "tf32x3+f64", "data": "synthetic",
            "config": {"workload": args.workload if args.mode == "opt" else "D=2..7, chi=5D^2",
                       "precision": args.precision, "J2": J2, "gradient": "unrolled",
                       "parallelism": f"replicas{world}"},
            "roofline": None,
            "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"],
            "sweep": rows,
        }
        print(json.dumps(line), flush=True)


def bench_chi_sweep(args, q, dist, world, rank, local):
    """Large-chi evaluations (Results: chi_eval up to 600-700 at D = 7, 8):
    iterations/s and the energy-per-site time at each chi, split precision."""
    import torch
    D, d = 8, 2
    rows = []
    X = torch.tensor(qi.raw_tensor(d, D, 0, True, 0.0), dtype=torch.float64, device="cuda")
    A = q.c4v_symmetrize(X, normalize=True)
    for chi in args.chis:
        ctx = q.QRCTM(d, D, chi, precision=args.precision, check_every=args.check_every)
        t0 = time.perf_counter()
        ctx.init_env(A)
        torch.cuda.synchronize()
        init_s = time.perf_counter() - t0
        ce = args.check_every

        def one_step(i):
            ctx.step(1, want_delta=(i % ce == ce - 1))

        for i in range(2):
            one_step(i)
        torch.cuda.synchronize()
        steps = max(ce, args.steps)
        ms, launches, clocks = timed_region(q, one_step, steps, dist, local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = ctx.energy(1.0, 0.0)
        e_ms = 1e3 * (time.perf_counter() - t0)
        rows.append({"chi": chi, "m": chi * D * D, "iter_per_s": job_rate(steps, world, ms),
                     "ms_per_step": ms / steps, "init_s": init_s, "energy_ms": e_ms,
                     "E_unconverged": E, "workspace_GB": ctx.workspace_bytes / 1e9,
                     "clocks": clocks, "gpu_launches": int(launches)})
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    if rank == 0:
        head = rows[-1]
        line = {
            "metric": f"QR-CTMRG iterations/s (d=2, D=8, chi={head['chi']}; chi sweep)",
            "value": head["iter_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": max(args.check_every, args.steps),
            "warmup": 2, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "tf32x3+f64", "data": "synthetic",
            "config": {"workload": "d2_D8 chi sweep", "chis": args.chis,
                       "precision": args.precision, "parallelism": f"replicas{world}"},
            "roofline": None, "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "sweep": rows,
        }
        print(json.dumps(line), flush=True)


def run_reference(args, w, rank):
    if rank != 0:
        return
    o_times, layers = oracle_sample(w, args.warmup + args.steps)
    timed = o_times[args.warmup:]
    tot = sum(timed)
    val = len(timed) / tot
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "d": w["d"], "D": w["D"], "chi": w["chi"],
                   "layers": layers, "parallelism": "replicas"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle QR-CTMRG iterations after "
                                   f"{args.warmup} untimed, NumPy FP64 on the host"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--method", default="qr", choices=["qr", "eigen"],
                    help="qr: QR-CTMRG; eigen: the standard step with a full "
                         "eigendecomposition (comparison method, FP64)")
    ap.add_argument("--workload", default="d2_D6_chi144",
                    choices=sorted(qi.WORKLOADS) + sorted(qi.NETWORK_WORKLOADS))
    ap.add_argument("--check-every", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=3, help="oracle steps in cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip time-to-convergence, dE vs FP64 and the energy gradient")
    ap.add_argument("--grad-tol", type=float, default=1e-6,
                    help="relative residual target of the implicit adjoint solve")
    ap.add_argument("--mode", default="step", choices=["step", "opt", "opt-sweep", "chi-sweep"],
                    help="step: CTMRG iterations (default); opt: optimisation steps on the "
                         "workload; opt-sweep: D = 2..7 at chi = 5 D^2; chi-sweep: D = 8 at "
                         "large chi")
    ap.add_argument("--j2", type=float, default=0.0, help="J2/J1 of the optimisation modes")
    ap.add_argument("--opt-steps", type=int, default=5, help="L-BFGS steps reported in opt mode")
    ap.add_argument("--chis", type=int, nargs="+", default=[300, 400, 500, 600, 700])
    ap.add_argument("--conv-tol", type=float, default=0.0,
                    help="spectrum tolerance for time-to-converged (default 1e-10; the split path "
                         "stops earlier at its precision floor)")
    ap.add_argument("--fp64-ttc-max-iter", type=int, default=4000,
                    help="iteration cap of the FP64 path's own run from the bulk boundary to the "
                         "tolerance (time-to-converged of the plain FP64 path); 0 skips it")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the energy-gradient extras (automatic when chi D^2 > 8192, where "
                         "the 2x2-patch buffers of the J2 term and the gradient tapes are large)")
    ap.add_argument("--oracle-sample-only", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    network = args.workload in qi.NETWORK_WORKLOADS
    if args.oracle_sample_only:
        times, _ = oracle_sample(qi.WORKLOADS[args.workload], args.cpu_sample)
        # the BLAS pool size set by the parent (threadpoolctl may be absent)
        cores = int(os.environ.get("OPENBLAS_NUM_THREADS") or cpu_threads())
        print(json.dumps({"value": len(times) / sum(times), "cores": cores}), flush=True)
        return
    w = qi.NETWORK_WORKLOADS[args.workload] if network else qi.WORKLOADS[args.workload]
    if network:
        args.precision = "fp64"
    if args.method == "eigen" and not network:
        args.precision = "fp64"
        args.no_extras = True
    if args.steps <= 0:
        if args.mode in ("opt", "opt-sweep"):
            args.steps = 5 if args.mode == "opt" else 3
        elif args.mode == "chi-sweep":
            args.steps = 10
        else:
            args.steps = 5 if args.method == "eigen" else (20 if args.precision == "fp64" else 200)
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if network:
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm times the oracle on the iPEPS "
                                             "workloads; the network workloads report their "
                                             "oracle sample in cpu_baseline"}), flush=True)
            return
        run_reference(args, w, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2505_00494_b300 import build
    if rank == 0 and not os.path.exists(build.LIB):
        build.build()
    if dist is not None:
        dist.barrier()
    import paper_2505_00494_b300 as q
    if args.mode in ("opt", "opt-sweep"):
        bench_opt(args, q, dist, world, rank, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.mode == "chi-sweep":
        bench_chi_sweep(args, q, dist, world, rank, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    if network:
        bench_network(args, w, q, dist, world, rank, local)
        if dist is not None:
            dist.destroy_process_group()
        return

    d, D, chi = w["d"], w["D"], w["chi"]
    # every replica runs the same seeded workload
    X = torch.tensor(qi.raw_tensor(d, D, w["seed"], w["decay"], w["bias"]), dtype=torch.float64,
                     device="cuda")
    A = q.c4v_symmetrize(X, normalize=True)
    ctx = q.QRCTM(d, D, chi, precision=args.precision, check_every=args.check_every,
                  with_nnn=chi * D * D <= 8192, method=args.method)
    ctx.init_env(A)
    ce = args.check_every

    def one_step(i):
        ctx.step(1, want_delta=(i % ce == ce - 1))

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    ms, launches, clocks = timed_region(q, one_step, args.steps, dist, local)
    ms_per_step = ms / args.steps
    value = job_rate(args.steps, world, ms)
    phases, prof_ms = phase_profile(ctx, one_step, max(ce, min(args.steps, 10 * ce)))

    # roofline of the dominant kernel.  Per-phase device times come from CUDA
    # events on the library's stream; the phases below are one kernel each
    # (qr_panel: the FP64 panel launches; absorb: the fused ket/bra kernel;
    # x1, project: one tensor-core contraction)
    fl = algorithmic_flops(d, D, chi)
    peaks = load_peaks()
    tf32_peak, tf32_note = tf32_peak_sustained(peaks)
    traffic = load_traffic(args.precision, args.workload)
    fp64_note = "fp64 nominal 1.25 TFLOP/s (CUDA-core FP64 pipe)"
    # the split path's panels take two columns per grid-wide exchange
    panel_k = "qr_panel2_kernel" if args.precision == "split" else "qr_panel_kernel"
    kernels = {"qr_panel": (panel_k, panel_flops(d, D, chi), "alu", FP64_PEAK_TFLOPS,
                            fp64_note)}
    if args.precision == "split":
        m = chi * D * D
        if D == 6:
            # both layers on the tensor cores in one kernel
            absorb = ("absorb_tc_kernel", fl["absorb"], "tensor", tf32_peak, tf32_note)
        elif D < 6:
            absorb = ("absorb_fused_k", fl["absorb"], "alu",
                      fp32_simt_peak(), "fp32 FMA nominal: 148 SMs x 128 FMA/clk x 2 x 2.032 GHz")
        else:
            # two tensor-core contractions of equal flops (ket: N = d D^2, K = D^2;
            # bra: N = D^2, K = d D^2)
            absorb = (tc_kernel_name(d * D * D, D * D) + " (ket), " +
                      tc_kernel_name(D * D, d * D * D) + " (bra)", fl["absorb"] / 2, "tensor",
                      tf32_peak, tf32_note)
        kernels.update({
            "absorb": absorb,
            "x1": (tc_kernel_name(m, chi, 2, m), fl["x1"], "tensor", tf32_peak, tf32_note),
            "project": (tc_kernel_name(chi, m, 1), fl["project"], "tensor", tf32_peak,
                        tf32_note),
        })
    else:
        kernels.update({
            "x1": ("gemm_f64_kernel", fl["x1"], "alu", FP64_PEAK_TFLOPS, fp64_note),
            "project": ("gemm_f64_kernel", fl["project"], "alu", FP64_PEAK_TFLOPS, fp64_note),
        })
    rows = roofline_rows(kernels, phases, prof_ms, traffic)
    dom = max(rows, key=lambda k: rows[k]["share_of_step"])
    share = {k: round(phases[k][0] / prof_ms, 4) for k in ("ct", "qr", "x1", "absorb", "project",
                                                      "corner", "symnorm", "spectrum",
                                                      "qr_panel")}

    # energy per site after the timed steps (Heisenberg, J2 = 0; and J1-J2 at 0.5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E = ctx.energy(1.0, 0.0)
    energy_ms = 1e3 * (time.perf_counter() - t0)
    # the 2x2-patch RDM costs 2 d^2 (chi D^2)^3 FP64 flops: skipped beyond
    # chi D^2 = 8192 (minutes at D = 8, chi = 512)
    E12, energy_j2_ms = None, None
    if chi * D * D <= 8192:
        t0 = time.perf_counter()
        E12 = ctx.energy(1.0, 0.5)
        energy_j2_ms = 1e3 * (time.perf_counter() - t0)

    # end to end through the C ABI with host buffers: per step the library
    # copies (A, C, T) in from pinned host memory (qrctm_init_env_host),
    # re-initialises from them, runs one iteration with its convergence test
    # and copies (C, T) back out (qrctm_get_env_host).
    C_d, T_d, _ = ctx.get_env(spectrum=False)
    hA = A.cpu().pin_memory()
    hC = C_d.cpu().pin_memory()
    hT = T_d.cpu().pin_memory()
    ctx2 = ctx
    oC, oT = torch.empty_like(hC).pin_memory(), torch.empty_like(hT).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx2.init_env_host(hA, hC, hT)
        ctx2.step(1, want_delta=True)
        ctx2.get_env_host(oC, oT)
        # the result becomes the next step's pinned input: swap the buffers
        hC, oC = oC, hC
        hT, oT = oT, hT
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    h2d = (hA.numel() + hC.numel() + hT.numel()) * 8
    d2h = (oC.numel() + oT.numel()) * 8 + 8

    # time to a converged environment from the bulk boundary (warm-up included),
    # the energy error of the split path against the FP64 path from that
    # environment, and the energy-gradient time (J1-J2 at J2/J1 = 0.5)
    extras = {}
    grad_extras = not args.no_grad and chi * D * D <= 8192
    if not args.no_extras:
        # time to a converged environment from the bulk boundary: until the
        # spectrum change falls below tol, or (split precision) until it stops
        # decreasing -- the FP32-class contractions leave a floor near 1e-6 at
        # this size, the summed rounding noise of the small singular values
        tol = args.conv_tol or 1e-10
        cctx = q.QRCTM(d, D, chi, precision=args.precision, check_every=ce,
                       with_nnn=grad_extras, with_grad=grad_extras, grad_tol=args.grad_tol,
                       grad_max_iter=300)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cctx.init_env(A)
        its, dl, stalled = converge(cctx, tol, 4000, floor=args.precision == "split")
        torch.cuda.synchronize()
        extras["time_to_converged_s"] = time.perf_counter() - t0
        extras["converged_iterations"] = its
        extras["converged_delta"] = dl
        extras["converged_tol"] = tol
        extras["converged_at_floor"] = stalled
        Cc, Tc, _ = cctx.get_env(spectrum=False)
        e_split = cctx.energy(1.0, 0.0)
        fctx = q.QRCTM(d, D, chi, precision="fp64", check_every=ce, with_nnn=grad_extras,
                       with_grad=grad_extras, grad_tol=args.grad_tol, grad_max_iter=300)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fctx.init_env(A, Cc, Tc)
        fits, fdl = fctx.run_to_convergence(tol=tol, max_iter=4000)
        if fits % 2:
            fctx.step(1, want_delta=False)
        torch.cuda.synchronize()
        extras["fp64_refine_s"] = time.perf_counter() - t0
        extras["fp64_refine_delta"] = fdl
        e_fp64 = fctx.energy(1.0, 0.0)
        extras["E_per_site_J2_0"] = e_fp64
        extras["dE_split_vs_fp64"] = (e_split - e_fp64) if args.precision == "split" else 0.0
        extras["fp64_refine_iterations"] = fits
        if args.precision == "split":
            extras["time_to_converged_split_polish_s"] = (extras["time_to_converged_s"] +
                                                          extras["fp64_refine_s"])
        if args.precision == "split" and grad_extras:
            # gradients with the contractions on the TF32x3 engine, taken at
            # the polished environment like the FP64 ones below: the implicit
            # gradient assumes an elementwise fixed point, which the split
            # floor meets only to ~4e-4 (at the floor environment itself the
            # FP64 implicit gradient moves by up to ~3e-3 from run to run)
            Cf, Tf, _ = fctx.get_env(spectrum=False)
            cctx.init_env(A, Cf, Tf)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, gs = cctx.energy_grad(1.0, 0.5, mode="implicit")
            torch.cuda.synchronize()
            extras["split_energy_grad_implicit_ms"] = 1e3 * (time.perf_counter() - t0)
            extras["split_energy_grad_applications"] = cctx.grad_iterations
            extras["split_energy_grad_adjoint_residual"] = cctx.grad_residual
            extras["split_grad_fixed_point_residual"] = cctx.grad_fixed_point_residual
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # an NVTX range for launch lists of the gradient alone
            # (ncu --nvtx --nvtx-include "split_grad_unroll20/")
            torch.cuda.nvtx.range_push("split_grad_unroll20")
            _, gsu = cctx.energy_grad(1.0, 0.5, mode="unroll", k_unroll=20)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            extras["split_energy_grad_unroll20_ms"] = 1e3 * (time.perf_counter() - t0)
            extras["split_energy_grad_ms"] = extras["split_energy_grad_unroll20_ms"]
        cctx.close()
        # the plain FP64 path on its own, from the same bulk boundary to the
        # same tolerance: the comparison of time to a converged environment
        # at equal energy accuracy (the split path's energy at its floor is
        # within dE_split_vs_fp64 of the converged FP64 energy)
        if args.precision == "split" and args.fp64_ttc_max_iter > 0:
            bctx = q.QRCTM(d, D, chi, precision="fp64", check_every=ce)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bctx.init_env(A)
            bits, bdl, _ = converge(bctx, tol, args.fp64_ttc_max_iter)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            e_b = bctx.energy(1.0, 0.0)
            bctx.close()
            reached = bdl < tol
            extras["fp64_time_to_converged_s"] = tb if reached else None
            extras["fp64_converged_iterations"] = bits
            extras["fp64_converged_delta"] = bdl
            extras["fp64_s_per_iteration"] = tb / max(1, bits)
            extras["dE_fp64_from_bulk_vs_polished"] = e_b - e_fp64
            if reached:
                extras["split_floor_speedup_vs_fp64"] = tb / extras["time_to_converged_s"]
                extras["split_polish_speedup_vs_fp64"] = (
                    tb / extras["time_to_converged_split_polish_s"])
            else:
                # capped: the same map needs about as many iterations from the
                # bulk as the split run plus its polish took
                extras["fp64_time_to_converged_estimate_s"] = (
                    extras["fp64_s_per_iteration"] * (its + fits))
        if not grad_extras:
            fctx.close()
    if not args.no_extras and grad_extras:
        # energy gradient at J2/J1 = 0.5 with FP64 reverse passes: the implicit
        # adjoint (GMRES on the two-step fixed point) and the unrolled
        # backpropagation through the last 20 steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Eg, g = fctx.energy_grad(1.0, 0.5, mode="implicit")
        torch.cuda.synchronize()
        extras["energy_grad_implicit_ms"] = 1e3 * (time.perf_counter() - t0)
        extras["energy_grad_adjoint_applications"] = fctx.grad_iterations
        extras["energy_grad_adjoint_residual"] = fctx.grad_residual
        extras["grad_fixed_point_residual"] = fctx.grad_fixed_point_residual
        extras["E_per_site_J2_0.5"] = Eg
        extras["grad_norm"] = float(g.norm().item())
        extras["grad_dot_A"] = float((g * A).sum().item())
        # the headline gradient: backpropagation through the last 20 steps
        # (the paper's scheme at D = 6); it needs no elementwise fixed point
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Eu, gu = fctx.energy_grad(1.0, 0.5, mode="unroll", k_unroll=20)
        torch.cuda.synchronize()
        extras["energy_grad_unroll20_ms"] = 1e3 * (time.perf_counter() - t0)
        extras["energy_grad_ms"] = extras["energy_grad_unroll20_ms"]
        extras["energy_grad_mode"] = "unroll20"
        extras["grad_implicit_vs_unroll20_rel"] = float((g - gu).norm() / g.norm())
        if args.precision == "split":
            # split and FP64 gradients at the same (polished) environment
            extras["grad_split_vs_fp64_rel"] = float((gs - g).norm() / g.norm())
            extras["grad_split_unroll20_vs_fp64_rel"] = float((gsu - gu).norm() / gu.norm())
        fctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, layers = oracle_sample(w, args.cpu_sample)
        cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": cpu_threads(),
               "kind": "oracle",
               "sample": f"{len(times)} oracle QR-CTMRG iterations ({layers} layers, NumPy FP64, "
                         f"d={d} D={D} chi={chi}) from a random symmetric environment"}
        # the same sample on 8 BLAS threads, the paper's CPU setting (8 cores):
        # a child process, since the BLAS pool size is fixed when NumPy loads
        cpu["threads_8"] = oracle_sample_threads(args.workload, args.cpu_sample, 8)

    if rank == 0:
        line = {
            "metric": (METRIC if args.workload == "d2_D6_chi144" else
                       f"QR-CTMRG iterations/s ({args.workload})") if args.method == "qr" else
            f"standard C4v CTMRG (eigendecomposition) iterations/s ({args.workload})",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "tf32x3+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "D": D, "chi": chi,
                       "precision": args.precision, "method": args.method,
                       "layers": "split" if 2 * d < D * D else "double",
                       "check_every": ce, "parallelism": f"replicas{world}",
                       "l2": "per-step intermediates larger than L2 (X1 alone "
                             f"{(chi * D * D) ** 2 * 8 / 1e6:.0f} MB)"},
            "roofline": rows[dom],
            "roofline_kernels": rows,
            "phase_share": share,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "energy_per_site": {"J2_0": E, "J2_0.5": E12, "energy_ms": energy_ms,
                                "energy_j2_ms": energy_j2_ms},
            "energy_grad_ms": extras.get("energy_grad_ms"),
            "split_energy_grad_ms": extras.get("split_energy_grad_ms"),
            "energy_grad_mode": extras.get("energy_grad_mode"),
            "convergence": extras,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
