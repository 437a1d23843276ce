#!/usr/bin/env python3
"""Benchmark of the eGPE ground-state solver hot path on one GB300 per rank.

Headline: NCG iterations per second on the 128^3 two-component dipolar eGPE
(the stripe/supersolid couplings on [-16,16]^2 x [-8,8]) with FP32 fields, sums
reduced to FP64 values and an FP64 controller, the FP64 path timed beside it, time to ground
state (mixed vs FP64, relative energy 1e-8), and the HBM roofline of the
dominant kernel.  One "step" is one attempt of the NCG loop body (precondition,
line-search coefficients, trial energy/gradient, controller); steps are timed
with CUDA events on the solver's stream, in chunks that each restart from the
seeded start so the solver never finishes inside a timed region.

  python bench.py --gpus N --steps K --warmup W          (this implementation)
  python bench.py --impl reference --steps K --warmup W  (the FP64 CPU oracle)

Under torchrun every rank solves its own instance (seed + rank: independent
problems, weak scaling, no collective on the data path); rank 0 prints one
JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-ground-state & NCG iters/s at 128^3 (mixed vs FP64), % HBM roofline"
UNIT = "NCG iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3p")
    ap.add_argument("--precond", default="kinetic+diagonal")
    ap.add_argument("--chunk", type=int, default=25)
    ap.add_argument("--no-tts", action="store_true", help="skip time-to-ground-state")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-ite", action="store_true", help="skip the NCG-vs-ITE comparison on the 64^3 workload")
    ap.add_argument("--no-scan", action="store_true", help="skip the 64-instance parameter scan")
    ap.add_argument("--no-tune", action="store_true", help="untuned launch shapes (no autotuning)")
    ap.add_argument("--no-cont", action="store_true", help="skip continuation along the scan")
    ap.add_argument("--no-pcstudy", action="store_true", help="skip the preconditioner study")
    ap.add_argument("--no-pgrad", action="store_true", help="skip the parameter-derivative timing")
    ap.add_argument("--fp32-switch", type=float, default=1e-4)
    ap.add_argument("--table", action="store_true",
                    help="per-workload table (oracle and GPU) instead of the benchmark line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples (200 ms) while the GPU work runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def snapshot(self):
        """Median SM clock of the samples taken so far (None if none)."""
        sm = []
        for ln in list(self.lines):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm)} if sm else None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alu_peaks(sm_count, sm_mhz):
    """CUDA-core peaks from the unit counts of this GPU (Blackwell SM: 128 FP32
    lanes, 2 FP64 FMA lanes per clock on GB300) at a given SM clock, 2
    operations per fused multiply-add, in TFLOP/s."""
    return {"fp32": sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12, "fp64": sm_count * 2 * 2 * sm_mhz * 1e6 / 1e12}


def eg_pass_flops(n):
    """FP64 operations of one energy/gradient pass counted as its six complex
    3D transforms (psi_1, psi_2 and the packed dipolar source, forward and
    inverse) at the standard 5 N log2 N each; the pointwise physics (a few
    hundred operations per point with the LHY tables) is left out, so this is
    a lower bound on the pass's arithmetic."""
    N = n[0] * n[1] * n[2]
    return 6 * 5 * N * math.log2(N)


def traffic_record(kernel_name, workload):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None
    if the summary is missing or was taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        from paper_2510_24543_gb300 import build as B
        with open(p) as f:
            d = json.load(f)
        rec = d.get("kernels", {}).get(kernel_name)
        if not rec or d.get("sources") != B._digest() or rec.get("workload") != workload:
            return None
        return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2510_24543_gb300 import build as B
    from paper_2510_24543_gb300 import egpe as E
    from paper_2510_24543_gb300 import inputs as I

    from paper_2510_24543_gb300 import autotune as AT
    from paper_2510_24543_gb300 import replicas as RP

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return RP.combine(dist, x, 0.0, device="cuda")[0]

    def sum_over_ranks(x):
        return RP.combine(dist, 0.0, x, device="cuda")[1]

    B.build()
    E.load()
    w0 = I.PRESETS[args.workload]
    w = RP.rank_workload(w0, rank)
    N = w.points
    psi0_np = I.gaussian_start(w)
    stream = torch.cuda.Stream()
    grid = E.make_grid(w.n, w.L)
    prm = E.params_from_workload(w)
    h = E.egpe_create([grid], [prm], E.EGPE_MIXED, stream.cuda_stream)
    psi64 = torch.from_numpy(psi0_np).to("cuda")
    psi32 = psi64.to(torch.complex64)
    pc = E.PRECOND[args.precond]
    device_name = torch.cuda.get_device_name(local)
    tuning = None
    if not args.no_tune:
        t0 = time.perf_counter()
        used = AT.tune_handle(h, [w.n], E.EGPE_MIXED, pc, lambda i, e: psi64 if e == 0 else psi32, device_name)
        tuning = {"seconds": round(time.perf_counter() - t0, 3),
                  "changed": [{"engine": k.split("|")[2], "kernel": f"{t['name']} L={t['L']}", "choice": t["choice"],
                               "default": t["default_choice"], "ms_best": round(t["ms_best"], 5),
                               "ms_default": round(t["ms_default"], 5)}
                              for k, v in used.items() for t in v if t["choice"] != t["default_choice"]]}
    clocks = Clocks(local)
    clocks.start()

    def opts(**kw):
        o = E.egpe_default_solve_opts()
        o.precond = pc
        o.tol_res = 0.0
        o.max_iter = 1 << 30
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def timed_steps(engine, psi, K, W, chunk):
        """K attempts of the NCG loop body timed with CUDA events on the solver
        stream, W untimed warm-up attempts before each chunk."""
        o = opts()
        tot_ms, iters, launches, done = 0.0, 0, 0, 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while done < K:
            n = min(chunk, K - done)
            E.egpe_solver_start(h, 0, engine, psi, o)
            E.egpe_solver_step(h, 0, engine, W)
            r0 = E.egpe_solver_read(h, 0, engine)
            torch.cuda.synchronize()
            barrier()
            ev0.record(stream)
            E.egpe_solver_step(h, 0, engine, n)
            ev1.record(stream)
            ev1.synchronize()
            torch.cuda.synchronize()
            barrier()
            r1 = E.egpe_solver_read(h, 0, engine)
            if r1["status"] != 5:
                raise RuntimeError(f"solver finished inside a timed region ({r1}); lower --chunk")
            tot_ms += ev0.elapsed_time(ev1)
            iters += r1["iters"] - r0["iters"]
            launches += r1["kernels"] - r0["kernels"] - 1  # minus the read's residual kernel
            done += n
        return tot_ms, iters, launches

    # ---- headline: FP32 fields (mixed precision) iterations per second
    ms32, it32, launch32 = timed_steps(1, psi32, args.steps, args.warmup, args.chunk)
    ms32 = max_over_ranks(ms32)
    it32_all = sum_over_ranks(it32)
    value = it32_all / (ms32 * 1e-3)
    ms_per_step = ms32 / args.steps

    # ---- FP64 path beside it
    k64 = min(args.steps, 10)
    ms64, it64, launch64 = timed_steps(0, psi64, k64, args.warmup, args.chunk)
    ms64 = max_over_ranks(ms64)
    fp64 = {"iters_per_s": sum_over_ranks(it64) / (ms64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64,
            "gpu_launches": launch64}

    # ---- the same rates from the ground state (the FP64 LHY cost depends on how many points
    # carry non-negligible density; the FP32 cost does not)
    at_gs = None
    try:
        hgs = E.egpe_create([grid], [prm], E.EGPE_FP64, stream.cuda_stream)
        try:
            og = opts(tol_res=1e-9, max_iter=5000)
            psi_gs = psi64.clone()
            E.egpe_ncg_solve(hgs, [psi_gs], og, 1)
        finally:
            E.egpe_destroy(hgs)
        ms_g32, it_g32, _ = timed_steps(1, psi_gs.to(torch.complex64), args.steps, args.warmup, args.chunk)
        ms_g64, it_g64, _ = timed_steps(0, psi_gs, k64, args.warmup, args.chunk)
        at_gs = {"fp32_iters_per_s": sum_over_ranks(it_g32) / (max_over_ranks(ms_g32) * 1e-3),
                 "fp64_iters_per_s": sum_over_ranks(it_g64) / (max_over_ranks(ms_g64) * 1e-3),
                 "state": "FP64 ground state, ||r|| < 1e-9, same workload"}
    except Exception as ex:  # reported, not fatal for the headline
        at_gs = {"error": str(ex)[:300]}
    fp64["at_ground_state"] = at_gs

    # ---- per-kernel device times (roofline of the dominant kernel)
    hbm, peak_kind = peaks()
    prof32 = E.egpe_profile_attempt(h, 0, 1, psi32, pc, reps=5)
    prof64 = E.egpe_profile_attempt(h, 0, 0, psi64, pc, reps=3)
    att_ms = sum(t for _, t, _ in prof32)
    att_bytes = sum(b for _, _, b in prof32)
    dom = max(prof32, key=lambda x: x[1])
    gbs = dom[2] / (dom[1] * 1e-3) / 1e9
    attempt = {"ms": round(att_ms, 4), "algorithmic_bytes": att_bytes,
               "achieved_GBs": round(att_bytes / (att_ms * 1e-3) / 1e9, 1),
               "frac_hbm": round(att_bytes / (att_ms * 1e-3) / 1e9 / hbm, 4)}
    common = {"kernel": dom[0], "ms_per_launch": dom[1], "share_of_attempt": round(dom[1] / att_ms, 4),
              "traffic": traffic_record(dom[0], args.workload), "algorithmic_bytes": dom[2],
              "hbm_view": {"achieved_GBs": round(gbs, 1), "frac": round(gbs / hbm, 4), "peak_GBs": hbm,
                           "peak_kind": peak_kind + " (burst copy)"},
              "attempt": attempt,
              "kernels": [{"name": n, "ms": round(t, 5), "GBs": round(b / (t * 1e-3) / 1e9, 1)} for n, t, b in prof32]}
    props = torch.cuda.get_device_properties(local)
    clk_mid = clocks.snapshot()
    sm_mhz = (clk_mid or {}).get("sm_mhz") or 2070.0
    pk = alu_peaks(props.multi_processor_count, sm_mhz)
    peak_src = f"derived: {props.multi_processor_count} SMs x {{lanes}} x 2 x {sm_mhz:.0f} MHz (median SM clock sampled so far)"
    roofline = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4), "peak_kind": peak_kind + " (burst copy)", **common}
    eg = prof32[-5:]  # the trial energy/gradient pass: x fwd, y, z fused, y, x inv
    eg_ms = sum(t for _, t, _ in eg)
    roofline["eg_pass"] = {"kernels": [n for n, _, _ in eg], "ms": round(eg_ms, 4),
                           "algorithmic_bytes": sum(b for _, _, b in eg),
                           "model_32SN_bytes": 32 * 8 * N,
                           "achieved_GBs": round(32 * 8 * N / (eg_ms * 1e-3) / 1e9, 1),
                           "frac_hbm_32SN": round(32 * 8 * N / (eg_ms * 1e-3) / 1e9 / hbm, 4)}
    dom64 = max(prof64, key=lambda x: x[1])
    fp64["dominant_kernel"] = {"name": dom64[0], "ms": dom64[1], "share": round(dom64[1] / sum(t for _, t, _ in prof64), 4),
                               "bound": "alu (FP64)"}
    eg64 = prof64[-5:]
    eg64_ms = sum(t for _, t, _ in eg64)
    fl64 = eg_pass_flops(w.n)
    fp64["roofline_eg_pass"] = {"bound": "alu (FP64)", "achieved": round(fl64 / (eg64_ms * 1e-3) / 1e12, 4),
                                "peak": round(pk["fp64"], 4), "unit": "TFLOP/s",
                                "frac": round(fl64 / (eg64_ms * 1e-3) / 1e12 / pk["fp64"], 4),
                                "peak_kind": peak_src.format(lanes="2 FP64 FMA lanes"),
                                "algorithmic_flops": fl64, "ms": round(eg64_ms, 4),
                                "flops_model": "6 complex 3D transforms x 5 N log2 N (pointwise work not counted)"}
    fp64["kernels"] = [{"name": n, "ms": round(t, 4)} for n, t, _ in prof64]
    roofline["fp32_alu_peak"] = {"value": round(pk["fp32"], 2), "unit": "TFLOP/s",
                                 "kind": peak_src.format(lanes="128 FP32 lanes")}

    # ---- end to end through the public solve call with host buffers
    h32 = E.egpe_create([grid], [prm], E.EGPE_FP32, stream.cuda_stream)
    if not args.no_tune:
        AT.tune_handle(h32, [w.n], E.EGPE_FP32, pc, lambda i, e: psi32, device_name)
    host32 = torch.from_numpy(psi0_np.astype("complex64")).pin_memory()
    calls = max(1, math.ceil(args.steps / args.chunk))
    e2e_iters, e2e_s = 0, 0.0
    o = opts(max_iter=args.chunk, psi_on_host=1)
    buf = host32.clone().pin_memory()
    E.egpe_ncg_solve(h32, [buf.data_ptr()], o, 1)  # warm-up call (graph capture)
    for _ in range(calls):
        buf.copy_(host32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, reps, _ = E.egpe_ncg_solve(h32, [buf.data_ptr()], o, 1)
        e2e_s += time.perf_counter() - t0
        e2e_iters += reps[0]["iters"]
    e2e_s = max_over_ranks(e2e_s)
    field_bytes = 2 * N * 8
    e2e = {"value": sum_over_ranks(e2e_iters) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": field_bytes / args.chunk, "d2h_bytes_per_step": field_bytes / args.chunk,
           "call": f"egpe_ncg_solve(FP32 fields, host psi) running {args.chunk} iterations per call; "
                   "per-call H2D psi and D2H psi+report amortised per iteration"}
    E.egpe_destroy(h32)

    # ---- time to ground state: mixed (FP32 phase + FP64 polish) vs plain FP64
    tts = None
    if not args.no_tts:
        try:
            tts = time_to_ground_state(E, h, grid, prm, psi64, pc, args.fp32_switch)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            tts = {"error": str(ex)[:300]}
    # single-GPU studies: only in a one-rank run (under torchrun every rank would repeat them)
    solo = world == 1
    ite = None
    if solo and not args.no_ite:
        try:
            ite = ncg_vs_ite(E, tune=not args.no_tune)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            ite = {"error": str(ex)[:300]}
    scan = None
    if solo and not args.no_scan:
        try:
            scan = scan_benchmark(E, tune=not args.no_tune)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            scan = {"error": str(ex)[:300]}
    pgrad = None
    if solo and not args.no_pgrad:
        try:
            pgrad = param_grad_timing(E)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            pgrad = {"error": str(ex)[:300]}
    pcs = None
    if solo and not args.no_pcstudy:
        try:
            pcs = precond_study(E)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            pcs = {"error": str(ex)[:300]}
    cont = None
    if solo and not args.no_cont:
        try:
            cont = continuation_benchmark(E, tune=not args.no_tune)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            cont = {"error": str(ex)[:300]}
    clk = clocks.stop()
    E.egpe_destroy(h)

    # the CPU leg: the oracle timed on the host, and the oracle's evaluation of
    # the mixed-precision results (rank 0 of a one-GPU run only)
    cpu = macc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w)
        try:
            macc = mixed_accuracy(E, w0, pc, args.fp32_switch)
        except Exception as ex:  # reported, not fatal for the iteration numbers
            macc = {"error": str(ex)[:300]}
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": "FP32 fields and transforms; sums reduced deterministically (float-float) to "
                             "FP64 values; FP64 controller",
                "data": "synthetic (seeded Gaussian + 1% noise start)",
                "config": {"workload": w0.name + " on [-16,16]^2x[-8,8], trap (0.5,1,2), g=300/300/280, "
                                       "g_dd=420/420/400, LHY c=100",
                           "grid": list(w.n), "precond": args.precond, "lhy_nodes": w.lhy_nodes,
                           "parallelism": f"replicas x{world} (one instance per GPU)",
                           "l2": "inputs larger than L2: ~25 complex64 fields of 16.8 MB resident per instance",
                           "step": "one NCG attempt (precondition + line coefficients + trial E/grad + controller)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launch32,
                "clocks": clk, "fp64": fp64, "time_to_ground_state": tts, "mixed_accuracy": macc,
                "ncg_vs_ite": ite,
                "scan": scan, "continuation": cont,
                "precond_study": pcs, "param_grad": pgrad, "autotune": tuning}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def time_to_ground_state(E, h, grid, prm, psi64, pc, fp32_switch):
    """Wall time of egpe_ncg_solve from the seeded start, FP64 fields against
    FP32 fields, to two targets; every returned state is re-evaluated by the
    GPU FP64 engine (egpe_energy_grad on an FP64 handle), and its relative
    energy error is taken against E_ref, the FP64 energy of a solve to
    ||r|| <= 1e-11:
      * "energy_1e-8": both stop at the residual r* at which the FP64 run first
        came within 1e-8 of E_ref (FP64 fields vs FP32 fields alone);
      * "residual_1e-8": both stop at ||r|| <= 1e-8, FP64 alone against mixed
        precision (FP32 fields until ||r|| < fp32_switch, then the FP64 polish).
    Timed solves run on handles that have solved once already, so none pays
    graph capture or first-launch set-up; the mixed handle's first solve is
    reported as seconds_cold."""
    import torch
    o = E.egpe_default_solve_opts()
    o.precond = pc
    o.tol_res = 1e-11
    o.max_iter = 5000
    o.max_iter_fp32 = 5000
    ref = psi64.clone()
    hd = E.egpe_create([grid], [prm], E.EGPE_FP64)
    h32 = E.egpe_create([grid], [prm], E.EGPE_FP32)
    try:
        st, reps, tr = E.egpe_ncg_solve(hd, [ref], o, 1, trace_cap=8000)
        Eref = E.egpe_energy_grad(hd, 0, ref)[0]
        rstar = None
        acc = [t for t in tr if t["flags"] & 1]
        for k, t in enumerate(acc):
            if abs(t["E_trial"] - Eref) <= 1e-8 * abs(Eref):
                rstar = acc[k + 1]["res"] if k + 1 < len(acc) else reps[0]["res"]
                break
        if rstar is None:
            raise RuntimeError("reference never reached the accuracy")

        def fp64_error(x):
            e64 = E.egpe_energy_grad(hd, 0, x.to(torch.complex128))[0]
            return abs(e64 - Eref) / abs(Eref)

        def run(handle, tol, switch=None, dtype=torch.complex128):
            o.tol_res = tol
            if switch is not None:
                o.tol_fp32_switch = switch
            x = psi64.clone().to(dtype)
            st, r, _ = E.egpe_ncg_solve(handle, [x], o, 1)
            r = r[0]
            return {"seconds": r["seconds"], "iters": r["iters"], "iters_fp32": r["iters_fp32"], "status": r["status"],
                    "res": r["res"], "rel_err_fp64_eval": fp64_error(x)}

        run(hd, rstar)  # warm-up of the FP64 handle at this tolerance (graphs by max_iter)
        run(h32, rstar, dtype=torch.complex64)  # warm-up: graph capture, first launches
        e_fp64 = run(hd, rstar)
        e_fp32 = run(h32, rstar, dtype=torch.complex64)
        cold = run(h, 1e-8, fp32_switch)  # the mixed handle's first solve
        r_fp64 = run(hd, 1e-8)
        r_mixed = run(h, 1e-8, fp32_switch)
        r_mixed["seconds_cold"] = cold["seconds"]
        r_mixed["fp32_switch"] = fp32_switch
        return {"E_ref": Eref, "ref_iters": reps[0]["iters"], "ref_status": reps[0]["status"],
                "energy_1e-8": {"res_target": rstar, "fp64": e_fp64, "fp32_fields": e_fp32,
                                "speedup": e_fp64["seconds"] / e_fp32["seconds"]},
                "residual_1e-8": {"fp64": r_fp64, "mixed": r_mixed,
                                  "speedup": r_fp64["seconds"] / r_mixed["seconds"]}}
    finally:
        E.egpe_destroy(hd)
        E.egpe_destroy(h32)


def mixed_accuracy(E, w, pc, fp32_switch=1e-4, tol_polish=1e-10):
    """Mixed-precision accuracy against the FP64 oracle: the state after the
    FP32 phase (FP32 fields to ||r|| < fp32_switch), the state after the FP64
    polish (||r|| < tol_polish) and an FP64 reference (||r|| <= 1e-11) are each
    evaluated by the oracle (the CPU-baseline leg may call it); reported are
    |E - E_ref|/|E_ref| and |mu_i - mu_ref,i| with E_ref, mu_ref the oracle's
    evaluation of the reference, and the GPU's own reported values against the
    oracle's evaluation of the same state."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2510_24543_gb300 import inputs as I

    g = O.Grid(w.n, w.L)
    op = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    grid, prm = E.make_grid(w.n, w.L), E.params_from_workload(w)
    psi0 = torch.from_numpy(I.gaussian_start(w)).to("cuda")
    states = {}
    for name, prec, tol in (("reference_fp64", E.EGPE_FP64, 1e-11), ("after_fp32_phase", E.EGPE_FP32, fp32_switch),
                            ("after_fp64_polish", E.EGPE_MIXED, tol_polish)):
        h = E.egpe_create([grid], [prm], prec)
        try:
            o = E.egpe_default_solve_opts()
            o.precond = pc
            o.tol_res = tol
            o.tol_fp32_switch = fp32_switch
            o.max_iter = 5000
            o.max_iter_fp32 = 5000
            x = psi0.clone() if prec != E.EGPE_FP32 else psi0.to(torch.complex64)
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            states[name] = (reps[0], x.to(torch.complex128).cpu().numpy())
        finally:
            E.egpe_destroy(h)
    evs = {k: O.evaluate(g, op, v[1]) for k, v in states.items()}
    ref = evs["reference_fp64"]
    out = {"workload": w.name, "E_ref_oracle": ref.E, "mu_ref_oracle": list(ref.mu)}
    for k in ("after_fp32_phase", "after_fp64_polish"):
        rep, psi = states[k]
        ev = evs[k]
        r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
        out[k] = {"iters": rep["iters"], "iters_fp32": rep["iters_fp32"], "status": rep["status"],
                  "rel_err_E": abs(ev.E - ref.E) / abs(ref.E),
                  "abs_err_mu": [abs(ev.mu[i] - ref.mu[i]) for i in range(2)],
                  "res_oracle": float(np.sqrt(sum(O.inner(g, r[i], r[i]).real for i in range(2)))),
                  "reported_vs_oracle_rel_E": abs(rep["E"] - ev.E) / abs(ev.E)}
    return out


def ncg_vs_ite(E, tune=True):
    """The paper's comparison of NCG with imaginary-time evolution (Sec. VI.B),
    both on the GPU in FP64 on the 64^3 droplet workload from the same seeded
    start, both stopped at |E^{k+1} - E^k| < 1e-6 (Sec. VI.A): iterations or
    steps, transforms and wall time, for a few ITE steps dtau.  Each energy is
    also compared with a tight NCG solve (||r|| < 1e-10)."""
    import torch

    from paper_2510_24543_gb300 import inputs as I

    w = I.PRESETS["c2"]
    psi0 = torch.from_numpy(I.gaussian_start(w)).to("cuda")
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], E.EGPE_FP64)
    try:
        if tune:
            from paper_2510_24543_gb300 import autotune as AT
            AT.tune_handle(h, [w.n], E.EGPE_FP64, E.PRECOND["kinetic+diagonal"], lambda i, e: psi0,
                           torch.cuda.get_device_name())

        def ncg(tol_res, tol_dE):
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND["kinetic+diagonal"]
            o.tol_res = tol_res
            o.tol_dE = tol_dE
            o.max_iter = 20000
            x = psi0.clone()
            torch.cuda.synchronize()
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            return reps[0]
        ncg(1e-10, 0.0)  # warm-up: graphs captured, code paged in
        tight = ncg(1e-10, 0.0)
        Estar = tight["E"]
        cg = ncg(1e-14, 1e-6)
        out = {"workload": w.name, "stop": "|dE| < 1e-6", "E_star": Estar,
               "ncg": {"iters": cg["iters"], "ffts": cg["ffts"], "seconds": cg["seconds"], "status": cg["status"],
                       "rel_err_E": abs(cg["E"] - Estar) / abs(Estar)},
               "ite": []}
        for dtau in (1e-3, 2e-3, 4e-3):
            o = E.egpe_default_ite_opts()
            o.dtau = dtau
            o.tol_dE = 1e-6
            o.max_steps = 50000
            x = psi0.clone()
            torch.cuda.synchronize()
            st, reps = E.egpe_ite_solve(h, [x], o)
            r = reps[0]
            out["ite"].append({"dtau": dtau, "steps": r["iters"], "ffts": r["ffts"], "seconds": r["seconds"],
                               "status": r["status"], "rel_err_E": abs(r["E"] - Estar) / abs(Estar),
                               "steps_per_ncg_iter": r["iters"] / max(cg["iters"], 1),
                               "time_ratio": r["seconds"] / max(cg["seconds"], 1e-12)})
        return out
    finally:
        E.egpe_destroy(h)


def scan_benchmark(E, tol_res=1e-6, fp32_switch=1e-4, tune=True):
    """The 64-instance parameter scan (16 each of 48^3, 64^3, 80^3, 96^3; Latin
    hypercube over g12 and g_dd; P_Delta o P_V preconditioner): wall time to the
    ground states of all instances, mixed precision batched (FP32 phase to
    ||r|| < fp32_switch, FP64 polish; the grid shapes in sequence, and for
    comparison as concurrent graph branches) against plain FP64 one instance
    after the other, all stopped at ||r|| < tol_res.  Accuracy: each energy against the
    lower of the two methods' energies for that instance (the two can settle in
    different local minima of this multistable problem)."""
    import torch

    from paper_2510_24543_gb300 import inputs as I

    ws = I.scan_workloads()
    grids = [E.make_grid(w.n, w.L) for w in ws]
    prms = [E.params_from_workload(w) for w in ws]
    starts = [torch.from_numpy(I.gaussian_start(w)) for w in ws]

    from paper_2510_24543_gb300 import autotune as AT
    device = torch.cuda.get_device_name()

    def run(prec, batch, tol):
        h = E.egpe_create(grids, prms, prec)
        try:
            if tune:
                AT.tune_handle(h, [w.n for w in ws], prec, E.PRECOND[ws[0].precond],
                               lambda i, e: starts[i].to("cuda").to(torch.complex128 if e == 0 else torch.complex64),
                               device)
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND[ws[0].precond]
            o.tol_res = tol
            o.tol_fp32_switch = fp32_switch
            o.max_iter = 6000
            o.max_iter_fp32 = 6000
            o.batch = batch
            xs = [s.to("cuda") for s in starts]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, reps, _ = E.egpe_ncg_solve(h, xs, o, len(ws))
            torch.cuda.synchronize()
            return time.perf_counter() - t0, reps
        finally:
            E.egpe_destroy(h)

    run(E.EGPE_MIXED, 1, 1e-3)  # warm-up: code paged in, occupancy queries cached
    out = {"instances": len(ws), "grids": "16 each of 48^3, 64^3, 80^3, 96^3", "precond": ws[0].precond,
           "tol_res": tol_res, "fp32_switch": fp32_switch, "accuracy_target": 1e-8}
    runs = {}
    for name, prec, batch in (("fp64_one_by_one", E.EGPE_FP64, 0), ("mixed_batched", E.EGPE_MIXED, 1),
                              ("mixed_batched_concurrent_shapes", E.EGPE_MIXED, 2)):
        runs[name] = run(prec, batch, tol_res)
    Ebest = [min(runs[k][1][i]["E"] for k in runs) for i in range(len(ws))]
    for name, (secs, reps) in runs.items():
        d = [(r["E"] - b) / abs(b) for r, b in zip(reps, Ebest)]
        iters = sum(r["iters"] for r in reps)
        out[name] = {"seconds": round(secs, 4), "iters_total": iters, "iters_fp32_total": sum(r["iters_fp32"] for r in reps),
                     "instances_within_1e-8_of_best": sum(x <= 1e-8 for x in d),
                     "worse_than_best": {str(i): x for i, x in enumerate(d) if x > 1e-8},
                     "all_converged": all(r["status"] == 0 for r in reps)}
    out["speedup_mixed_batched_vs_fp64_one_by_one"] = round(runs["fp64_one_by_one"][0] / runs["mixed_batched"][0], 3)
    out["batching"] = ("mixed_batched: one launch per pass for the instances of each grid shape, the shapes one "
                       "after the other (batch=1, the default); mixed_batched_concurrent_shapes: the four shapes' "
                       "launch chains as concurrent graph branches (batch=2)")
    return out


def param_grad_timing(E, reps=5):
    """Device time of the parameter-derivative pass (dE/d(g, g_dd, kappa, eta_s,
    lambda), the autograd extension) on the 256x256x128 workload beside one
    energy/gradient evaluation, FP64 and FP32 fields; wall time per call with a
    synchronisation on both sides."""
    import torch

    from paper_2510_24543_gb300 import inputs as I

    w = I.PRESETS["c5"]
    psi64 = torch.from_numpy(I.gaussian_start(w)).to("cuda")
    out = {"workload": w.name, "points": w.points}
    for name, prec, psi in (("fp64", E.EGPE_FP64, psi64), ("fp32", E.EGPE_FP32, psi64.to(torch.complex64))):
        h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
        try:
            grad = torch.empty_like(psi)
            E.egpe_param_grad(h, 0, psi)
            E.egpe_energy_grad(h, 0, psi, grad)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                E.egpe_param_grad(h, 0, psi)
            torch.cuda.synchronize()
            t_pg = (time.perf_counter() - t0) / reps
            t0 = time.perf_counter()
            for _ in range(reps):
                E.egpe_energy_grad(h, 0, psi, grad)
            torch.cuda.synchronize()
            t_eg = (time.perf_counter() - t0) / reps
        finally:
            E.egpe_destroy(h)
        out[name] = {"param_grad_ms": round(t_pg * 1e3, 3), "energy_grad_ms": round(t_eg * 1e3, 3)}
    return out


def precond_study(E, tol_res=1e-6, per_grid=4):
    """Iterations and time to ||r|| < tol_res per preconditioner (Sec. IV.B and
    the paper's Fig. 1a/b comparison of P_V and P_Delta, here on synthetic scan
    instances): 4 instances of each scan grid, FP64, solved together."""
    import torch

    from paper_2510_24543_gb300 import inputs as I

    scan = I.scan_workloads()
    ws = [scan[16 * g + k] for g in range(4) for k in range(per_grid)]
    grids = [E.make_grid(w.n, w.L) for w in ws]
    prms = [E.params_from_workload(w) for w in ws]
    out = {"instances": len(ws), "tol_res": tol_res, "precision": "fp64", "modes": {}}
    for mode in ("kinetic", "diagonal", "kinetic+diagonal", "blend"):
        h = E.egpe_create(grids, prms, E.EGPE_FP64)
        try:
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND[mode]
            o.tol_res = tol_res
            o.max_iter = 6000
            o.pc_blend = 0.5
            xs = [torch.from_numpy(I.gaussian_start(w)).to("cuda") for w in ws]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, reps, _ = E.egpe_ncg_solve(h, xs, o, len(ws))
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        finally:
            E.egpe_destroy(h)
        its = sorted(r["iters"] for r in reps)
        out["modes"][mode] = {"seconds": round(secs, 3), "iters_total": sum(its), "iters_median": its[len(its) // 2],
                              "iters_max": its[-1], "converged": sum(r["status"] == 0 for r in reps)}
    return out


def continuation_benchmark(E, tol_res=1e-6, tune=True):
    """Continuation along the 64-instance scan (the paper's proposal for
    phase-diagram sweeps): per grid size, the 16 parameter points are chained
    nearest-neighbour in the normalised (g12, g_dd) plane and solved with
    egpe_ncg_continuation (each solve warm-started from the previous ground
    state), against cold solves of the same points from their seeded starts;
    mixed precision, P_Delta o P_V, ||r|| < tol_res."""
    import torch

    from paper_2510_24543_gb300 import autotune as AT
    from paper_2510_24543_gb300 import inputs as I

    ws = I.scan_workloads()
    device = torch.cuda.get_device_name()
    out = {"instances": len(ws), "tol_res": tol_res, "groups": []}
    tot = {"cold_s": 0.0, "warm_s": 0.0, "cold_iters": 0, "warm_iters": 0}
    same = lower = higher = 0
    for size in (48, 64, 80, 96):
        grp = [w for w in ws if w.n[0] == size]
        pts = [((w.g[0][1] - 100.0) / 250.0, (w.gdd[0][0] - 250.0) / 200.0) for w in grp]
        order, left = [min(range(len(grp)), key=lambda i: pts[i][0])], set(range(len(grp)))
        left.discard(order[0])
        while left:
            last = pts[order[-1]]
            nxt = min(left, key=lambda i: (pts[i][0] - last[0]) ** 2 + (pts[i][1] - last[1]) ** 2)
            order.append(nxt)
            left.discard(nxt)
        path = [grp[i] for i in order]
        prms = [E.params_from_workload(w) for w in path]
        h = E.egpe_create([E.make_grid(path[0].n, path[0].L)], [prms[0]], E.EGPE_MIXED)
        try:
            if tune:
                AT.tune_handle(h, [path[0].n], E.EGPE_MIXED, E.PRECOND[path[0].precond],
                               lambda i, e: torch.from_numpy(I.gaussian_start(path[0])).to("cuda").to(
                                   torch.complex128 if e == 0 else torch.complex64), device)
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND[path[0].precond]
            o.tol_res = tol_res
            o.max_iter = 6000
            o.max_iter_fp32 = 6000
            cold = []
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for w, p in zip(path, prms):
                E.egpe_set_params(h, 0, p)
                x = torch.from_numpy(I.gaussian_start(w)).to("cuda")
                st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
                cold.append(reps[0])
            torch.cuda.synchronize()
            t_cold = time.perf_counter() - t0
            x = torch.from_numpy(I.gaussian_start(path[0])).to("cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, warm = E.egpe_ncg_continuation(h, 0, prms, x, o)
            torch.cuda.synchronize()
            t_warm = time.perf_counter() - t0
        finally:
            E.egpe_destroy(h)
        for c, wr in zip(cold, warm):
            best = min(c["E"], wr["E"])
            dc, dw = (c["E"] - best) / abs(best), (wr["E"] - best) / abs(best)
            if dc <= 1e-8 and dw <= 1e-8:
                same += 1
            elif dw <= 1e-8:
                lower += 1
            else:
                higher += 1
        g = {"grid": size, "cold_s": round(t_cold, 3), "warm_s": round(t_warm, 3),
             "cold_iters": sum(r["iters"] for r in cold), "warm_iters": sum(r["iters"] for r in warm),
             "all_converged": all(r["status"] == 0 for r in cold + warm)}
        out["groups"].append(g)
        for k in tot:
            tot[k] += g[k]
    out.update({k: round(v, 3) if isinstance(v, float) else v for k, v in tot.items()})
    out["speedup"] = round(tot["cold_s"] / tot["warm_s"], 3)
    out["points_same_minimum"] = same
    out["points_warm_lower"] = lower
    out["points_warm_higher"] = higher
    return out


def host_cpu():
    """Core count and CPU model of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model or "unknown"


def cpu_baseline(w):
    """The FP64 oracle as it stands on this host: one NCG iteration (precondition,
    line coefficients, trial evaluation) of the same 128^3 workload, its
    transforms on every host core (scipy.fft workers), its pointwise NumPy code
    on one."""
    import numpy as np  # noqa: F401

    import oracle as O
    from paper_2510_24543_gb300 import inputs as I

    cores, model = host_cpu()
    O.egpe.set_fft_workers(cores)
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    psi = I.gaussian_start(w)
    O.evaluate(g, prm, psi)  # warm-up: imports, transform plans, page-in
    t0 = time.perf_counter()
    O.evaluate(g, prm, psi)
    t_eval = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, rep = O.ncg_solve(g, prm, psi, O.SolveOpts(precond=w.precond if w.precond in O.PRECOND_MODES else "kinetic",
                                                   max_iter=1, tol_res=0.0))
    t_solve = time.perf_counter() - t0
    t_it = max(t_solve - t_eval, 1e-9)
    O.egpe.set_fft_workers(None)
    return {"value": round(1.0 / t_it, 5), "unit": UNIT, "cores": cores, "cpu_model": model, "kind": "oracle",
            "sample": f"one oracle NCG iteration on the full {w.n[0]}x{w.n[1]}x{w.n[2]} workload "
                      f"({t_it:.1f} s; its initial evaluation, {t_eval:.1f} s, timed separately and excluded); "
                      f"transforms on {cores} threads (scipy.fft), pointwise NumPy code on one"}


# ---------------------------------------------------------------------------
def run_reference(args):
    """The FP64 CPU oracle timed on this host on the same workload and metric."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_2510_24543_gb300 import inputs as I

    w = I.PRESETS[args.workload]
    cores, model = host_cpu()
    O.egpe.set_fft_workers(cores)
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    psi = I.gaussian_start(w)
    budget = 150.0
    O.evaluate(g, prm, psi)  # warm-up: imports, transform plans, page-in
    t0 = time.perf_counter()
    ev = O.evaluate(g, prm, psi)
    t_eval = time.perf_counter() - t0
    # warm-up: one evaluation counts as the oracle's warm-up (no JIT, no cache to fill)
    per_it = 2.0 * t_eval
    k = max(1, min(args.steps, int(budget / max(per_it, 1e-3))))
    t0 = time.perf_counter()
    _, rep = O.ncg_solve(g, prm, psi, O.SolveOpts(precond=args.precond, max_iter=k, tol_res=0.0))
    t_solve = time.perf_counter() - t0 - t_eval
    done = rep["iters"]
    value = done / t_solve
    line = {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": done,
            "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_solve / done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian + 1% noise start)", "impl": "reference",
            "config": {"workload": w.name, "grid": list(w.n), "precond": args.precond},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "cpu_model": model,
                             "kind": "oracle",
                             "sample": f"first {done} oracle NCG iterations on the full workload (bounded to "
                                       f"~{int(budget)} s), initial evaluation excluded; transforms on {cores} "
                                       "threads (scipy.fft), pointwise NumPy code on one"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_table(args):
    """Per-workload figures: the FP64 oracle's seconds per NCG iteration and per
    ITE step and its time to ground state (single host thread), the GPU's time
    to ground state at 1e-8 relative energy (plain FP64 and mixed precision),
    and the FP32 energy/gradient pass against the measured HBM peak.  Oracle
    times to ground state on the larger workloads are seconds per iteration
    times the iterations the GPU FP64 solve needed (labelled)."""
    import torch

    from paper_2510_24543_gb300 import egpe as E
    from paper_2510_24543_gb300 import inputs as I

    if not args.no_cpu:
        import oracle as O  # the CPU baseline columns only
    E.load()
    hbm, _ = peaks()
    rows = {}
    for key in ("c1", "c2", "c3", "c3p", "c5"):
        w = I.PRESETS[key]
        grid, prm = E.make_grid(w.n, w.L), E.params_from_workload(w)
        pc = E.PRECOND[w.precond]
        psi0 = I.gaussian_start(w)
        psi64 = torch.from_numpy(psi0).to("cuda")
        h = E.egpe_create([grid], [prm], E.EGPE_MIXED)
        try:
            tts = time_to_ground_state(E, h, grid, prm, psi64, pc, args.fp32_switch)
            prof = E.egpe_profile_attempt(h, 0, 1, psi64.to(torch.complex64), pc, reps=3)
        finally:
            E.egpe_destroy(h)
        eg = prof[-5:]  # the trial energy/gradient pass: x fwd, y, z fused, y, x inv
        eg_gbs = sum(b for _, _, b in eg) / (sum(t for _, t, _ in eg) * 1e-3) / 1e9
        en, rs = tts["energy_1e-8"], tts["residual_1e-8"]
        gpu_cols = {"grid": list(w.n),
                    "gpu_fp64_tts_energy_s": round(en["fp64"]["seconds"], 4),
                    "gpu_fp32_tts_energy_s": round(en["fp32_fields"]["seconds"], 4),
                    "fp32_energy_err_fp64_eval": en["fp32_fields"]["rel_err_fp64_eval"],
                    "gpu_fp64_tts_res_s": round(rs["fp64"]["seconds"], 4),
                    "gpu_mixed_tts_res_s": round(rs["mixed"]["seconds"], 4),
                    "gpu_mixed_iters": [rs["mixed"]["iters_fp32"], rs["mixed"]["iters"]],
                    "gpu_fp64_iters": rs["fp64"]["iters"], "fp32_eg_pass_frac_hbm": round(eg_gbs / hbm, 3)}
        if key in ("c3", "c3p") and not args.no_cpu:
            gpu_cols["mixed_accuracy"] = mixed_accuracy(E, w, pc, args.fp32_switch)
        if args.no_cpu:  # GPU columns only
            rows[key] = gpu_cols
            print(json.dumps({key: rows[key]}), flush=True)
            continue
        g = O.Grid(w.n, w.L)
        op = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
        t0 = time.perf_counter()
        O.evaluate(g, op, psi0)
        t_eval = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.ncg_solve(g, op, psi0, O.SolveOpts(precond=w.precond, tol_res=0.0, max_iter=1))
        s_iter = max(time.perf_counter() - t0 - t_eval, 1e-9)
        row = {"oracle_s_per_iter": round(s_iter, 3), "fp32_eg_pass_GBs": round(eg_gbs, 1), **gpu_cols}
        if key in ("c1", "c2"):
            t0 = time.perf_counter()
            O.ite_solve(g, op, psi0, dtau=1e-3, tol_dE=0.0, max_steps=2)
            row["oracle_s_per_ite_step"] = round((time.perf_counter() - t0 - 2 * t_eval) / 2, 3)
            t0 = time.perf_counter()
            _, rep = O.ncg_solve(g, op, psi0, O.SolveOpts(precond=w.precond, tol_res=en["res_target"]))
            row["oracle_tts_s"] = round(time.perf_counter() - t0, 2)
            row["oracle_tts_iters"] = rep["iters"]
        else:
            row["oracle_tts_s_extrapolated"] = round(s_iter * en["fp64"]["iters"] + t_eval, 1)
        rows[key] = row
        print(json.dumps({key: row}), flush=True)
    if args.no_cpu:
        print(json.dumps({"table": rows}))
        return
    # the 64-instance scan: oracle seconds per iteration on one sampled instance per grid size
    scan = I.scan_workloads()
    c4 = {}
    for k in (0, 16, 32, 48):
        w = scan[k]
        g = O.Grid(w.n, w.L)
        op = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
        psi0 = I.gaussian_start(w)
        t0 = time.perf_counter()
        O.evaluate(g, op, psi0)
        t_eval = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.ncg_solve(g, op, psi0, O.SolveOpts(precond=w.precond, tol_res=0.0, max_iter=1))
        c4[f"{w.n[0]}^3"] = round(max(time.perf_counter() - t0 - t_eval, 1e-9), 3)
    rows["c4_oracle_s_per_iter_sampled"] = c4
    print(json.dumps({"table": rows}))


def main():
    args = parse()
    if args.table:
        config_table(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
