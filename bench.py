#!/usr/bin/env python
"""Throughput of the pseudospectral ImEx-ARK phase-field hot path on GB300.

Workload (FP64 against FP32-bulk integrated to a fixed simulated time, with
the error per field): 256^3 periodic grid, 4 fields (X, phi_1..3), 32 seeded
spherical gamma'' nuclei (radius 4-10 cells, composition at the precipitate
value inside),
ARK4(3)6L[2]SA with the embedded-error WRMS controller at rtol 1e-4,
atol 1e-8, integrated from t = 0 (h0 = 1 s) to t_final = 60 s.  One bench
step = one such integration: every controller-driven step attempt (6 stages,
each a full explicit RHS evaluation -- 14 real 3D FFTs with the physics fused
in -- plus the implicit stage solves, the step completion, the embedded local
error, its WRMS norm and the accept/reject decision) until t_final.

Headline value: Gpt-stage/s (grid points x RHS evaluations per second,
rejected attempts included) of the FP32-bulk form (FFTs/RHS in FP32; state,
norm and controller in FP64; stage vectors and their combinations in
double-float, ~47 significant bits).  The same line carries, for the same
integration: simulated seconds per wall second of the FP32-bulk form and of
the plain FP64 GPU path, their ratio (the gain at the same end time and
tolerance), the FP32-bulk final state's error per field against the FP64
final state, and both forms' errors against a tight-tolerance FP64
integration (rtol 1e-6), which shows the two reach the same final-state
error.  Every array a step streams (the FP64 state alone is 512 MiB at
256^3; ~7 GB of step buffers in all) is far larger than the 129 MB L2, so no
flush is needed between steps.

Further legs on the same line: the 640^3 / 300-nucleus workload (the
largest single-GPU configuration) over a bounded stretch of simulated time,
the uneven-grid ensemble advanced to 60 s, the surrogate, the measured FMA
peaks, and the FP64 oracle on the host cores.

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on bounded samples of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated s per wall s at fixed tol vs plain FP64 GPU; Gpt-stage/s; % HBM BW"
UNIT = "Gpt-stage/s"
WORKLOAD2 = ("256^3 gamma'' KKS phase field (4 fields), 32 seeded nuclei r 4-10 cells, ARK4(3)6L[2]SA adaptive "
             "rtol 1e-4 atol 1e-8 from t=0 (h0=1 s) to t_final=60 s; FP32-bulk (FP64 state/norms) vs plain FP64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5, help="timed integrations to t_final")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--t-final", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 integration")
    ap.add_argument("--no-tight", action="store_true", help="skip the tight-tolerance FP64 reference")
    ap.add_argument("--big", type=int, default=640, help="side of the largest-grid leg (0: skip)")
    ap.add_argument("--big-t", type=float, default=20.0, help="simulated seconds of the largest-grid leg")
    ap.add_argument("--ensemble", type=int, default=64, help="members of the batched-ensemble measurement (0: skip)")
    ap.add_argument("--ensemble-t", type=float, default=60.0, help="simulated seconds of the ensemble measurement")
    ap.add_argument("--surrogate", type=int, default=24, help="training trajectories of the surrogate measurement (0: skip)")
    ap.add_argument("--sweep", action="store_true", help="add the work-precision sweep of the two-particle test")
    ap.add_argument("--hc", type=int, default=128, help="side of the phase-dependent-stiffness leg (0: skip)")
    ap.add_argument("--elastic-form", default="-1",
                    help="after autotuning, run this form of the elastic pass in the FP32-bulk main leg "
                         "(0 fused stage, 1 stages over three fields, 2 three-CTA cluster; -1: the autotuner's), "
                         "optionally with its tile width as FORM:COLUMNS")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler over the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
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
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def traffic_from_profiles(kernel, precision, n):
    """ncu DRAM bytes per launch of `kernel` on the n^3 workload, recorded
    under profiles/ for the current kernel source, or None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(precision, {}).get(kernel)
        if e is None or int(e.get("grid", 0)) != n:
            return None
        return float(e["dram_bytes_per_launch_full"])
    except Exception:
        return None


def relerr(a, b):
    import numpy as np
    return [float(np.linalg.norm((a[f] - b[f]).ravel()) / np.linalg.norm(b[f].ravel())) for f in range(a.shape[0])]


# nominal FP64 flops of one explicit RHS evaluation per grid point: 14 real
# 3D transforms at 2.5 log2(N) flops per point each (half of the 5 N log2 N
# of a complex transform) plus ~300 flops of pointwise physics and elastic
# kernel; the stage sums add ~50
def nominal_flops_per_point_stage(N):
    import math
    return 14 * 2.5 * math.log2(N) + 350.0


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_2609_36100_gb300 as pfg
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    pfg.build()
    p = synth.load_params()
    n = args.n
    T = args.t_final
    y0 = synth.ic_spheres(n, 32 if n >= 256 else max(4, 32 * n ** 3 // 256 ** 3), 4.0, 10.0, 2, p)
    stream = torch.cuda.current_stream()
    N = n ** 3

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    y0_dev = torch.from_numpy(y0).to("cuda")

    def new_sim(prec, rtol=1e-4, tune=True):
        sim = pfg.Simulation((n, n, n), p, "ark4", prec)
        sim.set_state(y0_dev)
        tuning = sim.autotune(reps=2) if tune else None
        form, _, width = str(args.elastic_form).partition(":")
        if tune and prec == "fp32bulk" and int(form) >= 0:
            cfg = sim.tuning()
            cfg[40] = int(form)
            if width:
                cfg[2] = int(width)
            sim.set_tuning(cfg)
            tuning = dict(tuning, cfg=sim.tuning(), elastic_form_forced=args.elastic_form)
        return sim, tuning, sim.state_hat()

    def integrate(sim, y0h, rtol=1e-4):
        sim.set_state_hat(y0h)
        sim.set_time(0.0, 1.0)
        return sim.advance(T, rtol, 1e-8)

    def timed(sim, y0h, K, W, clocks=False, rtol=1e-4):
        """W untimed integrations, then K timed ones (CUDA events on the
        launching stream, barrier + synchronize on both sides)."""
        clk = Clocks(local) if (clocks and rank == 0) else None
        for _ in range(W):
            integrate(sim, y0h, rtol)
        barrier()
        st0 = sim.stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include timed/ selects these launches
        e0.record(stream)
        for _ in range(K):
            integrate(sim, y0h, rtol)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        st1 = sim.stats()
        att = sim.attempts()
        rhs = (st1["rhs_evals"] - st0["rhs_evals"]) // K
        return {"ms_per_integration": ms / K, "rhs_per_integration": rhs,
                "accepted": sum(1 for a in att if a[3]), "rejected": sum(1 for a in att if not a[3]),
                "h_last": att[-1][1] if att else None, "h_max": max((a[1] for a in att if a[3]), default=None),
                "gpt_stage_s": rhs * N * world / (ms / K / 1e3) / 1e9,
                "sim_s_per_wall_s": T / (ms / K / 1e3),
                "clocks": clk.stop() if clk else None}

    K, W = args.steps, args.warmup
    s32, tun32, y0h = new_sim("fp32bulk")
    r32 = timed(s32, y0h, K, W, clocks=True)
    final32 = s32.get_state()
    # per-kernel CUDA events over one more integration (kept out of the headline)
    s32.profile(True)
    barrier()
    integrate(s32, y0h)
    barrier()
    prof = s32.profile_read()
    s32.profile(False)
    top = max(prof.items(), key=lambda kv: kv[1][0])
    kname, (kms, kbytes, klaunch) = top
    hbm, src = peaks()
    achieved = kbytes / (kms / 1e3) / 1e9
    launches = int(sum(v[2] for v in prof.values()))
    # end to end through the public API with host buffers: the real-space
    # initial state copied host -> device, the integration to t_final, the
    # real-space final state copied device -> host, every step
    host_in = torch.from_numpy(y0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def e2e_step():
        s32.set_state(host_in)
        s32.set_time(0.0, 1.0)
        s32.advance(T, 1e-4, 1e-8)
        s32.get_state(host_out)

    e2e_step()
    barrier()
    st0 = s32.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    Ke = max(2, K // 2)
    e0.record(stream)
    for _ in range(Ke):
        e2e_step()
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))
    st1 = s32.stats()
    e2e_value = (st1["rhs_evals"] - st0["rhs_evals"]) * N * world / (ms_e2e / 1e3) / 1e9
    s32.close()
    del y0h
    out = {}
    fp64 = None
    if not args.no_fp64:
        s64, _, y0h = new_sim("fp64", tune=False)
        r64 = timed(s64, y0h, 1, 1)
        final64 = s64.get_state()
        fl = nominal_flops_per_point_stage(N)
        fp64 = dict(r64, nominal_tflops=r64["gpt_stage_s"] * 1e9 * fl / 1e12,
                    nominal_flops_per_point_stage=fl)
        out["error_per_field_fp32bulk_vs_fp64"] = relerr(final32, final64)
        if not args.no_tight:
            # tight-tolerance FP64 integration: both forms' final-state errors
            s64.set_state_hat(y0h)
            s64.set_time(0.0, 0.25)
            stt = s64.advance(T, 1e-6, 1e-10)
            tight = s64.get_state()
            out["final_state_error_vs_rtol1e-6_fp64"] = {
                "fp64": relerr(final64, tight), "fp32bulk": relerr(final32, tight),
                "tight_attempts": int(stt["steps_accepted"] + stt["steps_rejected"])}
        s64.close()
        del y0h
    fma = {"fp64_tflops": pfg.fma_peak("fp64"), "fp32_tflops": pfg.fma_peak("fp32")}
    if fp64:
        fp64["frac_of_measured_fp64_fma_peak"] = fp64["nominal_tflops"] / fma["fp64_tflops"]
    line = {
        "metric": METRIC, "value": r32["gpt_stage_s"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": r32["ms_per_integration"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 transforms/RHS, f64 state/norms", "data": "synthetic",
        "config": {"workload": WORKLOAD2.replace("256^3", "%d^3" % n).replace("t_final=60 s", "t_final=%g s" % T),
                   "grid": [n, n, n], "fields": 4, "method": "ARK4(3)6L[2]SA", "precision": "fp32bulk",
                   "rtol": 1e-4, "atol": 1e-8, "t_final": T, "step": "one integration from t=0 to t_final",
                   "l2": "inputs larger than L2 (FP64 k-space state %.0f MiB; no flush needed)" % (
                       4 * n * n * (n // 2 + 1) * 16 / 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "sim_s_per_wall_s": r32["sim_s_per_wall_s"],
        "fp32bulk": {k: v for k, v in r32.items() if k != "clocks"},
        "fp64_plain": fp64,
        "gain_at_equal_time": (r32["sim_s_per_wall_s"] / fp64["sim_s_per_wall_s"]) if fp64 else None,
        "autotune": {"fp32bulk": {k: tun32[k] for k in ("ms_before", "ms_after", "cfg")}},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": src,
                     "algorithmic_bytes_per_launch": kbytes / klaunch, "launches": int(klaunch),
                     "traffic": traffic_from_profiles(kname, "fp32bulk", n),
                     "timing": "CUDA events around every launch over one further integration"},
        "kernels": {k: {"ms": v[0], "launches": int(v[2]), "GBps": v[1] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None,
                        "frac_of_hbm": v[1] / (v[0] / 1e3) / 1e9 / hbm if v[0] > 0 else None,
                        "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()},
        "gpu_launches": launches * K,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(y0.nbytes),
                "d2h_bytes_per_step": int(y0.nbytes), "steps": Ke},
        "fma_peak_measured": fma,
        "clocks": r32["clocks"],
    }
    line.update(out)
    return line


def run_big(n, t_final, rank=0, world=1):
    """The largest single-GPU configuration: n^3 grid, 300 non-overlapping
    nuclei of radius 4-12 cells, ARK4 adaptive at rtol 1e-4 in FP32-bulk from
    t = 0 (h0 = 1 s) to t_final (a bounded stretch of the configuration's
    300 s), with per-kernel rooflines; the plain FP64 path over two attempts
    for the throughput ratio."""
    import torch

    import paper_2609_36100_gb300 as pfg
    import synth

    p = synth.load_params()
    w0 = time.perf_counter()
    y0 = synth.ic_spheres(n, 300, 4.0, 12.0, 5, p)
    t_ic = time.perf_counter() - w0
    N = n ** 3
    hbm, _ = peaks()
    y0d = torch.from_numpy(y0).to("cuda")
    del y0
    res = {"grid": [n, n, n], "nuclei": 300, "t_final": t_final, "ic_s": t_ic}
    for prec in ("fp32bulk", "fp64"):
        sim = pfg.Simulation((n, n, n), p, "ark4", prec)
        sim.set_state(y0d)
        if prec == "fp32bulk":
            res["autotune"] = sim.autotune(reps=1)
        sim.set_time(0.0, 1.0)
        sim.advance_attempts(1)  # warm-up
        torch.cuda.synchronize()
        sim.set_state(y0d)
        sim.set_time(0.0, 1.0)
        st0 = sim.stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        if prec == "fp32bulk":
            sim.advance(t_final, 1e-4, 1e-8)
        else:
            sim.advance_attempts(2, t_final, 1e-4, 1e-8)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st1 = sim.stats()
        rhs = st1["rhs_evals"] - st0["rhs_evals"]
        r = {"ms": ms, "attempts": len(sim.attempts()), "sim_s": st1["t"] - st0["t"],
             "gpt_stage_s": rhs * N / (ms / 1e3) / 1e9, "sim_s_per_wall_s": (st1["t"] - st0["t"]) / (ms / 1e3)}
        if prec == "fp32bulk":
            sim.profile(True)
            sim.set_time(0.0, 1.0)
            sim.advance_attempts(2, 1e30, 1e-4, 1e-8)
            prof = sim.profile_read()
            sim.profile(False)
            r["kernels"] = {k: {"ms": v[0], "launches": int(v[2]),
                                "GBps": v[1] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None,
                                "frac_of_hbm": v[1] / (v[0] / 1e3) / 1e9 / hbm if v[0] > 0 else None,
                                "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}
        res[prec] = r
        sim.close()
        torch.cuda.synchronize()
    res["gain_fp32bulk_vs_fp64_gpt_stage_s"] = res["fp32bulk"]["gpt_stage_s"] / res["fp64"]["gpt_stage_s"]
    return res


def run_hc(n=128, t_final=20.0):
    """Phase-dependent stiffness (Hu-Chen iterations, FP64) on an n^3 state of
    the 256^3 recipe scaled down (32 n^3/256^3 nuclei, at least 4), with a
    precipitate stiffer than the matrix (C11, C12, C44 up 30, 10, 20 %):
    ARK4 adaptive at rtol 1e-4 from t = 0 (h0 = 1 s) to t_final with the
    loose elastic tolerance of Sec. 2.3 (1e-6) and a tight one (1e-12), and
    the homogeneous modulus on the same state for the cost of the iterations.
    Returns wall time, RHS evaluations and elastic solves per RHS evaluation
    (each attempt's RHS evaluations counted at the solve count of its last
    one, which the library reports)."""
    import torch

    import paper_2609_36100_gb300 as pfg
    import synth

    p = synth.load_params()
    y0 = synth.ic_spheres(n, max(4, 32 * n ** 3 // 256 ** 3), 4.0, 10.0, 2, p)
    y0d = torch.from_numpy(y0).to("cuda")
    base = dict(p, C11_v=1.3 * p["C11"], C12_v=1.1 * p["C12"], C44_v=1.2 * p["C44"], el_max_iter=200)
    res = {"grid": [n, n, n], "t_final": t_final, "contrast": "C11 +30 %, C12 +10 %, C44 +20 % in the precipitate",
           "runs": []}
    for prec in ("fp32bulk", "fp64"):
        for label, extra in (("homogeneous", {"el_inhom": 0}), ("loose 1e-6", {"el_inhom": 1, "el_tol": 1e-6}),
                             ("tight 1e-12", {"el_inhom": 1, "el_tol": 1e-12})):
            q = dict(base, **extra)
            with pfg.Simulation((n, n, n), q, "ark4", prec) as sim:
                sim.set_state(y0d)
                sim.set_time(0.0, 1.0)
                sim.advance_attempts(1)  # warm-up
                sim.set_state(y0d)
                sim.set_time(0.0, 1.0)
                torch.cuda.synchronize()
                st0 = sim.stats()
                w0 = time.perf_counter()
                solves = 0
                rhs = 0
                # attempt by attempt, to count the elastic solves of every RHS
                while sim.time()[0] < t_final - 1e-9:
                    r0 = sim.stats()["rhs_evals"]
                    sim.advance_attempts(1, t_final, 1e-4, 1e-8)
                    d = sim.stats()["rhs_evals"] - r0
                    rhs += d
                    solves += d * sim.elastic_iterations()
                torch.cuda.synchronize()
                wall = time.perf_counter() - w0
                st1 = sim.stats()
                res["runs"].append({"precision": prec, "elastic": label, "wall_s": wall,
                                    "attempts": int(st1["steps_accepted"] + st1["steps_rejected"]
                                                    - st0["steps_accepted"] - st0["steps_rejected"]),
                                    "rhs_evals": rhs, "elastic_solves_per_rhs": solves / max(rhs, 1),
                                    "ms_per_rhs": wall * 1e3 / max(rhs, 1),
                                    "sim_s_per_wall_s": t_final / wall})
    return res


def run_ensemble(K, t_final, rank=0, world=1):
    """Ensembles advanced to t_final (ARK4 adaptive, rtol 1e-4, atol 1e-8):
    every member one after another with pf_advance, then the same states
    together with pf_batch_advance (one launch of the device-looped graph).

    - "uneven": members 0..K-1 of the seeded uneven-grid recipe (sides from
      {64,96,120,128,160}, 4-24 nuclei, T0 +/- 20 K), FP32-bulk, and the plain
      FP64 path advanced member by member as the comparison point;
    - "small": K members of 32^3 and 48^3 (4 nuclei each), FP32-bulk, where a
      single member's kernels no longer fill the GPU."""
    import torch

    import paper_2609_36100_gb300 as pfg
    import synth
    from paper_2609_36100_gb300.dist import max_over_ranks, shard, sum_over_ranks

    p = synth.load_params()
    ids = shard(K, rank, world)  # members shard across ranks (no collective on the data path)
    recipes = {
        "uneven": [synth.ensemble_member(i) for i in ids],
        "small": [(synth.ic_spheres((32, 48)[i % 2], 4, 3.0, 5.0, 300 + i, p), p) for i in ids],
    }
    stream = torch.cuda.current_stream()
    dev = "cuda"
    tuned = {}

    def timed(mem, prec, fn):
        sims = []
        for y0, q in mem:
            s = pfg.Simulation(y0.shape[1:], q, "ark4", prec)
            s.set_state(y0)
            key = (y0.shape[1:], prec)  # one autotuned schedule per grid size
            if key not in tuned:
                tuned[key] = s.autotune(reps=1)["cfg"]
            s.set_tuning(tuned[key])
            s.set_time(0.0, 1.0)
            sims.append(s)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(sims)
        e1.record(stream)
        torch.cuda.synchronize()
        st = [s.stats() for s in sims]
        for s in sims:
            s.close()
        ms = max_over_ranks(e0.elapsed_time(e1), dev)
        ps = sum_over_ranks(sum(x["point_stages"] for x in st), dev)
        return {"ms": ms, "gpt_stage_s": ps / (ms / 1e3) / 1e9, "sim_s_per_wall_s": K * t_final / (ms / 1e3)}

    out = {"members": K, "ranks": world, "t_final": t_final}
    for name, mem in recipes.items():
        r = {"sides_rank0": sorted({int(y0.shape[1]) for y0, _ in mem}),
             "points": int(sum_over_ranks(sum(y0[0].size for y0, _ in mem), dev))}
        r["sequential"] = timed(mem, "fp32bulk", lambda sims: [s.advance(t_final, 1e-4, 1e-8) for s in sims])
        r["batched"] = timed(mem, "fp32bulk", lambda sims: pfg.batch_advance(sims, t_final, 1e-4, 1e-8))
        r["batched"]["rounds"], r["batched"]["device_looped"] = pfg.batch_last()
        r["gain_batched_vs_sequential"] = r["sequential"]["ms"] / r["batched"]["ms"]
        if name == "uneven":
            r["fp64_sequential"] = timed(mem, "fp64", lambda sims: [s.advance(t_final, 1e-4, 1e-8) for s in sims])
            r["gain_batched_fp32bulk_vs_fp64"] = r["fp64_sequential"]["ms"] / r["batched"]["ms"]
        out[name] = r
    return out


def run_surrogate(ntraj, n=128, dt=1.0, nsnap=25, epochs=1):
    """FNO (4 spectral layers, 12 modes, width 32, BF16 spectral weights)
    trained with the library's kernels on `ntraj` solver trajectories of the
    8-ellipsoid recipe scaled to n^3 (8 nuclei; ARK4 FP32-bulk, dt = 1 s,
    snapshots every tau = 8 s, 0-200 s), then rollouts of two held-out seeds
    to 200 s in windows of tau: each window proposed by the network and
    checked by the method's own adaptive integration of the window (rtol
    1e-4), against plain adaptive integration; final-state errors against an
    FP64 rtol 1e-8 reference."""
    import numpy as np
    import torch

    import synth
    from paper_2609_36100_gb300 import surrogate as S

    p = synth.load_params()
    ics = [(synth.ic_ellipsoids(n, 1000 + i, p), p) for i in range(ntraj)]
    w0 = time.perf_counter()
    traj = S.trajectories(ics, p, dt, nsnap)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - w0
    net = S.new_network((n, n, n))
    w0 = time.perf_counter()
    losses = S.train(net, traj, epochs, 1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - w0
    pairs = ntraj * nsnap * epochs
    del traj
    tau = 8 * dt
    t_end = nsnap * tau
    rows = []
    for seed in (2000, 2001):
        y0 = synth.ic_ellipsoids(n, seed, p)
        ref, _, _, _, _ = S.rollout(y0, p, t_end, tau, None, precision="fp64", rtol=1e-8, atol=1e-12)
        plain, wp, _, _, _ = S.rollout(y0, p, t_end, tau, None)
        sur, ws, acc, off, dists = S.rollout(y0, p, t_end, tau, net)
        e = lambda a: [float(np.linalg.norm(a[f] - ref[f]) / np.linalg.norm(ref[f])) for f in range(4)]  # noqa: E731
        rows.append({"seed": seed, "wall_plain_s": wp, "wall_surrogate_s": ws, "accepted": acc, "offered": off,
                     "proposal_wrms_distance": {"min": float(np.min(dists)), "median": float(np.median(dists)),
                                                "max": float(np.max(dists))},
                     "err_plain_per_field": e(plain), "err_surrogate_per_field": e(sur)})
    net.close()
    return {"grid": [n, n, n], "train_trajectories": ntraj,
            "train_note": "subsample of the 200-trajectory recipe (seeds 1000+), one Adam step per pair",
            "pairs_seen": pairs, "epochs": epochs, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "data_s": t_data, "train_s": t_train, "train_ms_per_pair": t_train / pairs * 1e3, "tau_s": tau,
            "t_end_s": t_end, "rollouts": rows,
            "wall_ratio_plain_over_surrogate": float(np.mean([r["wall_plain_s"] / r["wall_surrogate_s"] for r in rows])),
            "acceptance": "the method integrates every window itself; a proposal counts as accepted when its WRMS "
                     "distance to that verified state is <= 1, and the rollout always continues from the verified "
                     "state"}


def run_sweep(n=64, t_end=300.0):
    """Work-precision sweep on the two-particle geometry (Sec. 2.3, Fig. 4):
    the ImEx-ARK family of orders 1-4 at fixed step sizes and adaptively,
    FP64, each run's wall time and its L2 error at t_end against a
    tight-tolerance ARK4 reference (rtol 1e-8)."""
    import numpy as np
    import torch

    import paper_2609_36100_gb300 as pfg
    import synth

    p = synth.load_params()
    y0 = synth.ic_two_particle(n, p)
    shape = y0.shape[1:]

    def run(meth, dt=None, rtol=None):
        with pfg.Simulation(shape, p, meth, "fp64") as s:
            s.set_state(y0)
            s.set_time(0.0, dt if dt else 0.5)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            if dt:
                k = int(round(t_end / dt))
                for _ in range(k):
                    s.step(dt, want_lte=False)
            else:
                s.advance(t_end, rtol, rtol * 1e-4)
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
            st = s.stats()
            return s.get_state(), wall, st["rhs_evals"]

    ref, _, _ = run("ark4", rtol=1e-8)
    rows = []
    plan = [("euler", [0.0625, 0.125, 0.25, 0.5]), ("ark2", [0.25, 0.5, 1.0]), ("ark3", [0.5, 1.0, 1.5]),
            ("ark4", [1.0, 1.5, 2.0, 2.25])]
    for meth, dts in plan:
        for dt in dts:
            try:
                y, wall, rhs = run(meth, dt=dt)
                err = float(np.sqrt(np.mean((y - ref) ** 2)))
            except pfg.PFError as e:  # noqa: F841
                y, wall, rhs, err = None, None, None, None
            rows.append({"method": meth, "dt": dt, "wall_s": wall, "rhs_evals": rhs, "l2_error": err})
    for meth in ("ark2", "ark3", "ark4"):
        for rtol in (1e-4, 1e-6):
            y, wall, rhs = run(meth, rtol=rtol)
            rows.append({"method": meth, "adaptive_rtol": rtol, "wall_s": wall, "rhs_evals": rhs,
                         "l2_error": float(np.sqrt(np.mean((y - ref) ** 2)))})
    return {"grid": [n, n, n], "t_end": t_end, "reference": "ARK4 adaptive rtol 1e-8 atol 1e-12, FP64", "runs": rows}


def cpu_baseline(n, budget_s=15.0):
    """The FP64 oracle as it stands, timed on this host's cores on a bounded
    sample: explicit RHS evaluations of the same 256^3 workload."""
    import numpy as np  # noqa: F401

    import oracle
    import synth
    from oracle import model as om

    p = synth.load_params()
    y0 = synth.ic_spheres(n, 32 if n >= 256 else 4, 4.0, 10.0, 2, p)
    m = oracle.Model(y0.shape[1:], p)
    yh = m.to_k(y0)
    t0 = time.perf_counter()
    k = 0
    while True:
        m.rhs_explicit(yh)
        k += 1
        el = time.perf_counter() - t0
        if el > budget_s or k >= 8:
            break
    val = k * n ** 3 / el / 1e9
    return {"value": val, "unit": UNIT, "cores": om._WORKERS, "kind": "oracle",
            "sample": "%d explicit RHS evaluation(s) of the %d^3 32-sphere initial state (FP64 numpy/scipy, %.1f s)" % (k, n, el)}


def run_reference(args):
    import oracle
    import synth
    from oracle import model as om

    p = synth.load_params()
    n = args.n
    y0 = synth.ic_spheres(n, 32 if n >= 256 else 4, 4.0, 10.0, 2, p)
    m = oracle.Model(y0.shape[1:], p)
    yh = m.to_k(y0)
    # one bench step of the reference arm = one explicit RHS evaluation (one
    # stage of an ARK4 step) of the same workload
    for _ in range(args.warmup):
        m.rhs_explicit(yh)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m.rhs_explicit(yh)
    el = time.perf_counter() - t0
    val = args.steps * n ** 3 / el / 1e9
    sample = "%d explicit RHS evaluations (one ARK4 stage each) of the %d^3 workload" % (args.steps, n)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD2.replace("256^3", "%d^3" % n).replace("t_final=60 s", "t_final=%g s" % args.t_final),
                       "grid": [n, n, n], "implementation": "FP64 CPU oracle (numpy/scipy) on the host cores",
                       "step": "one explicit RHS evaluation (one ARK4 stage) of the initial state"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": om._WORKERS, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl")
        dist = td
    line = run_ours(args, rank, world, dist)
    if args.big > 0 and rank == 0:
        line["largest_grid"] = run_big(args.big, args.big_t)
    if args.ensemble > 0:
        line["ensemble"] = run_ensemble(args.ensemble, args.ensemble_t, rank, world)
    if args.sweep and rank == 0:
        line["work_precision"] = run_sweep()
    if args.hc > 0 and rank == 0:
        line["hu_chen"] = run_hc(args.hc)
    if args.surrogate > 0 and rank == 0:
        line["surrogate"] = run_surrogate(args.surrogate)
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.n)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
