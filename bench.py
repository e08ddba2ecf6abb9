#!/usr/bin/env python
"""Throughput of the pseudospectral ImEx-ARK phase-field hot path on GB300.

Workload: 256^3 periodic grid, 4 fields (X, phi_1..3), 32 seeded spherical
gamma'' nuclei (radius 4-10 cells, composition at the precipitate value
inside), ARK4(3)6L[2]SA with the embedded-error WRMS controller at rtol 1e-4,
atol 1e-8.  One bench step = one controller-driven step attempt: 6 stages
(each a full explicit RHS evaluation: 14 real 3D FFTs with the physics fused
in, plus the implicit stage solve), step completion, the embedded local
error, its WRMS norm and the accept/reject decision.

Headline value: Gpt-stage/s (grid points x RHS evaluations per second) of the
FP32-bulk form (FFTs/RHS in FP32; state, norm and controller in FP64; stage
vectors and their combinations in double-float, ~47 significant bits); the
plain FP64 GPU path is timed beside it.  Every array a step streams (the FP64
state alone is 512 MiB at 256^3; ~7 GB of step buffers in all) is far larger
than the 129 MB L2, so no flush is needed between steps.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the plain FP64 path")
    ap.add_argument("--ensemble", type=int, default=64, help="members of the batched-ensemble measurement (0: skip)")
    ap.add_argument("--ensemble-t", type=float, default=5.0, help="simulated seconds of the ensemble measurement")
    ap.add_argument("--surrogate", type=int, default=16, help="training trajectories of the surrogate measurement (0: skip)")
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
    if n == 640:
        y0 = synth.ic_config5(n, 5, p)  # 300 nuclei r in [4, 12] cells
    else:
        y0 = synth.ic_spheres(n, 32 if n >= 256 else max(4, 32 * n ** 3 // 256 ** 3), 4.0, 10.0, 2, p)
    stream = torch.cuda.current_stream()
    N = n ** 3
    out = {}

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

    def timed(prec, K, W, profile=False):
        """W warm-up attempts, K timed attempts (the headline), then -- with
        `profile` -- K more attempts with a CUDA event pair around every
        kernel (the per-kernel times and the roofline; the events add a few
        per cent to those attempts, so they are kept out of the headline)."""
        sim = pfg.Simulation((n, n, n), p, "ark4", prec)
        sim.set_state(y0)
        tuning = sim.autotune(reps=2)  # launch schedule picked by the autotuner
        sim.set_time(0.0, 1.0)
        # clocks sampled over the warm-up and timed attempts (identical work)
        clk = Clocks(local) if (profile and rank == 0) else None
        sim.advance_attempts(W)
        st0 = sim.stats()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include timed/ selects these launches
        e0.record(stream)
        sim.advance_attempts(K)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        wall = time.perf_counter() - w0
        ms = e0.elapsed_time(e1)
        st1 = sim.stats()
        prof, ms_prof = None, None
        if profile:
            sim.profile(True)
            barrier()
            e0.record(stream)
            sim.advance_attempts(K)
            e1.record(stream)
            barrier()
            ms_prof = e0.elapsed_time(e1)
            prof = sim.profile_read()
            sim.profile(False)
        clocks = clk.stop() if clk else None
        res = {"ms": max_over_ranks(ms), "wall": wall, "rhs": st1["rhs_evals"] - st0["rhs_evals"],
               "sim_s": st1["t"] - st0["t"], "accepted": st1["steps_accepted"] - st0["steps_accepted"],
               "rejected": st1["steps_rejected"] - st0["steps_rejected"], "prof": prof, "clocks": clocks,
               "sim": sim, "tuning": tuning, "ms_profiled": ms_prof}
        return res

    K, W = args.steps, args.warmup
    r32 = timed("fp32bulk", K, W, profile=True)
    units = r32["rhs"] * N * world
    value = units / (r32["ms"] / 1e3) / 1e9
    sim_rate = r32["sim_s"] / (r32["ms"] / 1e3)
    # dominant kernel and its live roofline
    prof = r32["prof"]
    top = max(prof.items(), key=lambda kv: kv[1][0])
    kname, (kms, kbytes, klaunch) = top
    hbm, src = peaks()
    achieved = kbytes / (kms / 1e3) / 1e9
    launches = int(sum(v[2] for v in prof.values()))
    # end to end through the public API with host buffers: H2D of the
    # real-space state, one step attempt, D2H of the real-space state
    sim = r32["sim"]
    host_in = torch.from_numpy(y0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for _ in range(2):
        sim.set_state(host_in)
        sim.advance_attempts(1)
        sim.get_state(host_out)
    barrier()
    st0 = sim.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    Ke = max(3, K // 2)
    e0.record(stream)
    for _ in range(Ke):
        sim.set_state(host_in)
        sim.advance_attempts(1)
        sim.get_state(host_out)
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))
    st1 = sim.stats()
    e2e_value = (st1["rhs_evals"] - st0["rhs_evals"]) * N * world / (ms_e2e / 1e3) / 1e9
    sim.close()
    out["fp32"] = r32
    fp64 = None
    if not args.no_fp64:
        r64 = timed("fp64", max(2, K // 2), 1, profile=True)
        v64 = r64["rhs"] * N * world / (r64["ms"] / 1e3) / 1e9
        p64 = r64["prof"]
        t64 = max(p64.items(), key=lambda kv: kv[1][0])
        fp64 = {"gpt_stage_s": v64, "ms_per_step": r64["ms"] / max(1, r64["rhs"] // 6),
                "sim_s_per_wall_s": r64["sim_s"] / (r64["ms"] / 1e3),
                "top_kernel": t64[0], "top_kernel_gbs": t64[1][1] / (t64[1][0] / 1e3) / 1e9}
        r64["sim"].close()
    r32["sim"].close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": r32["ms"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%d^3 gamma'' KKS phase field, %d seeded nuclei, ARK4(3)6L[2]SA adaptive "
                               "rtol 1e-4 atol 1e-8, FP32-bulk (FP64 state/norms)" % (n, 300 if n == 640 else 32),
                   "grid": [n, n, n], "fields": 4, "method": "ARK4(3)6L[2]SA", "precision": "fp32bulk",
                   "rtol": 1e-4, "atol": 1e-8, "l2": "inputs larger than L2 (FP64 k-space state %.0f MiB; no flush needed)" % (
                       4 * n * n * (n // 2 + 1) * 16 / 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "sim_s_per_wall_s": sim_rate,
        "autotune": {"fp32bulk": {k: r32["tuning"][k] for k in ("ms_before", "ms_after", "cfg")}},
        "attempts": {"accepted": r32["accepted"], "rejected": r32["rejected"], "sim_s": r32["sim_s"]},
        "fp64_plain": fp64,
        "gain_fp32bulk_vs_fp64": (value / fp64["gpt_stage_s"]) if fp64 else None,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": src,
                     "algorithmic_bytes_per_launch": kbytes / klaunch, "launches": int(klaunch),
                     "traffic": traffic_from_profiles(kname, "fp32bulk", n),
                     "timing": "CUDA events around every launch over %d further attempts (%.2f ms per attempt "
                               "with the events)" % (K, r32["ms_profiled"] / K)},
        "kernels": {k: {"ms": v[0], "launches": int(v[2]), "GBps": v[1] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None,
                        "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()},
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(y0.nbytes),
                "d2h_bytes_per_step": int(y0.nbytes), "steps": Ke},
        "clocks": r32["clocks"],
    }
    return line


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


def run_surrogate(ntraj, n=64, dt=1.0, nsnap=25, epochs=3):
    """FNO (4 spectral layers, 12 modes, width 32, BF16 spectral weights)
    trained with the library's kernels on `ntraj` solver trajectories of the
    64^3 8-nucleus recipe (ARK4 FP32-bulk, dt = 1 s, tau = 8 s, 0-200 s), then
    judged rollouts of two held-out seeds to 200 s: wall time, accepted
    proposals and final-state error against a dt = 0.25 s FP64 reference, with
    and without the network."""
    import numpy as np
    import torch

    import synth
    from paper_2609_36100_gb300 import surrogate as S

    p = synth.load_params()
    ics = [(synth.ic_config1(n, 1000 + i, p), p) for i in range(ntraj)]
    w0 = time.perf_counter()
    traj = S.trajectories(ics, p, dt, nsnap)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - w0
    net = S.new_network((n, n, n))
    w0 = time.perf_counter()
    losses = S.train(net, traj, epochs, 1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - w0
    del traj
    rows = []
    for seed in (2000, 2001):
        y0 = synth.ic_config1(n, seed, p)
        ref, _, _, _ = S.rollout(y0, p, nsnap * 8 * dt, 0.25, None, precision="fp64")
        plain, wp, _, _ = S.rollout(y0, p, nsnap * 8 * dt, dt, None)
        sur, ws, acc, off = S.rollout(y0, p, nsnap * 8 * dt, dt, net)
        e = lambda a: float(np.linalg.norm((a - ref)[1:]) / np.linalg.norm(ref[1:]))  # noqa: E731
        rows.append({"seed": seed, "wall_plain_s": wp, "wall_surrogate_s": ws, "accepted": acc, "offered": off,
                     "err_plain": e(plain), "err_surrogate": e(sur)})
    net.close()
    return {"grid": [n, n, n], "train_trajectories": ntraj, "pairs": ntraj * nsnap, "epochs": epochs,
            "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "data_s": t_data, "train_s": t_train,
            "tau_s": 8 * dt, "rollouts": rows,
            "speedup_wall": float(np.mean([r["wall_plain_s"] / r["wall_surrogate_s"] for r in rows])),
            "note": "proposals pass the integrator's judge (one ARK step from the proposal, ||LTE|| <= 1) but are "
                    "far less accurate than the steps they replace; no gain at equal final-state error"}


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
            "sample": "%d explicit RHS evaluation(s) of the %d^3 workload (FP64 numpy/scipy, %.1f s)" % (k, n, el)}


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
            "config": {"workload": "%d^3 gamma'' KKS phase field, 32 seeded nuclei, ARK4(3)6L[2]SA stage RHS, FP64 "
                                   "CPU oracle" % n, "grid": [n, n, n]},
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
    if args.ensemble > 0:
        line["ensemble"] = run_ensemble(args.ensemble, args.ensemble_t, rank, world)
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
