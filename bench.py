"""Benchmark of the periodized DMK hot path on B300.

Workload (the configuration the headline metric is quoted on): Laplace kernel, D = 2 (x, y
periodic), cell L = (1, 1, 0.25), N = 1e5 uniform points, neutral charges uniform in [-1, 1]
minus their mean, tol 1e-6 (p = 20, N_F = 27), n_s = 250.  One step = one full dmk_eval of
potentials and forces (tree build, upward pass, root far field, plane waves, shifts, leaf
stage) on inputs already resident in HBM.  value = targets/s of the mixed FP32/FP64 path; the
plain FP64 path is timed beside it.  The inputs (~4 MB) are smaller than L2, so L2 is
flushed (a 256 MB write) before every timed step and each step is timed on its own with
CUDA events on the library's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank evaluates its own independent problem (replicas; no
collective on the data path); the step time is the max over ranks and value counts the
targets of all ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

WORKLOAD = dict(kernel="laplace", D=2, L=[1.0, 1.0, 0.25], tol=1e-6, N=100_000, n_s=250)
STAGES = ["tree", "upward", "root", "planewave", "shift", "leaf", "total", "leaf_pair", "leaf_exp"]
METRIC = "targets/s at 1e-5 rel-L2, FP32+forces vs plain FP64 GPU; P2P Gpairs/s"
CONFIG = {"workload": "Laplace potential+forces, D=2 (x,y periodic), L=(1,1,0.25), N=1e5 uniform, "
                      "neutral uniform charges, tol 1e-6 (p=20, NF=27), n_s=250",
          "kernel": "laplace", "D": 2, "L": [1, 1, 0.25], "N": 100000, "tol": 1e-6, "n_s": 250,
          "l2": "flushed (256 MB write) before every timed step", "inputs": "resident in HBM"}


def peaks():
    try:
        return json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons during the timed region (into a temporary file)."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.out = os.path.join(tempfile.gettempdir(), f"dmk_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.out):
                f = [v.strip() for v in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except FileNotFoundError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def reference_arm(args, rank, world):
    """The oracle (FP64 numpy/scipy, this host's cores) on a bounded sample of the workload."""
    if rank != 0:
        return
    from oracle.dmk import evaluate
    from paper_2606_27134_b300 import workloads as Wl
    Ns = 4000
    x = Wl.uniform_points(Ns, WORKLOAD["L"], 12345)
    q = Wl.uniform_charges(Ns, 12346)
    # untimed warm-up evaluations of the same sample (at most 3, like the timed steps, so the
    # whole run stays within a few minutes)
    n_warm = max(0, min(args.warmup, 3))
    for _ in range(n_warm):
        evaluate("laplace", 2, WORKLOAD["L"], WORKLOAD["tol"], x, q, n_s=WORKLOAD["n_s"], grad=True)
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        t = time.perf_counter()
        evaluate("laplace", 2, WORKLOAD["L"], WORKLOAD["tol"], x, q, n_s=WORKLOAD["n_s"], grad=True)
        times.append(time.perf_counter() - t)
    dt = statistics.median(times)
    v = Ns / dt
    sample = (f"oracle (FP64 numpy) full evaluation with forces of N={Ns} uniform points in the same cell, "
              f"distribution and plan (25x sparser than the N=1e5 workload); median of {len(times)}")
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "targets/s", "n_gpus": args.gpus,
            "steps": len(times), "warmup": n_warm, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": v, "unit": "targets/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


EXTRA = [
    # (name, kernel, D, L, N, point generator, strengths) -- the other workload shapes, mixed path
    ("Stokeslet velocity+gradient, D=1, L=(8,1,1), N=1e6 uniform, N(0,1) forces minus mean, tol 1e-6",
     "stokeslet", 1, [8.0, 1.0, 1.0], 1_000_000, "uniform", "stokes"),
    ("Stresslet potential+gradient, D=3, L=(1,1,16) (16 cubes, DFT over the cube index), N=4e6 uniform, "
     "q (x) n strengths, tol 1e-6; k = 0 excluded, the 3P compensation term of the literature not applied",
     "stresslet", 3, [1.0, 1.0, 16.0], 4_000_000, "uniform", "stokes"),
    ("Rotlet potential+gradient, D=3, L=(1,1,16) (16 cubes, DFT over the cube index), N=4e6 uniform, "
     "N(0,1) torques, tol 1e-6", "rotlet", 3, [1.0, 1.0, 16.0], 4_000_000, "uniform", "stokes"),
    ("Laplace energy and forces through torch.autograd (two evaluations), D=3, L=(1,1,1), N=1e6 in 64 "
     "Gaussian clusters (sigma 0.02), balanced +-1 charges, tol 1e-6", "laplace-autograd", 3, [1.0, 1.0, 1.0],
     1_000_000, "clusters", "balanced"),
]


def extra_configs(dmk, Wl, dev, stream, steps=3, warmup=2):
    """Targets/s of the other workload shapes (mixed path, potentials and gradients), a few steps each."""
    import torch
    from paper_2606_27134_b300 import autograd as ag
    out = []
    for name, kernel, D, L, N, pg, sg in EXTRA:
        try:
            if pg == "uniform":
                x = Wl.uniform_points(N, L, 7001)
            else:
                x = Wl.clustered_points(N, L, 7001, n_centers=64, sigma=0.02)
            if sg == "stokes":
                rho = Wl.stokes_strengths(kernel, N, 7002)
            else:
                rho = Wl.balanced_charges(N, 7002).reshape(N, 1)
            xt = torch.tensor(x, dtype=torch.float64, device=dev)
            rt = torch.tensor(rho, dtype=torch.float64, device=dev)
            if kernel == "laplace-autograd":
                pot = ag.Potential("laplace", D, L, 1e-6, precision="mixed", n_s=250)

                def step():
                    xx = xt.detach().requires_grad_(True)
                    u = pot(xx, rt)
                    E = 0.5 * (rt * u).sum()
                    (gx,) = torch.autograd.grad(E, xx)
                    return gx
                plan = pot.plan
            else:
                plan = dmk.Plan(kernel, D, L, 1e-6, precision="mixed", n_s=250)   # default stream

                def step():
                    return plan.eval(xt, rt, grad=True)
            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            ms = []
            for _ in range(steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(torch.cuda.current_stream())
                step()
                b.record(torch.cuda.current_stream())
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            st = plan.stats()
            t = statistics.median(ms)
            # one more pass with per-stage events, in order (each kernel alone on the SMs)
            plan.set_timing(True)
            plan.set_pair_overlap(False)
            step()
            torch.cuda.synchronize()
            stage = plan.stats()["stage_ms"]
            plan.set_pair_overlap(True)
            plan.set_timing(False)
            out.append({"workload": name, "N": N, "ms_per_step": t, "targets_per_s": N / (t / 1e3),
                        "p": st["p"], "n_boxes": st["n_boxes"], "n_levels": st["n_levels"], "pairs": st["n_pairs"],
                        "stage_ms": dict(zip(STAGES,
                                             [round(v, 3) for v in stage])),
                        "steps": steps, "warmup": warmup})
            if kernel != "laplace-autograd":
                plan.close()
            # the plain FP64 path on the same workload (one warm-up, two steps), beside the mixed
            try:
                if kernel == "laplace-autograd":
                    pot = ag.Potential("laplace", D, L, 1e-6, precision="fp64", n_s=250)
                    plan = pot.plan
                else:
                    plan = dmk.Plan(kernel, D, L, 1e-6, precision="fp64", n_s=250)
                step()
                torch.cuda.synchronize()
                ms64 = []
                for _ in range(2):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(torch.cuda.current_stream())
                    step()
                    b.record(torch.cuda.current_stream())
                    torch.cuda.synchronize()
                    ms64.append(a.elapsed_time(b))
                t64 = statistics.median(ms64)
                out[-1]["fp64_path"] = {"ms_per_step": t64, "targets_per_s": N / (t64 / 1e3), "steps": 2, "warmup": 1,
                                        "mixed_over_fp64": t64 / t}
                if kernel != "laplace-autograd":
                    plan.close()
            except Exception as e:  # reported, never fatal
                out[-1]["fp64_path"] = {"error": str(e)[:200]}
            del xt, rt
            torch.cuda.empty_cache()
        except Exception as e:  # reported, never fatal
            out.append({"workload": name, "error": str(e)[:200]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="mixed,fp64", help="precision paths to time (profiling: mixed)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workload configurations (profiling)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    from paper_2606_27134_b300 import dmk, workloads as Wl

    torch.cuda.set_device(local_rank)
    from paper_2606_27134_b300 import peaks as pkmod
    measured_peaks = pkmod.measure(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    args.warmup = max(args.warmup, 3)
    W = WORKLOAD
    N = W["N"]
    x = Wl.uniform_points(N, W["L"], 2002 + rank)
    q = Wl.uniform_charges(N, 3002 + rank)
    dev = torch.device("cuda", local_rank)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    qt = torch.tensor(q, dtype=torch.float64, device=dev).reshape(N, 1)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(plan, steps, warmup, host=False):
        u = torch.empty((N, 1), dtype=torch.float64, device=dev)
        g = torch.empty((N, 3, 1), dtype=torch.float64, device=dev)
        if host:
            hx = xt.cpu().pin_memory()
            hq = qt.cpu().pin_memory()
            hu = torch.empty((N, 1), dtype=torch.float64).pin_memory()
            hg = torch.empty((N, 3, 1), dtype=torch.float64).pin_memory()

        def step():
            if host:
                plan.eval_host_ptr(N, hx.data_ptr(), hq.data_ptr(), hu.data_ptr(), hg.data_ptr())
            else:
                plan.eval_ptr(N, xt.data_ptr(), qt.data_ptr(), u.data_ptr(), g.data_ptr())

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stage = []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            stream.synchronize()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stage.append(plan.stats())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stage, wall, (u, g)

    prec_results = {}
    paths = [p for p in args.paths.split(",") if p]
    for prec in paths:
        plan = dmk.Plan("laplace", W["D"], W["L"], W["tol"], precision=prec, n_s=W["n_s"],
                        stream=stream.cuda_stream)
        with Clocks(local_rank) as ck:
            ms, stats, wall, _ = timed(plan, args.steps, args.warmup)
        # per-kernel times: the stage-timing pass runs in order (the residual kernel alone on the
        # SMs), the timed steps above with it beside the far field (the default)
        plan.set_timing(True)
        plan.set_pair_overlap(False)
        _, st_t, _, _ = timed(plan, 5, 1)
        plan.set_pair_overlap(True)
        plan.set_timing(False)
        # per-stage median over the timing steps (the tree stage holds host round trips and
        # varies from step to step)
        stage_med = [statistics.median(st["stage_ms"][i] for st in st_t) for i in range(len(st_t[0]["stage_ms"]))]
        prec_results[prec] = dict(ms=ms, stats=stats[-1], clocks=ck.summary(), stage=stage_med, wall=wall,
                                  plan=plan)
    # end-to-end through the host-buffer entry point (copies inside the timed region)
    plan_m = prec_results["mixed"]["plan"]
    ms_e2e = [float("nan")] if args.no_e2e else timed(plan_m, max(3, args.steps // 2), 2, host=True)[0]

    from paper_2606_27134_b300.replicas import max_over_ranks

    def agg(v):
        return max_over_ranks(v, dist, dev)

    mixed = prec_results["mixed"]
    step_ms = agg(statistics.mean(mixed["ms"]))
    fp64_ms = agg(statistics.mean(prec_results["fp64"]["ms"])) if "fp64" in prec_results else float("nan")
    e2e_ms = agg(statistics.mean(ms_e2e))
    value = world * N / (step_ms / 1e3)
    st = mixed["stats"]
    # leaf kernels: timed with per-stage events in a separate pass (stage 7 = the residual
    # kernel k_pair; stage 8 = the expansion kernel k_leafexp_parent; stage 5 = both)
    leaf_ms = mixed["stage"][5]
    pair_ms = mixed["stage"][7]
    pairs = st["n_pairs"]
    gpairs = pairs / (pair_ms / 1e3) / 1e9 if pair_ms > 0 else None
    # pairs inside the support of K_R (r < nu), counted on the host with a k-d tree: every
    # non-empty leaf of this workload sits at the deepest level, so nu = s / 2^(levels - 1) for
    # every listed pair (periodic along x1, x2)
    try:
        from scipy.spatial import cKDTree
        nu = 1.0 / 2 ** (int(st["n_levels"]) - 1)
        tree = cKDTree(x, boxsize=[W["L"][0], W["L"][1], 1e9])
        in_support = int(tree.count_neighbors(tree, nu)) - N
    except Exception:       # reported when available
        in_support = None
    # roofline of the dominant kernel, k_pair (FP32 ALU bound): algorithmic FLOPs per launch =
    # visited pairs x F_pair (roofline.pair_flops), over its CUDA-event duration; the peaks are
    # the pipe throughputs measured on this GPU in this run (paper_2606_27134_b300.peaks)
    from paper_2606_27134_b300 import roofline as rf
    pk_meas = measured_peaks
    pk = pk_meas["fp32_tflops"]
    flops = rf.pair_flops("laplace", st, grad=True)
    achieved = flops / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    exp_ms = mixed["stage"][8]
    exp_tf = rf.leafexp_flops(st, N, grad=True) / (exp_ms / 1e3) / 1e12 if exp_ms > 0 else None
    roof = {"bound": "alu", "kernel": "k_pair<float, Laplace, grad>", "achieved": achieved, "peak": pk,
            "unit": "TFLOP/s", "frac": (achieved / pk) if achieved else None, "traffic": rf.PAIR_TRAFFIC_BYTES,
            "peak_note": "of measured: FP32 FFMA throughput of this GPU, dmk_peak_measure in this run "
                         "(derived 148 SMs x 128 lanes x 2 x %.3f GHz = %.1f TFLOP/s)" % (
                             rf.MAX_SM_GHZ, rf.fp32_peak_tflops()),
            "per_unit": "%d FLOP per visited pair (22 + d_q, d_q = %d)" % (rf.pair_flops("laplace", {"n_pairs": 1,
                        "fit_terms": st["fit_terms"]}, grad=True), max(int(st["fit_terms"]) - 1, 0)),
            "second_kernel": {"kernel": "k_leafexp_parent<float, Laplace, grad>", "ms": exp_ms, "achieved": exp_tf,
                              "frac": (exp_tf / pk) if exp_tf else None}}
    fp64_line = {"value": world * N / (fp64_ms / 1e3), "unit": "targets/s", "ms_per_step": fp64_ms}
    if "fp64" in prec_results:
        st64 = prec_results["fp64"]["stats"]
        pair64 = prec_results["fp64"]["stage"][7]
        if pair64 > 0:
            a64 = rf.pair_flops("laplace", st64, grad=True) / (pair64 / 1e3) / 1e12
            fp64_line["roofline"] = {"bound": "alu", "kernel": "k_pair<double, Laplace, grad>", "achieved": a64,
                                     "peak": pk_meas["fp64_tflops"], "unit": "TFLOP/s",
                                     "frac": a64 / pk_meas["fp64_tflops"],
                                     "peak_note": "of measured: FP64 DFMA throughput, dmk_peak_measure in this run"}
        fp64_line["stage_ms"] = dict(zip(STAGES, prec_results["fp64"]["stage"]))
    line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(CONFIG, parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "fp64_path": fp64_line,
            "peaks": {k: pk_meas[k] for k in ("fp32_tflops", "fp64_tflops", "mufu_rsqrt_tops", "clocks")},
            "mixed_over_fp64": fp64_ms / step_ms,
            "p2p": {"gpairs_per_s": gpairs, "pairs_per_step": pairs, "pair_kernel_ms": pair_ms, "leaf_stage_ms": leaf_ms,
                    "pairs_in_support": in_support,
                    "support_fraction": (in_support / pairs) if in_support else None},
            "stage_ms": dict(zip(STAGES, mixed["stage"])),
            # the paper's timing convention (Sec. 6): the evaluation without the octree build,
            # from the stage-timing pass
            "ms_excluding_tree": mixed["stage"][6] - mixed["stage"][0],
            "tree": {k: st[k] for k in ("n_levels", "n_boxes", "n_leaves", "n_nonleaf", "n_direct_entries")},
            "roofline": roof,
            "clocks": mixed["clocks"],
            "e2e": {"value": world * N / (e2e_ms / 1e3), "unit": "targets/s",
                    "h2d_bytes_per_step": N * (3 + 1) * 8, "d2h_bytes_per_step": N * (1 + 3) * 8},
            "gpu_launches": int(st["kernel_launches"]) * args.steps}
    if not args.no_extra:
        line["other_configs"] = extra_configs(dmk, Wl, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            from oracle.dmk import evaluate
            Ns = 4000
            xs = Wl.uniform_points(Ns, W["L"], 12345)
            qs = Wl.uniform_charges(Ns, 12346)
            t = time.perf_counter()
            evaluate("laplace", 2, W["L"], W["tol"], xs, qs, n_s=W["n_s"], grad=True)
            dt = time.perf_counter() - t
            # the oracle is Python loops over boxes with numpy contractions: only the BLAS calls
            # inside numpy use more than one thread; timed again with BLAS on one thread (in a
            # child process whose BLAS is limited before numpy loads)
            code = ("import time, sys; sys.path.insert(0, %r); from oracle.dmk import evaluate; "
                    "from paper_2606_27134_b300 import workloads as Wl; L = %r; "
                    "x = Wl.uniform_points(%d, L, 12345); q = Wl.uniform_charges(%d, 12346); "
                    "t = time.perf_counter(); evaluate('laplace', 2, L, %r, x, q, n_s=%d, grad=True); "
                    "print(time.perf_counter() - t)" % (os.path.dirname(os.path.abspath(__file__)), list(W["L"]),
                                                        Ns, Ns, W["tol"], W["n_s"]))
            env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                       CUDA_VISIBLE_DEVICES="")
            r1 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
            dt1 = float(r1.stdout.strip().splitlines()[-1])
            line["cpu_baseline"] = {"value": Ns / dt, "unit": "targets/s", "cores": len(os.sched_getaffinity(0)),
                                    "kind": "oracle", "value_1_thread": Ns / dt1,
                                    "sample": f"oracle (FP64 numpy, single-threaded Python with numpy's BLAS "
                                              f"threads) full evaluation with forces of N={Ns} uniform points, same "
                                              f"cell/distribution/plan (25x sparser), one run ({dt:.1f} s; "
                                              f"{dt1:.1f} s with BLAS on one thread)"}
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
