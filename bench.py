"""Benchmark: decoupled (D-scheme) multicontinuum time stepping on GB300.

Workload: three continua on a 1024 x 1024 grid (correlated log-normal k with
geometric means 1, 1e2, 1e4, c = (1, 0.2, 0.05), sigma = (5, 1, 20),
tau = 1/200, point sources +-1), synthetic and seeded. One benchmark step is
one time step of the D-scheme: the fused exchange/right-hand-side pass and
the three per-continuum PCG solves to ||r|| <= rtol ||b|| (rtol 1e-10, which
keeps every step within rel-L2 1e-8 of the exact solve), one persistent
kernel launch per step. The coupled backward-Euler solve of the same steps is
timed beside it at the same tolerance.

Metric: continuum-cell updates per second = L * nx * ny * steps / time, and
the fraction of the measured HBM bandwidth the step kernel reaches on the
algorithmic traffic (88 B per continuum-cell PCG iteration, 8 (2L+1) B per
continuum-cell per step for the right-hand side).

--impl reference times the FP64 CPU oracle (sparse direct solves) on a
bounded crop of the same workload instead.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL_IT = 88.0          # 11 FP64 values per continuum-cell per PCG iteration
SMI_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-coupled", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--crop", type=int, default=384, help="oracle sample size (cells per side)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def crop(w, m):
    import mc_inputs as mi
    m = min(m, w.nx)
    return mi.Workload(w.name + "_crop%d" % m, m, m, w.L, [k[:m, :m].copy() for k in w.k], w.c,
                       w.sigma, w.tau, w.nsteps, [f[:m, :m].copy() for f in w.F],
                       [p[:m, :m].copy() for p in w.p0],
                       {kk: v[:m, :m].copy() for kk, v in w.sigma_cell.items()})


def oracle_timing(w, steps, warmup):
    """Time the oracle's D-scheme steps (factorisation once, before timing)."""
    from oracle.schemes import from_workload
    t0 = time.perf_counter()
    o = from_workload(w)
    for a in range(w.L):
        o._factor(a)
    t_fact = time.perf_counter() - t0
    F = [np.ravel(x) for x in w.F]
    p = [np.ravel(x).copy() for x in w.p0]
    for _ in range(warmup):
        p = o.step(p, F, "D")
    t0 = time.perf_counter()
    for _ in range(steps):
        p = o.step(p, F, "D")
    dt = time.perf_counter() - t0
    return w.L * w.nx * w.ny * steps / dt, dt, t_fact


def cores_used():
    # SuperLU in scipy runs on one thread; numpy reductions are single threaded too.
    return 1


class Clocks:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + SMI_QUERY, "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self, device_index):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != device_index:
                    continue
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_per_unit():
    """DRAM bytes per continuum-cell PCG iteration from the committed ncu
    summary, valid only while the step kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2209_01158_gb300", "csrc", "mc_step.cu")
    try:
        with open(path) as f:
            d = json.load(f)
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("source_sha256") != h:
            return None
        return float(d["dram_bytes_per_cell_iteration"])
    except Exception:
        return None


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import mc_inputs as mi
    w = crop(mi.triple_1024(n=args.n), args.crop)
    val, dt, tf = oracle_timing(w, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": "continuum-cell updates/s (D-scheme)", "value": val,
        "unit": "continuum-cell updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "triple_1024 (3 continua, 1024x1024, tau=1/200)", "scheme": "D",
                   "sample": "%dx%d crop" % (w.nx, w.ny)},
        "cpu_baseline": {"value": val, "unit": "continuum-cell updates/s", "cores": cores_used(),
                         "kind": "oracle",
                         "sample": "oracle D-scheme, %dx%d crop of the 1024x1024 workload, %d steps after "
                                   "%d warm-up; SuperLU factorisation (%.1f s) excluded"
                                   % (w.nx, w.ny, args.steps, args.warmup, tf)},
        "e2e": {"value": val, "unit": "continuum-cell updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import torch.distributed as dist

    import mc_inputs as mi
    import paper_2209_01158_gb300 as mc

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w = mi.triple_1024(n=args.n)
    L, Ncell = w.L, w.nx * w.ny
    opts = mc.mc_default_opts()
    opts.rtol = args.rtol

    def timed_run(scheme):
        ctx = mc.Context.from_workload(w, opts=opts, stream=stream)
        for _ in range(args.warmup):
            ctx.step(scheme, 1)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        its = []
        barrier()
        t0 = time.perf_counter()
        for e0, e1 in evs:
            e0.record(stream)
            st = ctx.step(scheme, 1)
            e1.record(stream)
            its.append(sum(st["iters"][:L]) if scheme != "coupled" else st["iters"][0])
        barrier()
        wall = time.perf_counter() - t0
        per = [e0.elapsed_time(e1) * 1e-3 for e0, e1 in evs]
        ctx.close()
        return sum(per), wall, per, its

    clocks = Clocks()
    clocks.start()
    dev_time, wall, per, its = timed_run("D")
    ck = clocks.stop(local)
    t = torch.tensor([dev_time], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_time = float(t.item())
    cells_steps = L * Ncell * args.steps
    value = ws * cells_steps / dev_time

    coupled = None
    if not args.no_coupled:
        cdev, cwall, cper, cits = timed_run("coupled")
        coupled = {"value": ws * cells_steps / cdev, "ms_per_step": 1e3 * cdev / args.steps,
                   "pcg_iterations_per_step": float(np.mean(cits)),
                   "unit": "continuum-cell updates/s"}

    # roofline of the step kernel (one launch per step)
    hbm, peak_kind = peaks()
    alg_bytes = [BYTES_PER_CELL_IT * Ncell * it + 8.0 * (2 * L + 1) * L * Ncell for it in its]
    achieved = sum(alg_bytes) / dev_time / 1e9 if ws == 1 else sum(alg_bytes) / sum(per) / 1e9
    tpu = traffic_per_unit()
    traffic = None if tpu is None else tpu * Ncell * float(np.mean(its))
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
            "kernel": "step_kernel<3,false> (D-scheme, one launch per time step)"}

    e2e = None
    if not args.no_e2e:
        ctx = mc.Context.from_workload(w, opts=opts, stream=stream)
        host_in = [torch.from_numpy(np.ravel(x).astype(np.float64)).pin_memory() for x in w.p0]
        host_out = [torch.empty(Ncell, dtype=torch.float64).pin_memory() for _ in range(L)]
        for _ in range(args.warmup):
            ctx.set_state(host_in)
            ctx.step("D", 1)
            ctx.get_state(host_out)
            host_in, host_out = host_out, host_in
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_state(host_in)
            ctx.step("D", 1)
            ctx.get_state(host_out)
            host_in, host_out = host_out, host_in
        barrier()
        et = time.perf_counter() - t0
        ctx.close()
        tt = torch.tensor([et], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * cells_steps / float(tt.item()), "unit": "continuum-cell updates/s",
               "h2d_bytes_per_step": 8 * L * Ncell, "d2h_bytes_per_step": 8 * L * Ncell}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        wc = crop(w, args.crop)
        v, dt, tf = oracle_timing(wc, 3, 1)
        cpu = {"value": v, "unit": "continuum-cell updates/s", "cores": cores_used(), "kind": "oracle",
               "sample": "oracle D-scheme, %dx%d crop of the workload, 3 steps after 1 warm-up "
                         "(%.1f s); SuperLU factorisation (%.1f s) excluded" % (wc.nx, wc.ny, dt, tf)}

    if rank == 0:
        line = {
            "metric": "continuum-cell updates/s (D-scheme, rel-L2 1e-8) and % HBM peak",
            "value": value, "unit": "continuum-cell updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_time / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded correlated log-normal fields)",
            "config": {"workload": "triple_1024: 3 continua, 1024x1024, tau=1/200, D-scheme, rtol %g"
                                   % args.rtol,
                       "l2": "working set %.0f MB > 129 MB L2 (no flush)"
                             % (8 * L * Ncell * 11 / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "pcg_iterations_per_step": float(np.mean(its))},
            "coupled": coupled,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
