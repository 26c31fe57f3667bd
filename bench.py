#!/usr/bin/env python
"""Benchmark of the synchronous island GA on the paper-scale workload.

Workload (one "step"): the 512x1024 torus of 32-agent islands (16,777,216 agents, 16-byte
records: trait, counter, 64 one-bit steady-curated hstrat sites), tournament size 5,
p_del = 0.01, one migrant from each neighbour every generation, 10,000 generations, for the
adaptive (p_ben = 0.01) and the purifying-only (p_ben = 0) treatment (Sec. 3 of the paper),
each started from its founder population and followed by pairwise MRCA bounds over 4,096
uniformly sampled end-state agents (8,386,560 pairs).

Prints one JSON line.  value = agent-generations per second over the timed steps (inputs
resident in HBM, CUDA events on the run's stream); e2e = the same job through the public API
with host buffers (create, step, MRCA into pinned host arrays, snapshot into pinned host
memory, destroy) timed on the host.  --impl reference times the CPU oracle on a bounded
sample of the same workload on the host cores.  Under torchrun each rank runs an
independent replica on its own GPU (the path is not sharded).
"""
import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "agent-gens/sec @16.8M agents on 1 GB300; % roofline; batched vs serial"
UNIT = "agent-gens/s"
# legs of the default line: main (the headline, 16.8M agents), e2e (the same job through the
# public API with host buffers), batch, async, resident (the 32x32 torus), peak (integer-pipe
# probe), variants (surface variants), treatments (the paper's float treatments), serve
# (1,000-request trace), cpu-baseline (the oracle on the host cores)
LEGS = ("main", "e2e", "batch", "async", "resident", "peak", "variants", "treatments", "serve",
        "cpu-baseline")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--rows", type=int, default=512)
    p.add_argument("--cols", type=int, default=1024)
    p.add_argument("--gens", type=int, default=10000)
    p.add_argument("--sample", type=int, default=4096)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--batch-runs", type=int, default=256)
    p.add_argument("--batch-gens", type=int, default=2000)
    p.add_argument("--serve-requests", type=int, default=1000)
    p.add_argument("--variant-gens", type=int, default=1000)
    p.add_argument("--treatment-gens", type=int, default=10000)
    p.add_argument("--async-gens", type=int, default=2000)
    p.add_argument("--resident-gens", type=int, default=1000)
    p.add_argument("--legs", default="all",
                   help="comma list of: " + ",".join(LEGS) + " (default all); the headline "
                        "value comes from 'main'")
    for leg in LEGS:
        p.add_argument(f"--no-{leg}", action="store_true", help=f"drop the {leg} leg")
    a = p.parse_args()
    chosen = set(LEGS) if a.legs == "all" else set(x.strip() for x in a.legs.split(",") if x.strip())
    unknown = chosen - set(LEGS)
    if unknown:
        p.error(f"unknown legs: {sorted(unknown)}")
    a.run = {leg: leg in chosen and not getattr(a, "no_" + leg.replace("-", "_")) for leg in LEGS}
    return a


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shapes(args, rank):
    from paper_2405_03605_gb300.workloads import PAPER_ADAPTIVE, PAPER_PURIFYING
    out = []
    for i, s in enumerate((PAPER_ADAPTIVE, PAPER_PURIFYING)):
        out.append(s.with_(rows=args.rows, cols=args.cols, generations=args.gens,
                           run_id=2 * rank + i))
    return out


def workload_config(args, sh):
    return {
        "workload": (f"island GA {args.rows}x{args.cols} torus x {sh.island_size} agents "
                     f"({sh.n_agents} agents), 16 B records (steady 64x1-bit hstrat), "
                     f"tournament {sh.tournament_size}, p_del 0.01, 1 migrant/neighbour/gen, "
                     f"{args.gens} gens, adaptive (p_ben 0.01) + purifying (p_ben 0) runs, "
                     f"then MRCA bounds over {args.sample} sampled agents"),
        "rows": args.rows, "cols": args.cols, "island_size": sh.island_size,
        "agents_per_run": sh.n_agents, "runs_per_step": 2, "generations": args.gens,
        "record_bytes": 16, "mrca_sample": args.sample,
        "l2": "no flush: every generation streams the 256 MiB population in and a second "
              "256 MiB buffer out, both larger than the 129 MB L2",
    }


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if shutil.which("nvidia-smi") is None:
            return
        visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
        if visible:
            ids = [x.strip() for x in visible.split(",") if x.strip()]
            if gpu_index < len(ids):
                gpu_index = ids[gpu_index]
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen(
            ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=self.f, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": reasons}


# Counters of one launch of the island step on the 512x1024x32 grid (migration every
# generation), from an ncu capture of this kernel build on the 256x1024 grid scaled by the
# islands processed (profiles/): DRAM bytes read + written,
# warp-instructions per island-generation (smsp__inst_executed.sum / islands), ALU-pipe
# warp-instructions per island-generation (sm__inst_executed_pipe_alu.sum / islands; each
# occupies the ALU pipe two cycles) and FMA-heavy pipe cycles per island-generation
# (sm__pipe_fmaheavy_cycles_active.sum / islands).
ISLAND_STEP_TRAFFIC = {"kernel": "island_units_kernel<32,5,0>", "bytes": 448.1e6,
                       "inst_per_island_gen": 36143104 / 262144,
                       "alu_inst_per_island_gen": 14254080 / 262144,
                       "fma_cycles_per_island_gen": 30867456 / 262144,
                       "rows": 512, "cols": 1024, "island_size": 32}
# warp-instructions per island-generation of the resident kernel on the 32x32 torus
# (smsp__inst_executed.sum of a 200-generation launch / (1,024 islands x 200), this build)
RESIDENT_INST = {"kernel": "resident_warp_kernel<32,5,0,4>", "inst_per_island_gen": 70550765 / 204800}


def aggregate_replicas(elapsed_ms, agent_gens, world, device="cpu"):
    """Whole-job figures over independent replicas (one per rank): the slowest rank's time
    and the sum of all ranks' agent-generations.  With world == 1 the inputs come back."""
    if world <= 1:
        return float(elapsed_ms), float(agent_gens)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(agent_gens)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(args, sh, seconds):
    """The oracle, as it stands, on the same grid: generations until `seconds` elapse."""
    from oracle import OracleRun
    threads = os.cpu_count() or 1
    o = OracleRun(sh.rows, sh.cols, island_size=sh.island_size,
                  tournament_size=sh.tournament_size, p_ben=sh.p_ben, p_del=sh.p_del,
                  surface_sites=sh.surface_sites, differentia_bits=sh.differentia_bits,
                  curation=sh.curation, migrate_every=sh.migrate_every, seed=sh.seed,
                  run_id=sh.run_id, threads=threads)
    gens = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        gens += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    o.close()
    return {"value": sh.n_agents * gens / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"adaptive run, full {sh.rows}x{sh.cols}x{sh.island_size} grid, first "
                      f"{gens} generations ({dt:.1f} s), OpenMP over islands"}


def run_reference(args, rank, world):
    """CPU oracle arm: each step = a bounded sample of the workload on the host cores."""
    if rank != 0:
        return
    sh = shapes(args, 0)[0]
    from oracle import OracleRun
    threads = os.cpu_count() or 1
    o = OracleRun(sh.rows, sh.cols, island_size=sh.island_size,
                  tournament_size=sh.tournament_size, p_ben=sh.p_ben, p_del=sh.p_del,
                  surface_sites=sh.surface_sites, differentia_bits=sh.differentia_bits,
                  curation=sh.curation, migrate_every=sh.migrate_every, seed=sh.seed,
                  run_id=sh.run_id, threads=threads)
    gens_per_step = 2
    for _ in range(args.warmup):
        o.step(gens_per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(gens_per_step)
    dt = time.perf_counter() - t0
    value = sh.n_agents * gens_per_step * args.steps / dt
    sample = (f"adaptive run, full {sh.rows}x{sh.cols}x{sh.island_size} grid, "
              f"{gens_per_step} generations per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1000 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args, sh),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2405_03605_gb300 import build as lib_build
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import sample_agent_ids

    lib_build.build()
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    shs = shapes(args, rank)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {**workload_config(args, shs[0]),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}}
    launches = 0
    clk = None
    if args.run["main"]:
        main, launches, clk = measure_main(args, shs, rank, world, local, barrier)
        line.update(main)

    extra = {}
    if args.run["e2e"]:
        ids_h = sample_agent_ids(shs[0].n_agents, args.sample, seed=42)
        extra["e2e"] = measure_e2e(args, shs, ids_h, world)
    if args.run["batch"]:
        extra["batched_vs_serial"] = measure_batch(args, rank)
    if rank == 0:
        if args.run["peak"]:
            extra["int_peak"] = measure_peak(args)
        if args.run["resident"]:
            extra["resident"] = measure_resident(args, extra.get("int_peak"))
        if args.run["async"]:
            extra["async"] = measure_async(args)
        if args.run["variants"]:
            extra["variants"] = measure_variants(args)
        if args.run["treatments"]:
            extra["paper_treatments"] = measure_treatments(args)
        if args.run["serve"]:
            extra["serving"] = measure_serve(args)
    if rank != 0:
        return
    issue = line.get("issue_roofline")
    if issue is not None:
        mhz = (clk or {}).get("sm_mhz") or 2070.0  # sampled median SM clock, else the maximum
        issue["peak"] = issue["sms"] * 4 * mhz * 1e6
        issue["frac"] = issue["achieved"] / issue["peak"]
        issue["clock_mhz"] = mhz
        # pipes: the ALU pipe takes a warp-instruction every two cycles per sub-partition (its
        # measured ceiling is the LOP3 stream of the integer probe), the FMA-heavy pipe is busy
        # the measured cycles per island-generation
        rate = issue["island_gens_per_s"]
        alu = ISLAND_STEP_TRAFFIC["alu_inst_per_island_gen"] * rate
        fma = ISLAND_STEP_TRAFFIC["fma_cycles_per_island_gen"] * rate
        subparts = issue["sms"] * 4 * mhz * 1e6
        issue["alu_pipe_frac"] = alu * 2 / subparts
        issue["fma_pipe_frac"] = fma / subparts
        peak = extra.get("int_peak")
        if peak:
            issue["alu_vs_measured_lop3_stream"] = alu / peak["lop3"]["warp_instr_per_s"]
    cpu = None
    if args.run["cpu-baseline"] and world == 1:
        cpu = cpu_baseline(args, shs[0], args.cpu_seconds)
    line.update(extra)
    line["gpu_launches"] = launches
    line["cpu_baseline"] = cpu
    line["clocks"] = clk
    line.setdefault("e2e", None)
    print(json.dumps(line), flush=True)


def measure_main(args, shs, rank, world, local, barrier):
    """The headline: for each treatment, reset to the founder population, --gens generations,
    MRCA bounds over --sample agents; --warmup untimed steps, then --steps timed."""
    import numpy as np
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import sample_agent_ids

    stream = torch.cuda.Stream()
    runs = [ga.Run(s, stream=stream) for s in shs]
    n = args.sample
    pairs = n * (n - 1) // 2
    ids_h = sample_agent_ids(shs[0].n_agents, n, seed=42)
    with torch.cuda.stream(stream):
        ids_d = torch.from_numpy(ids_h.view(np.int32)).cuda()
        outs = [(torch.empty(pairs, dtype=torch.int32, device="cuda"),
                 torch.empty(pairs, dtype=torch.int32, device="cuda")) for _ in runs]

    step_pairs, mrca_pairs = [], []

    def one_step(record):
        for r, (lo, hi) in zip(runs, outs):
            r.reset()
            if record:
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
            r.step(args.gens)
            if record:
                e1.record(stream)
            r.mrca_bounds_device(ids_d, lo, hi)
            if record:
                e2.record(stream)
                step_pairs.append((e0, e1))
                mrca_pairs.append((e1, e2))

    for _ in range(args.warmup):
        one_step(False)
    stream.synchronize()
    for r in runs:
        r.sync()

    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    launches0 = sum(r.launches for r in runs)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        one_step(True)
    t_end.record(stream)
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    for r in runs:
        r.sync()
    launches = sum(r.launches for r in runs) - launches0
    elapsed_ms = t_start.elapsed_time(t_end)
    local_agent_gens = args.steps * sum(s.n_agents * args.gens for s in shs)
    elapsed_ms, agent_gens = aggregate_replicas(elapsed_ms, local_agent_gens, world,
                                                device="cuda")
    value = agent_gens / (elapsed_ms / 1000.0)

    # roofline of the island-step kernel: one launch = one generation of one run (migration
    # every generation), algorithmic bytes per agent = record in + record out + 4 immigrant
    # records per island = 2G + 4G/N
    step_ms = sum(a.elapsed_time(b) for a, b in step_pairs)
    step_launches = args.gens * len(step_pairs)
    G, N = 16, shs[0].island_size
    bytes_per_launch = shs[0].n_agents * (2 * G + 4 * G / N)
    avg_launch_s = step_ms / 1000.0 / step_launches
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    mrca_ms = statistics.mean(a.elapsed_time(b) for a, b in mrca_pairs)
    same_shape = (args.rows, args.cols, shs[0].island_size) == (
        ISLAND_STEP_TRAFFIC["rows"], ISLAND_STEP_TRAFFIC["cols"], ISLAND_STEP_TRAFFIC["island_size"])
    traffic = ISLAND_STEP_TRAFFIC["bytes"] if same_shape else None

    # Sec. 3 treatment contrast from the last step's MRCA bounds: mean time since divergence
    # bounded below by T - hi (purifying-only runs should keep deeper genealogies)
    contrast = {}
    with torch.cuda.stream(stream):
        for sh, (lo, hi) in zip(shs, outs):
            depth = (args.gens - hi.to(torch.int64)).double().mean().item()
            contrast["adaptive" if sh.p_ben > 0 else "purifying"] = depth
    contrast["unit"] = "generations (mean over sampled pairs of T - hi)"

    # issue roofline of the same kernel: warp-instructions issued per second against the SM
    # issue limit (one warp-instruction per clock on each of the 4 sub-partitions of each SM)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    issue = None
    if same_shape:
        island_gens = shs[0].n_islands / avg_launch_s
        inst_rate = ISLAND_STEP_TRAFFIC["inst_per_island_gen"] * island_gens
        issue = {"bound": "alu", "unit": "warp-instr/s", "achieved": inst_rate,
                 "per_unit": ISLAND_STEP_TRAFFIC["inst_per_island_gen"],
                 "unit_of_work": "island-generation (ncu smsp__inst_executed.sum of this build)",
                 "sms": n_sm, "island_gens_per_s": island_gens}
    for r in runs:
        r.close()
    main = {
        "value": value, "ms_per_step": elapsed_ms / args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": ISLAND_STEP_TRAFFIC["kernel"],
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "bytes_per_launch": bytes_per_launch,
                     "avg_launch_us": avg_launch_s * 1e6},
        "issue_roofline": issue,
        "mrca": {"ms_per_run": mrca_ms, "pairs": pairs, "bytes_written": 8 * pairs,
                 "achieved": 8 * pairs / (mrca_ms / 1000.0) / 1e9, "peak": peak, "unit": "GB/s",
                 "frac": 8 * pairs / (mrca_ms / 1000.0) / 1e9 / peak,
                 "note": "every MRCA kernel of the call (closed-form rank table, pack, pairs); "
                         "bound by the (lo, hi) output writes"},
        "treatment_contrast": contrast,
    }
    return main, launches, clk


def measure_peak(args):
    """Integer-pipe probe (ga_int_peak): operations and warp-instructions per second of
    dependence-free LOP3, IMAD.WIDE and Philox-round streams, next to the nominal issue limit
    (4 warp-instructions per clock per SM)."""
    import torch
    from paper_2405_03605_gb300 import ga
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"nominal_issue_warp_instr_per_s_at_2070mhz": n_sm * 4 * 2070e6}
    for name, kind in (("lop3", ga.PEAK_LOP3), ("imad_wide", ga.PEAK_IMAD), ("philox_mix", ga.PEAK_MIX)):
        rate, sec = ga.int_peak(kind, iters=4096)
        out[name] = {"ops_per_s": rate, "warp_instr_per_s": rate / 32.0, "seconds": sec}
    return out


def measure_resident(args, peak):
    """The 32x32 torus of 32-agent islands (32,768 agents, 16-byte records, migration every
    generation) for --resident-gens generations from the founder population: resident (one
    cooperative launch, islands in registers, migrants through mailboxes) and streamed (one
    launch per generation), CUDA events on the run's stream, end states compared."""
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import SMALL_TORUS

    gens = args.resident_gens
    stream = torch.cuda.Stream()
    out = {"workload": "32x32 torus x 32 agents (32,768 agents), 16 B records, migration every "
                       f"generation, {gens} gens", "generations": gens}
    snaps = {}
    for name, mode in (("resident", ga.RESIDENT_ON), ("streamed", ga.RESIDENT_OFF)):
        r = ga.Run(SMALL_TORUS, stream=stream)
        r.resident_policy(mode)
        r.step(gens)  # warm-up
        r.reset()
        times = []
        for _ in range(3):
            r.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.step(gens)
            e1.record(stream)
            r.sync()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        with torch.cuda.stream(stream):
            snaps[name] = r.snapshot_device()
        stream.synchronize()
        out[name] = {"agent_gens_per_s": SMALL_TORUS.n_agents * gens / (ms / 1000.0),
                     "us_per_gen": ms * 1000.0 / gens, "launches": r.launches}
        r.close()
    with torch.cuda.stream(stream):
        out["identical"] = bool(torch.equal(snaps["resident"], snaps["streamed"]))
    stream.synchronize()
    out["resident_vs_streamed"] = (out["resident"]["agent_gens_per_s"] /
                                   out["streamed"]["agent_gens_per_s"])
    per = RESIDENT_INST["inst_per_island_gen"]
    if per:
        rate = per * SMALL_TORUS.n_islands * gens / (out["resident"]["us_per_gen"] * 1e-6 * gens)
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        issue = {"kernel": RESIDENT_INST["kernel"], "inst_per_island_gen": per,
                 "warp_instr_per_s": rate, "nominal_issue_frac": rate / (n_sm * 4 * 2070e6)}
        if peak:
            issue["vs_measured_lop3_stream"] = rate / peak["lop3"]["warp_instr_per_s"]
            issue["vs_measured_philox_mix"] = rate / peak["philox_mix"]["warp_instr_per_s"]
        out["issue"] = issue
    return out


def measure_batch(args, rank):
    """Heterogeneous replicate runs (grid sides from {16..256}, islands of 16/32/64, p_ben and
    p_del log-uniform on [1e-4, 1e-1], tournament size 2..8), each for the same generation
    count: once as one autotuned batch (shared launches, CUDA-graph chunks), once as serial
    per-run launches of the same runs on the same stream.  Both timed with CUDA events from
    founder populations; end states compared on the device."""
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import batch_shapes

    shapes = [s.with_(run_id=s.run_id + 100000 * rank)
              for s in batch_shapes(args.batch_runs, seed=42, generations=args.batch_gens)]
    gens = args.batch_gens
    stream = torch.cuda.Stream()
    runs = [ga.Run(s, stream=stream) for s in shapes]
    batch = ga.Batch(runs, stream=stream)
    tune = batch.autotune(trial_gens=8)
    batch.step(tune["chunk"])  # capture and warm the graph
    batch.sync()
    for r in runs:
        r.reset()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = batch.launches
    e0.record(stream)
    batch.step(gens)
    e1.record(stream)
    batch.sync()
    batched_ms = e0.elapsed_time(e1)
    batched_launches = batch.launches - l0

    alone = [ga.Run(s, stream=stream) for s in shapes]
    for r in alone:
        r.step(2)
        r.reset()
    torch.cuda.synchronize()
    l0 = sum(r.launches for r in alone)
    e0.record(stream)
    for r in alone:
        r.step(gens)
    e1.record(stream)
    stream.synchronize()
    serial_ms = e0.elapsed_time(e1)
    serial_launches = sum(r.launches for r in alone) - l0
    with torch.cuda.stream(stream):
        identical = all(torch.equal(a.snapshot_device(), b.snapshot_device())
                        for a, b in zip(runs, alone))
    stream.synchronize()
    agent_gens = float(sum(s.n_agents for s in shapes)) * gens
    batch.close()
    for r in runs + alone:
        r.close()
    return {
        "workload": (f"{len(shapes)} runs, grid sides from {{16,32,64,128,256}}, islands of "
                     f"16/32/64, p log-uniform [1e-4,1e-1], tournament 2..8, {gens} gens"),
        "agents_total": int(sum(s.n_agents for s in shapes)),
        "batched": agent_gens / (batched_ms / 1000.0),
        "serial": agent_gens / (serial_ms / 1000.0),
        "unit": UNIT,
        "ratio": serial_ms / batched_ms,
        "batched_ms": batched_ms, "serial_ms": serial_ms,
        "batched_launches": batched_launches, "serial_launches": serial_launches,
        "autotune": tune,
        "identical": bool(identical),
    }


def measure_variants(args):
    """4,194,304-agent surface/genome variants (256-site steady, 32-site 8-bit tilted, 64-site
    hybrid), islands of 16/32/64, migration every 1/4/16 generations: agent-generations/s
    from founder populations, CUDA events on the run's stream, with the algorithmic HBM
    bytes per agent-generation (record in and out once per launch plus the immigrant
    records, 2G/k + 4G/(N k)) turned into a fraction of the measured copy bandwidth."""
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import variant_shapes

    peak, _ = measured_peaks()
    gens = args.variant_gens
    stream = torch.cuda.Stream()
    out = []
    for n in (16, 32, 64):
        for k in (1, 4, 16):
            for name, sh in variant_shapes(n, migrate_every=k, generations=gens).items():
                r = ga.Run(sh, stream=stream)
                r.step(2 * k)
                r.reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.step(gens)
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1)
                rate = sh.n_agents * gens / (ms / 1000.0)
                G = r.record_bytes
                b_alg = 2 * G / k + 4 * G / (n * k)
                out.append({"variant": name, "island_size": n, "migrate_every": k,
                            "record_bytes": G, "agent_gens_per_s": rate,
                            "hbm_frac": rate * b_alg / 1e9 / peak})
                r.close()
    return {"agents": 4194304, "generations": gens, "runs": out}


def measure_treatments(args):
    """The paper's own treatments (Sec. 3) on the 512x1024x32 grid: float fitness, 33% of
    births lose a normally distributed amount (purifying-only), plus 0.3% that gain one
    (adaptive); each run from founders for --treatment-gens generations, then MRCA bounds over
    4,096 sampled agents.  Reports agent-generations/s and the mean MRCA depth (T - hi)."""
    import numpy as np
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import (PAPER_FITNESS_ADAPTIVE,
                                                  PAPER_FITNESS_PURIFYING, sample_agent_ids)

    gens = args.treatment_gens
    stream = torch.cuda.Stream()
    out = {"generations": gens}
    for name, sh in (("purifying", PAPER_FITNESS_PURIFYING), ("adaptive", PAPER_FITNESS_ADAPTIVE)):
        r = ga.Run(sh, stream=stream)
        r.step(3)
        r.reset()
        ids = torch.from_numpy(sample_agent_ids(sh.n_agents, 4096, seed=7).view(np.int32))
        with torch.cuda.stream(stream):
            ids = ids.cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.step(gens)
        e1.record(stream)
        lo, hi = r.mrca_bounds_device(ids)
        r.sync()
        ms = e0.elapsed_time(e1)
        with torch.cuda.stream(stream):
            depth = (gens - hi.to(torch.int64)).double().mean().item()
            fit = r.snapshot_device()[:, 0:4].contiguous().view(torch.float32)
            mean_fit = fit.double().mean().item()
        stream.synchronize()
        out[name] = {"agent_gens_per_s": sh.n_agents * gens / (ms / 1000.0),
                     "mean_mrca_depth": depth, "mean_fitness": mean_fit}
        r.close()
    return out


def measure_async(args):
    """The asynchronous mode (send buffers, Sec. 2 loop) on the 512x1024x32 grid: each
    treatment from founders for --async-gens generations at window 1 (neighbours at most a
    generation apart) and window 16 (islands kept in registers 16 generations per launch),
    then mixed-counter MRCA bounds over 4,096 sampled agents.  Reports agent-generations/s,
    the median counter over the generation (1 when no lineage outruns the schedule), the
    mean MRCA depth min(Ta, Tb) - hi and the MRCA time."""
    import numpy as np
    import torch
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import (ASYNC, PAPER_ADAPTIVE, PAPER_PURIFYING,
                                                  sample_agent_ids)

    gens = args.async_gens
    stream = torch.cuda.Stream()
    n = 4096
    ids_h = sample_agent_ids(args.rows * args.cols * 32, n, seed=9)
    with torch.cuda.stream(stream):
        ids = torch.from_numpy(ids_h.view(np.int32)).cuda()
        iu = torch.triu_indices(n, n, 1, device="cuda")
    out = {"generations": gens, "workload": f"{args.rows}x{args.cols} islands x 32 agents"}
    base = {"adaptive": PAPER_ADAPTIVE.with_(rows=args.rows, cols=args.cols),
            "purifying": PAPER_PURIFYING.with_(rows=args.rows, cols=args.cols)}
    for window in (1, 16):
        for name, sh in base.items():
            sh = sh.with_(mode=ASYNC, async_window=window)
            r = ga.Run(sh, stream=stream)
            r.step(window)  # warm-up launch
            r.reset()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            r.step(gens)
            e1.record(stream)
            lo, hi = r.mrca_bounds_device(ids)
            e2.record(stream)
            r.sync()
            with torch.cuda.stream(stream):
                cnt = r.snapshot_device()[:, 4:8].contiguous().view(torch.int32).view(-1)
                c = cnt[ids.long()].to(torch.int64)
                T = torch.minimum(c[iu[0]], c[iu[1]])
                depth = (T - hi.to(torch.int64)).double().mean().item()
                med = cnt.to(torch.int64).median().item()
            stream.synchronize()
            out[f"window{window}_{name}"] = {
                "agent_gens_per_s": sh.n_agents * gens / (e0.elapsed_time(e1) / 1000.0),
                "median_counter_over_generation": med / gens,
                "mean_mrca_depth": depth, "mrca_ms": e1.elapsed_time(e2)}
            r.close()
    # the asynchronous figure: window 1, where no island gets more than a generation ahead of
    # another (window 16 lets lineages run ahead of the schedule: reported, not the figure)
    w1 = [out["window1_adaptive"], out["window1_purifying"]]
    out["agent_gens_per_s"] = statistics.mean(x["agent_gens_per_s"] for x in w1)
    out["median_counter_over_generation"] = max(x["median_counter_over_generation"] for x in w1)
    out["figure"] = "window 1, mean of both treatments; drift = largest median counter / generation"
    return out


def measure_serve(args):
    """Poisson stream (mean 50 requests/s) of GA runs with agents log-uniform on [1e4, 1e7]
    and generations log-uniform on [100, 10000], served with continuous batching under an
    HBM budget, then the same trace one run at a time.  Latency = completion - arrival."""
    import torch
    from paper_2405_03605_gb300 import serve
    from paper_2405_03605_gb300.workloads import serve_trace

    trace = serve_trace(n_requests=args.serve_requests, rate_hz=50.0, seed=42)
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(160e9, 0.8 * free))
    cont = serve.serve_continuous(trace, budget, chunk_gens=64, autotune=True)
    single = serve.serve_one_at_a_time(trace)
    out = {}
    for name, rep in (("continuous", cont), ("one_at_a_time", single)):
        out[name] = {"throughput": rep.throughput, "unit": UNIT,
                     "p50_s": rep.percentile(50), "p99_s": rep.percentile(99),
                     "makespan_s": rep.makespan, "launches": rep.launches}
    out["requests"] = len(trace)
    out["hbm_budget_bytes"] = budget
    out["peak_resident_bytes"] = cont.peak_bytes
    out["throughput_ratio"] = cont.throughput / single.throughput
    return out


def measure_e2e(args, shs, ids_h, world):
    """Same job through the public API with host buffers: create (library-allocated
    workspace), step, MRCA from pinned host ids into pinned host (lo, hi), snapshot into
    pinned host memory, destroy -- timed on the host around each step."""
    import numpy as np
    import torch
    from paper_2405_03605_gb300 import ga

    n = ids_h.size
    pairs = n * (n - 1) // 2
    pin = lambda nbytes: torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()
    ids_pin = pin(ids_h.nbytes).view(np.uint32)
    ids_pin[:] = ids_h
    lo_pin = pin(pairs * 4).view(np.uint32)
    hi_pin = pin(pairs * 4).view(np.uint32)
    rb = 16
    snaps = [pin(s.n_agents * rb).reshape(s.n_agents, rb) for s in shs]
    stream = torch.cuda.Stream()

    def job():
        for s, snap in zip(shs, snaps):
            r = ga.Run(s, stream=stream, workspace="library")
            r.step(args.gens)
            r.mrca_bounds(ids_pin, lo_pin, hi_pin)
            r.snapshot(snap)
            r.close()

    job()  # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        job()
        times.append(time.perf_counter() - t0)
    agent_gens = sum(s.n_agents * args.gens for s in shs) * world
    dt = statistics.mean(times)
    return {"value": agent_gens / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(len(shs) * ids_h.nbytes),
            "d2h_bytes_per_step": int(sum(s.n_agents * rb for s in shs) + len(shs) * 2 * pairs * 4),
            "steps": args.e2e_steps, "ms_per_step": dt * 1000}


def main():
    args = parse_args()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
