#!/usr/bin/env python
"""Benchmark of the CUBICS hot path: search nodes propagated per second.

A step is one complete search of the workload (every node labelled, propagated to its
fixpoint and backtracked on the GPU).  Default workload: 16-queens, all solutions (the
N-queens configuration at N = 16: 16 variables, 360 int_ne constraints, one uint32 word
per domain).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload queens16|queens14|rb4096]
  python bench.py --impl reference      # the CPU oracle on a bounded sample of the workload

Multi-GPU (torchrun): every rank solves its own copy of the workload (independent
problems, no data-path collective); value = all ranks' nodes / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "search nodes propagated/sec and time-to-all/first-solution vs plain GPU first-fail"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE = os.path.join(ROOT, "profiles", "search_kernel_queens16.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1909_09213_gb300", "csrc", f)
                  for f in ("search.cuh", "device.cuh", "internal.h", "kernels_w1.cu")]


def kernel_digest() -> str:
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


def golden_row(N):
    path = os.path.join(ROOT, "tests", "golden", "queens_oracle.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            f = ln.split()
            if int(f[0]) == N:
                return {"nodes": int(f[1]), "fails": int(f[2]), "solutions": int(f[3]),
                        "hash_sum": int(f[4]), "hash_xor": int(f[5]), "ne_evals": int(f[6]),
                        "work_bytes": float(f[7])}
    return None


def bytes_per_node(N):
    """Algorithmic bytes per search node: read the parent state and write the child
    (2 n W 4 bytes) plus 12 B per int_ne wake of the oracle's event-driven fixpoint."""
    g = golden_row(N)
    if g is None:
        return None
    return 2 * N * 1 * 4 + g["work_bytes"] / g["nodes"]


def traffic_from_profile():
    """DRAM bytes per search launch from the committed ncu summary, if it was taken on the
    current kernel sources."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    for ln in open(PROFILE):
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_digest") != kernel_digest():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (self.out or "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workloads

def make_workload(name):
    from paper_1909_09213_gb300 import instances as I
    if name == "queens16":
        return "16-queens, all solutions (16 vars, 360 int_ne, 1 uint32 word per domain)", I.queens(16)
    if name == "queens14":
        return "14-queens, all solutions (14 vars, 273 int_ne, 1 uint32 word per domain)", I.queens(14)
    raise SystemExit(f"unknown workload {name}")


def oracle_sample(N, depth=2):
    """A bounded sample of the N-queens search: the subtree under x0 = 0, x1 = 2 (or x0 = 0
    with depth 1), solved by the oracle; returns (nodes, seconds, description)."""
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    m = I.queens(N)
    fixed = [(0, 0), (1, 2), (2, 4)][:depth]
    for (v, a) in fixed:
        m.removed += [(v, u) for u in range(N) if u != a]
    om = O.OracleModel(m)
    t = time.perf_counter()
    r = O.solve(om, variant=1, W=1)
    dt = time.perf_counter() - t
    desc = f"{N}-queens subtree " + ", ".join(f"x{v}={a}" for v, a in fixed)
    return r.nodes, dt, desc


# ----------------------------------------------------------------------------- arms

def run_reference(args, rank, world):
    """The oracle as it stands, timed on this host, on the same metric and workload."""
    if rank != 0:
        return
    N = 16 if args.workload == "queens16" else 14
    desc, _ = make_workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(N, depth=3)
    nodes, secs = 0, 0.0
    sample = ""
    for _ in range(args.steps):
        n, dt, sample = oracle_sample(N, depth=3)
        nodes += n
        secs += dt
    value = nodes / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nodes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample}, {nodes // args.steps} nodes per step"},
            "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1909_09213_gb300 import cubics as K

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    desc, model = make_workload(args.workload)
    N = model.n
    stream = torch.cuda.Stream()
    p = K.Csp(model)
    p.stream = stream
    p.bind(K.CSP_ALL, 0, stream)
    p.upload(K.CSP_ALL, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # > 129 MB of L2

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1)                                              # untimed L2 flush
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.launch()
            e1.record(stream)
        rc = p.collect()
        if rc != 0:
            raise RuntimeError(f"search failed: {rc}")
        st = p.stats()
        return e0.elapsed_time(e1), st

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, kms, nodes = [], [], 0
    st = None
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            ms, st = step()
            times.append(ms)
            kms.append(st["ms"])
            nodes += st["nodes"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms, float(nodes)], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_max, nodes_all = float(mx[0]), float(t[1])
    else:
        total_ms_max, nodes_all = total_ms, float(nodes)
    value = nodes_all / (total_ms_max * 1e-3)

    # end to end through csp_solve: encode + pinned host-to-device copy + search + read-back
    e2e_nodes, e2e_secs = 0, 0.0
    for _ in range(max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        rc, est, _ = p.solve(K.CSP_ALL, 0)
        e2e_secs += time.perf_counter() - t0
        e2e_nodes += est["nodes"]
    e2e = {"value": e2e_nodes / e2e_secs, "unit": "nodes/s",
           "h2d_bytes_per_step": int(est["h2d_bytes"]), "d2h_bytes_per_step": int(est["d2h_bytes"])}

    if rank != 0:
        return
    golden = golden_row(N)
    parity = None
    if golden is not None:
        parity = (st["nodes"], st["fails"], st["solutions"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
            golden["nodes"], golden["fails"], golden["solutions"], golden["hash_sum"], golden["hash_xor"])
    smem_peak = K.probe_smem_bandwidth(stream)
    bpn = bytes_per_node(N)
    kernel_ms = sum(kms) / len(kms)
    roof = None
    if bpn is not None:
        achieved = bpn * st["nodes"] / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved / smem_peak, "traffic": traffic_from_profile(),
                "peak_source": "measured: csp_probe_smem_bandwidth (128-bit ld.shared, all SMs)",
                "bytes_per_node": bpn, "kernel": "search_kernel<1>", "kernel_ms": kernel_ms}
    cpu = None
    if not args.no_cpu_baseline:
        n_s, dt, sample = oracle_sample(N, depth=2)
        cpu = {"value": n_s / dt, "unit": "nodes/s", "cores": 1, "kind": "oracle",
               "sample": f"{sample} ({n_s} nodes, {dt:.1f} s on one host core)"}
    line = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": desc, "nodes_per_step": st["nodes"],
                       "solutions_per_step": st["solutions"],
                       "time_to_all_solutions_ms": total_ms_max / args.steps,
                       "l2": "flushed before every step (256 MiB write, untimed)",
                       "workers": st["workers"], "blocks": st["blocks"],
                       "parity_with_oracle_reference": parity},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": 2 * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="queens16", choices=["queens16", "queens14"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
