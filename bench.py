#!/usr/bin/env python
"""Benchmark of the CUBICS hot path: search nodes propagated per second.

A step is one complete search of the workload (every node labelled, propagated to its
fixpoint and backtracked on the GPU).  Workloads:

* queens16 (default) / queens15 / queens14: N-queens, all solutions (N vars, 3 C(N,2) int_ne,
  one uint32 word per domain), one problem per step;
* rb4096: 4096 seeded model-RB instances (n ~ U[20,60], d ~ U[8,32], tables), first solution
  or UNSAT proof for each, all in one persistent launch replayed from a CUDA graph, with the
  launch shape chosen by the autotuner;
* linad256: 256 mixed linear/alldifferent instances (200 vars on 0..255), first solution;
* rb_learned: 1024 held-out model-RB instances (n = 80, d = 20) with the learned brancher,
  trained first on subtree logs of 20 000 exhaustive searches, against first-fail;
* linad_learned: the mixed batch with the learned brancher, trained first on the levels that
  first-solution searches of 2048 training-seed instances refute, against first-fail;
* lns: one round of parallel large neighbourhood search on a mixed instance.

With the default workload the batch workloads also run once, after the timed steps, and are
reported under config.secondary: verdicts against the oracle, per-instance time to solution,
batched against one-at-a-time first-fail search, learned against first-fail ordering, and
the propagation of large nodes with a warp or a whole block per node.  The
CPU baseline is the oracle on one host core and, for N-queens, on every host core.

Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--no-secondary]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "search nodes propagated/sec and time-to-all/first-solution vs plain GPU first-fail"
GOLDEN = os.path.join(ROOT, "tests", "golden")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1909_09213_gb300", "csrc", f)
                  for f in ("search.cuh", "device.cuh", "internal.h", "kernels_w1.cu",
                            "kernels_w1r.cu")]


def note(msg):
    """progress on stderr (the JSON line alone goes to stdout)"""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def kernel_digest() -> str:
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


def traffic_from_profile(name):
    """DRAM bytes per search launch from a committed ncu summary, if it was taken on the
    current kernel sources."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
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
        self.out = ""

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

def _time_to_solution(res):
    """median / p90 / max of the instances' own search times (csp_result.ms), by verdict"""
    out = {}
    for name, sel in (("", lambda r: True), ("_sat", lambda r: r["status"] == 1),
                      ("_unsat", lambda r: r["status"] == 0)):
        ms = sorted(r["ms"] for r in res if sel(r))
        if ms:
            out[f"time_to_solution_ms{name}"] = {
                "median": float(np.median(ms)), "p90": float(np.percentile(ms, 90)),
                "max": float(ms[-1])}
    return out


def cpu_description():
    """host CPU model and core count (lscpu where it exists)"""
    model = ""
    try:
        for ln in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def _queens_subtree_nodes(args):
    """pool worker: the oracle's all-solution search of the N-queens subtree below `prefix`
    (x_0 .. x_{k-1} fixed); returns its node count"""
    N, prefix = args
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    m = I.queens(N)
    for v, a in enumerate(prefix):
        m.removed += [(v, u) for u in range(N) if u != a]
    return O.solve(O.OracleModel(m), variant=1, W=1).nodes


def queens_oracle_all_cores(N, budget_s=15.0):
    """The oracle as it stands, run on every host core at once over N-queens subtrees with
    x_0, x_1, x_2 fixed (queens-consistent prefixes in lexicographic order), one subtree per
    process, until about budget_s of wall time has passed.  A spawn pool, so that no process
    is forked from one that holds a CUDA context."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    prefixes = [(a, b, c) for a in range(N) for b in range(N) for c in range(N)
                if a != b and b != c and a != c and abs(a - b) != 1 and abs(b - c) != 1
                and abs(a - c) != 2]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_queens_subtree_nodes, [(6, (0,))] * cores)       # start-up, untimed
        t = time.perf_counter()
        nodes, k, dt = 0, 0, 0.0
        # subtrees are fed one at a time to whichever process is free; counted until the
        # budget is spent (the ones still running then are dropped, their time included)
        for c in pool.imap_unordered(_queens_subtree_nodes, [(N, p) for p in prefixes]):
            nodes += c
            k += 1
            dt = time.perf_counter() - t
            if dt >= budget_s:
                break
        pool.terminate()
    return {"value": nodes / dt, "unit": "nodes/s", "cores": cores, "kind": "oracle",
            "sample": (f"{N}-queens subtrees with x0, x1, x2 fixed, consistent prefixes in "
                       f"lexicographic order fed to {cores} processes: {k} finished "
                       f"({nodes} nodes, {dt:.1f} s wall)")}


def huge_node_propagation(K, count=2048, reps=3):
    """Constraint-parallel propagation of large nodes: fixpoints of `count` random sub-states
    (each present value kept with probability 7/8) of two 1000-variable instances, one
    csp_propagate call per shape: a warp per state, or a block of 128..1024 threads per state
    sharing out the constraints.  Kernel time from the call's events (best of `reps`); every
    shape must give the same fixpoints, and a sample of states is checked against the oracle."""
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    from paper_1909_09213_gb300 import tune
    out = {}
    rng = np.random.default_rng(20190920)
    cases = (("mixed: 1000 vars on 0..255 (8 words), 300 rows, 100 alldifferent groups of 10",
              I.lin_alldiff(I.seed_for(I.CFG_LINAD, 77), n=1000, dmax=255, rows=300, groups=100,
                            gsize=10)),
             ("model RB: 1000 vars, d = 32 (1 word), 4835 tables",
              I.model_rb(I.seed_for(I.CFG_RB, 999_001), 1000, 32)))
    for desc, m in cases:
        p = K.Csp(m)
        n, W, lo0 = p.layout()
        root = p.root_domains().ravel()
        r = [rng.integers(0, 1 << 32, size=(count, n * W), dtype=np.uint64).astype(np.uint32)
             for _ in range(3)]
        states = root[None, :] & (r[0] | r[1] | r[2])
        shapes, ref = {}, None
        for tpn in (32, 128, 256, 512, 1024):
            p.set_tiling(K.tiling(threads_per_node=tpn))
            try:
                best = None
                for _ in range(reps):
                    dout, failed = p.propagate(states)
                    ms = p.stats()["ms"]
                    best = ms if best is None else min(best, ms)
            except K.CspError as e:
                shapes[tpn] = {"error": str(e)}
                continue
            if ref is None:
                ref = (dout, failed)
            same = bool(np.array_equal(failed, ref[1]) and np.array_equal(dout[~failed], ref[0][~failed]))
            shapes[tpn] = {"kernel_ms": best, "states_per_s": count / (best * 1e-3),
                           "failed": int(failed.sum()), "same_fixpoints": same}
        om = O.OracleModel(m)
        ok = True
        for k in range(4):
            flags = np.zeros(int(om.off[-1]), dtype=np.uint8)
            for i in range(n):
                for j in range(int(om.size[i])):
                    b = int(om.lo[i]) + j - lo0
                    flags[om.off[i] + j] = (int(states[k, i * W + b // 32]) >> (b % 32)) & 1
            of, od = O.propagate(om, flags, variant=1)
            ok &= of == bool(ref[1][k])
            if not of:
                for i in range(n):
                    for j in range(int(om.size[i])):
                        b = int(om.lo[i]) + j - lo0
                        ok &= bool((int(ref[0][k, i * W + b // 32]) >> (b % 32)) & 1) == bool(od[om.off[i] + j])
        t, entry = tune.tune_propagate(m, states[:512], reps=1, use_cache=False)
        out[desc] = {"states": count, "state_bytes": n * W * 4, "shapes": shapes,
                     "oracle_sample_parity": bool(ok), "tuned_threads_per_node": t.threads_per_node}
    return out


class Queens:
    """N-queens, all solutions: one problem per step."""

    def __init__(self, N):
        from paper_1909_09213_gb300 import instances as I
        self.N = N
        self.model = I.queens(N)
        self.desc = (f"{N}-queens, all solutions ({N} vars, {len(self.model.ne)} int_ne, "
                     "1 uint32 word per domain)")
        self.profile = f"search_kernel_queens{N}.md"
        # one-word int_ne problems of at most 32 variables: domains held in registers
        self.kernel = "search_kernel_reg<true>" if N <= 32 else "search_kernel<1, true>"

    def golden(self):
        path = os.path.join(GOLDEN, "queens_oracle.txt")
        for ln in open(path):
            if ln.strip() and not ln.startswith("#"):
                f = ln.split()
                if int(f[0]) == self.N:
                    return {"nodes": int(f[1]), "fails": int(f[2]), "solutions": int(f[3]),
                            "hash_sum": int(f[4]), "hash_xor": int(f[5]), "work_bytes": float(f[7])}
        return None

    def bytes_per_node(self):
        """2 n W 4 (read the parent record's domains, write the child's) + 12 B per int_ne wake
        of the oracle's event-driven fixpoint, from the full-size oracle run."""
        g = self.golden()
        return None if g is None else 2 * self.N * 4 + g["work_bytes"] / g["nodes"]

    def setup(self, K, stream):
        self.p = K.Csp(self.model)
        self.p.stream = stream
        self.p.bind(K.CSP_ALL, 0, stream)
        self.p.upload(K.CSP_ALL, 0)

    def launch(self, K):
        self.p.launch()

    def launches_per_step(self):
        """the split search of the first 3 levels (per level: the fixpoint, then the counting,
        scan and writing passes of the expansion), the queues' set-up kernel and the search"""
        return 2 + 4 * 3

    def collect(self, K):
        rc = self.p.collect()
        if rc != 0:
            raise RuntimeError(f"search failed: {rc}")
        return self.p.stats()

    def e2e_step(self, K):
        rc, st, _ = self.p.solve(K.CSP_ALL, 0)
        return st

    def parity(self, st):
        g = self.golden()
        if g is None:
            return None
        return (st["nodes"], st["fails"], st["solutions"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
            g["nodes"], g["fails"], g["solutions"], g["hash_sum"], g["hash_xor"])

    def extra(self, K, st):
        """untimed: the autotuner's shapes for this problem (warps per block x two nodes or
        one node per warp x the problem's own or a twice wider bitset) with their nodes/s"""
        from paper_1909_09213_gb300 import tune
        out = {"solutions_per_step": st["solutions"],
               "time_to_all_solutions_ms": st["ms"]}
        t, entry = tune.tune_single(self.model, reps=1, use_cache=False)
        name = lambda c: (f"warps{c['warps_per_block']}/"
                          f"{'two_nodes' if c['threads_per_node'] == 16 else 'one_node'}_per_warp/"
                          f"words{c['domain_words'] or 1}")
        out["tuned_shape"] = name(entry["tiling"])
        out["shape_nodes_per_s"] = {name(c): round(st["nodes"] / (ms * 1e-3))
                                    for ms, c in entry["candidates"]}
        return out

    def oracle_sample(self, depth):
        """The subtree under x0=0, x1=2 (, x2=4): a bounded piece of the same search."""
        from oracle import oracle as O
        from paper_1909_09213_gb300 import instances as I
        m = I.queens(self.N)
        fixed = [(0, 0), (1, 2), (2, 4)][:depth]
        for (v, a) in fixed:
            m.removed += [(v, u) for u in range(self.N) if u != a]
        t = time.perf_counter()
        r = O.solve(O.OracleModel(m), variant=1, W=1)
        dt = time.perf_counter() - t
        return r.nodes, dt, f"{self.N}-queens subtree " + ", ".join(f"x{v}={a}" for v, a in fixed)

    def cpu_sample(self):
        return self.oracle_sample(2)

    def reference_step(self):
        return self.oracle_sample(3)


class RBBatch:
    """4096 model-RB instances, first solution or UNSAT proof each, one launch per step."""

    def __init__(self, count=4096):
        from paper_1909_09213_gb300 import instances as I
        self.count = count
        self.models = I.rb_batch(count)
        self.desc = (f"{count} model-RB instances, n~U[20,60], d~U[8,32], alpha 0.8, r 0.7, "
                     f"p {I.rb_tightness():.6f}, first solution or UNSAT each, one launch (CUDA graph)")
        self.profile = "search_kernel_rb4096.md"
        self.kernel = "search_kernel<1, true>"

    def golden(self):
        path = os.path.join(GOLDEN, "rb4096_oracle.txt")
        if not os.path.exists(path):
            return None
        rows = {}
        for ln in open(path):
            if ln.strip() and not ln.startswith("#"):
                i, n, d, status, nodes = map(int, ln.split())
                rows[i] = (status, nodes)
        return rows

    def bytes_per_node(self):
        """2 n W 4 + 4 (|D(x)| + 2) per table direction woken, from the oracle's event-driven
        fixpoint on the first 32 instances (first-solution searches, 2 000 nodes at most)."""
        from oracle import oracle as O
        nodes, by = 0, 0.0
        for m in self.models[:32]:
            r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, W=1, node_limit=2000)
            nodes += r.nodes
            by += r.work_bytes + r.nodes * 2 * m.n * 4
        return by / max(nodes, 1)

    def setup(self, K, stream):
        from paper_1909_09213_gb300 import tune
        self.tiling, self.tune_entry = tune.tune_batch(self.models, K.CSP_FIRST, calib=256, reps=1)
        self.probs = [K.Csp(m) for m in self.models]
        self.b = K.Batch(self.probs)
        self.b.stream = stream
        self.b.set_tiling(self.tiling)
        self.b.bind(K.CSP_FIRST, stream)
        self.rc, self.res = self.b.solve(K.CSP_FIRST, use_graph=True, bind=False)

    def launch(self, K):
        K._check(K.lib().csp_batch_launch(self.b.b, None, 1), "csp_batch_launch")

    def collect(self, K):
        import ctypes as C
        import numpy as np
        res = (K.csp_result * self.count)()
        words = K.lib().csp_batch_solution_words(self.b.b)
        self.sol = np.zeros(max(words, 1), dtype=np.int32)
        rc = K.lib().csp_batch_collect(self.b.b, res, self.sol.ctypes.data_as(K._I32P))
        if rc != 0:
            raise RuntimeError(f"batch failed: {rc}")
        self.res = [{f: getattr(r, f) for f, _ in K.csp_result._fields_} for r in res]
        st = self.b.stats()
        st["solutions"] = sum(r["status"] == 1 for r in self.res)
        st["nodes"] = sum(r["nodes"] for r in self.res)
        return st

    def e2e_step(self, K):
        rc, res = self.b.solve(K.CSP_FIRST, use_graph=True, bind=False)
        st = self.b.stats()
        st["nodes"] = sum(r["nodes"] for r in res)
        st["h2d_bytes"] = 0
        st["d2h_bytes"] = self.count * 40 + 4 * K.lib().csp_batch_solution_words(self.b.b)
        return st

    def parity(self, st):
        from oracle import oracle as O
        g = self.golden()
        if g is None:
            return None
        ok = True
        for i, (m, r) in enumerate(zip(self.models, self.res)):
            status, _ = g[i]
            if status >= 0 and r["status"] != status:
                ok = False
            if r["status"] == 1:
                s = self.sol[r["sol_offset"]:r["sol_offset"] + r["n"]]
                ok &= O.check_solution(O.OracleModel(m), s)
        return ok

    def extra(self, K, st):
        sat = sum(r["status"] == 1 for r in self.res)
        out = {"instances": self.count, "sat": sat, "unsat": self.count - sat,
               "time_to_all_first_solutions_ms": st["ms"],
               "tiling": {f: getattr(self.tiling, f) for f, _ in K.csp_tiling._fields_},
               "tuned_on": self.tune_entry.get("calib")}
        # plain first-fail GPU search on a sample: the first 512 instances one csp_solve at a
        # time, against the same 512 batched (one launch, same tiling)
        sample = self.probs[:512]
        note(f"plain first-fail on {len(sample)} instances")
        t0 = time.perf_counter()
        plain_nodes = 0
        for p in sample:
            rc, ps, _ = p.solve(K.CSP_FIRST)
            plain_nodes += ps["nodes"]
        out["plain_first_fail_gpu_ms_sample512"] = 1e3 * (time.perf_counter() - t0)
        out["plain_first_fail_gpu_nodes_sample512"] = plain_nodes
        b = K.Batch(sample)
        b.set_tiling(self.tiling)
        b.stream = self.b.stream
        b.bind(K.CSP_FIRST, self.b.stream)
        t0 = time.perf_counter()
        rc, res = b.solve(K.CSP_FIRST, use_graph=False, bind=False)
        out["batched_gpu_ms_sample512"] = 1e3 * (time.perf_counter() - t0)
        out["batched_gpu_kernel_ms_sample512"] = b.stats()["ms"]
        return out

    def secondary(self, K, stream):
        """One batched launch of the whole workload, as a secondary line of the default run:
        verdicts against the oracle's file, per-instance time to solution, the node count
        against the oracle's sequential search, and plain one-at-a-time first-fail search."""
        t0 = time.time()
        self.setup(K, stream)
        setup_s = time.time() - t0
        self.collect(K)
        st = self.b.stats()
        res = self.res
        nodes = sum(r["nodes"] for r in res)
        out = {"workload": self.desc, "setup_s": round(setup_s, 1),
               "tiling": {f: getattr(self.tiling, f) for f, _ in K.csp_tiling._fields_},
               "launch_ms": st["ms"], "nodes": nodes, "nodes_per_s": nodes / (st["ms"] * 1e-3),
               "sat": sum(r["status"] == 1 for r in res), "unsat": sum(r["status"] == 0 for r in res),
               "undecided": sum(r["status"] < 0 for r in res)}
        out.update(_time_to_solution(res))
        out.update(self._oracle_comparison(res))
        out.update(self.extra(K, st))                  # before parity: it may set references
        out["parity_with_oracle_reference"] = self.parity(st)
        return out

    def _oracle_comparison(self, res):
        """verdicts against the oracle's file, and nodes against its sequential first-solution
        search, on the instances the oracle decided within its node budget"""
        g = self.golden()
        if g is None:
            return {}
        dec = [(r, g[i]) for i, r in enumerate(res) if g[i][0] >= 0]
        mism = sum(r["status"] != s for r, (s, _) in dec)
        out = {"oracle_decided": len(dec), "verdict_mismatches": mism}
        for name, sel in (("all", lambda s: True), ("sat", lambda s: s == 1), ("unsat", lambda s: s == 0)):
            pairs = [(r["nodes"], n) for r, (s, n) in dec if sel(s)]
            if pairs:
                out[f"gpu_over_oracle_nodes_{name}"] = sum(a for a, _ in pairs) / max(1, sum(b for _, b in pairs))
                out[f"gpu_over_oracle_nodes_{name}_median"] = float(np.median([a / max(b, 1) for a, b in pairs]))
        return out

    def _oracle_instances(self, start, budget_s, node_limit=100_000):
        from oracle import oracle as O
        nodes, secs, k = 0, 0.0, start
        while secs < budget_s and k < self.count:
            t = time.perf_counter()
            r = O.solve(O.OracleModel(self.models[k]), mode=1, cap=1, variant=1, node_limit=node_limit)
            secs += time.perf_counter() - t
            nodes += r.nodes
            k += 1
        return nodes, secs, (f"instances {start}..{k - 1} of the batch, first solution each "
                             f"(at most {node_limit} nodes each)")

    def cpu_sample(self):
        return self._oracle_instances(0, 12.0)

    def reference_step(self):
        return self._oracle_instances(0, 1.5)


class LearnedRB(RBBatch):
    """The learning configuration: the network is trained on subtree logs of 20000 exhaustive
    searches (n = 30, d = 16); a step solves 1024 held-out instances (n = 80, d = 20, first
    solution) in one launch with the learned brancher.  The same batch under first-fail is
    timed alongside (time-to-solution at identical verdicts)."""

    def __init__(self, train_count=20000, eval_count=1024):
        from paper_1909_09213_gb300 import instances as I
        self.count = eval_count
        self.train_count = train_count
        self.models = I.rb_batch(eval_count, n_range=(80, 80), d_range=(20, 20), config_id=I.CFG_RB_EVAL)
        self.desc = (f"{eval_count} held-out model-RB instances n=80, d=20, first solution, learned "
                     f"brancher trained on {train_count} exhaustive searches (n=30, d=16)")
        self.profile = "search_kernel_rb_learned.md"
        self.kernel = "search_kernel_ext<1, true>"

    def golden(self):
        return None

    def bytes_per_node(self):
        """as for the model-RB batch, from the oracle's first-fail searches of 4 held-out
        instances (the learned order does not change what one node moves)"""
        from oracle import oracle as O
        nodes, by = 0, 0.0
        for m in self.models[:4]:
            r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, W=1, node_limit=20000)
            nodes += r.nodes
            by += r.work_bytes + r.nodes * 2 * m.n * 4
        return by / max(nodes, 1)

    def setup(self, K, stream):
        from paper_1909_09213_gb300 import instances as I
        from paper_1909_09213_gb300 import learn
        t0 = time.time()
        train_models = I.rb_batch(self.train_count, n_range=(30, 30), d_range=(16, 16),
                                  config_id=I.CFG_RB_TRAIN)
        data, self.cinfo = learn.collect(train_models, cap=8_000_000, sample=1)
        self.params, self.tinfo = learn.train(data, epochs=8)
        self.prep_s = time.time() - t0
        self.tiling = K.tiling(warps_per_block=4, smem_levels=8)
        self.tune_entry = {"calib": None}
        self.probs = [K.Csp(m) for m in self.models]
        self.b = K.Batch(self.probs)
        self.b.stream = stream
        self.b.set_tiling(self.tiling)
        w = np.ascontiguousarray(self.params, dtype=np.uint16)
        K._check(K.lib().csp_batch_set_brancher(self.b.b, K.CSP_BR_LEARNED, w.ctypes.data_as(K._U16P)),
                 "csp_batch_set_brancher")
        self.b.bind(K.CSP_FIRST, stream)
        self.rc, self.res = self.b.solve(K.CSP_FIRST, use_graph=True, bind=False)

    def parity(self, st):
        # the verdicts must equal first-fail's on every instance; SAT solutions are checked
        from oracle import oracle as O
        ok = [r["status"] for r in self.res] == [r["status"] for r in self.ff_res]
        for m, r in zip(self.models, self.res):
            if r["status"] == 1:
                ok &= O.check_solution(O.OracleModel(m), self.sol[r["sol_offset"]:r["sol_offset"] + r["n"]])
        return ok

    def threshold_variant(self, K):
        """The same evaluation at the first-moment threshold p* = 1 - exp(-ln d / (r ln n))
        of n = 80, d = 20 (0.6234) instead of the configured p (0.6811, where every instance
        is UNSAT): other held-out seeds, the same trained network, learned against first-fail
        (2 M nodes at most per instance), and the SAT fraction."""
        from oracle import oracle as O
        from paper_1909_09213_gb300 import instances as I
        p_star = I.rb_threshold_tightness(80, 20)
        models = I.rb_batch(self.count, n_range=(80, 80), d_range=(20, 20), config_id=I.CFG_RB_EVAL,
                            p=p_star, first=100_000)
        lim = K.limits(node_limit=2_000_000)
        out = {"p": p_star, "instances": self.count}
        for name in ("first_fail", "learned"):
            b = K.Batch([K.Csp(m) for m in models])
            b.stream = self.b.stream
            b.set_tiling(self.tiling)
            if name == "learned":
                w = np.ascontiguousarray(self.params, dtype=np.uint16)
                K._check(K.lib().csp_batch_set_brancher(b.b, K.CSP_BR_LEARNED, w.ctypes.data_as(K._U16P)),
                         "csp_batch_set_brancher")
            best = None
            for _ in range(2):
                rc, res = b.solve(K.CSP_FIRST, lim=lim, use_graph=True)
                ms = b.stats()["ms"]
                if best is None or ms < best[0]:
                    best = (ms, res)
            ms, res = best
            ok = all(O.check_solution(O.OracleModel(m), r["solution"])
                     for m, r in zip(models, res) if r["status"] == 1)
            out[name] = {"ms": ms, "nodes": sum(r["nodes"] for r in res),
                         "sat": sum(r["status"] == 1 for r in res),
                         "unsat": sum(r["status"] == 0 for r in res),
                         "undecided": sum(r["status"] < 0 for r in res), "solutions_valid": ok,
                         "status": [r["status"] for r in res]}
        f, l = out["first_fail"].pop("status"), out["learned"].pop("status")
        out["verdicts_agree_where_both_decide"] = all(a == b for a, b in zip(f, l) if a >= 0 and b >= 0)
        out["sat_fraction"] = out["first_fail"]["sat"] / self.count
        out["speedup_vs_first_fail"] = out["first_fail"]["ms"] / max(out["learned"]["ms"], 1e-9)
        return out

    def extra(self, K, st):
        b = K.Batch([K.Csp(m) for m in self.models])
        b.stream = self.b.stream
        b.set_tiling(self.tiling)
        b.bind(K.CSP_FIRST, self.b.stream)
        times = []
        for _ in range(4):
            rc, self.ff_res = b.solve(K.CSP_FIRST, use_graph=True, bind=False)
            times.append(b.stats()["ms"])
        ff_ms = min(times[1:])
        ff_nodes = sum(r["nodes"] for r in self.ff_res)
        sat = sum(r["status"] == 1 for r in self.res)
        return {"instances": self.count, "sat": sat, "unsat": self.count - sat,
                "sat_fraction": sat / self.count,
                "time_to_all_first_solutions_ms": st["ms"],
                "first_fail_gpu_ms": ff_ms, "first_fail_gpu_nodes": ff_nodes,
                "learned_nodes": st["nodes"], "speedup_vs_first_fail": ff_ms / st["ms"],
                "threshold_p": self.threshold_variant(K),
                "training": {"logged_subtrees": self.cinfo["entries"], "train_nodes": self.cinfo["nodes"],
                             "adam_steps": self.tinfo["steps"], "mse": self.tinfo["mse_per_epoch"][-1],
                             "target_variance": self.tinfo["target_variance"],
                             "collect_and_train_s": self.prep_s}}


class LinAdBatch(RBBatch):
    """256 mixed linear/alldifferent instances (200 vars on 0..255, 8-word domains, 60 rows of
    5-20 terms, 20 alldifferent groups of 10), first solution each, one launch per step, a
    node limit per instance (instances that reach it are reported undecided)."""

    NODE_LIMIT = 2_000_000

    def __init__(self, count=256):
        from paper_1909_09213_gb300 import instances as I
        self.count = count
        self.models = I.linad_batch(count)
        self.desc = (f"{count} mixed instances: 200 vars on 0..255 (8 words), 60 int_lin_le rows of "
                     f"5-20 terms, 20 alldifferent groups of 10, rhs theta {I.LINAD_THETA}, first "
                     f"solution, {self.NODE_LIMIT} nodes at most per instance")
        self.profile = "search_kernel_linad256.md"
        self.kernel = "search_kernel<8, false>"

    def golden(self):
        return None

    def bytes_per_node(self):
        """2 n W 4 + 4 W (2k + changed) per row wake + 4 W 2k per alldifferent wake, from the
        oracle's event-driven fixpoint on the first solution search of 2 instances (500 nodes)"""
        from oracle import oracle as O
        nodes, by = 0, 0.0
        for m in self.models[:2]:
            r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, W=8, node_limit=500)
            nodes += r.nodes
            by += r.work_bytes + r.nodes * 2 * m.n * 8 * 4
        return by / max(nodes, 1)

    def setup(self, K, stream):
        self.tiling = K.tiling(warps_per_block=4, smem_levels=4)
        self.tune_entry = {"calib": None}
        self.lim = K.limits(node_limit=self.NODE_LIMIT)
        self.probs = [K.Csp(m) for m in self.models]
        self.b = K.Batch(self.probs)
        self.b.stream = stream
        self.b.set_tiling(self.tiling)
        self.b.bind(K.CSP_FIRST, stream)
        self.rc, self.res = self.b.solve(K.CSP_FIRST, lim=self.lim, use_graph=True, bind=False)

    def launch(self, K):
        import ctypes
        K._check(K.lib().csp_batch_launch(self.b.b, ctypes.byref(self.lim), 1), "csp_batch_launch")

    def e2e_step(self, K):
        rc, res = self.b.solve(K.CSP_FIRST, lim=self.lim, use_graph=True, bind=False)
        st = self.b.stats()
        st["nodes"] = sum(r["nodes"] for r in res)
        st["h2d_bytes"] = 0
        st["d2h_bytes"] = self.count * 40 + 4 * K.lib().csp_batch_solution_words(self.b.b)
        return st

    def parity(self, st):
        # every reported solution satisfies every constraint (oracle check)
        from oracle import oracle as O
        ok = True
        for m, r in zip(self.models, self.res):
            if r["status"] == 1:
                ok &= O.check_solution(O.OracleModel(m), self.sol[r["sol_offset"]:r["sol_offset"] + r["n"]])
        return ok

    def extra(self, K, st):
        sat = sum(r["status"] == 1 for r in self.res)
        unsat = sum(r["status"] == 0 for r in self.res)
        return {"instances": self.count, "sat": sat, "unsat": unsat,
                "undecided_at_node_limit": self.count - sat - unsat,
                "time_to_all_first_solutions_ms": st["ms"]}

    def cpu_sample(self):
        return self._oracle_instances(0, 12.0)

    def reference_step(self):
        return self._oracle_instances(0, 1.5)


class LearnedLinAd(LinAdBatch):
    """The mixed linear/alldifferent batch with learned ordering: the network is trained on
    the refuted levels of first-solution searches of 2048 training-seed instances (40 000
    nodes at most each); a step solves the 256 graded instances in one launch with the
    learned brancher.  The same batch under first-fail is timed alongside."""

    # measured: 2048 x 40 000 nodes, 16 epochs gives the best network within ~30 s of
    # collection and training (4096 x 10 000 and 3072 x 20 000 are slower at evaluation)
    TRAIN, TRAIN_NODES, EPOCHS = 2048, 40_000, 16

    def __init__(self, count=256):
        super().__init__(count)
        self.desc = (f"{count} mixed instances (200 vars on 0..255, 60 int_lin_le rows, 20 "
                     f"alldifferent groups of 10), first solution, learned brancher trained on "
                     f"first-solution searches of {self.TRAIN} training-seed instances, "
                     f"{self.NODE_LIMIT} nodes at most per instance")
        self.profile = "search_kernel_linad_learned.md"
        self.kernel = "search_kernel_ext<8, false>"

    def setup(self, K, stream):
        from paper_1909_09213_gb300 import learn
        t0 = time.time()
        self.params, self.tinfo = learn.linad_training(self.TRAIN, self.TRAIN_NODES, self.EPOCHS)
        self.prep_s = time.time() - t0
        self.tiling = K.tiling(warps_per_block=4, smem_levels=4)
        self.tune_entry = {"calib": None}
        self.lim = K.limits(node_limit=self.NODE_LIMIT)
        self.probs = [K.Csp(m) for m in self.models]
        self.b = K.Batch(self.probs)
        self.b.stream = stream
        self.b.set_tiling(self.tiling)
        w = np.ascontiguousarray(self.params, dtype=np.uint16)
        K._check(K.lib().csp_batch_set_brancher(self.b.b, K.CSP_BR_LEARNED, w.ctypes.data_as(K._U16P)),
                 "csp_batch_set_brancher")
        self.b.bind(K.CSP_FIRST, stream)
        self.rc, self.res = self.b.solve(K.CSP_FIRST, lim=self.lim, use_graph=True, bind=False)

    def parity(self, st):
        # every solution satisfies the model (oracle check); where both orderings decide an
        # instance, they agree on SAT / UNSAT
        from oracle import oracle as O
        ok = True
        for m, r, f in zip(self.models, self.res, self.ff_res):
            if r["status"] == 1:
                ok &= O.check_solution(O.OracleModel(m), self.sol[r["sol_offset"]:r["sol_offset"] + r["n"]])
            if r["status"] >= 0 and f["status"] >= 0:
                ok &= r["status"] == f["status"]
        return ok

    def extra(self, K, st):
        b = K.Batch([K.Csp(m) for m in self.models])
        b.stream = self.b.stream
        b.set_tiling(self.tiling)
        b.bind(K.CSP_FIRST, self.b.stream)
        best = None
        for _ in range(3):
            rc, res = b.solve(K.CSP_FIRST, lim=self.lim, use_graph=True, bind=False)
            ms = b.stats()["ms"]
            if best is None or ms < best[0]:
                best = (ms, res)
        ff_ms, self.ff_res = best
        out = super().extra(K, st)
        out.update({"first_fail_gpu_ms": ff_ms,
                    "first_fail_gpu_nodes": sum(r["nodes"] for r in self.ff_res),
                    "first_fail_undecided": sum(r["status"] < 0 for r in self.ff_res),
                    "first_fail_time_to_solution_ms": _time_to_solution(self.ff_res).get("time_to_solution_ms"),
                    "learned_nodes": st["nodes"], "speedup_vs_first_fail": ff_ms / st["ms"],
                    "training": {"instances": self.tinfo["train_instances"],
                                 "node_limit": self.tinfo["node_limit"],
                                 "logged_subtrees": self.tinfo["collect"]["entries"],
                                 "train_nodes": self.tinfo["collect"]["nodes"],
                                 "adam_steps": self.tinfo["train"]["steps"],
                                 "mse": self.tinfo["train"]["mse_per_epoch"][-1],
                                 "target_variance": self.tinfo["train"]["target_variance"],
                                 "collect_and_train_s": self.prep_s}})
        return out


class LNSRound(RBBatch):
    """Parallel large neighbourhood search on a mixed instance (200 vars on 0..255, 60 rows,
    20 alldifferent groups) with objective min sum w_i x_i, w_i ~ U[1, 9]: one step is one
    search round, 256 neighbourhoods (about 10 % of the variables reset, the others fixed to
    the incumbent, objective <= incumbent - 1) in one launch, first solution each."""

    COPIES, FRAC, NODE_LIMIT, WARM_ROUNDS = 256, 0.1, 5000, 3

    def __init__(self):
        from paper_1909_09213_gb300 import instances as I
        self.model = I.lin_alldiff(I.seed_for(I.CFG_LINAD, 0))
        self.obj = I.objective_weights(0, self.model.n)
        self.count = self.COPIES
        self.desc = (f"LNS round on a mixed instance (200 vars on 0..255, 60 int_lin_le rows, 20 "
                     f"alldifferent groups of 10), objective min sum w_i x_i (w ~ U[1,9]): "
                     f"{self.COPIES} neighbourhoods, {self.FRAC:.0%} of the vars reset, "
                     f"{self.NODE_LIMIT} nodes at most each, first solution, one launch (CUDA graph)")
        self.profile = "search_kernel_lns_linad.md"
        self.kernel = "search_kernel<8, false>"

    def golden(self):
        return None

    def bytes_per_node(self):
        """2 n W 4 + the oracle's wake bytes, from first-solution searches of 4 neighbourhoods
        of the round (500 nodes at most each)"""
        from oracle import lns_ref as L
        from oracle import oracle as O
        nodes, by = 0, 0.0
        for mk in self.masks[:4]:
            m = L.neighbourhood_model(self.model, self.inc, mk, self.obj, self.bound)
            r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, W=8, node_limit=500)
            nodes += r.nodes
            by += r.work_bytes + r.nodes * 2 * m.n * 8 * 4
        return by / max(nodes, 1)

    def setup(self, K, stream):
        from paper_1909_09213_gb300 import instances as I
        from paper_1909_09213_gb300 import lns
        self.lns_mod = lns
        # a mid-search incumbent: the first solution, improved by a few rounds (untimed)
        self.search = lns.LNS(self.model, self.obj, copies=self.COPIES, frac=self.FRAC,
                              node_limit=self.NODE_LIMIT, seed=1, share=False)
        self.initial_value = self.search.initial()
        for r in range(self.WARM_ROUNDS):
            self.search.round(r)
        self.inc = self.search.incumbent.copy()
        self.value = self.search.value
        self.bound = self.value - 1
        self.masks = I.relax_masks(self.model.n, self.COPIES, self.FRAC, 1000, 1)
        self.bounded = self.search.base.clone()
        self.bounded.post_lin(self.obj[0], self.obj[1], self.bound)
        _, _, lo0 = self.bounded.layout()
        roots = lns.neighbourhood_roots(self.bounded.root_domains(), lo0, self.inc, self.masks)
        self.tiling = K.tiling(warps_per_block=4, smem_levels=4)
        self.tune_entry = {"calib": None}
        self.lim = K.limits(node_limit=self.NODE_LIMIT)
        self.b = K.Batch.from_roots(self.bounded, roots)
        self.b.stream = stream
        self.b.set_tiling(self.tiling)
        self.b.bind(K.CSP_FIRST, stream)
        self.rc, self.res = self.b.solve(K.CSP_FIRST, lim=self.lim, use_graph=True, bind=False)

    def launch(self, K):
        import ctypes
        K._check(K.lib().csp_batch_launch(self.b.b, ctypes.byref(self.lim), 1), "csp_batch_launch")

    def e2e_step(self, K):
        """A whole round through the public API: draw the neighbourhoods, build the copies
        (one encoding, per-copy roots), upload, search, read the results back."""
        from paper_1909_09213_gb300 import instances as I
        self.e2e_round = getattr(self, "e2e_round", 2000) + 1
        masks = I.relax_masks(self.model.n, self.COPIES, self.FRAC, self.e2e_round, 1)
        _, _, lo0 = self.bounded.layout()
        roots = self.lns_mod.neighbourhood_roots(self.bounded.root_domains(), lo0, self.inc, masks)
        b = K.Batch.from_roots(self.bounded, roots)
        b.set_tiling(self.tiling)
        b.stream = self.b.stream
        rc, res = b.solve(K.CSP_FIRST, lim=self.lim)
        if rc != 0:
            raise RuntimeError(f"LNS round failed: {rc}")
        st = b.stats()
        st["nodes"] = sum(r["nodes"] for r in res)
        self.e2e_note = ("each end-to-end step is a whole round on fresh neighbourhoods (other "
                         "copies than the device-timed launch), workspace allocation included")
        return st

    def parity(self, st):
        # every solution satisfies the model, the fixings and the bound; the verdicts of the
        # first 8 neighbourhoods equal the oracle's where it decides them within 5 000 nodes
        from oracle import lns_ref as L
        from oracle import oracle as O
        om = O.OracleModel(self.model)
        ok = True
        for mk, r in zip(self.masks, self.res):
            if r["status"] == 1:
                s = self.sol[r["sol_offset"]:r["sol_offset"] + r["n"]]
                ok &= O.check_solution(om, s) and L.objective(self.obj, s) <= self.bound
                ok &= all(s[x] == self.inc[x] for x in range(self.model.n) if not mk[x])
        for mk, r in list(zip(self.masks, self.res))[:8]:
            want = L.verdict(L.neighbourhood_model(self.model, self.inc, mk, self.obj, self.bound),
                             node_limit=5_000)
            if want >= 0 and r["status"] >= 0:
                ok &= want == r["status"]
        return ok

    def extra(self, K, st):
        sat = sum(r["status"] == 1 for r in self.res)
        unsat = sum(r["status"] == 0 for r in self.res)
        e2e_note = getattr(self, "e2e_note", None)
        # the whole search from scratch, 20 s at most (untimed by the events; wall clock)
        note("full LNS run")
        # rank 0 alone runs this part: no exchange with the other ranks
        res = self.lns_mod.LNS(self.model, self.obj, copies=self.COPIES, frac=self.FRAC,
                               node_limit=self.NODE_LIMIT, seed=2, share=False).run(
                                   rounds=200, time_budget_s=20)
        return {"copies": self.count, "sat": sat, "unsat": unsat, "e2e_note": e2e_note,
                "undecided_at_node_limit": self.count - sat - unsat,
                "incumbent_of_the_timed_round": int(self.value),
                "full_search": {"initial": res.initial, "best": res.best, "optimal": res.optimal,
                                "rounds": len(res.rounds), "nodes": res.nodes,
                                "kernel_ms": res.kernel_ms, "wall_ms": res.wall_ms,
                                "trajectory": [(r.round, r.best, round(r.wall_ms, 1))
                                               for r in res.rounds if r.improved]}}

    def _oracle_copies(self, budget_s, node_limit=20_000):
        from oracle import lns_ref as L
        from oracle import oracle as O
        if not hasattr(self, "inc"):
            # the reference arm has no GPU incumbent: the oracle's first solution instead
            from paper_1909_09213_gb300 import instances as I
            r = O.solve(O.OracleModel(self.model), mode=1, cap=1, variant=1)
            self.inc = r.sols[0].copy()
            self.value = L.objective(self.obj, self.inc)
            self.bound = self.value - 1
            self.masks = I.relax_masks(self.model.n, self.COPIES, self.FRAC, 1000, 1)
        nodes, secs, k = 0, 0.0, 0
        while secs < budget_s and k < len(self.masks):
            m = L.neighbourhood_model(self.model, self.inc, self.masks[k], self.obj, self.bound)
            t = time.perf_counter()
            r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, node_limit=node_limit)
            secs += time.perf_counter() - t
            nodes += r.nodes
            k += 1
        return nodes, secs, (f"neighbourhoods 0..{k - 1} of the round, first solution each "
                             f"(at most {node_limit} nodes each)")

    def cpu_sample(self):
        return self._oracle_copies(12.0)

    def reference_step(self):
        return self._oracle_copies(1.5)


def make_workload(name):
    if name == "queens16":
        return Queens(16)
    if name in ("queens14", "queens15"):
        return Queens(int(name[6:]))
    if name == "rb4096":
        return RBBatch(4096)
    if name == "linad256":
        return LinAdBatch(256)
    if name == "rb_learned":
        return LearnedRB()
    if name == "linad_learned":
        return LearnedLinAd()
    if name == "lns":
        return LNSRound()
    raise SystemExit(f"unknown workload {name}")


# ----------------------------------------------------------------------------- arms

def run_reference(args, rank, world):
    """The oracle as it stands, timed on this host, on the same metric and workload."""
    if rank != 0:
        return
    wl = make_workload(args.workload)
    for _ in range(args.warmup):
        wl.reference_step()
    nodes, secs, sample = 0, 0.0, ""
    for _ in range(args.steps):
        n, dt, sample = wl.reference_step()
        nodes += n
        secs += dt
    value = nodes / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nodes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": wl.desc, "sample": sample},
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
    wl = make_workload(args.workload)
    stream = torch.cuda.Stream()
    note(f"setup {args.workload}")
    wl.setup(K, stream)
    note("setup done; warm-up and timed steps")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # > 129 MB of L2

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1)                                              # untimed L2 flush
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wl.launch(K)
            e1.record(stream)
        st = wl.collect(K)
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
            kms.append(st.get("kernel_ms") or st["ms"])     # the search kernel alone
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

    # end to end through the public API: host-to-device copies, search, read-back
    note("timed steps done; end-to-end steps")
    e2e_nodes, e2e_secs = 0, 0.0
    est = None
    for _ in range(max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        est = wl.e2e_step(K)
        e2e_secs += time.perf_counter() - t0
        e2e_nodes += est["nodes"]
    e2e = {"value": e2e_nodes / e2e_secs, "unit": "nodes/s",
           "h2d_bytes_per_step": int(est["h2d_bytes"]), "d2h_bytes_per_step": int(est["d2h_bytes"])}

    if rank != 0:
        return
    note("workload extras, parity, roofline, CPU baseline")
    extra = wl.extra(K, st)
    parity = wl.parity(st)
    smem_peak = K.probe_smem_bandwidth(stream)
    bpn = wl.bytes_per_node()
    kernel_ms = sum(kms) / len(kms)
    roof = None
    if bpn is not None:
        achieved = bpn * st["nodes"] / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved / smem_peak, "traffic": traffic_from_profile(wl.profile),
                "peak_source": "measured: csp_probe_smem_bandwidth (volatile 128-bit ld.shared, all SMs)",
                "bytes_per_node": bpn, "kernel": wl.kernel, "kernel_ms": kernel_ms}
    cpu = None
    if not args.no_cpu_baseline:
        n_s, dt, sample = wl.cpu_sample()
        cpu = {"value": n_s / dt, "unit": "nodes/s", "cores": 1, "kind": "oracle",
               "sample": f"{sample} ({n_s} nodes, {dt:.1f} s on one host core)"}
        cpu.update(cpu_description())
        if isinstance(wl, Queens):
            note("oracle on every host core")
            cpu["all_cores"] = queens_oracle_all_cores(wl.N)
    secondary = None
    if args.secondary and world == 1 and args.workload == "queens16":
        secondary = {}
        for name, make in (("rb4096", lambda: RBBatch(4096)), ("linad256", lambda: LinAdBatch(256)),
                           ("rb_learned", lambda: LearnedRB()), ("linad_learned", lambda: LearnedLinAd())):
            note(f"secondary workload {name}")
            t0 = time.time()
            secondary[name] = make().secondary(K, stream)
            secondary[name]["wall_s"] = round(time.time() - t0, 1)
        note("secondary: propagation of large nodes, warp or block per node")
        t0 = time.time()
        secondary["huge_node_propagation"] = huge_node_propagation(K)
        secondary["huge_node_propagation"]["wall_s"] = round(time.time() - t0, 1)
    config = {"workload": wl.desc, "nodes_per_step": st["nodes"],
              "search_ms_per_step_device": sum(kms) / len(kms),
              "l2": "flushed before every step (256 MiB write, untimed)",
              "workers": st["workers"], "blocks": st["blocks"],
              "idle_fraction": st["wait_ns"] / max(1.0, st["workers"] * kernel_ms * 1e6),
              "parity_with_oracle_reference": parity}
    config.update(extra)
    if secondary is not None:
        config["secondary"] = secondary
    line = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": config, "clocks": clk.summary(), "e2e": e2e,
            "gpu_launches": getattr(wl, "launches_per_step", lambda: 2)() * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="queens16",
                    choices=["queens16", "queens15", "queens14", "rb4096", "rb_learned", "linad256",
                             "linad_learned", "lns"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--secondary", dest="secondary", action="store_true", default=True,
                    help="with the default workload: also run the batch workloads once "
                         "(model RB, mixed linear/alldifferent, learned branching) and report "
                         "them under config.secondary")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false")
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
