"""Write rb4096_oracle.txt: the oracle's verdict on every instance of the batched model-RB
workload (4096 instances, n ~ U[20,60], d ~ U[8,32], alpha 0.8, r 0.7, first solution).

Runs only the CPU oracle (FIFO fixpoint, first-fail, d-way), instances in parallel
processes.  Columns: index n d status nodes, status 1 SAT / 0 UNSAT / -5 undecided within the
node budget; nodes is the oracle's sequential count up to its first solution.  Verdicts are
appended to a work file as they arrive, so an interrupted run resumes where it stopped.

usage: python tests/golden/make_rb_reference.py [count] [node_budget]
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "rb4096_oracle.txt")
PARTIAL = OUT + ".partial"


def verdict(args):
    i, budget = args
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    m = I.rb_batch(1, first=i)[0]
    r = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1, node_limit=budget)
    return i, m.n, m.hi[0] + 1, r.status, r.nodes


def main(count=4096, budget=2_000_000):
    done = {}
    if os.path.exists(PARTIAL):
        for ln in open(PARTIAL):
            f = ln.split()
            if len(f) == 5:
                done[int(f[0])] = tuple(int(x) for x in f)
    todo = [(i, budget) for i in range(count) if i not in done]
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool, open(PARTIAL, "a") as part:
        for r in pool.imap_unordered(verdict, todo):
            done[r[0]] = r
            part.write(" ".join(str(int(x)) for x in r) + "\n")
            part.flush()
    rows = [done[i] for i in range(count)]
    with open(OUT, "w") as f:
        f.write("# Oracle verdicts on the batched model-RB workload (instances.rb_batch: 4096 instances, "
                "n~U[20,60], d~U[8,32]),\n"
                f"# first solution, node budget {budget}; written by tests/golden/make_rb_reference.py.\n"
                "# index n d status nodes   (status 1 SAT, 0 UNSAT, -5 undecided)\n")
        for r in rows:
            f.write(" ".join(str(int(x)) for x in r) + "\n")
    os.remove(PARTIAL)
    print(f"{count} instances: {sum(r[3] == 1 for r in rows)} SAT, {sum(r[3] == 0 for r in rows)} "
          f"UNSAT, {sum(r[3] < 0 for r in rows)} undecided", flush=True)


if __name__ == "__main__":
    a = [int(x) for x in sys.argv[1:]]
    main(*a)
