"""Write queens_oracle.txt: full-size oracle results for N-queens, all solutions.

Runs only the CPU oracle.  The search tree is split at the root: the root's fixpoint leaves
every domain full, first-fail picks x0, and each child x0 = v is the root of the model with
D(x0) = {v}; so nodes = 1 + sum of the children's nodes, and fails, solutions, hash sums
and work bytes add up (hash xors combine by xor).  Children run in parallel processes.

usage: python tests/golden/make_queens_reference.py 14 16
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def child(args):
    N, v = args
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    m = I.queens(N)
    m.removed += [(0, u) for u in range(N) if u != v]
    r = O.solve(O.OracleModel(m), variant=1, W=1)
    return r.nodes, r.fails, r.solutions, r.hash_sum, r.hash_xor, r.evals[0], r.work_bytes


def main(Ns):
    out = os.path.join(HERE, "queens_oracle.txt")
    rows = {}
    if os.path.exists(out):
        for ln in open(out):
            if ln.strip() and not ln.startswith("#"):
                rows[int(ln.split()[0])] = ln.strip()
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool:
        for N in Ns:
            res = pool.map(child, [(N, v) for v in range(N)])
            nodes = 1 + sum(r[0] for r in res)
            fails = sum(r[1] for r in res)
            sols = sum(r[2] for r in res)
            hsum = sum(r[3] for r in res) % (1 << 64)
            hxor = 0
            for r in res:
                hxor ^= r[4]
            evals = sum(r[5] for r in res)
            wbytes = sum(r[6] for r in res)
            rows[N] = f"{N} {nodes} {fails} {sols} {hsum} {hxor} {evals} {wbytes:.0f}"
            print(rows[N], flush=True)
    with open(out, "w") as f:
        f.write("# Oracle (oracle/cubics_oracle.c, FIFO fixpoint, W = 1) on N-queens, all solutions,\n"
                "# written by tests/golden/make_queens_reference.py (root split, children summed).\n"
                "# work_bytes: algorithmic bytes of all propagator wakes (12 B per int_ne wake);\n"
                "# the root's own fixpoint is not included.\n"
                "# N nodes fails solutions hash_sum hash_xor ne_evals work_bytes\n")
        for N in sorted(rows):
            f.write(rows[N] + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [14, 16])
