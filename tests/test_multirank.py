"""Multi-rank host logic on CPU (gloo, world size 2): sharing one search tree between ranks
and combining their statistics, plus a rank that fails before the exchange.

The ranks run the oracle on their share of the root's children (each child x0 = v is the
root of the model with D(x0) = {v}); rank 0 also counts the root.  The combined statistics
must equal the undivided oracle search.  No GPU is involved.
"""
import datetime
import json
import os
import socket
import tempfile

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_share(N, rank, world):
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    from paper_1909_09213_gb300 import shard
    part, nparts = shard.partition(rank, world)
    st = {"nodes": 1 if part == 0 else 0, "fails": 0, "solutions": 0, "sol_hash_sum": 0,
          "sol_hash_xor": 0}
    children = list(range(N))                     # the root's fixpoint leaves D(x0) = 0..N-1
    for v in children[part::nparts]:
        m = I.queens(N)
        m.removed += [(0, u) for u in range(N) if u != v]
        r = O.solve(O.OracleModel(m), variant=1)
        st = shard.combine([st, {"nodes": r.nodes, "fails": r.fails, "solutions": r.solutions,
                                 "sol_hash_sum": r.hash_sum, "sol_hash_xor": r.hash_xor}])
    return st


def _worker(rank, world, port, outdir, N, fail_rank):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    from paper_1909_09213_gb300 import shard
    result = {"rank": rank}
    try:
        st = _rank_share(N, rank, world)
        if rank == fail_rank:
            raise RuntimeError("injected failure before the exchange")
        result["combined"] = shard.combine_across_ranks(st)
    except Exception as e:                                       # noqa: BLE001
        result["error"] = f"{type(e).__name__}: {e}"
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(result, f)
    if "error" in result and rank == fail_rank:
        os._exit(3)                                              # leave without the collective
    try:
        dist.destroy_process_group()
    except Exception:                                            # noqa: BLE001
        pass


def _run(world, N, fail_rank):
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_worker, args=(r, world, port, d, N, fail_rank))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            if p.is_alive():
                p.kill()
                raise AssertionError("a rank did not finish")
        out = {}
        for r in range(world):
            path = os.path.join(d, f"rank{r}.json")
            out[r] = json.load(open(path)) if os.path.exists(path) else {}
        return out, [p.exitcode for p in procs]


def test_two_ranks_share_one_tree():
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    out, codes = _run(2, 8, fail_rank=-1)
    assert codes == [0, 0]
    full = O.solve(O.OracleModel(I.queens(8)), variant=1)
    expect = {"nodes": full.nodes, "fails": full.fails, "solutions": full.solutions,
              "sol_hash_sum": full.hash_sum, "sol_hash_xor": full.hash_xor}
    for r in (0, 1):
        assert out[r]["combined"] == expect


def test_rank_failure_is_reported_not_hung():
    out, codes = _run(2, 6, fail_rank=1)
    assert codes[1] == 3
    assert "error" in out[0], out            # the surviving rank's exchange fails, it does not hang


def test_units_and_partition_cover_everything():
    from paper_1909_09213_gb300 import shard
    for world in (1, 2, 3, 8):
        got = sorted(u for r in range(world) for u in shard.units_of(r, world, 37))
        assert got == list(range(37))
    with pytest.raises(ValueError):
        shard.partition(2, 2)


# ----------------------------------------------------------------------------- depth-k split

def _oracle_tools(m):
    """The library's layout and root domains (host-only calls) and a propagate function with
    the oracle's fixpoint standing in for the device's (same (count, n*W) bitset layout)."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    from _util import bits_to_flags, flags_to_bits
    from oracle import oracle as O
    from paper_1909_09213_gb300 import cubics as K
    p = K.Csp(m)
    n, W, lo0 = p.layout()
    om = O.OracleModel(m)

    def propagate(states):
        out, failed = [], []
        for s in states:
            f, d = O.propagate(om, bits_to_flags(om, s, n, W, lo0), variant=1)
            failed.append(f)
            out.append(flags_to_bits(om, d, n, W, lo0) if not f else s)
        return np.array(out, dtype=np.uint32), np.array(failed)

    def solve_unit(u, mode=0):
        return O.solve(om, mode=mode, cap=1, variant=1, dom=bits_to_flags(om, u, n, W, lo0))

    return p, n, W, om, propagate, solve_unit


def _share(m, depth, part, nparts):
    from paper_1909_09213_gb300 import shard
    p, n, W, om, propagate, solve_unit = _oracle_tools(m)
    units, nodes, fails = shard.split_units(propagate, p.root_domains().ravel(), n, W, depth)
    st = {"nodes": nodes if part == 0 else 0, "fails": fails if part == 0 else 0,
          "solutions": 0, "sol_hash_sum": 0, "sol_hash_xor": 0}
    for u in units[part::nparts]:
        r = solve_unit(u)
        st = shard.combine([st, {"nodes": r.nodes, "fails": r.fails, "solutions": r.solutions,
                                 "sol_hash_sum": r.hash_sum, "sol_hash_xor": r.hash_xor}])
    return st, len(units)


def _tiny_mixed():
    from paper_1909_09213_gb300 import instances as I
    return I.random_tiny(I.seed_for(I.CFG_TINY, 70003))


@pytest.mark.parametrize("depth", [1, 2, 3, 5])
def test_depth_k_split_sums_to_the_whole_search(depth):
    """Every rank count and depth: the ranks' shares of a tree cut at depth k combine to the
    undivided search (nodes, fails, solutions, both hashes)."""
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    from paper_1909_09213_gb300 import shard
    for m in (I.queens(8), I.worked_example("lin", "table"), _tiny_mixed()):
        full = O.solve(O.OracleModel(m), variant=1)
        want = {"nodes": full.nodes, "fails": full.fails, "solutions": full.solutions,
                "sol_hash_sum": full.hash_sum, "sol_hash_xor": full.hash_xor}
        for nparts in (1, 2, 3, 8):
            parts = [_share(m, depth, r, nparts)[0] for r in range(nparts)]
            assert shard.combine(parts) == want, (m.name, depth, nparts)
    # 8-queens at depth 3: the units are the consistent placements of the first three queens
    _, count = _share(I.queens(8), 3, 0, 1)
    assert count > 100


def _split_worker(rank, world, port, outdir, depth):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    from paper_1909_09213_gb300 import instances as I
    from paper_1909_09213_gb300 import shard
    st, _ = _share(I.queens(9), depth, rank, world)
    res = {"combined": shard.combine_across_ranks(st)}
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_three_ranks_share_a_tree_cut_at_depth_3():
    from oracle import oracle as O
    from paper_1909_09213_gb300 import instances as I
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_split_worker, args=(r, 3, port, d, 3)) for r in range(3)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert not p.is_alive() and p.exitcode == 0
        out = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(3)]
    full = O.solve(O.OracleModel(I.queens(9)), variant=1)
    for o in out:
        assert o["combined"] == {"nodes": full.nodes, "fails": full.fails,
                                 "solutions": full.solutions, "sol_hash_sum": full.hash_sum,
                                 "sol_hash_xor": full.hash_xor}


def _first_worker(rank, world, port, outdir, which):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    from paper_1909_09213_gb300 import instances as I
    from paper_1909_09213_gb300 import shard
    m = I.queens(10) if which == "sat" else I.queens(3)
    p, n, W, om, propagate, solve_unit = _oracle_tools(m)
    units, _, _ = shard.split_units(propagate, p.root_domains().ravel(), n, W, 3)

    def solve_chunk(piece):
        nodes = 0
        for u in piece:
            r = solve_unit(u, mode=1)
            nodes += r.nodes
            st = {"nodes": nodes, "fails": 0, "solutions": 0, "sol_hash_sum": 0, "sol_hash_xor": 0}
            if r.status == 1:
                return True, [int(v) for v in r.sols[0]], st
        return False, None, {"nodes": nodes, "fails": 0, "solutions": 0, "sol_hash_sum": 0,
                             "sol_hash_xor": 0}

    found, sol, st, ran = shard.first_over_ranks(units, rank, world, solve_chunk,
                                                 shard.any_rank, chunk=4)
    from oracle import oracle as O
    res = {"found": found, "sol": sol, "ran": ran, "units": len(units),
           "valid": bool(sol is None or O.check_solution(om, sol))}
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("which", ["sat", "unsat"])
def test_first_solution_stops_every_rank(which):
    """FIRST mode over a shared tree: the ranks OR a found flag after each chunk of units,
    so every rank stops after the same chunk once one has a solution (10-queens, SAT); when
    there is none (3-queens, UNSAT) every unit is searched and no rank reports one."""
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_first_worker, args=(r, 2, port, d, which)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert not p.is_alive() and p.exitcode == 0
        out = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(2)]
    assert all(o["valid"] for o in out)
    if which == "sat":
        assert all(o["found"] for o in out)
        assert any(o["sol"] is not None for o in out)
        # the first chunk already holds solutions: nobody searched its whole share
        assert all(o["ran"] <= 1 for o in out) and out[0]["units"] > 8
    else:
        assert not any(o["found"] for o in out)
