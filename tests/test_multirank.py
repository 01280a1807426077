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
