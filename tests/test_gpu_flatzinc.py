"""GPU: problems read by the FlatZinc front end, searched by the library, against the oracle
(solution count, solution-set hash, node and fail counts)."""
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import flatzinc as F
from paper_1909_09213_gb300 import instances as I

from test_flatzinc import WORKED, queens_fzn

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _parity(model):
    r = O.solve(O.OracleModel(model), variant=1)
    rc, st, _ = K.Csp(model).solve(K.CSP_ALL, 0)
    assert rc == 0
    assert st["solutions"] == r.solutions
    assert (st["sol_hash_sum"], st["sol_hash_xor"]) == (r.hash_sum, r.hash_xor)
    assert (st["nodes"], st["fails"]) == (r.nodes, r.fails)
    return st


@pytest.mark.parametrize("N,want", [(6, 4), (8, 92), (10, 724)])
def test_flat_queens(N, want):
    assert _parity(F.parse(queens_fzn(N)).model)["solutions"] == want


def test_flat_worked_example():
    assert _parity(F.parse(WORKED).model)["solutions"] == 11


def test_written_models_search_like_their_sources():
    for k in range(30):
        m = I.random_tiny(I.seed_for(I.CFG_TINY, 93000 + k))
        _parity(F.parse(F.write(m)).model)
