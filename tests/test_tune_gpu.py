"""The autotuner on the device: it times its candidates, records the winner,
and the factorizations that leave their options at zero follow the table (the
launch trace shows the outer panel width in use); results stay those of the
oracle."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import EPS64, dev

pytestmark = pytest.mark.gpu


@pytest.fixture()
def clean_table():
    import paper_1611_06365_gb300 as lu
    lu.lu_tune_clear()
    yield
    lu.lu_tune_clear()


def _panels_traced(fn):
    import torch

    import paper_1611_06365_gb300 as lu
    lu.lu_trace(True)
    fn()
    torch.cuda.synchronize()
    ev = lu.lu_trace_read()
    lu.lu_trace(False)
    return sum(1 for e in ev if e["kind"] == "panel")


def _factor(A0, **kw):
    import torch

    import paper_1611_06365_gb300 as lu
    n = A0.shape[0]
    A = A0.clone()
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev())
    info = torch.zeros(1, dtype=torch.int32, device=dev())
    lu.lu_factor(A, ipiv, info, n, **kw)
    return A, ipiv, info


def test_table_entry_sets_panel_width(clean_table):
    """An entry for order 700 with b_o = 16 doubles the panels of the default
    plan (b_o = 32); an entry for another order changes nothing."""
    import torch

    import paper_1611_06365_gb300 as lu
    n = 700
    A0 = li.uniform_colmajor_torch(n, n, 4100, dev(), torch.float64)
    base = _panels_traced(lambda: _factor(A0))
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 701, nb=16)
    assert _panels_traced(lambda: _factor(A0)) == base
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, n, nb=16)
    tuned = _panels_traced(lambda: _factor(A0))
    assert tuned == (n + 15) // 16 and base == (n + 31) // 32
    # an explicit option wins over the table
    assert _panels_traced(lambda: _factor(A0, nb=32)) == base


@pytest.mark.parametrize("dtype,update,n", [("f64", 0, 1024), ("f32", 0, 2048), ("f32", 2, 2048), ("f32", 3, 1536)])
def test_autotune_records_the_winner(oracle_mod, clean_table, dtype, update, n):
    import torch

    import paper_1611_06365_gb300 as lu
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    r = lu.lu_autotune(code, n, update=update)
    assert r["candidates"] >= 4 and r["ms"] > 0.0 and r["opts"]["nb"] > 0
    got = lu.lu_tune_get(lu.TUNE_FACTOR, code, n, update=update)
    assert got == r["opts"]
    # the default call now runs the winner: same bits as the explicit options
    tdt = torch.float64 if dtype == "f64" else torch.float32
    A0 = li.uniform_colmajor_torch(n, n, 4200 + n, dev(), torch.float64).to(tdt)
    Ad, pd, infod = _factor(A0, update=update)
    o = r["opts"]
    Ae, pe, infoe = _factor(A0, nb=o["nb"], nb_inner=o["nb_inner"], panel_ctas=o["panel_ctas"],
                            lookahead=o["lookahead"], update=update, update_ctas=o["update_ctas"])
    torch.cuda.synchronize()
    assert int(infod.item()) == 0 and torch.equal(pd, pe) and torch.equal(Ad.view(torch.uint8), Ae.view(torch.uint8))
    if dtype == "f64":
        A_f = A0.cpu().numpy().T
        LUo, pivo, _ = oracle_mod.getrf(np.asfortranarray(A_f))
        assert np.array_equal(pd.cpu().numpy(), pivo)
        r_, a_ = oracle_mod.lu_residual_fro(A_f, Ad.cpu().numpy().T, pd.cpu().numpy())
        assert r_ / a_ <= 10 * n * EPS64


def test_autotune_budget_stops_early(clean_table):
    import paper_1611_06365_gb300 as lu
    r = lu.lu_autotune(lu.LU_F64, 512, budget_ms=1e-6)
    assert r["candidates"] == 1


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_autotune_batched(clean_table, dtype):
    import torch

    import paper_1611_06365_gb300 as lu
    sizes = li.batch_sizes(400, 16, 256, seed=li.BASE_SEED + 4300)
    ns = torch.tensor(sizes, dtype=torch.int32, device=dev())
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    r = lu.lu_autotune_batched(code, ns, 256)
    assert r["candidates"] == 3 and r["opts"]["nb"] in (1, 16, 32) and r["ms"] > 0
    assert lu.lu_tune_get(lu.TUNE_BATCHED, code, 256)["nb"] == r["opts"]["nb"]
    # orders above 256 have only the unblocked kernel
    r2 = lu.lu_autotune_batched(code, torch.tensor([300, 17], dtype=torch.int32, device=dev()), 300)
    assert r2["candidates"] == 1 and r2["opts"]["nb"] == 1


@pytest.mark.parametrize("update", [1, 2, 3])
def test_update_grid_cap_keeps_bits(update):
    """Capping the remainder update's persistent grid (the SM split between panel
    and update) changes which CTA computes a tile, not its arithmetic."""
    import torch

    n = 1536
    A0 = li.uniform_colmajor_torch(n, n, 4400 + update, dev(), torch.float32)
    ref = _factor(A0, nb=64, update=update)
    for cap in (1, 37, 96):
        got = _factor(A0, nb=64, update=update, update_ctas=cap)
        torch.cuda.synchronize()
        assert torch.equal(got[1], ref[1]) and torch.equal(got[0].view(torch.uint8), ref[0].view(torch.uint8)), cap
