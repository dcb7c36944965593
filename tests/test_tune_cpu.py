"""The autotuner's table (host logic, no GPU): entries are validated, stored
under (kind, dtype, update, order), written and read back as text, and a file
with any malformed or out-of-range line is refused whole."""
import ctypes

import pytest

import paper_1611_06365_gb300 as lu


@pytest.fixture()
def L():
    lu.build()
    L = lu.lib()
    lu.lu_tune_clear()
    yield L
    lu.lu_tune_clear()


def test_put_get_clear(L):
    assert lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 4096) is None
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 4096, nb=16, panel_ctas=8, ms=12.5)
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F32, 4096, nb=128, update=lu.LU_UPDATE_BF16X3, ms=3.0)
    lu.lu_tune_put(lu.TUNE_BATCHED, lu.LU_F32, 256, nb=32, ms=5.0)
    assert lu.lu_tune_count() == 3
    got = lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 4096)
    assert got == {"nb": 16, "nb_inner": 0, "panel_ctas": 8, "lookahead": 0, "update": 0, "update_ctas": 0, "sm_share": 0,
                   "tile": 0, "early_term": 0}
    # the key includes the update kind and the exact order
    assert lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F32, 4096) is None
    assert lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F32, 4096, update=lu.LU_UPDATE_BF16X3)["nb"] == 128
    assert lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 4095) is None
    assert lu.lu_tune_get(lu.TUNE_BATCHED, lu.LU_F32, 256)["nb"] == 32
    # a second put replaces the entry
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 4096, nb=64, ms=11.0)
    assert lu.lu_tune_count() == 3 and lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 4096)["nb"] == 64
    lu.lu_tune_clear()
    assert lu.lu_tune_count() == 0


@pytest.mark.parametrize("kind,dt,n,kw,code", [
    (2, 0, 64, {}, -1),                                           # unknown kind
    (0, 5, 64, {}, -2),                                           # unknown dtype
    (0, 0, 64, {"update": 1}, -3),                                # tensor-core update on FP64
    (0, 0, -1, {}, -4),                                           # negative order
    (0, 0, 64, {"panel_ctas": 17}, -5),                           # team larger than a cluster
    (0, 0, 64, {"lookahead": 5}, -5),                             # deeper than the deepest look-ahead (4)
    (0, 1, 64, {"update": 4}, -3),                                # emulated FP64 update on FP32
    (1, 1, 64, {"nb": 8}, -5),                                    # batched widths are 1, 16, 32
])
def test_put_rejects(L, kind, dt, n, kw, code):
    with pytest.raises(lu.LuError) as e:
        lu.lu_tune_put(kind, dt, n, **kw)
    assert e.value.code == code
    assert lu.lu_tune_count() == 0


def test_save_load_round_trip(L, tmp_path):
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 16384, nb=32, panel_ctas=16, lookahead=1, ms=2650.25)
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F32, 8192, nb=64, update=lu.LU_UPDATE_FP8, update_ctas=120, ms=40.0)
    lu.lu_tune_put(lu.TUNE_BATCHED, lu.LU_F64, 256, nb=16, ms=41.5)
    p = tmp_path / "tune.txt"
    assert lu.lu_tune_save(p) == 3
    text = p.read_text().splitlines()
    assert text[0].startswith("#") and len([t for t in text if not t.startswith("#")]) == 3
    before = {k: lu.lu_tune_get(*k[:3], update=k[3]) for k in
              [(0, 0, 16384, 0), (0, 1, 8192, 3), (1, 0, 256, 0)]}
    lu.lu_tune_clear()
    assert lu.lu_tune_load(p) == 3
    after = {k: lu.lu_tune_get(*k[:3], update=k[3]) for k in before}
    assert after == before and None not in after.values()


def test_load_accepts_both_table_versions(L, tmp_path):
    """A v1 line (no tile field) loads with tile 0; a v2 line keeps its tile shape."""
    p = tmp_path / "mixed.txt"
    p.write_text("# v1 and v2 lines\n0 0 0 1024 16 0 16 1 0 5.0\n0 0 4 2048 64 0 8 1 0 2 7.5\n")
    assert lu.lu_tune_load(p) == 2
    assert lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 1024)["tile"] == 0
    got = lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 2048, update=lu.LU_UPDATE_F64EMU)
    assert got["tile"] == 2 and got["nb"] == 64
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 4096, nb=32, tile=1, ms=1.0)
    q = tmp_path / "again.txt"
    lu.lu_tune_save(q)
    lu.lu_tune_clear()
    assert lu.lu_tune_load(q) == 3 and lu.lu_tune_get(lu.TUNE_FACTOR, lu.LU_F64, 4096)["tile"] == 1


@pytest.mark.parametrize("line", [
    "0 0 0 512 32 0 16 1 0",               # a field missing
    "0 0 0 512 32 0 16 1 0 2.0 extra",     # a field too many
    "0 0 1 512 32 0 16 1 0 2.0",           # BF16 update on FP64
    "1 1 0 256 24 0 0 0 0 1.0",            # batched width 24
    "0 0 0 512 32 0 99 1 0 2.0",           # panel team 99
    "0 1 1 512 64 0 16 1 -3 2.0",          # negative update grid
    "zero 0 0 512 32 0 16 1 0 2.0",
    "0 0 0 512 32 0 16 1 0 3 2.0",         # tile shape 3
    "0 0 0 512 32 0 16 1 0 1 2.0 extra",   # a field too many (v2)
])
def test_load_refuses_whole_file(L, tmp_path, line):
    p = tmp_path / "bad.txt"
    p.write_text("# header\n0 0 0 1024 16 0 16 1 0 5.0\n" + line + "\n")
    with pytest.raises(lu.LuError) as e:
        lu.lu_tune_load(p)
    assert e.value.code == -2
    assert lu.lu_tune_count() == 0


def test_load_missing_file(L, tmp_path):
    with pytest.raises(lu.LuError) as e:
        lu.lu_tune_load(tmp_path / "absent.txt")
    assert e.value.code == -1


def test_autotune_argument_errors(L):
    """Argument errors return before any CUDA call."""
    r = lu.TuneResult()
    dummy = ctypes.c_void_p(16)
    assert L.lu_autotune(7, 64, 0, 0.0, ctypes.byref(r), None) == -1
    assert L.lu_autotune(0, 0, 0, 0.0, ctypes.byref(r), None) == -2
    assert L.lu_autotune(0, 64, lu.LU_UPDATE_BF16, 0.0, ctypes.byref(r), None) == -3
    assert L.lu_autotune(1, 64, 9, 0.0, ctypes.byref(r), None) == -3
    assert L.lu_autotune(1, 64, 0, 0.0, None, None) == -5
    assert L.lu_autotune_batched(0, 0, dummy, 64, ctypes.byref(r), None) == -2
    assert L.lu_autotune_batched(0, 4, None, 64, ctypes.byref(r), None) == -3
    assert L.lu_autotune_batched(0, 4, dummy, 2000, ctypes.byref(r), None) == -4
    assert L.lu_autotune_batched(0, 4, dummy, 64, None, None) == -5


def test_plan_info_follows_table(L):
    rc, p = lu.lu_plan_info(lu.LU_F64, 4096)
    assert rc == 0 and p["nb"] == 32 and p["lookahead"] == 1 and p["panel_ctas"] == 8
    assert lu.lu_plan_info(lu.LU_F64, 16384)[1]["nb"] == 64
    lu.lu_tune_put(lu.TUNE_FACTOR, lu.LU_F64, 4096, nb=64, panel_ctas=4)
    rc, p = lu.lu_plan_info(lu.LU_F64, 4096)
    assert rc == 0 and p["nb"] == 64 and p["panel_ctas"] == 4
    rc, p = lu.lu_plan_info(lu.LU_F64, 4096, nb=16)          # explicit fields win
    assert rc == 0 and p["nb"] == 16 and p["panel_ctas"] == 4
    rc, p = lu.lu_plan_info(lu.LU_F64, 4097)
    assert p["nb"] == 32


def test_plan_info_worker_sharing_option(L):
    """sm_share: on unless -1; values outside -1..1 are refused like other bad options."""
    assert lu.lu_plan_info(lu.LU_F32, 4096, update=lu.LU_UPDATE_BF16)[1]["sm_share"] == 1
    assert lu.lu_plan_info(lu.LU_F32, 4096, update=lu.LU_UPDATE_BF16, sm_share=1)[1]["sm_share"] == 1
    assert lu.lu_plan_info(lu.LU_F64, 4096, update=lu.LU_UPDATE_F64EMU, sm_share=-1)[1]["sm_share"] == -1
    for bad in (-2, 2):
        with pytest.raises(lu.LuError):
            lu.lu_plan_info(lu.LU_F64, 4096, sm_share=bad)
    assert lu.lu_plan_info(lu.LU_F64, 4096, tile=2)[1]["tile"] == 2
    for bad in (-1, 3):
        with pytest.raises(lu.LuError):
            lu.lu_plan_info(lu.LU_F64, 4096, tile=bad)


def test_plan_info_early_termination_option(L):
    """early_term: 0..2, only with look-ahead of depth 1; the plan reports it, and
    the fit check then covers panels starting at any column."""
    for et in (1, 2):
        rc, p = lu.lu_plan_info(lu.LU_F64, 1000, nb=64, nb_inner=16, early_term=et)
        assert rc == 0 and p["early_term"] == et and p["lookahead"] == 1 and p["nb_inner"] == 16
    rc, p = lu.lu_plan_info(lu.LU_F32, 4096, nb=64, nb_inner=16, early_term=1, update=lu.LU_UPDATE_BF16X3)
    assert rc == 0 and p["early_term"] == 1
    assert lu.lu_plan_info(lu.LU_F64, 1000)[1]["early_term"] == 0
    for kw in ({"early_term": -1}, {"early_term": 3}, {"early_term": 1, "lookahead": 2},
               {"early_term": 1, "lookahead": -1}):
        with pytest.raises(lu.LuError):
            lu.lu_plan_info(lu.LU_F64, 1000, **kw)


@pytest.mark.parametrize("dt,update,widths", [
    (0, 0, (0, 16, 32, 64)), (0, 4, (0, 32, 64)), (1, 0, (0, 64, 128, 256)), (1, 1, (0, 64, 128, 256)),
    (1, 2, (0, 64, 128, 256)), (1, 3, (0, 64, 128, 256)),
])
def test_every_tuner_candidate_fits(L, dt, update, widths):
    """Each plan the autotuner may time, at orders that give ragged last panels
    and panels of at most 512 rows (one CTA), fits a cluster's shared memory."""
    for n in (17, 100, 257, 511, 512, 513, 700, 1000, 1536, 2048, 3001, 4096, 8192, 16384, 32768, 65536):
        for nb in widths:
            if nb > n:
                continue
            for pc in (0, 8, 4):
                for la in (0, -1, 2):
                    rc, p = lu.lu_plan_info(dt, n, nb=nb, panel_ctas=pc, lookahead=la, update=update)
                    assert rc == 0, (dt, update, n, nb, pc, la, p)
                    assert p["nb"] == (nb or p["nb"]) and 1 <= p["nb_inner"] <= p["nb"]


def test_plan_info_reports_a_panel_that_cannot_fit(L):
    """FP64, b_o = 256 at n = 500: the second panel (244 rows, 244 columns) does
    not fit; lu_factor would refuse the plan before launching anything."""
    rc, p = lu.lu_plan_info(lu.LU_F64, 500, nb=256)
    assert rc == lu.LU_ERR_UNSUPPORTED
