"""Per-CTA trace of the factorization kernels (lu_cta_trace): the GPU form of
the paper's execution traces (section 4), and the evidence for worker sharing
(section 4.1): SMs that ran the cluster of panel k+1 later run CTAs of the
remainder update RU2 of step k that take update tiles."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import factor_gpu

pytestmark = pytest.mark.gpu


def _trace(n, dtype, **opts):
    import paper_1611_06365_gb300 as lu
    lu.lu_cta_trace(1 << 21)
    try:
        A = li.uniform(n, n, seed=li.BASE_SEED + 77)
        LU, ipiv, info, _, _ = factor_gpu(A, dtype, **opts)
        made, ev = lu.lu_cta_trace_read(1 << 21)
    finally:
        lu.lu_cta_trace(0)
    assert info == 0 and made == len(ev)
    return ev


def _sharing(ev):
    """Steps k with an RU2(k) CTA that took tiles on an SM a panel(k+1) CTA had
    left, starting after that panel CTA ended."""
    panels = {}
    for e in ev:
        if e["kind"] == "panel":
            panels.setdefault(e["step"], []).append(e)
    steps = set()
    for e in ev:
        if e["kind"] != "ru2" or e["tiles"] < 1:
            continue
        for p in panels.get(e["step"] + 1, []):
            if p["smid"] == e["smid"] and e["t0"] >= p["t1"]:
                steps.add(e["step"])
    return steps


def _timeline(ev, steps):
    """Per early step: panel(k+1) interval, RU2(k) first start / last end (us from
    the first record), and how many RU2(k) CTAs started after the panel ended."""
    t00 = min(e["t0"] for e in ev)
    out = []
    for k in range(steps):
        p = [e for e in ev if e["kind"] == "panel" and e["step"] == k + 1]
        r = [e for e in ev if e["kind"] == "ru2" and e["step"] == k]
        if not p or not r:
            continue
        pend = max(e["t1"] for e in p)
        late = [e for e in r if e["t0"] >= pend]
        out.append((k, (min(e["t0"] for e in p) - t00) / 1e3, (pend - t00) / 1e3,
                    (min(e["t0"] for e in r) - t00) / 1e3, (max(e["t1"] for e in r) - t00) / 1e3,
                    len(r), len(late), sum(e["tiles"] for e in late)))
    return out


def _well_formed(ev, nsteps):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert all(e["t1"] >= e["t0"] and 0 <= e["smid"] < sms for e in ev)
    kinds = {e["kind"] for e in ev}
    assert {"panel", "ru1", "ru2", "pf1", "pf2"} <= kinds
    assert sorted({e["step"] for e in ev if e["kind"] == "panel"}) == list(range(nsteps))


@pytest.mark.parametrize("dtype,update,n,nb", [("f64", 0, 4096, 64), ("f32", 2, 16384, 64), ("f64", 4, 16384, 64)])
def test_panel_sms_join_the_remainder_update(dtype, update, n, nb):
    """Worker sharing needs a remainder update that outlasts the panel: the early
    steps of these orders (RU2 of step k is the larger task there; with the
    emulated FP64 update that takes n = 16384, as an 8192-row FP64 panel on 8
    SMs runs about as long as the update of step 0).  The DFMA
    update is a grid of short CTAs the hardware hands to freed SMs; the
    persistent tensor-core updates give a panel placement's SMs back on request
    and take them again with a joining grid (SmShare)."""
    ev = _trace(n, dtype, nb=nb, update=update)
    _well_formed(ev, (n + nb - 1) // nb)
    shared = _sharing(ev)
    assert len(shared) >= 1, ("no step shows a panel SM taking update tiles afterwards", _timeline(ev, 4))


@pytest.mark.parametrize("dtype,update,n,nb", [("f32", 2, 16384, 64), ("f64", 4, 8192, 64)])
def test_panel_overlaps_persistent_update(dtype, update, n, nb):
    """With worker sharing the panel k+1 cluster runs while RU2(k) is still
    working in most early steps, instead of waiting for the persistent grid to
    drain; with sm_share = -1 the trace still records every task (the flag
    changes the schedule, not the work)."""
    ev = _trace(n, dtype, nb=nb, update=update)
    tl = _timeline(ev, 8)
    overlapped = [r for r in tl if r[1] < r[4]]        # panel(k+1) started before RU2(k) ended
    assert len(overlapped) >= len(tl) // 2, tl
    off = _trace(n, dtype, nb=nb, update=update, sm_share=-1)
    for e in (ev, off):
        assert sum(x["tiles"] for x in e if x["kind"] == "ru2" and x["step"] == 0) > 0


def test_trace_off_records_nothing():
    import paper_1611_06365_gb300 as lu
    A = li.uniform(300, 300, seed=3)
    factor_gpu(A, "f64")
    lu.lu_cta_trace(1024)
    made, ev = lu.lu_cta_trace_read(1024)
    lu.lu_cta_trace(0)
    assert made == 0 and ev == []
