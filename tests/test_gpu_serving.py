"""Serving loop (continuous batching) through the C ABI.

* each result is the same alone (dpgmg_setup + dpgmg_solve on an idle device)
  and in the mix (submitted together with requests of other meshes, orders
  and frequencies that run concurrently on the device);
* admission by device memory: a request whose footprint exceeds the serving
  budget is refused with NOMEM at submission, requests that fit only a few at
  a time all complete;
* latency (completion - submission) is reported per request.
"""
import time

import numpy as np
import pytest

from paper_2304_01728_gb300 import dpgmg as D

pytestmark = pytest.mark.gpu

MIX = [
    (dict(n=(4, 4, 4), p=2, omega=5.0, src_center=(0.4, 0.5, 0.6), src_width=0.15), dict(n_levels=3, p_min=1)),
    (dict(n=(4, 4, 4), p=3, omega=9.0, src_center=(0.5, 0.5, 0.5), src_width=0.1), dict(n_levels=3, p_min=2)),
    (dict(n=(3, 5, 4), p=2, omega=3.0, x1=(1.0, 1.5, 1.2), src_center=(0.5, 0.7, 0.6), src_width=0.2,
          wavespeed=np.linspace(0.5, 1.5, 60)), dict(n_levels=2, p_min=1)),
    (dict(n=(6, 6, 6), p=2, omega=12.0, src_center=(0.3, 0.3, 0.6), src_width=0.1), dict(n_levels=3, p_min=2)),
    (dict(n=(4, 4, 4), p=2, omega=6.0, source="plane_wave", wave_dir=(1.0, 1.0, 0.5)), dict(n_levels=2, p_min=1)),
]


def _alone(pk, ok):
    with D.Solver(pk, **ok) as s:
        x, f, st, code = s.solve()
    assert code == D.DPGMG_OK
    return x, f, st.iters


def _wait(h, ticket, n_trace, n_field, timeout=120.0):
    x = np.zeros(n_trace, dtype=np.complex128)
    f = np.zeros(n_field, dtype=np.complex128)
    t0 = time.time()
    while True:
        code, st, lat = D.dpgmg_poll(h, ticket, x, f)
        if code != D.DPGMG_ERR_PENDING:
            return code, x, f, st, lat
        assert time.time() - t0 < timeout
        time.sleep(0.002)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-7)])
def test_same_alone_and_in_the_mix(precision, tol):
    ref = [_alone(pk, dict(ok, precision=precision)) for pk, ok in MIX]
    h = D.dpgmg_create(0)
    try:
        D.dpgmg_serve_start(h, 3)
        keep, tickets = [], []
        for pk, ok in MIX * 2:                      # every request twice, all in flight together
            pb, k = D.make_problem(**pk)
            op = D.make_opts(**dict(ok, precision=precision))
            keep.append((pb, op, k))
            nt, nf, _ = D.dpgmg_query_sizes(pb, op)
            tickets.append((D.dpgmg_submit(h, pb, op), nt, nf))
        lats = []
        for i, (t, nt, nf) in enumerate(tickets):
            code, x, f, st, lat = _wait(h, t, nt, nf)
            assert code == D.DPGMG_OK, (i, code, D.lib().dpgmg_last_error().decode())
            xr, fr, it = ref[i % len(MIX)]
            assert st.iters == it
            assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < tol
            assert np.linalg.norm(f - fr) / np.linalg.norm(fr) < tol
            assert lat > 0
            lats.append(lat)
        assert np.percentile(lats, 99) >= np.percentile(lats, 50) > 0
    finally:
        D.dpgmg_destroy(h)


def test_admission_by_memory():
    pk, ok = MIX[3]
    pb, keep = D.make_problem(**pk)
    op = D.make_opts(**ok)
    _, _, est = D.dpgmg_query_sizes(pb, op)
    # a serving budget that holds two such requests at a time
    h = D.dpgmg_create(0, mem_budget_bytes=int(2.5 * est))
    try:
        D.dpgmg_serve_start(h, 4)
        nt, nf, _ = D.dpgmg_query_sizes(pb, op)
        tickets = [D.dpgmg_submit(h, pb, op) for _ in range(6)]
        for t in tickets:
            code, x, f, st, lat = _wait(h, t, nt, nf)
            assert code == D.DPGMG_OK, (code, D.lib().dpgmg_last_error().decode())
            assert 0 < st.dev_bytes_peak <= est          # the admission estimate bounds the footprint
        big, keep2 = D.make_problem(n=(24, 24, 24), p=4, omega=20.0)
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_submit(h, big, op)
        assert e.value.code == D.DPGMG_ERR_NOMEM
        assert D.dpgmg_poll(h, tickets[0])[0] == D.DPGMG_ERR_ARG   # collected tickets are forgotten
    finally:
        D.dpgmg_destroy(h)


def test_one_ledger_for_setup_and_serving():
    """Systems set up with dpgmg_setup and running requests share the
    handle's memory budget: a request that fits the budget on its own waits
    while a set-up system holds memory, and runs once the system is released."""
    pk, ok = MIX[3]
    pb, keep = D.make_problem(**pk)
    op = D.make_opts(**ok)
    nt, nf, est = D.dpgmg_query_sizes(pb, op)
    h = D.dpgmg_create(0, mem_budget_bytes=est + (1 << 20))
    try:
        s = D.dpgmg_setup(h, pb, op)
        D.dpgmg_serve_start(h, 2)
        t = D.dpgmg_submit(h, pb, op)
        time.sleep(1.0)
        assert D.dpgmg_poll(h, t)[0] == D.DPGMG_ERR_PENDING   # held back by the set-up system
        D.dpgmg_release(h, s)
        code, x, f, st, lat = _wait(h, t, nt, nf)
        assert code == D.DPGMG_OK, D.lib().dpgmg_last_error().decode()
        s = D.dpgmg_setup(h, pb, op)                           # the budget is free again
        D.dpgmg_release(h, s)
    finally:
        D.dpgmg_destroy(h)
