"""Serving loop: runs queued from the host finish with results bit-identical to
the same grids stepped alone; the device-memory budget is respected; admission
is first come, first served; cancellation and per-run errors are reported; the
device-built collective initial state equals the host recipe."""
import time

import numpy as np
import pytest

from paper_2203_12866_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

FD, WENO = binding.COSENU_FDKO, binding.COSENU_WENO7
FP64, MIXED = binding.COSENU_FP64, binding.COSENU_MIXED


@pytest.fixture(scope="module", autouse=True)
def _built(oracle):
    from paper_2203_12866_gb300 import build
    build.build()
    binding.load()


def _solo(nz, nv, L, scheme, prec, nsteps, state=None, coll=None, **params):
    with binding.Solver(nz, nv, L, scheme, prec, **params) as s:
        if state is not None:
            s.set_state(state)
        else:
            binding.cosenu_set_state_collective(s.h, **coll)
        s.step(nsteps)
        s.sync()
        return s.state(), s.conserved()


def test_collective_state_matches_host_recipe():
    nz, nv = 300, 48
    with binding.Solver(nz, nv, 30.0, FD, FP64) as s:
        binding.cosenu_set_state_collective(s.h, alpha=0.8, sigma_nu=0.55, sigma_nubar=0.45,
                                            eps0=1e-6, seed=4242)
        got = s.state()
    ref = inputs.collective_state(nz, nv, alpha=0.8, sigma_nu=0.55, sigma_nubar=0.45, eps0=1e-6,
                                  seed=4242)
    # same formulas; exp/cos/sin and the normalising sum may round differently by an ulp or two
    assert np.allclose(got, ref, rtol=4e-15, atol=0.0)
    assert np.array_equal(got[:, 1], ref[:, 1])


def _mix_requests(outs):
    reqs = []
    specs = [(200, 32, FD, MIXED, 7), (64, 16, WENO, FP64, 3), (513, 64, WENO, MIXED, 5),
             (37, 8, FD, FP64, 9), (1000, 32, FD, MIXED, 1), (90, 128, WENO, MIXED, 4),
             (5, 8, FD, MIXED, 6), (300, 64, FD, FP64, 2)]
    for i, (nz, nv, scheme, prec, n) in enumerate(specs):
        params = dict(mu=0.5 + 0.3 * i, omega=0.1 * (i % 2), theta=0.2)
        out = np.empty((2, 4, nz, nv))
        outs.append(out)
        if i % 2 == 0:
            st = inputs.random_state(nz, nv, seed=700 + i, offdiag=0.05)
            r = binding.make_request(nz, nv, 0.2 * nz, scheme, prec, nsteps=n, state=st,
                                     out_state=out, **params)
            solo = dict(state=st)
        else:
            coll = dict(alpha=0.7 + 0.05 * i, sigma_nu=0.6, sigma_nubar=0.5, eps0=1e-6,
                        seed=800 + i)
            r = binding.make_request(nz, nv, 0.2 * nz, scheme, prec, nsteps=n, out_state=out,
                                     **coll, **params)
            solo = dict(coll=coll)
        reqs.append((r, (nz, nv, 0.2 * nz, scheme, prec, n), solo, params))
    return reqs


@pytest.mark.parametrize("round_steps", [0, 2])
def test_served_runs_bitwise_equal_solo(round_steps):
    outs = []
    reqs = _mix_requests(outs)
    with binding.Server(1 << 30, round_steps=round_steps) as srv:
        tickets = [srv.submit(r) for r, *_ in reqs]
        results = [srv.wait(t, 60.0) for t in tickets]
        st = srv.stats()
    for (r, args, solo, params), out, (rc, res) in zip(reqs, outs, results):
        assert rc == binding.COSENU_OK and res["status"] == binding.COSENU_OK, args
        assert res["steps"] == args[5]
        assert 0 <= res["t_submit"] <= res["t_admit"] <= res["t_done"]
        ref, cons = _solo(*args, **solo, **params)
        assert np.array_equal(out, ref), args
        assert res["conserved"]["tr_nu"] == cons["tr_nu"]
    assert st["finished"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
    assert st["bytes_in_use"] == 0


def test_budget_fifo_and_peak():
    """Runs that do not fit together wait; peak workspace use stays within the budget;
    admission follows submission order."""
    nz, nv = 4096, 64
    ws = binding.cosenu_workspace_bytes(nz, nv, FD, MIXED)
    budget = int(2.5 * ws)  # two runs at a time
    with binding.Server(budget, round_steps=4) as srv:
        tickets = [srv.submit(binding.make_request(nz, nv, 100.0, FD, MIXED, nsteps=8,
                                                   seed=i)) for i in range(6)]
        res = [srv.wait(t, 60.0)[1] for t in tickets]
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["peak_bytes"] <= budget and st["peak_bytes"] == 2 * ws
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)
    # never more than two runs at once (a leaving run's t_done precedes the next admission)
    for t in admits:
        assert sum(1 for r in res if r["t_admit"] <= t < r["t_done"]) <= 2


def test_over_budget_and_invalid_requests_rejected():
    with binding.Server(1 << 20) as srv:
        with pytest.raises(binding.CosenuError) as e:
            srv.submit(binding.make_request(4096, 64, 10.0, FD, MIXED, nsteps=1))
        assert e.value.code == binding.COSENU_ENOMEM
        with pytest.raises(binding.CosenuError):
            srv.submit(binding.make_request(16, 6, 10.0, FD, MIXED, nsteps=1))  # nv % 4
        with pytest.raises(binding.CosenuError):
            srv.submit(binding.make_request(16, 8, 10.0, FD, MIXED, nsteps=-1))
        with pytest.raises(binding.CosenuError):
            srv.poll(12345)


def test_cancel_and_max_running():
    with binding.Server(1 << 30, max_running=1, round_steps=1) as srv:
        t0 = srv.submit(binding.make_request(2048, 64, 50.0, WENO, MIXED, nsteps=10 ** 5))
        t1 = srv.submit(binding.make_request(64, 16, 10.0, FD, MIXED, nsteps=3))
        t2 = srv.submit(binding.make_request(64, 16, 10.0, FD, MIXED, nsteps=3))
        srv.cancel(t1)  # queued behind t0 (one run at a time)
        time.sleep(0.05)
        srv.cancel(t0)  # running: leaves at the end of its round
        r0 = srv.wait(t0, 60.0)[1]
        r1 = srv.wait(t1, 60.0)[1]
        r2 = srv.wait(t2, 60.0)[1]
    assert r0["status"] == binding.COSENU_ECANCELLED and r0["steps"] < 10 ** 5
    assert r1["status"] == binding.COSENU_ECANCELLED and r1["steps"] == 0
    assert r2["status"] == binding.COSENU_OK and r2["steps"] == 3


def test_nonfinite_run_reported_alone():
    bad = inputs.random_state(64, 16, seed=1, offdiag=0.05)
    bad[0, 2, 10, 3] = np.nan
    good = inputs.random_state(64, 16, seed=2, offdiag=0.05)
    out = np.empty_like(good)
    with binding.Server(1 << 30) as srv:
        tb = srv.submit(binding.make_request(64, 16, 10.0, FD, FP64, nsteps=4, state=bad))
        tg = srv.submit(binding.make_request(64, 16, 10.0, FD, FP64, nsteps=4, state=good,
                                             out_state=out))
        rb = srv.wait(tb, 60.0)[1]
        rg = srv.wait(tg, 60.0)[1]
    assert rb["status"] == binding.COSENU_ENONFINITE
    assert rg["status"] == binding.COSENU_OK
    ref, _ = _solo(64, 16, 10.0, FD, FP64, 4, state=good)
    assert np.array_equal(out, ref)


def test_poll_pending_then_done_and_destroy_cancels():
    srv = binding.Server(1 << 30, round_steps=1)
    t = srv.submit(binding.make_request(256, 32, 20.0, FD, MIXED, nsteps=50))
    rc, res = srv.poll(t)
    assert rc in (binding.COSENU_PENDING, binding.COSENU_OK)
    rc, res = srv.wait(t, 60.0)
    assert rc == binding.COSENU_OK and res["steps"] == 50
    with pytest.raises(binding.CosenuError):
        srv.poll(t)  # collected already
    srv.submit(binding.make_request(256, 32, 20.0, FD, MIXED, nsteps=10 ** 6))
    srv.close()  # cancels the unfinished run and returns


def _rel_by_component(got, ref):
    worst = 0.0
    for s in range(2):
        for c in range(4):
            scale = float(np.max(np.abs(ref[s, c])))
            if scale > 0.0:
                worst = max(worst, float(np.max(np.abs(got[s, c] - ref[s, c]))) / scale)
    return worst


def test_served_runs_match_oracle(oracle):
    """Twelve runs served together -- each scheme in each precision, from a (smooth)
    host state and from the device-built collective state -- against the FP64 oracle
    stepping the same initial state: FP64 runs to 1e-12 (max |delta rho|), mixed
    runs to 1e-5 relative per component, over 6-10 steps (half of the runs have a
    vacuum term, whose off-diagonals reach a few percent).  The runs differ in
    size, nv and parameters, so they share the batch's launches with runs of the
    other precision and scheme."""
    FD3 = binding.COSENU_FDKO3
    runs = []
    i = 0
    for scheme in (FD, WENO, FD3):
        for prec in (FP64, MIXED):
            for host in (True, False):
                nz, nv = 64 + 24 * i, (16, 32, 8)[i % 3]
                L = 0.25 * nz
                n = 6 + (i % 5)
                params = dict(mu=1.0 + 0.1 * i, omega=0.3 * (i % 2), theta=0.2)
                coll = dict(alpha=0.8 + 0.02 * i, sigma_nu=0.6, sigma_nubar=0.5, eps0=1e-6,
                            seed=900 + i)
                u0 = inputs.collective_state(nz, nv, **coll)
                if host:  # a smooth host state that is not the collective recipe's
                    z = np.arange(nz) / nz
                    u0 = u0 * (1.0 + 1e-3 * np.sin(2 * np.pi * (z + 0.1 * i)))[None, None, :, None]
                out = np.empty((2, 4, nz, nv))
                req = binding.make_request(nz, nv, L, scheme, prec, nsteps=n,
                                           state=u0 if host else None, out_state=out,
                                           **({} if host else coll), **params)
                runs.append((req, out, u0, (nz, nv, L, scheme, prec, n, params)))
                i += 1
    with binding.Server(1 << 30, round_steps=4) as srv:
        tickets = [srv.submit(r) for r, *_ in runs]
        results = [srv.wait(t, 60.0)[1] for t in tickets]
    for (req, out, u0, (nz, nv, L, scheme, prec, n, params)), res in zip(runs, results):
        assert res["status"] == binding.COSENU_OK and res["steps"] == n
        p = oracle.params(nz, nv, L, scheme, **params)
        ref = oracle.step(p, u0, n)
        if prec == FP64:
            err = float(np.max(np.abs(out - ref)))
            assert err <= 1e-12, (nz, nv, scheme, prec, err)
        else:
            err = _rel_by_component(out, ref)
            assert err <= 1e-5, (nz, nv, scheme, prec, err)
