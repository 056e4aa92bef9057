"""Batched solver: every member's result is bit-identical to the same grid
stepped alone, whatever else is in the batch, whatever launch shape the tuner
picks, and across membership changes; members also match the FP64 oracle like
single grids do.  Error flags are reported per member."""
import numpy as np
import pytest

from paper_2203_12866_gb300 import binding, inputs
from parity_util import max_abs, run_oracle

pytestmark = pytest.mark.gpu

FD, WENO, FD3 = binding.COSENU_FDKO, binding.COSENU_WENO7, binding.COSENU_FDKO3
FP64, MIXED = binding.COSENU_FP64, binding.COSENU_MIXED


@pytest.fixture(scope="module", autouse=True)
def _built(oracle):
    from paper_2203_12866_gb300 import build
    build.build()
    binding.load()


def _mix():
    """Uneven grids over both schemes, both precisions and several nv, with
    different parameters each; sizes span several CTAs, ragged tails, and
    grids shorter than the stencil."""
    specs = []
    for i, (nz, nv, scheme, prec) in enumerate([
            (37, 8, FD, FP64), (200, 32, FD, MIXED), (513, 32, FD, MIXED),
            (64, 32, WENO, MIXED), (1031, 64, WENO, MIXED), (3, 8, FD, MIXED),
            (96, 64, FD, FP64), (250, 32, WENO, FP64), (5, 8, WENO, MIXED),
            (777, 32, FD, MIXED), (2048, 128, FD, MIXED), (131, 128, WENO, MIXED),
            (300, 32, FD3, MIXED), (70, 16, FD3, FP64), (4, 8, FD3, MIXED)]):
        params = dict(mu=0.5 + 0.25 * i, omega=0.1 * (i % 3), theta=0.05 * i, ko_eps=0.1)
        params["lambda"] = 0.02 * (i % 2)
        u0 = inputs.random_state(nz, nv, seed=500 + i, offdiag=0.05)
        specs.append(dict(nz=nz, nv=nv, L=0.15 * nz, scheme=scheme, prec=prec, params=params,
                          u0=u0))
    return specs


def _alone(sp, nsteps):
    with binding.Solver(sp["nz"], sp["nv"], sp["L"], sp["scheme"], sp["prec"],
                        **sp["params"]) as s:
        s.set_state(sp["u0"])
        s.step(nsteps)
        s.sync()
        return s.state()


def _batch(specs):
    b = binding.Batch()
    ms = []
    for sp in specs:
        m = b.add(sp["nz"], sp["nv"], sp["L"], sp["scheme"], sp["prec"], **sp["params"])
        m.set_state(sp["u0"])
        ms.append(m)
    return b, ms


@pytest.mark.parametrize("nsteps", [1, 5])
def test_batch_bitwise_equals_alone(nsteps):
    specs = _mix()
    ref = [_alone(sp, nsteps) for sp in specs]
    b, ms = _batch(specs)
    with b:
        assert len(b.classes()) == len({(sp["scheme"], sp["prec"], sp["nv"]) for sp in specs})
        b.step(nsteps)
        assert b.sync() == (binding.COSENU_OK, -1)
        for sp, m, r in zip(specs, ms, ref):
            got = m.state()
            assert np.array_equal(got, r), (sp["nz"], sp["nv"], sp["scheme"], sp["prec"])
            assert m.conserved()["step"] == nsteps


def test_batch_tuned_bitwise_and_graph():
    """The tuner's trial steps are real steps; any launch shape gives the same bits."""
    specs = _mix()
    b, ms = _batch(specs)
    with b:
        taken = b.tune(reps=1)
        assert taken >= 5
        b.step(3)  # odd count: a graph replay plus a direct step
        assert b.sync()[0] == binding.COSENU_OK
        total = taken + 3
        for sp, m in zip(specs, ms):
            assert np.array_equal(m.state(), _alone(sp, total)), (sp["nz"], sp["nv"])
        for c in b.classes():
            assert all(g >= 1 for g in c["grid"]) and all(r >= 1 for r in c["ring"])


def test_batch_membership_changes_and_solo_steps():
    specs = _mix()
    b, ms = _batch(specs)
    with b:
        b.step(2)
        # drop three members, step one member alone (odd: moves its FP64 parity)
        for k in (1, 4, 8):
            b.remove(ms[k])
        keep = [i for i in range(len(specs)) if i not in (1, 4, 8)]
        solo = 0  # an FP64 member
        binding.cosenu_step(ms[solo].h, 1)
        b.step(3)
        # add a new member mid-run
        extra = dict(nz=300, nv=32, L=45.0, scheme=FD, prec=MIXED, params=dict(mu=2.0),
                     u0=inputs.random_state(300, 32, seed=77, offdiag=0.05))
        me = b.add(extra["nz"], extra["nv"], extra["L"], extra["scheme"], extra["prec"],
                   **extra["params"])
        me.set_state(extra["u0"])
        b.step(2)
        assert b.sync()[0] == binding.COSENU_OK
        for i in keep:
            n = 2 + 3 + 2 + (1 if i == solo else 0)
            assert np.array_equal(ms[i].state(), _alone(specs[i], n)), i
        assert np.array_equal(me.state(), _alone(extra, 2))


def test_batch_params_change_rebuilds_plan():
    specs = _mix()[:4]
    b, ms = _batch(specs)
    with b:
        b.step(2)
        binding.cosenu_set_params(ms[2].h, mu=3.0)
        b.step(2)
        for i, (sp, m) in enumerate(zip(specs, ms)):
            if i == 2:
                with binding.Solver(sp["nz"], sp["nv"], sp["L"], sp["scheme"], sp["prec"],
                                    **sp["params"]) as s:
                    s.set_state(sp["u0"])
                    s.step(2)
                    binding.cosenu_set_params(s.h, mu=3.0)
                    s.step(2)
                    ref = s.state()
            else:
                ref = _alone(sp, 4)
            assert np.array_equal(m.state(), ref), i


@pytest.mark.parametrize("scheme", [FD, WENO, FD3])
def test_batch_members_match_oracle(scheme):
    """Members of a mixed-size FP64 batch against the oracle (FP64 bound 1e-12)."""
    sizes = [(40, 16), (97, 16), (16, 8), (130, 32)]
    b = binding.Batch()
    with b:
        ms, u0s = [], []
        for i, (nz, nv) in enumerate(sizes):
            u0 = inputs.random_state(nz, nv, seed=900 + i, offdiag=0.1)
            m = b.add(nz, nv, 0.2 * nz, scheme, FP64, mu=1.0 + i, omega=0.3, theta=0.2)
            m.set_state(u0)
            ms.append(m)
            u0s.append(u0)
        b.step(4)
        for i, (nz, nv) in enumerate(sizes):
            ref = run_oracle(u0s[i], 0.2 * nz, scheme, 4, mu=1.0 + i, omega=0.3, theta=0.2)
            assert max_abs(ms[i].state(), ref) <= 1e-12, i


def test_batch_c4_recipe_small():
    """Grids drawn from the batched-workload recipe at reduced sizes, mixed precision:
    bitwise equal to the same grids alone after a tuned run."""
    specs = inputs.batch_instances(10, nz_range=(64, 2048))
    b = binding.Batch()
    with b:
        ms = []
        for sp in specs:
            m = b.add(sp["nz"], sp["nv"], sp["L"], sp["scheme"], MIXED, mu=sp["mu"], dt=sp["dt"])
            m.set_state(inputs.collective_state(sp["nz"], sp["nv"], alpha=sp["alpha"],
                                                sigma_nu=sp["sigma_nu"],
                                                sigma_nubar=sp["sigma_nubar"], seed=sp["seed"]))
            ms.append(m)
        taken = b.tune(reps=1)
        b.step(4)
        for sp, m in zip(specs, ms):
            with binding.Solver(sp["nz"], sp["nv"], sp["L"], sp["scheme"], MIXED, mu=sp["mu"],
                                dt=sp["dt"]) as s:
                s.set_state(inputs.collective_state(sp["nz"], sp["nv"], alpha=sp["alpha"],
                                                    sigma_nu=sp["sigma_nu"],
                                                    sigma_nubar=sp["sigma_nubar"],
                                                    seed=sp["seed"]))
                s.step(taken + 4)
                assert np.array_equal(m.state(), s.state())


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_batch_nonfinite_flag_names_member(prec):
    b = binding.Batch()
    with b:
        ms = []
        for i in range(3):
            m = b.add(64, 16, 10.0, FD, prec)
            u0 = inputs.random_state(64, 16, seed=i, offdiag=0.05)
            if i == 1:
                u0[0, 0, 5, 3] = np.inf
            m.set_state(u0)
            ms.append(m)
        b.step(1)
        rc, bad = b.sync()
        assert rc == binding.COSENU_ENONFINITE and bad == 1
        assert b.sync() == (binding.COSENU_OK, -1)  # flags cleared


def test_batch_member_handle_rules():
    b = binding.Batch()
    with b:
        m = b.add(32, 8, 5.0)
        binding.cosenu_destroy(m.h)  # ignored: the batch owns it
        assert "batch" in binding.cosenu_last_error(None)
        with pytest.raises(binding.CosenuError):
            binding.cosenu_set_stream(m.h, 0)
        assert binding.cosenu_batch_size(b.b) == 1
        assert binding.cosenu_batch_member(b.b, 0) == m.h
        assert binding.cosenu_batch_member(b.b, 1) is None
        with pytest.raises(binding.CosenuError):
            binding.cosenu_batch_add(b.b, 0, 8, 1.0)
        with pytest.raises(binding.CosenuError):
            binding.cosenu_batch_step(b.b, -1)
        b.step(0)
        assert b.device_bytes() >= binding.cosenu_workspace_bytes(32, 8, 0, 1)


def test_empty_batch():
    b = binding.Batch()
    with b:
        b.step(3)
        assert b.sync() == (binding.COSENU_OK, -1)
        assert b.classes() == []
        assert b.tune() == 0
