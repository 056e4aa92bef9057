"""Checkpoint and resume through the C ABI: the state read back with
cosenu_get_state and written into a fresh handle continues the run.  FP64 carries
no state besides y, so the resumed run is bitwise the uninterrupted one; the mixed
path rebuilds its float copy of y and its running FP64 v-moments from y on
cosenu_set_state, where the uninterrupted run carries moments summed from its
increments, so the two agree to rounding (checked per component)."""
import numpy as np
import pytest

from paper_2203_12866_gb300 import binding, inputs
from parity_util import PRECS, SCHEMES, rel_by_component

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_from_checkpoint(scheme, prec):
    nz, nv, L = 96, 32, 18.75
    u0 = inputs.collective_state(nz, nv, eps0=1e-3)
    kw = dict(mu=1.0, omega=0.1, theta=0.2)
    with binding.Solver(nz, nv, L, SCHEMES[scheme], PRECS[prec], **kw) as a:
        a.set_state(u0)
        a.step(10)
        a.sync()
        ckpt = a.state()
        a.step(7)
        a.sync()
        straight = a.state()
    with binding.Solver(nz, nv, L, SCHEMES[scheme], PRECS[prec], **kw) as b:
        b.set_state(ckpt)
        b.step(7)
        b.sync()
        resumed = b.state()
    if prec == "fp64":
        assert np.array_equal(resumed, straight)
    else:
        assert rel_by_component(resumed, straight) <= 1e-6
