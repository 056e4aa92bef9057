"""Parity at the benchmark's full size (nz = 2^20, nv = 256, mu = 10, the roofline
workload) in the launch configuration bench.py times.

The oracle cannot step the whole grid, but the method is local in z: after n RK4
steps a row depends only on rows within n * 4 * lag (lag = 2 for FD4+KO, 3 for
FD4+KO r = 3, 4 for WENO7; the v-moments are per row).  So for each sampled row z0 the oracle runs
the same n steps on a periodic patch of 128 rows centred on z0, and the 33 rows
around z0 -- farther than 2 * 4 * 4 = 32 rows from the patch edges' wrap -- must
match the GPU's rows element by element.  Samples include both ends of the
periodic domain and a CTA boundary.
"""
import numpy as np
import pytest

import oracle
from paper_2203_12866_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

NZ, NV = 1 << 20, 256
DZ = 3200.0 / 65536.0
L = NZ * DZ
MU = 10.0
NSTEPS = 2
HALF = 64          # patch = rows z0 - 64 .. z0 + 63
KEEP = 16          # compared rows z0 - 16 .. z0 + 16


def gpu_rows(h, z0):
    rows = (np.arange(z0 - KEEP, z0 + KEEP + 1)) % NZ
    out = np.empty((2, 4, rows.size, NV))
    # contiguous runs (at most two, across the periodic seam)
    start = 0
    while start < rows.size:
        end = start
        while end + 1 < rows.size and rows[end + 1] == rows[end] + 1:
            end += 1
        blk = np.empty((2, 4, end - start + 1, NV))
        binding.cosenu_get_rows(h, int(rows[start]), end - start + 1, blk)
        out[:, :, start:end + 1] = blk
        start = end + 1
    return out


@pytest.fixture(scope="module")
def state_dev():
    import torch
    torch.cuda.set_device(0)
    s = inputs.collective_state_device(NZ, NV, "cuda")
    torch.cuda.synchronize()
    yield s
    del s
    torch.cuda.empty_cache()


@pytest.mark.parametrize("scheme,prec", [("fdko", "mixed"), ("fdko", "fp64"),
                                         ("weno7", "mixed"), ("weno7", "fp64"),
                                         ("fdko3", "mixed"), ("fdko3", "fp64")])
def test_fullsize_sampled_rows(state_dev, scheme, prec, oracle):
    sc = {"fdko": binding.COSENU_FDKO, "weno7": binding.COSENU_WENO7,
          "fdko3": binding.COSENU_FDKO3}[scheme]
    pr = {"fp64": binding.COSENU_FP64, "mixed": binding.COSENU_MIXED}[prec]
    h = binding.cosenu_create(NZ, NV, L, sc, pr)
    try:
        binding.cosenu_set_params(h, mu=MU)
        dt = binding.cosenu_get_params(h).dt
        binding.cosenu_set_state_device(h, state_dev.data_ptr(), state_dev.numel())
        binding.cosenu_step(h, NSTEPS)
        binding.cosenu_sync(h)
        # 3450 and 6899 are CTA boundaries of the 304- and 152-CTA launch shapes
        samples = [0, 5, NZ - 3, 3450, 6899, NZ // 2 + 12345, 777777]
        for z0 in samples:
            got = gpu_rows(h, z0)
            patch = np.arange(z0 - HALF, z0 + HALF) % NZ
            u0 = inputs.collective_rows(patch, NV)
            p = oracle.params(2 * HALF, NV, 2 * HALF * DZ, sc, mu=MU, dt=dt)
            ref = oracle.step(p, u0, NSTEPS)[:, :, HALF - KEEP:HALF + KEEP + 1]
            if prec == "fp64":
                assert np.max(np.abs(got - ref)) <= 1e-12, z0
            else:
                worst = 0.0
                for sp in range(2):
                    for c in range(4):
                        scale = np.max(np.abs(ref[sp, c]))
                        if scale > 0:
                            worst = max(worst, np.max(np.abs(got[sp, c] - ref[sp, c])) / scale)
                assert worst <= 1e-5, (z0, worst)
    finally:
        binding.cosenu_destroy(h)
