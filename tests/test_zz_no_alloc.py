"""The allocation-free diagnostics entry point, cosenu_conserved_noalloc.

It serves callers that cannot call cudaMalloc (device memory already handed to
another allocator or held to a fixed budget): its scratch is a static device
array of the library.  The test calls it through the C ABI on a state held by a solver and
compares its eight outputs with those of cosenu_conserved, the allocating entry
point, on two calls in a row (the second after more steps, so stale scratch
would show), and that the second call leaves the device's free memory unchanged.  It also
checks the rejection of grids larger than the scratch.
The file is collected last; it needs nothing from the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_conserved_noalloc_matches_allocating_entry_point():
    import torch

    from paper_2203_12866_gb300 import binding, build, inputs

    build.build()
    binding.load()
    torch.cuda.set_device(0)
    nz, nv, L, theta = 3000, 64, 40.0, 0.3  # 192000 cells: 12 scratch rows, the last one partial
    u0 = inputs.random_state(nz, nv, seed=9, offdiag=0.3)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    with binding.Solver(nz, nv, L, binding.COSENU_FDKO, binding.COSENU_FP64, mu=1.0, omega=0.2,
                        theta=theta) as s:
        s.set_state(u0)
        for call in range(2):
            if call == 1:
                s.step(3)
                s.sync()
            ref = s.conserved()  # waits for the solver's stream
            expect = [ref["tr_nu"], ref["tr_nubar"], *ref["M"], ref["M_vac"], ref["dP_max"],
                      ref["dP_mean"]]
            y_dev = binding.cosenu_state_device(s.h)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            binding.cosenu_conserved_noalloc(y_dev, nz, nv, L, theta, out.data_ptr(), 0)
            torch.cuda.synchronize()
            if call == 1:  # the first call may load the library's device code; later ones take nothing
                assert torch.cuda.mem_get_info()[0] == free_before
            got = out.cpu().numpy()
            assert np.allclose(got, expect, rtol=1e-12, atol=1e-15), (call, got, expect)

        with pytest.raises(binding.CosenuError) as e:
            binding.cosenu_conserved_noalloc(y_dev, 1 << 21, 256, L, theta, out.data_ptr(), 0)
        assert e.value.code == binding.COSENU_EINVAL
        assert "static scratch limit" in binding.cosenu_last_error(None)
