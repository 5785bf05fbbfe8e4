"""The allocation-free acceleration entry point (fsi_accel_noalloc), for callers that
cannot allocate device memory, against the context-based fsi_accel.

Collected last on purpose (file name), so a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2210_02472_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12     # the FP64 tolerance of the parity tests (per particle, of |a_i|)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(got, ref):
    return (np.abs(got - ref).max(axis=0) / np.linalg.norm(ref, axis=0)).max()


def test_noalloc_matches_fsi_accel_on_two_calls():
    from paper_2210_02472_b300 import fsi as F
    cases = [inputs.plummer(20000, 91, imf="kroupa"), inputs.plummer(3001, 92)]
    with F.Context("fp64") as ctx:
        for eps2, c in zip((0.0, 1e-4), cases):          # two calls in a row, different sizes
            pos, mass = dev(c.pos), dev(c.mass)
            out = torch.empty((3, c.n), dtype=torch.float64, device="cuda")
            # through the C ABI directly (argument marshalling only)
            code = F._lib.fsi_accel_noalloc(c.n, ctypes.c_void_p(pos.data_ptr()),
                                            ctypes.c_void_p(mass.data_ptr()), eps2,
                                            ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert code == F.FSI_OK
            ref = F.fsi_accel(ctx, pos, mass, eps2=eps2)
            torch.cuda.synchronize()
            assert F.fsi_sync_status(ctx) == F.FSI_OK
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel(got, want) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2210_02472_b300 import fsi as F
    n = 32769
    pos = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    mass = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FsiError) as e:
        F.fsi_accel_noalloc(pos, mass)
    assert e.value.code == F.FSI_ERR_ARG
    assert "32768" in str(e.value)
