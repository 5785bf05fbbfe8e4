"""The allocation-free acceleration entry point (fsi_accel_noalloc).

Some callers cannot allocate device memory: code under a host framework that owns every
device allocation, or code that must not allocate while a CUDA graph capture is being
set up.  fsi_accel_noalloc serves them with a fixed scratch array in the library, and
these tests check it through the C ABI against the context-based fsi_accel and against
the FP64 oracle, on calls in a row of different sizes (one source slice, several slices,
the 32768-particle capacity), in a fresh process whose first library call is this one, and
with the device's free memory unchanged across a call.

Collected last on purpose (file name), so a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes
import os
import subprocess
import sys
import textwrap
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
from paper_2210_02472_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12     # the FP64 tolerance of the parity tests (per particle, of |a_i|)
ROOT = Path(__file__).resolve().parent.parent


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(got, ref):
    return (np.abs(got - ref).max(axis=0) / np.linalg.norm(ref, axis=0)).max()


def call_noalloc(F, n, pos, mass, eps2, out):
    """fsi_accel_noalloc through the C ABI (argument marshalling only)."""
    return F._lib.fsi_accel_noalloc(n, ctypes.c_void_p(pos.data_ptr()),
                                    ctypes.c_void_p(mass.data_ptr()), float(eps2),
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# (N, eps2): one source slice (N = 1000), several slices (3001, 20000), the capacity edge
CASES = [(20000, 0.0), (3001, 1e-4), (1000, 0.0), (32768, 0.0)]


def test_noalloc_matches_fsi_accel_and_oracle_on_calls_in_a_row():
    from paper_2210_02472_b300 import fsi as F
    oracle.set_threads(os.cpu_count() or 1)
    with F.Context("fp64") as ctx:
        for k, (n, eps2) in enumerate(CASES):        # calls in a row, different sizes
            c = inputs.plummer(n, 91 + k, imf="kroupa")
            pos, mass = dev(c.pos), dev(c.mass)
            out = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
            assert call_noalloc(F, n, pos, mass, eps2, out) == F.FSI_OK
            ref = F.fsi_accel(ctx, pos, mass, eps2=eps2)
            torch.cuda.synchronize()
            assert F.fsi_sync_status(ctx) == F.FSI_OK
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel(got, want) <= TOL
            rows = inputs.random_subset(n, min(n, 512), 93 + k)
            exact = oracle.acc(c.pos, c.mass, rows, None, eps2=eps2)
            assert rel(got[:, rows], exact) <= TOL


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which may load the kernels), a call changes neither torch's
    allocator count nor the device's free memory."""
    from paper_2210_02472_b300 import fsi as F
    n = 20000
    c = inputs.plummer(n, 95)
    pos, mass = dev(c.pos), dev(c.mass)
    out = torch.empty((3, n), dtype=torch.float64, device="cuda")
    assert call_noalloc(F, n, pos, mass, 0.0, out) == F.FSI_OK
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call_noalloc(F, n, pos, mass, 0.0, out) == F.FSI_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0


def test_noalloc_first_call_in_a_fresh_process():
    """A process whose first library call is fsi_accel_noalloc (no context ever created):
    the scratch address and the SM count are looked up on that call."""
    script = textwrap.dedent(f"""
        import ctypes, sys
        sys.path.insert(0, {str(ROOT)!r})
        import numpy as np, torch
        import oracle
        from paper_2210_02472_b300 import inputs
        from paper_2210_02472_b300 import fsi as F
        c = inputs.plummer(5000, 97)
        pos = torch.as_tensor(c.pos).cuda()
        mass = torch.as_tensor(c.mass).cuda()
        out = torch.empty((3, c.n), dtype=torch.float64, device="cuda")
        code = F._lib.fsi_accel_noalloc(c.n, ctypes.c_void_p(pos.data_ptr()),
                                        ctypes.c_void_p(mass.data_ptr()), 0.0,
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == F.FSI_OK, code
        got = out.cpu().numpy()
        rows = inputs.random_subset(c.n, 256, 98)
        ref = oracle.acc(c.pos, c.mass, rows, None)
        err = (np.abs(got[:, rows] - ref).max(axis=0) / np.linalg.norm(ref, axis=0)).max()
        assert err <= {TOL!r}, err
        print("fresh-process noalloc ok", err)
    """)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True,
                       timeout=600, cwd=str(ROOT))
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process noalloc ok" in r.stdout


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2210_02472_b300 import fsi as F
    n = 32769
    pos = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    mass = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FsiError) as e:
        F.fsi_accel_noalloc(pos, mass)
    assert e.value.code == F.FSI_ERR_ARG
    assert "32768" in str(e.value)


def test_noalloc_binding_rejects_tensors_off_the_current_device():
    """The C side launches on the current device; the binding refuses tensors that live
    elsewhere (CPU tensors here; another GPU's tensors the same way)."""
    from paper_2210_02472_b300 import fsi as F
    n = 64
    pos = torch.zeros((3, n), dtype=torch.float64)
    mass = torch.ones(n, dtype=torch.float64)
    with pytest.raises(TypeError):
        F.fsi_accel_noalloc(pos, mass)
