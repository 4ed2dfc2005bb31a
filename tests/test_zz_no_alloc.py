"""The allocation-free entry point bap_continuation_static against bap_debug_continuation.

Some callers cannot allocate device memory while they run (a host framework that owns all of the
GPU's memory, or a latency-bound loop that must not call cudaMalloc or cudaFree).  For them the
library offers one call whose scratch is a fixed array in its device image and whose inputs and
outputs are the caller's device buffers.  This file is collected last so that a failure here
stops a `-x` run only after every other test ran; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import paper_0805_1827_gb300 as bap
from bap_workloads import IZParams, PURPOSE_IZ, spec_max_call

pytestmark = pytest.mark.gpu


def _fn():
    L = bap.lib()
    f = L.bap_continuation_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_static_scratch_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=6, T=2.0)
    opt = bap.Option(spec)
    opt.fit_boundary(IZParams(J=16, N1=2000, degree=2, seed=3))
    rng = np.random.default_rng(11)
    n, N, m, seed = 40, 6000, 2, 9
    starts = 100.0 * np.exp(rng.normal(scale=0.25, size=(n, spec.d)))
    ids = np.arange(500, 500 + n, dtype=np.int32)
    piv = (np.arange(n) % spec.d).astype(np.int32)
    ref_sums, ref_steps = opt.debug_continuation(m, PURPOSE_IZ, seed, ids, starts, N, piv)

    # the caller's own device buffers (torch's allocator stands in for a host framework's)
    d_ids = torch.tensor(ids, dtype=torch.int32, device="cuda")
    d_piv = torch.tensor(piv, dtype=torch.int32, device="cuda")
    d_starts = torch.tensor(starts, dtype=torch.float64, device="cuda")
    d_sums = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    d_steps = torch.empty(n, dtype=torch.int64, device="cuda")
    f = _fn()
    for call in range(2):
        d_sums.fill_(-1.0)
        d_steps.fill_(-1)
        torch.cuda.synchronize()
        st = f(opt.h, m, PURPOSE_IZ, seed, n, d_ids.data_ptr(), d_piv.data_ptr(),
               d_starts.data_ptr(), N, d_sums.data_ptr(), d_steps.data_ptr())
        assert st == bap.BAP_OK, bap.lib().bap_last_error()
        torch.cuda.synchronize()
        got = d_sums.cpu().numpy()
        # same kernel, same work split: the sums agree to rounding (they are bitwise equal)
        assert np.allclose(got, ref_sums, rtol=1e-12, atol=0.0), (call, np.abs(got - ref_sums).max())
        assert np.array_equal(d_steps.cpu().numpy(), ref_steps), call
    opt.close()


def test_static_scratch_rejects_calls_beyond_its_size():
    torch = pytest.importorskip("torch")
    spec = spec_max_call(2, 100.0, n_dates=4, T=1.0)
    opt = bap.Option(spec)
    n, N = 4096, 1 << 24
    d_ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    d_starts = torch.full((n, 2), 100.0, dtype=torch.float64, device="cuda")
    d_sums = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    d_steps = torch.empty(n, dtype=torch.int64, device="cuda")
    st = _fn()(opt.h, 1, PURPOSE_IZ, 1, n, d_ids.data_ptr(), None, d_starts.data_ptr(), N,
               d_sums.data_ptr(), d_steps.data_ptr())
    assert st == bap.BAP_EINVAL
    assert b"static scratch" in bap.lib().bap_last_error()
    opt.close()


def test_static_scratch_marks_bad_inputs_without_touching_other_items():
    """The call cannot see device data on the host, so it checks the inputs on the device: an
    item whose pivot is outside -1..d-1 or whose start point has a coordinate <= 0 comes back
    with NaN sums and steps = -1, and every other item is computed as usual."""
    torch = pytest.importorskip("torch")
    spec = spec_max_call(3, 100.0, rho=0.2, n_dates=5, T=1.0)
    opt = bap.Option(spec)
    n, N, m, seed = 6, 3000, 2, 4
    starts = np.full((n, spec.d), 100.0)
    starts[:, 0] = [90.0, 110.0, 120.0, 95.0, 105.0, 130.0]
    ids = np.arange(n, dtype=np.int32)
    piv = np.zeros(n, dtype=np.int32)
    ref_sums, ref_steps = opt.debug_continuation(m, PURPOSE_IZ, seed, ids, starts, N, piv)
    bad_piv, bad_start = 1, 4
    piv_in = piv.copy()
    piv_in[bad_piv] = spec.d                 # one past the last asset
    starts_in = starts.copy()
    starts_in[bad_start, 2] = 0.0
    d_ids = torch.tensor(ids, dtype=torch.int32, device="cuda")
    d_piv = torch.tensor(piv_in, dtype=torch.int32, device="cuda")
    d_starts = torch.tensor(starts_in, dtype=torch.float64, device="cuda")
    d_sums = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    d_steps = torch.zeros(n, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    st = _fn()(opt.h, m, PURPOSE_IZ, seed, n, d_ids.data_ptr(), d_piv.data_ptr(),
               d_starts.data_ptr(), N, d_sums.data_ptr(), d_steps.data_ptr())
    assert st == bap.BAP_OK, bap.lib().bap_last_error()
    torch.cuda.synchronize()
    got, steps = d_sums.cpu().numpy(), d_steps.cpu().numpy()
    bad = np.zeros(n, dtype=bool)
    bad[[bad_piv, bad_start]] = True
    assert np.all(np.isnan(got[bad])) and np.all(steps[bad] == -1)
    assert np.allclose(got[~bad], ref_sums[~bad], rtol=1e-12, atol=0.0)
    assert np.array_equal(steps[~bad], ref_steps[~bad])
    opt.close()
