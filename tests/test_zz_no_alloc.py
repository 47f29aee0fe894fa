"""hlbm_fit_static -- the sine fit for callers that cannot allocate device memory.

Callers running under a fixed device-memory budget, inside a framework that
owns every allocation, or unable to take the synchronisation of cudaMalloc
use this entry point: it reads the caller's device samples and keeps its
partial sums in a file-scope device array.  Its results must equal those of
the allocating path (hlbm_gamma) on the same force history, call after call.
This file is collected last so that a failure here never hides the others.
"""
import math

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build
    from paper_2006_13631_gb300 import Solver

    build()
    w = inputs.workload("lamina-256-f64")
    s = Solver(w)
    s.step(w.steps)
    return w, s


def _window(omega, discard, fit):
    Tp = 2.0 * math.pi / omega
    return int(math.ceil(discard * Tp)), int(math.floor((discard + fit) * Tp))


def test_fit_static_matches_allocating_path_on_consecutive_calls(solver):
    from paper_2006_13631_gb300 import hlbm_fit_static

    w, s = solver
    fx, fy = s.force()
    hist = torch.tensor(np.stack([fx, fy], axis=1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    N = 0.25 * math.pi * w.rho0 * w.omega ** 2 * w.L ** 2 * w.A
    y_ptr = hist.data_ptr() + 8  # F_y column of the interleaved history
    results = []
    for discard, fit in ((1.0, 3.0), (2.0, 2.0), (1.0, 3.0)):
        t0, t1 = _window(w.omega, discard, fit)
        torch.cuda.synchronize()
        alloc_before = torch.cuda.memory_allocated()
        reserved_before = torch.cuda.memory_reserved()
        free_before = torch.cuda.mem_get_info()[0]
        a, b, rms = hlbm_fit_static(y_ptr, 2, t0, t1, w.omega, stream)
        torch.cuda.synchronize()
        # nothing went through torch's allocator
        assert torch.cuda.memory_allocated() == alloc_before
        assert torch.cuda.memory_reserved() == reserved_before
        if results:
            # device-wide free memory (other processes included) as a
            # secondary signal: the first call may load the module; after it
            # no cudaMalloc of the call's size (>= 2 MiB granules) shows up
            assert torch.cuda.mem_get_info()[0] >= free_before - (2 << 20)
        re, im, rms_ref = s.gamma(discard, fit)
        assert a / N == pytest.approx(re, rel=1e-12, abs=1e-14)
        assert b / N == pytest.approx(im, rel=1e-12, abs=1e-14)
        assert rms / N == pytest.approx(rms_ref, rel=1e-9, abs=1e-14)
        results.append((a, b))
    assert results[0] == results[2]  # the shared scratch leaves no trace between calls


def test_fit_static_rejects_oversized_and_invalid_windows(solver):
    from paper_2006_13631_gb300 import HLBMError, hlbm_fit_static

    w, s = solver
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(HLBMError):
        hlbm_fit_static(buf.data_ptr(), 1, 0, (1 << 26) + 5, w.omega)
    with pytest.raises(HLBMError):
        hlbm_fit_static(buf.data_ptr(), 1, 5, 5, w.omega)
    with pytest.raises(HLBMError):
        hlbm_fit_static(buf.data_ptr(), 0, 0, 10, w.omega)
    # w = pi: sin(w t) vanishes at every integer t, so no unique fit exists
    with pytest.raises(HLBMError):
        hlbm_fit_static(buf.data_ptr(), 1, 0, 15, math.pi)
