"""fh_apply_noalloc: the operator product for callers that cannot allocate.

Some callers cannot call cudaMalloc (a framework that owns every device
allocation through its own pool, a latency-critical loop that cannot afford
cudaMalloc's implicit synchronisation, a fixed device-memory budget).  For
them the library offers fh_apply_noalloc, whose scratch lives in fixed arrays
inside the library.  This file checks, through the C ABI, that calls in a row
(different grids, so each call reuses scratch the previous one left behind)
give the oracle's product (I + B) e or (I + B^T) e element by element within
the operator tolerance of tests/test_gpu_operator.py, for both products on
both grids, in place (e_in == e_out) as well as out of place, with phase ids
beyond the table (which act as L = L0), and that oversize grids are refused.

The file name sorts last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle

from gpu_util import cuda_or_skip, spd

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def _noalloc(lib, phase_t, nphase, L, L0, e_t, out_t, transpose, Y, stream):
    d = e_t.shape[0]
    N = (ctypes.c_int * d)(*phase_t.shape)
    Lh = np.ascontiguousarray(L[:nphase], dtype=np.float64)
    L0h = np.ascontiguousarray(L0, dtype=np.float64)
    Yh = None if Y is None else np.ascontiguousarray(Y, dtype=np.float64)
    buf = ctypes.create_string_buffer(256)
    pD = ctypes.POINTER(ctypes.c_double)
    rc = lib.fh_apply_noalloc(d, N, None if Yh is None else Yh.ctypes.data_as(pD),
                              ctypes.c_void_p(phase_t.data_ptr()), nphase, Lh.ctypes.data_as(pD),
                              L0h.ctypes.data_as(pD), ctypes.c_void_p(e_t.data_ptr()),
                              ctypes.c_void_p(out_t.data_ptr()), int(transpose), ctypes.c_void_p(stream),
                              buf, 256)
    return rc, buf.value.decode()


def test_noalloc_matches_oracle_on_calls_in_a_row():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    lib = fh.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [((81, 45), (1.0, 2.0), 11), ((15, 21, 9), None, 12)]
    calls = 0
    for N, Y, seed in cases:
        rng = np.random.default_rng(seed)
        d = len(N)
        nphase = 3
        # ids 3 and 4 have no tensor in the call: they must act as L = L0
        phase = rng.integers(0, nphase + 2, size=N).astype(np.uint8)
        L0 = spd(rng, d, 1.0, 3.0)
        L = np.stack([spd(rng, d) for _ in range(nphase)] + [L0, L0])
        e = rng.normal(size=(d,) + N)
        phase_t = torch.from_numpy(phase).cuda()
        tol = 64 * U64 * (1.0 + np.max(np.abs(L - L0[None]))) * np.max(np.abs(e))
        for transpose in (False, True):
            ref = (oracle.apply_AT if transpose else oracle.apply_A)(e, phase, L, L0, Y)
            for in_place in (False, True):
                e_t = torch.from_numpy(e).cuda()
                out_t = e_t if in_place else torch.empty_like(e_t)
                rc, msg = _noalloc(lib, phase_t, nphase, L, L0, e_t, out_t, transpose, Y, stream)
                torch.cuda.synchronize()
                assert rc == 0, msg
                calls += 1
                err = np.max(np.abs(out_t.cpu().numpy() - ref))
                assert err <= tol, (N, transpose, in_place, err, tol)
    assert calls == 8


def test_noalloc_refuses_grids_beyond_its_scratch():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    lib = fh.load_library()
    N = (2187, 729)
    phase_t = torch.zeros(N, dtype=torch.uint8, device="cuda")
    e_t = torch.zeros((2,) + N, dtype=torch.float64, device="cuda")
    rc, msg = _noalloc(lib, phase_t, 1, np.eye(2)[None], 2.0 * np.eye(2), e_t, e_t, False, None,
                       torch.cuda.current_stream().cuda_stream)
    assert rc == 9 and "scratch" in msg
