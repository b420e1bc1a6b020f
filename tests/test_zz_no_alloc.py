"""laGP_knn_noalloc, the kNN search for callers that may not allocate device
memory (a framework-owned memory pool, a latency-bound serving loop, a fixed
memory budget): its scratch lives in a static device array of the library.

Checked through the C ABI against laGP_knn (which uses a caller workspace) on
two calls in a row with different sizes, so that the second call also shows
that nothing left over from the first one leaks into its result.  The file
is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp
    L = lagp.load()
    f = L.laGP_knn_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    return lagp


def _reference(lagp, X, Xr, nc):
    import torch
    N, p = X.shape
    M = Xr.shape[0]
    ws = torch.empty(lagp.laGP_knn_workspace_bytes(N, p, M, nc), dtype=torch.uint8,
                     device="cuda")
    cand = torch.empty((M, nc), dtype=torch.int32, device="cuda")
    lagp.laGP_knn(X, Xr, nc, cand, ws)
    rc, st = lagp.laGP_status(ws)
    assert rc == 0 and st == 0
    return cand.cpu().numpy()


def test_noalloc_knn_matches_workspace_entry_twice(lib):
    import torch
    lagp = lib
    fn = lagp.load().laGP_knn_noalloc
    rng = np.random.default_rng(11)
    cases = [(30000, 4, 333, 700), (12345, 8, 97, 256)]
    stream = torch.cuda.current_stream()
    for N, p, M, nc in cases:
        X = torch.from_numpy(rng.random((N, p))).cuda()
        Xr = torch.from_numpy(rng.random((M, p)) * 1.1 - 0.05).cuda()
        expect = _reference(lagp, X, Xr, nc)
        cand = torch.full((M, nc), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
        rc = fn(X.data_ptr(), N, p, Xr.data_ptr(), M, nc, cand.data_ptr(), status.data_ptr(),
                stream.cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_array_equal(cand.cpu().numpy(), expect)


def test_noalloc_empty_request_clears_the_status_word(lib):
    """M = 0 enqueues no search, yet the caller's status word reports the call."""
    import torch
    fn = lib.load().laGP_knn_noalloc
    X = torch.from_numpy(np.random.default_rng(3).random((500, 3))).cuda()
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = fn(X.data_ptr(), 500, 3, X.data_ptr(), 0, 50, None, status.data_ptr(),
            stream.cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_noalloc_rejects_requests_beyond_its_scratch(lib):
    fn = lib.load().laGP_knn_noalloc
    need = lib.laGP_knn_workspace_bytes(4_000_000, 8, 1000, 1000)
    assert need > (64 << 20)
    # rejected before any device work: the pointers are never dereferenced
    assert fn(4096, 4_000_000, 8, 4096, 1000, 1000, 4096, None, None) == -2
    assert fn(4096, 1000, 0, 4096, 10, 10, 4096, None, None) == -1
