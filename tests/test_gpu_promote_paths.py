"""Precision promotion (LAGP_PROMOTE) on the two other ways into the path: a
CUDA-graph plan replay and a serving-context request must give the direct
call's results bit for bit, with the binary64 re-solve of the promoted
locations inside (the 4-d workload promotes every location)."""
import numpy as np
import pytest

from gpu_helpers import to_dev
from paper_1409_0074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M, N0, N, NC, NRAYS = 48, 6, 50, 1000, 4


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


@pytest.fixture(scope="module")
def w4():
    return W.paper_scale_4d(M=M)


@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_plan_replay_with_promotion(lagp, w4, search):
    import torch
    X, Y, xr = to_dev(w4.X), to_dev(w4.Y), to_dev(w4.Xref)
    direct = lagp.predict(X, Y, xr, N0, N, NC, w4.theta, w4.g, search=search, nrays=NRAYS,
                          precision="fp32_promote", want_promoted=True)
    assert direct["promoted"] >= M - 1
    s, pr = lagp.SEARCH[search], lagp.PRECISION["fp32_promote"]
    ws = torch.empty(lagp.laGP_workspace_bytes(w4.N, w4.p, M, N, NC, NRAYS, s, pr),
                     dtype=torch.uint8, device="cuda")
    mean = torch.full((M,), -1.0, dtype=torch.float64, device="cuda")
    s2 = torch.full((M,), -1.0, dtype=torch.float64, device="cuda")
    plan = lagp.Plan(X, Y, xr, N0, N, NC, w4.theta, w4.g, s, NRAYS, pr, mean, s2, ws)
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        assert lagp.laGP_status(ws)[0] == 0
        assert lagp.laGP_promoted(ws) == direct["promoted"]
        assert torch.equal(mean, direct["mean"]) and torch.equal(s2, direct["s2"])
    plan.close()


def test_serving_context_with_promotion(lagp, w4):
    import torch
    X, Y = to_dev(w4.X), to_dev(w4.Y)
    pr = lagp.PRECISION["fp32_promote"]
    L = lagp.load()
    arena = (L.laGP_ctx_design_bytes(w4.N, w4.p) +
             L.laGP_ctx_request_bytes(w4.N, w4.p, M, N, NC, NRAYS, lagp.LAGP_RAY, pr, 0) +
             (1 << 20))
    ctx = lagp.Context(X, Y, w4.theta, w4.g, N0, NC, lagp.LAGP_RAY, NRAYS, pr, arena,
                       max_inflight=2)
    mean = torch.empty(M, dtype=torch.float64, pin_memory=True).numpy()
    s2 = torch.empty(M, dtype=torch.float64, pin_memory=True).numpy()
    t = ctx.submit(np.ascontiguousarray(w4.Xref), N, mean, s2)
    assert t is not None
    ctx.wait(t)
    ref = lagp.predict(X, Y, to_dev(w4.Xref), N0, N, NC, w4.theta, w4.g, search="ray",
                       nrays=NRAYS, precision="fp32_promote")
    np.testing.assert_array_equal(mean, ref["mean"].cpu().numpy())
    np.testing.assert_array_equal(s2, ref["s2"].cpu().numpy())
    ctx.close()
