"""Pre-scaled inputs (Sec 5.3) on the GPU, through the C ABI: the separable
global lengthscales of laGP_sep_mle against the oracle's maximiser
(oracle/sep_mle.py), laGP_prescale against numpy, and the local path on
pre-scaled inputs against the oracle's FP64 designs on the same inputs."""
import numpy as np
import pytest

import oracle
from oracle import sep_mle as SM
from gpu_helpers import to_dev
from paper_1409_0074_gb300 import workloads as W
from test_gpu_parity import assert_fp64_parity, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

TMIN, TMAX = 1e-3, 100.0


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


@pytest.fixture(scope="module")
def w4():
    return W.paper_scale_4d(M=2000)


@pytest.mark.parametrize("n_sub", [200, 600])
def test_separable_lengthscales_match_the_oracle(lagp, w4, n_sub):
    """The GPU's BFGS fit (Gauss-Jordan inverses, its own summation order)
    and the oracle's (Cholesky) reach the same maximiser: theta within 1e-6,
    and the oracle's gradient at the GPU's estimate vanishes."""
    sub = W.subset(w4.N, n_sub, seed=1)
    th, (it, ev, st) = lagp.sep_mle(to_dev(w4.X), to_dev(w4.Y), to_dev(sub), w4.g, 1.0, TMIN,
                                    TMAX)
    th = th.cpu().numpy()
    assert st == 0 and 1 < it < 200 and ev >= it
    S, y = w4.X[sub], w4.Y[sub]
    to, _, _, lo = SM.sep_mle(S, y, w4.g, 1.0, TMIN, TMAX)
    np.testing.assert_allclose(th, to, rtol=1e-6)
    l, gr = SM.sep_loglik(S, y, th, w4.g)
    assert abs(l - lo) <= 1e-9 * abs(lo)
    interior = (th > TMIN * 1.01) & (th < TMAX * 0.99)
    assert np.all(np.abs(gr * th)[interior] <= 1e-5 * abs(l))


def test_prescale_is_exact(lagp, w4):
    th = np.array([0.03, 0.4, 2.5, 0.11])
    got = lagp.prescale(to_dev(w4.X[:5000]), to_dev(th)).cpu().numpy()
    np.testing.assert_array_equal(got, SM.prescale(w4.X[:5000], th))


def test_sep_mle_rejects_bad_subsets(lagp, w4):
    """A row index outside the design is reported (status 2), not read."""
    sub = W.subset(w4.N, 50, seed=1)
    sub[7] = w4.N + 3
    with pytest.raises(lagp.LagpError):
        lagp.sep_mle(to_dev(w4.X), to_dev(w4.Y), to_dev(sub), w4.g, 1.0, TMIN, TMAX)


@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_local_path_on_prescaled_inputs(lagp, w4, search):
    """The whole variant: global fit on a 400-row subset, inputs scaled on
    the GPU, then the FP64 local path at theta = 1; the oracle runs on the
    same scaled inputs and its designs are bit-identical."""
    sub = W.subset(w4.N, 400, seed=1)
    th, _ = lagp.sep_mle(to_dev(w4.X), to_dev(w4.Y), to_dev(sub), w4.g, 1.0, TMIN, TMAX)
    s = W.Workload(**{k: getattr(w4, k) for k in ("name", "N", "p", "M", "n0", "n", "nc",
                                                  "theta", "g", "search", "nrays", "response")})
    idx = np.linspace(0, w4.M - 1, 24).astype(int)
    s.X = lagp.prescale(to_dev(w4.X), th).cpu().numpy()
    s.Xref = lagp.prescale(to_dev(w4.Xref[idx]), th).cpu().numpy()
    s.Y, s.Ytrue, s.M, s.theta = w4.Y, w4.Ytrue[idx], len(idx), 1.0
    g = gpu_run(lagp, s, search, "fp64", nrays=4)
    o = oracle_run(s, search, nrays=4)
    ident, _ = assert_fp64_parity(g, o, s.n0, s.M)
    assert ident >= s.M - 1
