"""The C-ABI library builds, loads and exports every entry point that
include/lagp.h declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lagp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(laGP_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp
    return lagp.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 7
    for name in names:
        assert hasattr(lib, name), name
    from paper_1409_0074_gb300 import lagp
    assert set(lagp.EXPORTED) <= set(names)


def test_workspace_sizes_and_argument_checks(lib):
    from paper_1409_0074_gb300 import lagp
    ok = lagp.laGP_workspace_bytes(100000, 4, 10000, 50, 1000, 4, lagp.LAGP_RAY, lagp.LAGP_FP64)
    assert ok > 0
    # exhaustive FP64 keeps a correlation cache: larger
    ex = lagp.laGP_workspace_bytes(100000, 4, 10000, 50, 1000, 4, lagp.LAGP_EXHAUSTIVE,
                                   lagp.LAGP_FP64)
    assert ex > ok
    bad = [
        (100000, 0, 10, 50, 1000, 4, 1, 0),      # p < 1
        (100000, 17, 10, 50, 1000, 4, 1, 0),     # p > 16
        (100000, 4, 10, 50, 40, 4, 1, 0),        # n > N_close
        (500, 4, 10, 50, 1000, 4, 1, 0),         # N_close > N
        (100000, 4, 10, 129, 1000, 4, 1, 0),     # n > 128
        (100000, 4, 10, 50, 1000, 17, 1, 0),     # too many rays
        (100000, 4, 10, 50, 52, 4, 1, 0),        # nrays > N_close - n
        (100000, 4, 10, 50, 1000, 4, 3, 0),      # bad search
        (100000, 4, 10, 50, 1000, 4, 1, 3),      # bad precision
        (100000, 4, 10, 50, 1000, 4, 1, -1),     # bad precision
        (100000, 4, 10, 50, 1000, 4, 1, 16),     # promotion of the FP64 form
        (100000, 4, 10, 50, 1000, 4, 1, 3 | 16), # bad form with the promotion flag
        (100000, 4, 10, 50, 1000, 4, 1, 32),     # unknown flag
    ]
    for args in bad:
        assert lagp.laGP_workspace_bytes(*args) == 0, args
    # both FP32-scoring forms are valid; the tensor-core form also keeps its
    # operand tiles per slot
    f32 = [lagp.laGP_workspace_bytes(100000, 8, 10000, 50, 1000, 8, lagp.LAGP_EXHAUSTIVE, pr)
           for pr in (lagp.LAGP_FP32_SCORE, lagp.LAGP_FP32_SCORE_TC)]
    assert 0 < f32[0] < f32[1]
    # LAGP_PROMOTE adds the re-solve list, and for exhaustive search the
    # binary64 correlation cache of its 608 CTAs
    for search in (lagp.LAGP_RAY, lagp.LAGP_EXHAUSTIVE):
        off = lagp.laGP_workspace_bytes(100000, 8, 10000, 50, 1000, 8, search,
                                        lagp.LAGP_FP32_SCORE)
        on = lagp.laGP_workspace_bytes(100000, 8, 10000, 50, 1000, 8, search,
                                       lagp.LAGP_FP32_SCORE | lagp.LAGP_PROMOTE)
        assert 0 < off < on
        if search == lagp.LAGP_EXHAUSTIVE:
            assert on - off >= 8 * 608 * 50 * 1000
    assert lagp.laGP_knn_workspace_bytes(1000, 3, 10, 1) > 0
    assert lagp.laGP_host_workspace_bytes(1000, 3, 10, 10, 100, 2, 1, 1) > \
        lagp.laGP_workspace_bytes(1000, 3, 10, 10, 100, 2, 1, 1)


def test_invalid_calls_return_before_touching_the_device(lib):
    vp = C.c_void_p
    f = lib.laGP_build_and_predict
    f.restype = C.c_int
    f.argtypes = [vp, vp, C.c_int64, C.c_int, vp, C.c_int64, C.c_int, C.c_int, C.c_int,
                  C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp,
                  vp, C.c_size_t, vp]
    fake = 4096
    common = [fake, fake, 1000, 2, fake, 10]
    # theta <= 0
    assert f(*common, 3, 10, 100, 0.0, 1e-6, 0, 2, 0, None, None, fake, fake, None, None, None,
             fake, 1 << 30, None) == -1
    # n0 > n
    assert f(*common, 11, 10, 100, 0.1, 1e-6, 0, 2, 0, None, None, fake, fake, None, None, None,
             fake, 1 << 30, None) == -1
    # null output
    assert f(*common, 3, 10, 100, 0.1, 1e-6, 0, 2, 0, None, None, None, fake, None, None, None,
             fake, 1 << 30, None) == -1
    # workspace too small
    assert f(*common, 3, 10, 100, 0.1, 1e-6, 0, 2, 0, None, None, fake, fake, None, None, None,
             fake, 16, None) == -2
    # M == 0 is a no-op
    assert f(fake, fake, 1000, 2, fake, 0, 3, 10, 100, 0.1, 1e-6, 0, 2, 0, None, None, fake, fake,
             None, None, None, fake, 1 << 30, None) == 0


def test_mle_argument_checks_return_before_touching_the_device(lib):
    """laGP_mle_predict rejects out-of-range sizes, ranges and a missing status
    word before any device work (returns -1 without a GPU)."""
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    f = lib.laGP_mle_predict
    f.restype = C.c_int
    f.argtypes = [vp, vp, i64, i32, vp, i64, vp, i32, dbl, dbl, dbl, dbl, vp, vp, vp, vp, vp, vp]
    fake = 4096

    def call(N=1000, p=2, M=10, n=30, theta0=0.1, g=1e-6, tmin=1e-3, tmax=2.0, status=fake):
        return f(fake, fake, N, p, fake, M, fake, n, theta0, g, tmin, tmax, fake, fake, fake,
                 None, status, None)

    assert call(n=65) == -1          # n above 64
    assert call(n=0) == -1
    assert call(p=17) == -1
    assert call(N=20) == -1          # n > N
    assert call(tmin=0.0) == -1
    assert call(tmax=1e-3) == -1     # tmax <= tmin
    assert call(theta0=0.0) == -1
    assert call(g=-1.0) == -1
    assert call(status=None) == -1


def test_host_only_entry_points_of_tuning_plans_and_contexts(lib):
    """Sizes, the launch-choice table and argument checks of the plan and
    serving-context entry points need no device."""
    from paper_1409_0074_gb300 import lagp
    vp = C.c_void_p
    d = lib.laGP_ctx_design_bytes(1_000_000, 8)
    assert d >= 1_000_000 * 8 * 4          # at least the FP32 design copy
    r1 = lib.laGP_ctx_request_bytes(1_000_000, 8, 500, 50, 1000, 8, 1, 1, 0)
    r2 = lib.laGP_ctx_request_bytes(1_000_000, 8, 1000, 50, 1000, 8, 1, 1, 0)
    r3 = lib.laGP_ctx_request_bytes(1_000_000, 8, 500, 50, 1000, 8, 1, 1, 1)
    assert 0 < r1 < r2 and r3 > r1
    assert lib.laGP_ctx_request_bytes(1_000_000, 8, 0, 50, 1000, 8, 1, 1, 0) == 0
    # launch-choice table: defaults, set, get, invalid codes
    assert lagp.laGP_tune_get(3, 40, 500, 3, 1, 0) == 2 | 16
    lagp.laGP_tune_set(3, 40, 500, 3, 1, 0, 4 | 32)
    assert lagp.laGP_tune_get(3, 40, 500, 3, 1, 0) == 4 | 32
    assert lagp.laGP_tune_get(3, 40, 500, 3, 1, 1) == 2 | 16        # other key untouched
    for bad in (0, 3, 5, 2 | 64):
        assert lib.laGP_tune_set(3, 40, 500, 3, 1, 0, bad) == -1
    # plans and contexts reject invalid arguments before touching a device
    h = vp(0)
    assert lib.laGP_plan_create(None, None, 1000, 2, None, 10, 3, 10, 100, 0.1, 1e-6, 1, 2, 1,
                                None, None, None, None, None, None, None, None, 0,
                                C.byref(h)) == -1
    assert lib.laGP_ctx_create(None, None, 1000, 2, 0.1, 1e-6, 6, 100, 1, 2, 1, None, 0, 4,
                               C.byref(h)) == -1
    fake = 4096
    assert lib.laGP_ctx_create(fake, fake, 1000, 2, 0.1, 1e-6, 6, 100, 1, 2, 1, fake, 1 << 30,
                               0, C.byref(h)) == -1                 # no slots
    assert lib.laGP_ctx_create(fake, fake, 1000, 2, 0.1, 1e-6, 6, 100, 1, 2, 1, fake + 8,
                               1 << 30, 4, C.byref(h)) == -1        # misaligned arena
    assert lib.laGP_ctx_create(fake, fake, 1000, 2, 0.1, 1e-6, 6, 100, 1, 2, 1, fake, 64, 4,
                               C.byref(h)) == -2                    # arena below the design part
    done = C.c_int(0)
    assert lib.laGP_ctx_poll(None, 1, C.byref(done)) == -1
    assert lib.laGP_plan_launch(None, None) == -1


def test_mle_entry_argument_checks(lib):
    """laGP_build_and_predict_mle: local designs up to 64 points, one or two
    stages, a valid theta range; checked before any device work (the
    pointers below are never dereferenced)."""
    from paper_1409_0074_gb300 import lagp
    ok = lagp.laGP_mle_workspace_bytes(100000, 4, 1000, 64, 1000, 4, lagp.LAGP_RAY, lagp.LAGP_FP64)
    base = lagp.laGP_workspace_bytes(100000, 4, 1000, 64, 1000, 4, lagp.LAGP_RAY, lagp.LAGP_FP64)
    assert ok >= base + 1000 * 64 * 4
    assert lagp.laGP_mle_workspace_bytes(100000, 4, 1000, 65, 1000, 4, 1, 0) == 0
    assert lagp.laGP_mle_workspace_bytes(100000, 17, 1000, 50, 1000, 4, 1, 0) == 0
    f = lib.laGP_build_and_predict_mle
    p = 4096
    common = (p, p, 1000, 2, p, 10, 6, 30, 100)
    #             theta0 g     tmin  tmax stages search nrays prec  theta mean s2 sel ws  bytes
    assert f(*common, 0.5, 1e-6, 1e-3, 2.0, 3, 1, 2, 0, p, p, p, None, p, 1 << 30, None) == -1
    assert f(*common, 0.5, 1e-6, 2.0, 1e-3, 1, 1, 2, 0, p, p, p, None, p, 1 << 30, None) == -1
    assert f(*common, -1.0, 1e-6, 1e-3, 2.0, 1, 1, 2, 0, p, p, p, None, p, 1 << 30, None) == -1
    assert f(*common, 0.5, 1e-6, 1e-3, 2.0, 1, 1, 2, 0, None, p, p, None, p, 1 << 30, None) == -1
    small = lagp.laGP_mle_workspace_bytes(1000, 2, 10, 30, 100, 2, 1, 0)
    assert f(*common, 0.5, 1e-6, 1e-3, 2.0, 1, 1, 2, 0, p, p, p, None, p, small - 1, None) == -2
    m0 = (p, p, 1000, 2, p, 0, 6, 30, 100)
    assert f(*m0, 0.5, 1e-6, 1e-3, 2.0, 2, 1, 2, 0, None, None, None, None, None, 0, None) == 0


def test_prescaling_argument_checks_return_before_touching_the_device(lib):
    """laGP_sep_mle and laGP_prescale reject bad sizes and NULL pointers on the
    host (the fake pointers below are never dereferenced)."""
    from paper_1409_0074_gb300 import lagp
    L = lagp.load()
    assert L.laGP_sep_mle_workspace_bytes(1000, 8) >= 8 * 1000 * 1000
    for n, p in ((1, 8), (1025, 8), (100, 0), (100, 17)):
        assert L.laGP_sep_mle_workspace_bytes(n, p) == 0
    fake = 4096
    ws = L.laGP_sep_mle_workspace_bytes(100, 4)
    good = [fake, fake, 1000, 4, fake, 100, 1e-6, 1.0, 1e-3, 10.0, 50, fake, None, fake, ws, None]
    bad = [
        dict(i=0, v=None),           # design NULL
        dict(i=4, v=None),           # subset NULL
        dict(i=11, v=None),          # theta_out NULL
        dict(i=5, v=1),              # n_sub < 2
        dict(i=5, v=2000),           # n_sub > 1024
        dict(i=2, v=50),             # N < n_sub
        dict(i=7, v=0.0),            # theta0 <= 0
        dict(i=8, v=0.0),            # tmin <= 0
        dict(i=9, v=1e-4),           # tmax < tmin
        dict(i=10, v=0),             # maxit < 1
        dict(i=6, v=-1.0),           # g < 0
    ]
    for b in bad:
        a = list(good)
        a[b["i"]] = b["v"]
        assert L.laGP_sep_mle(*a) == -1, b
    a = list(good)
    a[14] = ws - 1
    assert L.laGP_sep_mle(*a) == -2
    assert L.laGP_prescale(fake, 10, 0, fake, fake, None) == -1
    assert L.laGP_prescale(None, 10, 3, fake, fake, None) == -1
    assert L.laGP_prescale(None, 0, 3, None, None, None) == 0
