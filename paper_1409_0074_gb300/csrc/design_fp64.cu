// design_fp64.cu -- plain FP64 greedy local design and prediction, one CTA per
// predictive location (Gramacy & Haaland: Sec 2.2 greedy ALC design with the
// partitioned-inverse update, Eq. alc, Sec 4 ray search, Eq. predgp/preds2).
//
// This is the parity form.  Every floating-point operation is an explicitly
// rounded binary64 operation (__dadd_rn, __dmul_rn, ...) and every sum runs in
// ascending index order, the order a plain serial implementation of the
// paper's formulas uses; correlations use exp_cw.  Block reductions combine
// only exact operations (max/min with index tie-breaks).  The results are
// therefore reproducible bit for bit by any IEEE-754 implementation of the
// same formulas in the same order.
//
// State per location (shared memory): K_j^{-1} (n_max x n_max, leading
// dimension n_max), the selected coordinates S, k_j(x), selection flags over
// the N' candidates.  The exhaustive search keeps the candidates' correlation
// rows K(S_i, c_r) in a global cache laid out [i][r] so that consecutive
// threads (candidates) read consecutive addresses.
#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "kdtree.cuh"
#include "lagp_internal.h"

namespace lagp {

#define D64_THREADS 256
#define D64_WARPS (D64_THREADS / 32)

enum { SEARCH_EXHAUSTIVE = 0, SEARCH_RAY = 1 };

struct D64Params {
  const double* X;
  const double* Y;
  int p;
  const double* xref;
  int64_t M;
  const int32_t* cand;
  int nc_max;
  const int32_t* nc_loc;
  int n0, n_max;
  const int32_t* n_loc;
  double theta, g;
  const double* theta_loc;   // per-location lengthscale [M] or null
  int R;
  const double* lo;
  const double* hi;
  double* mean;
  double* s2;
  int32_t* selected;
  double* tie_gap;
  int32_t* nevals;
  double* Kc;          // exhaustive correlation cache [M][n_max][nc_max], or per CTA
                       // [grid][n_max][nc_max] when the locations come from a list
  unsigned* status;
  const int32_t* list; // locations to solve (list[0 .. *count - 1]), or null: CTA b solves b
  const unsigned* count;
  int full;            // ray snaps over all of X_N through the k-d tree
  KdView<double> kd;   // the tree in binary64 (full scope)
};

// ----- exact top-2 reductions ------------------------------------------------
struct Top2 {
  double b1, b2;
  int i1;
};

// larger value wins, ties to the lower index; b2 keeps the second largest value
__device__ __forceinline__ Top2 merge_max(Top2 a, Top2 b) {
  Top2 r;
  if (b.b1 > a.b1 || (b.b1 == a.b1 && b.i1 >= 0 && (a.i1 < 0 || b.i1 < a.i1))) {
    r.b1 = b.b1; r.i1 = b.i1; r.b2 = fmax(a.b1, b.b2);
  } else {
    r.b1 = a.b1; r.i1 = a.i1; r.b2 = fmax(a.b2, b.b1);
  }
  return r;
}
// smaller value wins, ties to the lower index; b2 keeps the second smallest value
__device__ __forceinline__ Top2 merge_min(Top2 a, Top2 b) {
  Top2 r;
  if (b.b1 < a.b1 || (b.b1 == a.b1 && b.i1 >= 0 && (a.i1 < 0 || b.i1 < a.i1))) {
    r.b1 = b.b1; r.i1 = b.i1; r.b2 = fmin(a.b1, b.b2);
  } else {
    r.b1 = a.b1; r.i1 = a.i1; r.b2 = fmin(a.b2, b.b1);
  }
  return r;
}

template <bool MAX>
__device__ Top2 block_top2(Top2 t, Top2* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    Top2 u;
    u.b1 = __shfl_xor_sync(0xffffffffu, t.b1, o);
    u.b2 = __shfl_xor_sync(0xffffffffu, t.b2, o);
    u.i1 = __shfl_xor_sync(0xffffffffu, t.i1, o);
    t = MAX ? merge_max(t, u) : merge_min(t, u);
  }
  if (lane == 0) scratch[warp] = t;
  __syncthreads();
  Top2 r = scratch[0];
  for (int w = 1; w < D64_WARPS; ++w) r = MAX ? merge_max(r, scratch[w]) : merge_min(r, scratch[w]);
  __syncthreads();
  return r;
}

// ----- per-location shared state ------------------------------------------------
struct Loc {
  double* Kinv;      // [n_max][n_max]
  double* S;         // [n_max][p]
  double* kx;        // [n_max]
  double* a;         // [n_max] update work (a, then gv)
  double* kvec;      // [n_max]
  double* xq;        // [p]
  double* lo;        // [p]
  double* hi;        // [p]
  double* rkz;       // [WARPS][n_max]
  double* ru;        // [WARPS][n_max]
  double* rz;        // [WARPS][p] evaluation point per warp
  double* rA;        // [R][p]
  double* rE;        // [R][p]
  double* ralc;      // [R]
  double* rs;        // [R]
  double* rgap;      // [R]
  double* xs;        // [p]
  double* scal;      // [4] broadcast scalars
  Top2* red;         // [WARPS]
  int* sel;          // [n_max] selected ranks (-1: not a candidate)
  int* gsel;         // [n_max] selected design indices
  int* stk;          // [KD_STACK] k-d tree walk (full scope): nodes
  double* bnd;       // [KD_STACK] and their box distances
  int* rnev;         // [R]
  int* starts;       // [R]
  int* iscal;        // [4]
  unsigned char* used;  // [nc_max]
  int j;
  double theta;         // this location's lengthscale
};

__device__ __forceinline__ const double* cand_coords(const D64Params& P, const int32_t* cl, int r) {
  return P.X + (int64_t)cl[r] * P.p;
}

// Adds candidate rank r (partitioned-inverse step).  Returns false when v <= 0.
template <int SEARCH>
__device__ bool add_point(const D64Params& P, Loc& L, const int32_t* cl, int nc, int gi, int r,
                          double* Kc_loc) {
  const int tid = threadIdx.x, p = P.p, j = L.j, ld = P.n_max;
  const double* c = P.X + (int64_t)gi * p;
  if (tid < p) L.S[j * p + tid] = c[tid];
  __syncthreads();
  for (int i = tid; i < j; i += blockDim.x) L.kvec[i] = corr64(L.S + i * p, L.S + j * p, p, L.theta);
  __syncthreads();
  for (int i = tid; i < j; i += blockDim.x) {
    const double* Ki = L.Kinv + i * ld;
    double acc = 0.0;
    for (int k = 0; k < j; ++k) acc = __dadd_rn(acc, __dmul_rn(Ki[k], L.kvec[k]));
    L.a[i] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    double ka = 0.0;
    for (int i = 0; i < j; ++i) ka = __dadd_rn(ka, __dmul_rn(L.kvec[i], L.a[i]));
    L.scal[0] = __dsub_rn(__dadd_rn(1.0, P.g), ka);
  }
  __syncthreads();
  const double v = L.scal[0];
  if (!(v > 0.0)) return false;
  for (int i = tid; i < j; i += blockDim.x) L.a[i] = __ddiv_rn(-L.a[i], v);
  __syncthreads();
  for (int e = tid; e < j * j; e += blockDim.x) {
    int i = e / j, k = e - i * j;
    L.Kinv[i * ld + k] = __dadd_rn(L.Kinv[i * ld + k], __dmul_rn(__dmul_rn(L.a[i], L.a[k]), v));
  }
  for (int i = tid; i < j; i += blockDim.x) {
    L.Kinv[i * ld + j] = L.a[i];
    L.Kinv[j * ld + i] = L.a[i];
  }
  if (tid == 0) {
    L.Kinv[j * ld + j] = __ddiv_rn(1.0, v);
    L.kx[j] = corr64(L.S + j * p, L.xq, p, L.theta);
    L.sel[j] = r;
    L.gsel[j] = gi;
    if (r >= 0) L.used[r] = 1;
  }
  if (SEARCH == SEARCH_EXHAUSTIVE) {
    double* row = Kc_loc + (int64_t)j * P.nc_max;
    for (int q = tid; q < nc; q += blockDim.x)
      row[q] = corr64(L.S + j * p, cand_coords(P, cl, q), p, L.theta);
  }
  __syncthreads();
  L.j = j + 1;
  return true;
}

// ----- exhaustive search (Sec 2.2; Eq. alc at every unselected candidate) -----
__device__ int search_exhaustive(const D64Params& P, Loc& L, const int32_t* cl, int nc,
                                 const double* Kc_loc, double* gap_out) {
  const int j = L.j, ld = P.n_max, p = P.p;
  const double onepg = __dadd_rn(1.0, P.g);
  Top2 t;
  t.b1 = -1.0; t.b2 = -1.0; t.i1 = -1;
  for (int r = threadIdx.x; r < nc; r += blockDim.x) {
    if (L.used[r]) continue;
    const double* kc = Kc_loc + r;
    double ku = 0.0, ukx = 0.0;
    for (int i = 0; i < j; ++i) {
      const double* Ki = L.Kinv + i * ld;
      double acc = 0.0;
      for (int k = 0; k < j; ++k) acc = __dadd_rn(acc, __dmul_rn(Ki[k], kc[(int64_t)k * P.nc_max]));
      ku = __dadd_rn(ku, __dmul_rn(kc[(int64_t)i * P.nc_max], acc));
      ukx = __dadd_rn(ukx, __dmul_rn(acc, L.kx[i]));
    }
    const double v = __dsub_rn(onepg, ku);
    const double num = __dsub_rn(ukx, corr64(cand_coords(P, cl, r), L.xq, p, L.theta));
    const double alc = (v > 0.0) ? __ddiv_rn(__dmul_rn(num, num), v) : 0.0;
    if (alc > t.b1) { t.b2 = t.b1; t.b1 = alc; t.i1 = r; }
    else if (alc > t.b2) t.b2 = alc;
  }
  Top2 b = block_top2<true>(t, L.red);
  *gap_out = (b.b1 > 0.0 && b.b2 >= 0.0) ? __ddiv_rn(__dsub_rn(b.b1, b.b2), b.b1) : 0.0;
  return b.i1;
}

// ----- ray search (Sec 4) --------------------------------------------------------
// ALC at the warp's point z = rz[warp] (warp-collective, exact oracle order).
__device__ double warp_alc(const D64Params& P, Loc& L, const double* z) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = L.j, ld = P.n_max, p = P.p;
  double* kz = L.rkz + warp * ld;
  double* u = L.ru + warp * ld;
  for (int i = lane; i < j; i += 32) kz[i] = corr64(L.S + i * p, z, p, L.theta);
  __syncwarp();
  for (int i = lane; i < j; i += 32) {
    const double* Ki = L.Kinv + i * ld;
    double acc = 0.0;
    for (int k = 0; k < j; ++k) acc = __dadd_rn(acc, __dmul_rn(Ki[k], kz[k]));
    u[i] = acc;
  }
  __syncwarp();
  double val = 0.0;
  if (lane == 0) {
    for (int i = 0; i < j; ++i) val = __dadd_rn(val, __dmul_rn(kz[i], u[i]));      // k'.u
  } else if (lane == 1) {
    for (int i = 0; i < j; ++i) val = __dadd_rn(val, __dmul_rn(u[i], L.kx[i]));    // u.k(x)
  } else if (lane == 2) {
    val = corr64(z, L.xq, p, L.theta);                                              // K(z, x)
  }
  const double ku = __shfl_sync(0xffffffffu, val, 0);
  const double ukx = __shfl_sync(0xffffffffu, val, 1);
  const double kap = __shfl_sync(0xffffffffu, val, 2);
  __syncwarp();
  const double v = __dsub_rn(__dadd_rn(1.0, P.g), ku);
  const double num = __dsub_rn(ukx, kap);
  return (v > 0.0) ? __ddiv_rn(__dmul_rn(num, num), v) : 0.0;
}

// -ALC at A + s (E - A) for the warp's ray.
__device__ double ray_f(const D64Params& P, Loc& L, const double* A, const double* E, double s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* z = L.rz + warp * P.p;
  if (lane < P.p) z[lane] = __dadd_rn(A[lane], __dmul_rn(s, __dsub_rn(E[lane], A[lane])));
  __syncwarp();
  return -warp_alc(P, L, z);
}

// Brent (1973) minimisation of the ray's -ALC on [0, 1]: golden-section steps
// safeguarding parabolic interpolation, tol = 2^-13, sqrt(eps) = 2^-26.
// Warp-uniform; returns f(xmin), writes xmin, evaluation count, smallest gap.
__device__ double brent_ray(const D64Params& P, Loc& L, const double* A, const double* E,
                            double* xmin, int* nev, double* mingap) {
  const double tol = 0x1p-13, sqrt_eps = 0x1p-26;
  const double golden = __dmul_rn(__dsub_rn(3.0, __dsqrt_rn(5.0)), 0.5);
  const double tol3 = __ddiv_rn(tol, 3.0);
  double a = 0.0, b = 1.0;
  double x = __dadd_rn(a, __dmul_rn(golden, __dsub_rn(b, a)));
  double w = x, v = x;
  double fx = ray_f(P, L, A, E, x);
  double fw = fx, fv = fx, d = 0.0, e = 0.0;
  int evals = 1;
  double gap = __longlong_as_double(0x7ff0000000000000ll);
  for (int it = 0; it < 1000; ++it) {
    const double m = __dmul_rn(__dadd_rn(a, b), 0.5);
    const double tol1 = __dadd_rn(__dmul_rn(sqrt_eps, fabs(x)), tol3);
    const double tol2 = __dmul_rn(2.0, tol1);
    if (fabs(__dsub_rn(x, m)) <= __dsub_rn(tol2, __dmul_rn(__dsub_rn(b, a), 0.5))) break;
    bool golden_step = true;
    if (fabs(e) > tol1) {
      double r = __dmul_rn(__dsub_rn(x, w), __dsub_rn(fx, fv));
      double q = __dmul_rn(__dsub_rn(x, v), __dsub_rn(fx, fw));
      double pn = __dsub_rn(__dmul_rn(__dsub_rn(x, v), q), __dmul_rn(__dsub_rn(x, w), r));
      q = __dmul_rn(2.0, __dsub_rn(q, r));
      if (q > 0.0) pn = -pn; else q = -q;
      const double e_prev = e;
      e = d;
      if (fabs(pn) < fabs(__dmul_rn(__dmul_rn(0.5, q), e_prev)) &&
          pn > __dmul_rn(q, __dsub_rn(a, x)) && pn < __dmul_rn(q, __dsub_rn(b, x))) {
        d = __ddiv_rn(pn, q);
        const double u_try = __dadd_rn(x, d);
        if (__dsub_rn(u_try, a) < tol2 || __dsub_rn(b, u_try) < tol2)
          d = (__dsub_rn(m, x) >= 0.0) ? tol1 : -tol1;
        golden_step = false;
      }
    }
    if (golden_step) {
      e = (x < m) ? __dsub_rn(b, x) : __dsub_rn(a, x);
      d = __dmul_rn(golden, e);
    }
    double u;
    if (fabs(d) >= tol1) u = __dadd_rn(x, d);
    else if (d >= 0.0) u = __dadd_rn(x, tol1);
    else u = __dsub_rn(x, tol1);
    const double fu = ray_f(P, L, A, E, u);
    ++evals;
    gap = fmin(gap, relgap64(fu, fx));
    if (fu <= fx) {
      if (u < x) b = x; else a = x;
      v = w; fv = fw;
      w = x; fw = fx;
      x = u; fx = fu;
    } else {
      if (u < x) a = u; else b = u;
      gap = fmin(gap, relgap64(fu, fw));
      if (fu <= fw || w == x) {
        v = w; fv = fw;
        w = u; fw = fu;
      } else {
        gap = fmin(gap, relgap64(fu, fv));
        if (fu <= fv || v == x || v == w) { v = u; fv = fu; }
      }
    }
  }
  *xmin = x;
  *nev = evals;
  *mingap = gap;
  return fx;
}

// Returns the chosen design index; *rank_out its candidate rank (-1: none).
__device__ int search_ray(const D64Params& P, Loc& L, const int32_t* cl, int nc, double* gap_out,
                          int* nev_out, int* rank_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = P.p, R = P.R, j = L.j;
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  if (tid == 0) {
    // starts: unselected candidates of rank k0, k0+1, ... (mod |U|)
    const int nU = nc - j;
    const int k0 = ray_offset(j, P.n0);
    for (int i = 0; i < R; ++i) {
      int target = (k0 + i) % nU, seen = 0, r = 0;
      for (; r < nc; ++r) {
        if (L.used[r]) continue;
        if (seen == target) break;
        ++seen;
      }
      L.starts[i] = r < nc ? r : nc - 1;
    }
  }
  __syncthreads();
  for (int i = warp; i < R; i += D64_WARPS) {
    double* A = L.rA + i * p;
    double* E = L.rE + i * p;
    const double* c = cand_coords(P, cl, L.starts[i]);
    if (lane < p) A[lane] = c[lane];
    __syncwarp();
    if (lane == 0) {
      double tau = 1.0;
      for (int k = 0; k < p; ++k) {
        const double bk = __dadd_rn(A[k], __dmul_rn(10.0, __dsub_rn(A[k], L.xq[k])));
        const double dk = __dsub_rn(bk, A[k]);
        double t;
        if (dk > 0.0) { t = __ddiv_rn(__dsub_rn(L.hi[k], A[k]), dk); if (t < tau) tau = t; }
        else if (dk < 0.0) { t = __ddiv_rn(__dsub_rn(L.lo[k], A[k]), dk); if (t < tau) tau = t; }
      }
      if (tau < 0.0) tau = 0.0;
      for (int k = 0; k < p; ++k) {
        const double bk = __dadd_rn(A[k], __dmul_rn(10.0, __dsub_rn(A[k], L.xq[k])));
        E[k] = __dadd_rn(A[k], __dmul_rn(tau, __dsub_rn(bk, A[k])));
      }
    }
    __syncwarp();
    const double alc0 = warp_alc(P, L, A);
    int evals = 1;
    double mg = inf, s_star = 0.0, alc_star = alc0;
    if (sqdist64(A, E, p) > 0.0) {
      double sb, bg;
      int ne;
      const double fb = brent_ray(P, L, A, E, &sb, &ne, &bg);
      evals += ne;
      mg = fmin(mg, bg);
      const double alc_b = -fb;
      mg = fmin(mg, relgap64(alc0, alc_b));
      if (!(alc0 >= alc_b)) { s_star = sb; alc_star = alc_b; }
    }
    if (lane == 0) {
      L.ralc[i] = alc_star;
      L.rs[i] = s_star;
      L.rgap[i] = mg;
      L.rnev[i] = evals;
    }
    __syncwarp();
  }
  __syncthreads();
  if (tid == 0) {
    int ib = 0;
    for (int i = 1; i < R; ++i) if (L.ralc[i] > L.ralc[ib]) ib = i;
    double mg = inf;
    int ev = 0;
    for (int i = 0; i < R; ++i) {
      mg = fmin(mg, L.rgap[i]);
      ev += L.rnev[i];
      if (i != ib) mg = fmin(mg, relgap64(L.ralc[i], L.ralc[ib]));
    }
    const double* A = L.rA + ib * p;
    const double* E = L.rE + ib * p;
    for (int k = 0; k < p; ++k) L.xs[k] = __dadd_rn(A[k], __dmul_rn(L.rs[ib], __dsub_rn(E[k], A[k])));
    L.scal[1] = mg;
    L.iscal[0] = ev;
  }
  __syncthreads();
  if (P.full) {
    // snap over all of X_N outside the design (warp 0 walks the k-d tree); the
    // step's starts are forbidden unless they equal x*; ties to the point
    // nearer x, then to the lower design index
    if (warp == 0) {
      const KdView<double>& V = P.kd;
      auto excluded = [&](int32_t gi, int64_t, bool allow_starts) -> bool {
        for (int i = 0; i < j; ++i) if (L.gsel[i] == gi) return true;
        if (allow_starts) return false;
        const double* c = P.X + (int64_t)gi * p;
        for (int t = 0; t < R; ++t) {
          if (cl[L.starts[t]] != gi) continue;
          for (int k = 0; k < p; ++k) if (c[k] != L.xs[k]) return true;
        }
        return false;
      };
      auto dist = [&](int64_t, int32_t gi) { return sqdist64(P.X + (int64_t)gi * p, L.xs, p); };
      auto distx = [&](int64_t, int32_t gi) { return sqdist64(P.X + (int64_t)gi * p, L.xq, p); };
      const KdTop<double> b = kd_nearest<double>(V, L.xs, 1e-12, L.stk, L.bnd, excluded, dist, distx);
      if (lane == 0) {
        L.iscal[1] = b.i1;
        L.iscal[2] = 0x7fffffff;
        double mg = L.scal[1];
        if (b.d2 < inf) mg = fmin(mg, relgap64(b.d1, b.d2));
        L.scal[2] = mg;
      }
    }
    __syncthreads();
    const int gi = L.iscal[1];
    for (int r = tid; r < nc; r += blockDim.x)
      if (cl[r] == gi) atomicMin(&L.iscal[2], r);
    __syncthreads();
    *rank_out = L.iscal[2] != 0x7fffffff ? L.iscal[2] : -1;
    *gap_out = L.scal[2];
    *nev_out = L.iscal[0];
    __syncthreads();
    return gi;
  }
  // snap: nearest allowed unselected candidate, ties to the lower rank
  Top2 t;
  t.b1 = inf; t.b2 = inf; t.i1 = -1;
  for (int r = tid; r < nc; r += blockDim.x) {
    if (L.used[r]) continue;
    const double* c = cand_coords(P, cl, r);
    bool forbidden = false;
    for (int i = 0; i < R; ++i) {
      if (L.starts[i] != r) continue;
      bool same = true;
      for (int k = 0; k < p; ++k) if (c[k] != L.xs[k]) { same = false; break; }
      if (!same) forbidden = true;
    }
    if (forbidden) continue;
    const double d = sqdist64(c, L.xs, p);
    if (d < t.b1) { t.b2 = t.b1; t.b1 = d; t.i1 = r; }
    else if (d < t.b2) t.b2 = d;
  }
  Top2 b = block_top2<false>(t, L.red);
  if (b.i1 < 0) {   // every unselected candidate is a start: snap over all of them
    t.b1 = inf; t.b2 = inf; t.i1 = -1;
    for (int r = tid; r < nc; r += blockDim.x) {
      if (L.used[r]) continue;
      const double d = sqdist64(cand_coords(P, cl, r), L.xs, p);
      if (d < t.b1) { t.b2 = t.b1; t.b1 = d; t.i1 = r; }
      else if (d < t.b2) t.b2 = d;
    }
    b = block_top2<false>(t, L.red);
  }
  double mg = L.scal[1];
  if (b.b2 < inf) mg = fmin(mg, relgap64(b.b1, b.b2));
  *gap_out = mg;
  *nev_out = L.iscal[0];
  *rank_out = b.i1;
  return b.i1 >= 0 ? cl[b.i1] : -1;
}

// ----- predictive equations (Eq. predgp, preds2) -------------------------------
__device__ void predict(const D64Params& P, Loc& L, const int32_t* cl, double* mean, double* s2) {
  const int tid = threadIdx.x, n = L.j, ld = P.n_max;
  double* yS = L.rkz;        // reuse ray buffers: [n] each
  double* ky = L.ru;
  double* kk = L.rkz + ld;
  for (int i = tid; i < n; i += blockDim.x) yS[i] = P.Y[L.gsel[i]];
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const double* Ki = L.Kinv + i * ld;
    double a1 = 0.0, a2 = 0.0;
    for (int k = 0; k < n; ++k) a1 = __dadd_rn(a1, __dmul_rn(Ki[k], yS[k]));
    for (int k = 0; k < n; ++k) a2 = __dadd_rn(a2, __dmul_rn(Ki[k], L.kx[k]));
    ky[i] = a1;
    kk[i] = a2;
  }
  __syncthreads();
  if (tid < 3) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      if (tid == 0) acc = __dadd_rn(acc, __dmul_rn(L.kx[i], ky[i]));   // mu
      if (tid == 1) acc = __dadd_rn(acc, __dmul_rn(yS[i], ky[i]));     // psi
      if (tid == 2) acc = __dadd_rn(acc, __dmul_rn(L.kx[i], kk[i]));   // k^T K^-1 k
    }
    L.scal[tid] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    *mean = L.scal[0];
    *s2 = __ddiv_rn(__dmul_rn(L.scal[1], __dsub_rn(__dadd_rn(1.0, P.g), L.scal[2])), (double)n);
  }
  __syncthreads();
}

__device__ __forceinline__ size_t align8(size_t x) { return (x + 7) & ~(size_t)7; }

// One location by the whole CTA (all threads call it); Kc_loc: the CTA's
// correlation cache (exhaustive search).
template <int SEARCH>
__device__ void design64_location(const D64Params& P, const int64_t loc, double* Kc_loc,
                                  unsigned char* smem) {
  const int tid = threadIdx.x, p = P.p, ld = P.n_max, R = P.R;
  const int nc = P.nc_loc ? P.nc_loc[loc] : P.nc_max;
  const int n = P.n_loc ? P.n_loc[loc] : P.n_max;
  const int32_t* cl = P.cand + loc * P.nc_max;

  Loc L;
  double* dp = reinterpret_cast<double*>(smem);
  L.Kinv = dp; dp += ld * ld;
  L.S = dp; dp += ld * p;
  L.kx = dp; dp += ld;
  L.a = dp; dp += ld;
  L.kvec = dp; dp += ld;
  L.xq = dp; dp += p;
  L.lo = dp; dp += p;
  L.hi = dp; dp += p;
  L.rkz = dp; dp += D64_WARPS * ld;
  L.ru = dp; dp += D64_WARPS * ld;
  L.rz = dp; dp += D64_WARPS * p;
  L.rA = dp; dp += R * p;
  L.rE = dp; dp += R * p;
  L.ralc = dp; dp += R;
  L.rs = dp; dp += R;
  L.rgap = dp; dp += R;
  L.xs = dp; dp += p;
  L.scal = dp; dp += 4;
  L.bnd = dp; dp += KD_STACK;
  L.red = reinterpret_cast<Top2*>(dp); dp += 3 * D64_WARPS;
  int* ip = reinterpret_cast<int*>(dp);
  L.sel = ip; ip += ld;
  L.gsel = ip; ip += ld;
  L.stk = ip; ip += KD_STACK;
  L.rnev = ip; ip += R;
  L.starts = ip; ip += R;
  L.iscal = ip; ip += 4;
  L.used = reinterpret_cast<unsigned char*>(ip);
  L.j = 0;
  L.theta = P.theta_loc ? P.theta_loc[loc] : P.theta;

  for (int i = tid; i < ld * ld; i += blockDim.x) L.Kinv[i] = 0.0;
  for (int r = tid; r < nc; r += blockDim.x) L.used[r] = 0;
  if (tid < p) {
    L.xq[tid] = P.xref[loc * p + tid];
    L.lo[tid] = P.lo[tid];
    L.hi[tid] = P.hi[tid];
  }
  if (P.tie_gap)
    for (int i = tid; i < ld; i += blockDim.x) P.tie_gap[loc * ld + i] = 0.0;
  if (P.nevals)
    for (int i = tid; i < ld; i += blockDim.x) P.nevals[loc * ld + i] = 0;
  __syncthreads();

  bool ok = (n >= P.n0) && (n <= nc) && (n <= ld);
  for (int r = 0; r < P.n0 && ok; ++r) ok = add_point<SEARCH>(P, L, cl, nc, cl[r], r, Kc_loc);
  for (int j = P.n0; j < n && ok; ++j) {
    double gap = 0.0;
    int ne = 0;
    int r, gi;
    if (SEARCH == SEARCH_EXHAUSTIVE) {
      r = search_exhaustive(P, L, cl, nc, Kc_loc, &gap);
      gi = r >= 0 ? cl[r] : -1;
    } else {
      gi = search_ray(P, L, cl, nc, &gap, &ne, &r);
    }
    if (tid == 0) {
      if (P.tie_gap) P.tie_gap[loc * ld + (j - P.n0)] = gap;
      if (P.nevals) P.nevals[loc * ld + (j - P.n0)] = ne;
    }
    ok = (gi >= 0) && add_point<SEARCH>(P, L, cl, nc, gi, r, Kc_loc);
  }
  if (ok) {
    predict(P, L, cl, P.mean + loc, P.s2 + loc);
  } else if (tid == 0) {
    P.mean[loc] = __longlong_as_double(0x7ff8000000000000ll);
    P.s2[loc] = __longlong_as_double(0x7ff8000000000000ll);
    atomicOr(P.status, LAGP_DEV_BAD_UPDATE);
  }
  if (P.selected)
    for (int i = tid; i < ld; i += blockDim.x)
      P.selected[loc * ld + i] = (i < L.j) ? L.gsel[i] : -1;
  __syncthreads();
}

// Without a list, CTA b solves location b.  With a list (the locations an
// FP32 form hands over for a binary64 re-solve), the CTAs stride over its
// *count entries, each with its own slot of the exhaustive cache.
template <int SEARCH>
__global__ void __launch_bounds__(D64_THREADS) design64(D64Params P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t ldc = (int64_t)P.n_max * P.nc_max;
  if (!P.list) {
    const int64_t loc = blockIdx.x;
    if (loc >= P.M) return;
    design64_location<SEARCH>(P, loc, SEARCH == SEARCH_EXHAUSTIVE ? P.Kc + loc * ldc : nullptr,
                              smem);
    return;
  }
  const unsigned items = *P.count;
  double* Kc_slot = SEARCH == SEARCH_EXHAUSTIVE ? P.Kc + (int64_t)blockIdx.x * ldc : nullptr;
  for (unsigned it = blockIdx.x; it < items; it += gridDim.x)
    design64_location<SEARCH>(P, (int64_t)P.list[it], Kc_slot, smem);
}

static size_t smem_design64(int n_max, int p, int nc_max, int R) {
  size_t d = (size_t)n_max * n_max + (size_t)n_max * p + 3 * n_max + 3 * p +
             2 * D64_WARPS * n_max + D64_WARPS * p + 2 * R * p + 3 * R + p + 4 +
             3 * D64_WARPS * ((sizeof(Top2) + 7) / 8) + KD_STACK;
  size_t i = 2 * (size_t)n_max + KD_STACK + 2 * R + 4;
  return d * 8 + i * 4 + nc_max + 16;
}

cudaError_t launch_design_fp64(const DesignArgs& a, int search, cudaStream_t s,
                               const int32_t* list, const unsigned* count, double* kc_slots,
                               int grid_cap) {
  D64Params P;
  P.X = a.X; P.Y = a.Y; P.p = a.p; P.xref = a.xref; P.M = a.M; P.cand = a.cand;
  P.nc_max = a.nc_max; P.nc_loc = a.nc_loc; P.n0 = a.n0; P.n_max = a.n_max; P.n_loc = a.n_loc;
  P.theta = a.theta; P.theta_loc = a.theta_loc; P.g = a.g; P.R = a.nrays; P.lo = a.ws->lo; P.hi = a.ws->hi;
  P.mean = a.mean; P.s2 = a.s2; P.selected = a.selected; P.tie_gap = a.tie_gap;
  P.nevals = a.nevals; P.Kc = list ? kc_slots : a.ws->state64; P.status = a.ws->status;
  P.list = list; P.count = count;
  P.full = a.full_scope;
  if (P.full) {
    const KdTree& t = a.ws->kd;
    P.kd.box = t.box64; P.kd.stride = a.p; P.kd.p = a.p; P.kd.D = t.D; P.kd.N = a.N;
    P.kd.perm = t.perm; P.kd.pts = a.X; P.kd.by_design = true;
  } else {
    std::memset(&P.kd, 0, sizeof(P.kd));
  }
  size_t sm = smem_design64(a.n_max, a.p, a.nc_max, a.nrays);
  const int64_t grid = list ? (a.M < grid_cap ? a.M : grid_cap) : a.M;
  if (grid <= 0) return cudaSuccess;
  cudaError_t err;
  if (search == SEARCH_EXHAUSTIVE) {
    err = cudaFuncSetAttribute(design64<SEARCH_EXHAUSTIVE>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    prof_begin("design64_exhaustive", s);
    design64<SEARCH_EXHAUSTIVE><<<(unsigned)grid, D64_THREADS, sm, s>>>(P);
    prof_end(s);
  } else {
    err = cudaFuncSetAttribute(design64<SEARCH_RAY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
    if (err != cudaSuccess) return err;
    prof_begin("design64_ray", s);
    design64<SEARCH_RAY><<<(unsigned)grid, D64_THREADS, sm, s>>>(P);
    prof_end(s);
  }
  return cudaGetLastError();
}

}  // namespace lagp
