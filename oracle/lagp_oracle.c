/*
 * lagp_oracle.c -- plain, slow FP64 CPU oracle for local approximate GP
 * prediction with greedy ALC local design, exhaustive or by ray search
 * (Gramacy & Haaland, "Speeding up neighborhood search in local Gaussian
 * process prediction", arXiv:1409.0074).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only users of this library.  The CUDA
 * product path shares no code with it and never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off (see oracle/build.py).  Every floating-point
 * operation below is one IEEE-754 binary64 operation, evaluated in the order
 * written; every sum runs in ascending index order.  Nothing is blocked, fused
 * or reordered beyond what the paper's equations state.
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes of the repository):
 *   R1  correlation exp(-sum_k (x_k - x'_k)^2 / theta), literally (Sec 2.1).
 *   R2  a self-correlation is 1 + g everywhere it appears (the K_eta of the
 *       ALC denominator, Sec 3.1, and K(x,x) in the predictive scale, Eq.
 *       preds2); cross-correlations carry no nugget.
 *   R3  the printed g_j(x') = K_j^{-1} k_j(x') / v_j lacks a minus sign; with the
 *       partitioned inverse the ALC integrand reduces to
 *       (k_j(x)^T K_j^{-1} k_j(x') - K(x',x))^2 / v_j(x').
 *   R4  ALC is the unscaled correlation-scale reduction (the psi_j / j factor
 *       is common to all candidates and dropped).
 *   R5  zero mean, y is not centred (Sec 2.1).
 *   R6  kNN orders pairs (d, i) lexicographically; ties go to the lower index.
 *   R7  exhaustive argmax ties go to the lower candidate rank; v <= 0 scores 0.
 *   R8  ray starts: t = j - n0 + 1, k = t mod floor(sqrt(t)), starts are the
 *       unselected candidates of 0-based rank k, k+1, ..., k+R-1 (mod |U|).
 *   R9  ray end = start + 10 (start - x), cut at the first face of the bounding
 *       box of the whole design X_N; a zero-length segment evaluates s = 0 only.
 *   R10 Brent's fmin on [0,1] with tol = eps^(1/4) (R's optimize default), then
 *       the s = 0 check keeps s = 0 when ALC(0) >= ALC(s*).
 *   R11 the best continuous point over all rays (ties: lower ray) is snapped
 *       once, to the nearest unselected candidate (ties: lower rank) that is
 *       not a ray start of this step, unless that start equals x* exactly;
 *       when every unselected candidate is a start, over all of them.
 *   R12 K_{n0}^{-1} is built by n0 partitioned-inverse steps from the empty
 *       design, the same update the greedy loop uses.
 *   R13 the variance output is sigma^2 of Eq. preds2 with df = n.
 *   R14 (unlimited ray scope, off by default; lagp_oracle_set_snap_scope(1))
 *       the snap of R11 searches all of X_N minus the current design instead
 *       of the unselected candidates (Sec 5 places no N' limit on rays): the
 *       nearest such point to x*, ray starts of the step forbidden unless
 *       equal to x*; ties go to the point nearer to x, then the lower index.
 *       Ray starts still come from the N' candidates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* exp: Cody & Waite (1980) argument reduction x = k ln2 + r, |r| <= ln2/2,   */
/* then the Taylor series of e^r to degree 13 by Horner's rule and scaling by */
/* 2^k.  Arguments below -708 (results below the normal range) return 0.      */
/* Written out here, rather than taken from libm, so that the GPU path can    */
/* compute bit-identical correlations from its own copy of the same method.   */
/* ------------------------------------------------------------------------- */
double lagp_oracle_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -708.0) return 0.0;
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_hi = 0x1.62e42fee00000p-1; /* 32 significant bits */
    const double ln2_lo = 0x1.a39ef35793c76p-33;
    double kd = rint(x * inv_ln2);
    double r = (x - kd * ln2_hi) - kd * ln2_lo;
    double s = 1.0 / 6227020800.0;              /* 1/13! */
    s = s * r + 1.0 / 479001600.0;              /* 1/12! */
    s = s * r + 1.0 / 39916800.0;               /* 1/11! */
    s = s * r + 1.0 / 3628800.0;                /* 1/10! */
    s = s * r + 1.0 / 362880.0;                 /* 1/9!  */
    s = s * r + 1.0 / 40320.0;                  /* 1/8!  */
    s = s * r + 1.0 / 5040.0;                   /* 1/7!  */
    s = s * r + 1.0 / 720.0;                    /* 1/6!  */
    s = s * r + 1.0 / 120.0;                    /* 1/5!  */
    s = s * r + 1.0 / 24.0;                     /* 1/4!  */
    s = s * r + 1.0 / 6.0;                      /* 1/3!  */
    s = s * r + 0.5;                            /* 1/2!  */
    s = s * r + 1.0;
    s = s * r + 1.0;
    return ldexp(s, (int)kd);
}

/* Squared Euclidean distance, ascending k. */
double lagp_oracle_sqdist(const double* a, const double* b, int p)
{
    double acc = 0.0;
    for (int k = 0; k < p; ++k) {
        double t = a[k] - b[k];
        acc = acc + t * t;
    }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* Rounding-noise probe ("ulp jitter").  When a seed is set, every correlation */
/* value below is multiplied by 1 + 2^-52 or 1 - 2^-52, chosen by a counter-   */
/* based generator (SplitMix64 of Steele, Lea & Flood 2014, applied to the     */
/* seed, the location's index and the call count), so that repeated runs with */
/* different seeds show how far rounding alone can move the results.  Seed 0  */
/* (the default) leaves the oracle exact as described above.                  */
/* ------------------------------------------------------------------------- */
static uint64_t g_jitter_seed = 0;
static __thread uint64_t t_jitter_key = 0;
static __thread uint64_t t_jitter_ctr = 0;

static uint64_t splitmix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

void lagp_oracle_set_jitter(uint64_t seed) { g_jitter_seed = seed; }

static void jitter_location(int64_t m)
{
    t_jitter_key = splitmix64(g_jitter_seed ^ splitmix64((uint64_t)m));
    t_jitter_ctr = 0;
}

/* Isotropic Gaussian correlation (Sec 2.1): exp(-||a-b||^2 / theta). */
static double corr(const double* a, const double* b, int p, double theta)
{
    double k = lagp_oracle_exp(-(lagp_oracle_sqdist(a, b, p) / theta));
    if (g_jitter_seed) {
        uint64_t h = splitmix64(t_jitter_key + t_jitter_ctr++);
        k = k * ((h & 1) ? (1.0 + 0x1p-52) : (1.0 - 0x1p-52));
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* kNN candidate set (Sec 2.2: the N' nearest neighbours of x in X_N).        */
/* ------------------------------------------------------------------------- */
typedef struct { double d; int64_t i; } pair_t;

static int pair_cmp(const void* pa, const void* pb)
{
    const pair_t* a = (const pair_t*)pa;
    const pair_t* b = (const pair_t*)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    return (a->i < b->i) ? -1 : (a->i > b->i);
}

/* idx[r], dist[r] (dist may be NULL) for ranks r = 0..nc-1. Returns 0 or -1. */
int lagp_oracle_knn(const double* X, int64_t N, int p, const double* x, int nc,
                    int32_t* idx, double* dist)
{
    if (nc < 0 || nc > N) return -1;
    pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(N > 0 ? N : 1));
    if (!pr) return -1;
    for (int64_t i = 0; i < N; ++i) {
        pr[i].d = lagp_oracle_sqdist(X + i * p, x, p);
        pr[i].i = i;
    }
    qsort(pr, (size_t)N, sizeof(pair_t), pair_cmp);
    for (int r = 0; r < nc; ++r) {
        idx[r] = (int32_t)pr[r].i;
        if (dist) dist[r] = pr[r].d;
    }
    free(pr);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Partitioned-inverse step (Sec 2.2; the g_j and v_j of Eq. alc, with the    */
/* sign of R3).  Kinv holds K_j^{-1} (j x j, leading dimension ld).  kvec is  */
/* k_j(x_new), the new point's correlations with the current design.  On      */
/* success Kinv holds K_{j+1}^{-1}:                                           */
/*   a = K_j^{-1} k,  v = (1 + g) - k.a,  gv = -a / v,                         */
/*   K_{j+1}^{-1} = [[K_j^{-1} + gv gv^T v, gv], [gv^T, 1/v]].                 */
/* Returns v; when v <= 0 (or NaN) Kinv is left unchanged.  work: j doubles.  */
/* ------------------------------------------------------------------------- */
double lagp_oracle_update(double* Kinv, int j, int ld, const double* kvec, double g,
                          double* work)
{
    double* a = work;
    for (int i = 0; i < j; ++i) {
        double acc = 0.0;
        for (int k = 0; k < j; ++k) acc = acc + Kinv[i * ld + k] * kvec[k];
        a[i] = acc;
    }
    double ka = 0.0;
    for (int i = 0; i < j; ++i) ka = ka + kvec[i] * a[i];
    double v = (1.0 + g) - ka;
    if (!(v > 0.0)) return v;
    for (int i = 0; i < j; ++i) a[i] = -a[i] / v;          /* a now holds gv */
    for (int i = 0; i < j; ++i)
        for (int k = 0; k < j; ++k)
            Kinv[i * ld + k] = Kinv[i * ld + k] + (a[i] * a[k]) * v;
    for (int i = 0; i < j; ++i) {
        Kinv[i * ld + j] = a[i];
        Kinv[j * ld + i] = a[i];
    }
    Kinv[j * ld + j] = 1.0 / v;
    return v;
}

/* ------------------------------------------------------------------------- */
/* ALC at a point z (integrand of Eq. alc with the reading R3/R4):           */
/*   kz = k_j(z), u = K_j^{-1} kz, v = (1+g) - kz.u,                          */
/*   ALC(z) = (u.kx - K(z,x))^2 / v, and 0 when v <= 0.                       */
/* S: j x p design coordinates; kx = k_j(x).  work: 2j doubles.  v_out and    */
/* num_out (may be NULL) receive v and the bracketed numerator.               */
/* ------------------------------------------------------------------------- */
double lagp_oracle_alc(const double* S, int j, int p, const double* Kinv, int ld,
                       const double* kx, const double* x, const double* z,
                       double theta, double g, double* work, double* v_out,
                       double* num_out)
{
    double* kz = work;
    double* u = work + j;
    for (int i = 0; i < j; ++i) kz[i] = corr(S + i * p, z, p, theta);
    for (int i = 0; i < j; ++i) {
        double acc = 0.0;
        for (int k = 0; k < j; ++k) acc = acc + Kinv[i * ld + k] * kz[k];
        u[i] = acc;
    }
    double ku = 0.0;
    for (int i = 0; i < j; ++i) ku = ku + kz[i] * u[i];
    double v = (1.0 + g) - ku;
    double ukx = 0.0;
    for (int i = 0; i < j; ++i) ukx = ukx + u[i] * kx[i];
    double num = ukx - corr(z, x, p, theta);
    if (v_out) *v_out = v;
    if (num_out) *num_out = num;
    if (!(v > 0.0)) return 0.0;
    return (num * num) / v;
}

/* Relative gap between two compared values: |a-b| / max(|a|,|b|). */
static double relgap(double a, double b)
{
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m == 0.0) return 0.0;
    return fabs(a - b) / m;
}

/* ------------------------------------------------------------------------- */
/* One-dimensional minimisation on [lo, hi]: Brent (1973), "Algorithms for    */
/* Minimization without Derivatives", ch. 5 -- golden-section search          */
/* safeguarding successive parabolic interpolation; the method behind R's     */
/* optimize (Sec 4).  Keeps the bracket [a,b], the best point x, the second   */
/* best w and the previous w in v.  Stops when |x - m| <= 2 tol1 - (b-a)/2    */
/* with m the bracket midpoint and tol1 = sqrt(eps)|x| + tol/3.  A trial      */
/* point is never closer than tol1 to x.  At most max_iter evaluations after  */
/* the first.  Returns f(xmin); *xmin, *nevals and *mingap (the smallest      */
/* relative gap among the comparisons of f values made) are written.          */
/* ------------------------------------------------------------------------- */
typedef double (*lagp_fun1)(double s, void* ctx);

double lagp_oracle_brent(lagp_fun1 f, void* ctx, double lo, double hi, double tol,
                         int max_iter, double* xmin, int* nevals, double* mingap)
{
    const double golden = (3.0 - sqrt(5.0)) * 0.5;
    const double sqrt_eps = 0x1p-26;              /* sqrt(2^-52) */
    double a = lo, b = hi;
    double x = a + golden * (b - a);
    double w = x, v = x;
    double fx = f(x, ctx);
    double fw = fx, fv = fx;
    double d = 0.0, e = 0.0;
    int evals = 1;
    double gap = INFINITY;

    for (int it = 0; it < max_iter; ++it) {
        double m = (a + b) * 0.5;
        double tol1 = sqrt_eps * fabs(x) + tol / 3.0;
        double tol2 = 2.0 * tol1;
        if (fabs(x - m) <= tol2 - (b - a) * 0.5) break;

        int golden_step = 1;
        if (fabs(e) > tol1) {
            /* parabola through (x,fx), (w,fw), (v,fv); its vertex is x + p/q */
            double r = (x - w) * (fx - fv);
            double q = (x - v) * (fx - fw);
            double pn = (x - v) * q - (x - w) * r;
            q = 2.0 * (q - r);
            if (q > 0.0) pn = -pn; else q = -q;
            double e_prev = e;
            e = d;
            /* accept when it moves less than half the step before last and
               lands strictly inside the bracket */
            if (fabs(pn) < fabs(0.5 * q * e_prev) && pn > q * (a - x) && pn < q * (b - x)) {
                d = pn / q;
                double u_try = x + d;
                if ((u_try - a) < tol2 || (b - u_try) < tol2) d = (m - x >= 0.0) ? tol1 : -tol1;
                golden_step = 0;
            }
        }
        if (golden_step) {
            e = (x < m) ? (b - x) : (a - x);
            d = golden * e;
        }
        double u;
        if (fabs(d) >= tol1) u = x + d;
        else if (d >= 0.0) u = x + tol1;
        else u = x - tol1;
        double fu = f(u, ctx);
        ++evals;

        double gg = relgap(fu, fx);
        if (gg < gap) gap = gg;
        if (fu <= fx) {
            if (u < x) b = x; else a = x;
            v = w; fv = fw;
            w = x; fw = fx;
            x = u; fx = fu;
        } else {
            if (u < x) a = u; else b = u;
            gg = relgap(fu, fw);
            if (gg < gap) gap = gg;
            if (fu <= fw || w == x) {
                v = w; fv = fw;
                w = u; fw = fu;
            } else {
                gg = relgap(fu, fv);
                if (gg < gap) gap = gg;
                if (fu <= fv || v == x || v == w) {
                    v = u; fv = fu;
                }
            }
        }
    }
    if (xmin) *xmin = x;
    if (nevals) *nevals = evals;
    if (mingap) *mingap = gap;
    return fx;
}

/* ------------------------------------------------------------------------- */
/* Ray search pieces (Sec 4).                                                 */
/* ------------------------------------------------------------------------- */

/* Round-robin offset k = t mod floor(sqrt(t)), t = j - n0 + 1 (Sec 4). */
int lagp_oracle_ray_k(int j, int n0)
{
    int t = j - n0 + 1;
    if (t < 1) return 0;
    int q = 1;
    while ((q + 1) * (q + 1) <= t) ++q;          /* integer floor(sqrt(t)) */
    return t % q;
}

/* Segment of a ray (Sec 4, reading R9): B = A + 10 (A - x); E = A + tau (B - A)
   with tau in [0,1] the largest value keeping E inside [lo,hi].  Writes E and
   returns tau. */
double lagp_oracle_ray_segment(const double* A, const double* x, const double* lo,
                               const double* hi, int p, double* E)
{
    double tau = 1.0;
    for (int k = 0; k < p; ++k) {
        double bk = A[k] + 10.0 * (A[k] - x[k]);
        double dk = bk - A[k];
        double t;
        if (dk > 0.0) { t = (hi[k] - A[k]) / dk; if (t < tau) tau = t; }
        else if (dk < 0.0) { t = (lo[k] - A[k]) / dk; if (t < tau) tau = t; }
    }
    if (tau < 0.0) tau = 0.0;
    for (int k = 0; k < p; ++k) {
        double bk = A[k] + 10.0 * (A[k] - x[k]);
        E[k] = A[k] + tau * (bk - A[k]);
    }
    return tau;
}

/* Point of a segment at parameter s: A + s (E - A). */
static void ray_point(const double* A, const double* E, double s, int p, double* z)
{
    for (int k = 0; k < p; ++k) z[k] = A[k] + s * (E[k] - A[k]);
}

/* ------------------------------------------------------------------------- */
/* One predictive location.                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int p, nc, n0, n;
    double theta, g;
    const double* x;      /* predictive location            */
    const double* lo;     /* bounding box of X_N            */
    const double* hi;
    double* cx;           /* nc x p candidate coordinates   */
    double* S;            /* n x p selected coordinates     */
    double* Kinv;         /* n x n, leading dimension n     */
    double* kx;           /* n: k_j(x)                      */
    double* work;         /* 4n + 4p doubles                */
    unsigned char* used;  /* nc flags                       */
    int32_t* sel;         /* n selected ranks (-1: not a candidate) */
    int32_t* gsel;        /* n selected design indices      */
    const double* X;      /* the design X_N (N x p)         */
    int64_t N;
    const int32_t* cidx;  /* nc candidate design indices    */
    unsigned char* gused; /* N flags of the design, or NULL (candidate scope) */
    int j;                /* current design size            */
} loc_t;

/* Scope of the ray search's snap (R11 / R14): 0 the unselected candidates,
   1 all of X_N outside the current design. */
static int g_snap_scope = 0;
void lagp_oracle_set_snap_scope(int scope) { g_snap_scope = scope; }

typedef struct { loc_t* L; const double* A; const double* E; double* z; double* work; } rayfun_t;

static double ray_negalc(double s, void* vctx)
{
    rayfun_t* c = (rayfun_t*)vctx;
    loc_t* L = c->L;
    ray_point(c->A, c->E, s, L->p, c->z);
    return -lagp_oracle_alc(L->S, L->j, L->p, L->Kinv, L->n, L->kx, L->x, c->z,
                            L->theta, L->g, c->work, NULL, NULL);
}

/* Adds design point gi (candidate rank r, or -1 when it is not a candidate)
   to the design (update, Sec 2.2). Returns v. */
static double add_point_g(loc_t* L, int64_t gi, int r)
{
    const int p = L->p, j = L->j;
    const double* c = L->X + gi * p;
    double* kvec = L->work + 2 * L->n;
    for (int i = 0; i < j; ++i) kvec[i] = corr(L->S + i * p, c, p, L->theta);
    double v = lagp_oracle_update(L->Kinv, j, L->n, kvec, L->g, L->work);
    if (!(v > 0.0)) return v;
    memcpy(L->S + (size_t)j * p, c, sizeof(double) * p);
    L->kx[j] = corr(c, L->x, p, L->theta);
    L->sel[j] = r;
    L->gsel[j] = (int32_t)gi;
    if (r >= 0) L->used[r] = 1;
    if (L->gused) L->gused[gi] = 1;
    L->j = j + 1;
    return v;
}

/* Adds candidate rank r to the design. */
static double add_point(loc_t* L, int r) { return add_point_g(L, L->cidx[r], r); }

/* Candidate rank of design point gi, or -1. */
static int rank_of(const loc_t* L, int64_t gi)
{
    for (int r = 0; r < L->nc; ++r) if (L->cidx[r] == gi) return r;
    return -1;
}

/* Exhaustive search over unselected candidates (Sec 2.2). */
static int search_exhaustive(loc_t* L, double* gap)
{
    double best = -1.0, second = -1.0;
    int rbest = -1;
    for (int r = 0; r < L->nc; ++r) {
        if (L->used[r]) continue;
        double a = lagp_oracle_alc(L->S, L->j, L->p, L->Kinv, L->n, L->kx, L->x,
                                   L->cx + (size_t)r * L->p, L->theta, L->g, L->work,
                                   NULL, NULL);
        if (a > best) { second = best; best = a; rbest = r; }
        else if (a > second) second = a;
    }
    *gap = (best > 0.0 && second >= 0.0) ? (best - second) / best : 0.0;
    return rbest;
}

/* Ray search (Sec 4) with R rays; returns the chosen design index and its
   candidate rank in *rank_out (-1 when the snap left the candidates). */
static int64_t search_ray(loc_t* L, int R, double* gap, int* nevals_out, int* rank_out)
{
    const int p = L->p;
    int* U = (int*)malloc(sizeof(int) * (size_t)L->nc);
    double* Abuf = (double*)malloc(sizeof(double) * (size_t)R * p * 2 + sizeof(double) * 2 * p);
    double* sbest = (double*)malloc(sizeof(double) * (size_t)R * 2);
    int* starts = (int*)malloc(sizeof(int) * (size_t)R);
    int nU = 0;
    for (int r = 0; r < L->nc; ++r) if (!L->used[r]) U[nU++] = r;
    int k0 = lagp_oracle_ray_k(L->j, L->n0);
    double mingap = INFINITY;
    int evals = 0;
    double* z = Abuf + (size_t)R * p * 2;
    double* xs = z + p;
    double* wk = (double*)malloc(sizeof(double) * 2 * (size_t)L->n);
    double* alcs = sbest + R;

    for (int i = 0; i < R; ++i) {
        int r = U[(k0 + i) % nU];
        starts[i] = r;
        const double* A = L->cx + (size_t)r * p;
        double* E = Abuf + (size_t)i * 2 * p;
        memcpy(E + p, A, sizeof(double) * p);     /* keep a copy of A */
        lagp_oracle_ray_segment(A, L->x, L->lo, L->hi, p, E);
        double alc0 = lagp_oracle_alc(L->S, L->j, p, L->Kinv, L->n, L->kx, L->x, A,
                                      L->theta, L->g, wk, NULL, NULL);
        ++evals;
        double len2 = lagp_oracle_sqdist(A, E, p);
        double s_star = 0.0, alc_star = alc0;
        if (len2 > 0.0) {
            rayfun_t ctx = { L, A, E, z, wk };
            double sb; int ne; double bg;
            double fb = lagp_oracle_brent(ray_negalc, &ctx, 0.0, 1.0, 0x1p-13, 1000,
                                          &sb, &ne, &bg);
            evals += ne;
            if (bg < mingap) mingap = bg;
            double alc_b = -fb;
            double g0 = relgap(alc0, alc_b);
            if (g0 < mingap) mingap = g0;
            if (!(alc0 >= alc_b)) { s_star = sb; alc_star = alc_b; }
        }
        sbest[i] = s_star;
        alcs[i] = alc_star;
    }
    /* best continuous point over rays, ties to the lower ray index */
    int ib = 0;
    for (int i = 1; i < R; ++i) if (alcs[i] > alcs[ib]) ib = i;
    for (int i = 0; i < R; ++i) {
        if (i == ib) continue;
        double gg = relgap(alcs[i], alcs[ib]);
        if (gg < mingap) mingap = gg;
    }
    const double* Ab = Abuf + (size_t)ib * 2 * p + p;
    const double* Eb = Abuf + (size_t)ib * 2 * p;
    ray_point(Ab, Eb, sbest[ib], p, xs);

    /* snap: nearest unselected candidate, ray starts forbidden unless equal to x* */
    int rbest = -1;
    int64_t gbest = -1;
    double d1 = INFINITY, d2 = INFINITY;
    if (L->gused) {
        /* R14: the nearest point of X_N outside the design */
        double dxb = INFINITY;
        for (int pass = 0; pass < 2 && gbest < 0; ++pass) {
            for (int64_t c = 0; c < L->N; ++c) {
                if (L->gused[c]) continue;
                const double* cc = L->X + c * p;
                if (pass == 0) {
                    int forbidden = 0;
                    for (int i = 0; i < R; ++i) {
                        if (L->cidx[starts[i]] != c) continue;
                        int same = 1;
                        for (int k = 0; k < p; ++k) if (cc[k] != xs[k]) { same = 0; break; }
                        if (!same) forbidden = 1;
                    }
                    if (forbidden) continue;
                }
                double d = lagp_oracle_sqdist(cc, xs, p);
                if (d < d1) {
                    d2 = d1; d1 = d; gbest = c; dxb = lagp_oracle_sqdist(cc, L->x, p);
                } else if (d == d1) {
                    d2 = d;
                    double dx = lagp_oracle_sqdist(cc, L->x, p);
                    if (dx < dxb) { gbest = c; dxb = dx; }
                } else if (d < d2) {
                    d2 = d;
                }
            }
        }
        rbest = rank_of(L, gbest);
    }
    for (int u = 0; u < nU && !L->gused; ++u) {
        int r = U[u];
        const double* c = L->cx + (size_t)r * p;
        int forbidden = 0;
        for (int i = 0; i < R; ++i) {
            if (starts[i] != r) continue;
            int same = 1;
            for (int k = 0; k < p; ++k) if (c[k] != xs[k]) { same = 0; break; }
            if (!same) forbidden = 1;
        }
        if (forbidden) continue;
        double d = lagp_oracle_sqdist(c, xs, p);
        if (d < d1) { d2 = d1; d1 = d; rbest = r; }
        else if (d < d2) d2 = d;
    }
    if (rbest < 0 && !L->gused) {  /* every unselected point is a start: snap over U */
        for (int u = 0; u < nU; ++u) {
            double d = lagp_oracle_sqdist(L->cx + (size_t)U[u] * p, xs, p);
            if (d < d1) { d2 = d1; d1 = d; rbest = U[u]; }
            else if (d < d2) d2 = d;
        }
    }
    if (d2 < INFINITY) {
        double gg = relgap(d1, d2);
        if (gg < mingap) mingap = gg;
    }
    *gap = mingap;
    *nevals_out = evals;
    free(U); free(Abuf); free(sbest); free(starts); free(wk);
    *rank_out = rbest;
    if (!L->gused) gbest = rbest >= 0 ? L->cidx[rbest] : -1;
    return gbest;
}

/* Predictive equations (Eq. predgp, preds2) on the final design. */
static void predict(loc_t* L, const double* yS, double* mean, double* s2)
{
    const int n = L->j, ld = L->n;
    double* ky = L->work;
    double* kk = L->work + L->n;
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = acc + L->Kinv[i * ld + k] * yS[k];
        ky[i] = acc;
    }
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = acc + L->Kinv[i * ld + k] * L->kx[k];
        kk[i] = acc;
    }
    double mu = 0.0, psi = 0.0, q = 0.0;
    for (int i = 0; i < n; ++i) mu = mu + L->kx[i] * ky[i];
    for (int i = 0; i < n; ++i) psi = psi + yS[i] * ky[i];
    for (int i = 0; i < n; ++i) q = q + L->kx[i] * kk[i];
    *mean = mu;
    *s2 = (psi * ((1.0 + L->g) - q)) / (double)n;
}

/* Status bits per location. */
#define ST_BAD_UPDATE 1

/*
 * Whole path for one location: kNN candidates, n0 nearest start, greedy
 * selection for j = n0..n-1 (exhaustive: search = 0, ray: search = 1), then
 * the predictive equations.  sel_out[n] receives design indices in selection
 * order; gap_out[n-n0] the smallest relative gap of the step's decisions;
 * nevals_out[n-n0] the ALC evaluations a ray step made (0 when exhaustive).
 */
/* Allocates a location's state; the candidates must be filled in. */
static void loc_init(loc_t* L, const double* X, int64_t N, int p, const double* lo,
                     const double* hi, const double* x, int n0, int n, int nc, double theta,
                     double g, int32_t* cidx)
{
    L->p = p; L->nc = nc; L->n0 = n0; L->n = n; L->theta = theta; L->g = g;
    L->x = x; L->lo = lo; L->hi = hi; L->X = X; L->N = N; L->cidx = cidx;
    L->cx = (double*)malloc(sizeof(double) * (size_t)nc * p);
    L->S = (double*)malloc(sizeof(double) * (size_t)n * p);
    L->Kinv = (double*)calloc((size_t)n * n, sizeof(double));
    L->kx = (double*)malloc(sizeof(double) * (size_t)n);
    L->work = (double*)malloc(sizeof(double) * (size_t)(4 * n + 4 * p));
    L->used = (unsigned char*)calloc((size_t)nc, 1);
    L->sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    L->gsel = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    L->gused = g_snap_scope ? (unsigned char*)calloc((size_t)N, 1) : NULL;
    L->j = 0;
    lagp_oracle_knn(X, N, p, x, nc, cidx, NULL);
    for (int r = 0; r < nc; ++r)
        memcpy(L->cx + (size_t)r * p, X + (int64_t)cidx[r] * p, sizeof(double) * p);
}

static void loc_free(loc_t* L)
{
    free(L->cx); free(L->S); free(L->Kinv); free(L->kx); free(L->work);
    free(L->used); free(L->sel); free(L->gsel); free(L->gused);
}

/* One greedy step: the next point by the chosen search, added to the design.
   Returns 0 or ST_BAD_UPDATE. */
static int greedy_step(loc_t* L, int search, int nrays, double* gap, int* ne);

/*
 * Whole path for one location: kNN candidates, n0 nearest start, greedy
 * selection for j = n0..n-1 (exhaustive: search = 0, ray: search = 1), then
 * the predictive equations.  sel_out[n] receives design indices in selection
 * order; gap_out[n-n0] the smallest relative gap of the step's decisions;
 * nevals_out[n-n0] the ALC evaluations a ray step made (0 when exhaustive).
 */
static int one_location(const double* X, const double* Y, int64_t N, int p,
                        const double* lo, const double* hi, const double* x,
                        int n0, int n, int nc, double theta, double g, int search,
                        int nrays, double* mean, double* s2, int32_t* sel_out,
                        double* gap_out, int32_t* nevals_out)
{
    int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
    loc_t L;
    loc_init(&L, X, N, p, lo, hi, x, n0, n, nc, theta, g, cidx);
    int status = 0;

    for (int r = 0; r < n0 && !status; ++r)
        if (!(add_point(&L, r) > 0.0)) status |= ST_BAD_UPDATE;

    for (int j = n0; j < n && !status; ++j) {
        double gap = 0.0;
        int ne = 0;
        status |= greedy_step(&L, search, nrays, &gap, &ne);
        gap_out[j - n0] = gap;
        nevals_out[j - n0] = ne;
    }

    if (!status) {
        double* yS = (double*)malloc(sizeof(double) * (size_t)n);
        for (int i = 0; i < n; ++i) yS[i] = Y[L.gsel[i]];
        predict(&L, yS, mean, s2);
        free(yS);
        for (int i = 0; i < n; ++i) sel_out[i] = L.gsel[i];
    } else {
        *mean = NAN;
        *s2 = NAN;
        for (int i = 0; i < n; ++i) sel_out[i] = (i < L.j) ? L.gsel[i] : -1;
    }
    free(cidx);
    loc_free(&L);
    return status;
}

static int greedy_step(loc_t* L, int search, int nrays, double* gap, int* ne)
{
    int r = -1;
    int64_t gi = -1;
    if (search == 0) {
        r = search_exhaustive(L, gap);
        gi = r >= 0 ? L->cidx[r] : -1;
    } else {
        gi = search_ray(L, nrays, gap, ne, &r);
    }
    if (gi < 0 || !(add_point_g(L, gi, r) > 0.0)) return ST_BAD_UPDATE;
    return 0;
}

/* Bounding box of the design, per dimension. */
void lagp_oracle_bbox(const double* X, int64_t N, int p, double* lo, double* hi)
{
    for (int k = 0; k < p; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < p; ++k) {
            double v = X[i * p + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
}

/*
 * Batch driver over M locations (independent; OpenMP over locations when
 * nthreads != 1).  n_arr / nc_arr may be NULL (then n, nc apply to all);
 * otherwise they give each location's own n and N_close.  Row strides of
 * sel_out, gap_out and nevals_out are n_stride (>= every n).
 * status_out[M] receives per-location status bits.  Returns the number of
 * threads used.
 */
int lagp_oracle_predict(const double* X, const double* Y, int64_t N, int p,
                        const double* Xref, int64_t M, int n0, int n, int nc,
                        const int32_t* n_arr, const int32_t* nc_arr, int n_stride,
                        double theta, double g, int search, int nrays, double* mean,
                        double* s2, int32_t* sel_out, double* gap_out,
                        int32_t* nevals_out, int32_t* status_out, int nthreads)
{
    double* lo = (double*)malloc(sizeof(double) * (size_t)p);
    double* hi = (double*)malloc(sizeof(double) * (size_t)p);
    lagp_oracle_bbox(X, N, p, lo, hi);
    int used_threads = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t m = 0; m < M; ++m) {
#ifdef _OPENMP
        if (m == 0) used_threads = omp_get_num_threads();
#endif
        int nm = n_arr ? n_arr[m] : n;
        int ncm = nc_arr ? nc_arr[m] : nc;
        int R = nrays > 0 ? nrays : p;
        jitter_location(m);
        for (int i = 0; i < n_stride; ++i) {
            sel_out[m * n_stride + i] = -1;
            gap_out[m * n_stride + i] = 0.0;
            nevals_out[m * n_stride + i] = 0;
        }
        status_out[m] = one_location(X, Y, N, p, lo, hi, Xref + m * p, n0, nm, ncm, theta,
                                     g, search, R, mean + m, s2 + m, sel_out + m * n_stride,
                                     gap_out + m * n_stride, nevals_out + m * n_stride);
    }
    (void)nthreads;
    free(lo);
    free(hi);
    return used_threads;
}

/* ------------------------------------------------------------------------- */
/* Local inference for the lengthscale (Sec 2.1, Eq. gpk; Sec 5: local designs */
/* are coupled with Newton-like maximisation of the local posterior of theta, */
/* optionally followed by a second-stage re-design at the estimate).          */
/*                                                                            */
/* Readings (listed in the design notes):                                     */
/*   M1  the local posterior of theta is the marginal likelihood of Eq. gpk   */
/*       (reference prior on tau^2) with a flat prior on theta over a         */
/*       caller-given range [tmin, tmax]; the nugget g stays fixed.           */
/*   M2  K_theta carries 1 + g on its diagonal (R2), so dK/dtheta has a zero  */
/*       diagonal.                                                            */
/*   M3  Newton's method on theta from a start theta0, safeguarded: a bracket */
/*       [a, b] around the maximiser is kept from the sign of the first       */
/*       derivative, and a step that leaves the bracket, or is taken where    */
/*       the curvature is not negative, is replaced by the bracket's midpoint.*/
/*       It stops when a step or the bracket is below tol * theta, or after   */
/*       maxit iterations; a maximiser on a bound returns that bound.         */
/*   M4  two stages: the design built at theta0 gives theta_1; the design     */
/*       rebuilt at theta_1 gives theta_2; the prediction uses the last       */
/*       estimate on the last design (one stage: theta_1 on the first design).*/
/* ------------------------------------------------------------------------- */

/* log Gamma(n/2) for an integer n >= 1 from Gamma(1) = 1, Gamma(1/2) = sqrt(pi)
   and Gamma(z + 1) = z Gamma(z). */
static double log_gamma_half(int n)
{
    double s = 0.0;
    if (n % 2 == 0) {
        for (int i = 1; i < n / 2; ++i) s = s + log((double)i);
    } else {
        s = 0.5 * log(M_PI);
        for (int i = 0; i < (n - 1) / 2; ++i) s = s + log(0.5 + (double)i);
    }
    return s;
}

/* Plain Cholesky K = C C^T of an n x n symmetric matrix (row-major); C is
   written to the lower triangle of Cm.  Returns -1 when K is not positive
   definite. */
static int cholesky(const double* K, int n, double* Cm)
{
    for (int j = 0; j < n; ++j) {
        double s = K[j * n + j];
        for (int k = 0; k < j; ++k) s = s - Cm[j * n + k] * Cm[j * n + k];
        if (!(s > 0.0)) return -1;
        const double cjj = sqrt(s);
        Cm[j * n + j] = cjj;
        for (int i = j + 1; i < n; ++i) {
            double t = K[i * n + j];
            for (int k = 0; k < j; ++k) t = t - Cm[i * n + k] * Cm[j * n + k];
            Cm[i * n + j] = t / cjj;
        }
        for (int i = 0; i < j; ++i) Cm[i * n + j] = 0.0;
    }
    return 0;
}

/* K^{-1} = C^{-T} C^{-1} from the Cholesky factor; Ci receives C^{-1}. */
static void chol_inverse(const double* Cm, int n, double* Ci, double* Kinv)
{
    for (int i = 0; i < n * n; ++i) Ci[i] = 0.0;
    for (int c = 0; c < n; ++c) {              /* column c of C^{-1}: C w = e_c */
        for (int i = c; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) t = t - Cm[i * n + k] * Ci[k * n + c];
            Ci[i * n + c] = t / Cm[i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double t = 0.0;
            for (int k = 0; k < n; ++k) t = t + Ci[k * n + i] * Ci[k * n + j];
            Kinv[i * n + j] = t;
        }
}

/*
 * log p(y | K_theta) of Eq. gpk for the design S (n x p) and responses y:
 *   log Gamma(n/2) - (n/2) log(2 pi) - (1/2) log|K| - (n/2) log(psi / 2),
 *   psi = y^T K^{-1} y,
 * and, when d1 / d2 are not NULL, its first and second derivatives in theta:
 *   K'_ab = K_ab d_ab / theta^2, K''_ab = K_ab (d_ab^2 / theta^4 - 2 d_ab / theta^3),
 *   l'  = -(1/2) tr(K^{-1} K') - (n/2) psi' / psi,
 *   l'' = -(1/2) [tr(K^{-1} K'') - tr(K^{-1} K' K^{-1} K')]
 *         - (n/2) [psi'' / psi - (psi' / psi)^2],
 *   psi' = -alpha^T K' alpha, psi'' = 2 (K' alpha)^T K^{-1} (K' alpha) - alpha^T K'' alpha,
 *   alpha = K^{-1} y.
 * Returns NAN when K is not positive definite.
 */
double lagp_oracle_loglik(const double* S, const double* y, int n, int p, double theta,
                          double g, double* d1, double* d2)
{
    const size_t nn = (size_t)n * n;
    double* D = (double*)malloc(sizeof(double) * nn);      /* squared distances */
    double* K = (double*)malloc(sizeof(double) * nn);
    double* Cm = (double*)malloc(sizeof(double) * nn);
    double* Ci = (double*)malloc(sizeof(double) * nn);
    double* Ki = (double*)malloc(sizeof(double) * nn);
    double* K1 = (double*)malloc(sizeof(double) * nn);
    double* K2 = (double*)malloc(sizeof(double) * nn);
    double* A = (double*)malloc(sizeof(double) * nn);      /* K^{-1} K' */
    double* al = (double*)malloc(sizeof(double) * (size_t)n);
    double* u = (double*)malloc(sizeof(double) * (size_t)n);
    double ll = NAN;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const double d = lagp_oracle_sqdist(S + (size_t)a * p, S + (size_t)b * p, p);
            const double k = lagp_oracle_exp(-d / theta);
            D[a * n + b] = d;
            K[a * n + b] = (a == b) ? 1.0 + g : k;
            K1[a * n + b] = (a == b) ? 0.0 : k * d / (theta * theta);
            K2[a * n + b] = (a == b) ? 0.0
                : k * (d * d / (theta * theta * theta * theta) - 2.0 * d / (theta * theta * theta));
        }
    if (cholesky(K, n, Cm) == 0) {
        chol_inverse(Cm, n, Ci, Ki);
        double logdet = 0.0;
        for (int i = 0; i < n; ++i) logdet = logdet + 2.0 * log(Cm[i * n + i]);
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int k = 0; k < n; ++k) t = t + Ki[i * n + k] * y[k];
            al[i] = t;
        }
        double psi = 0.0;
        for (int i = 0; i < n; ++i) psi = psi + y[i] * al[i];
        const double hn = 0.5 * (double)n;
        ll = log_gamma_half(n) - hn * log(2.0 * M_PI) - 0.5 * logdet - hn * log(psi / 2.0);
        if (d1 || d2) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double t = 0.0;
                    for (int k = 0; k < n; ++k) t = t + Ki[i * n + k] * K1[k * n + j];
                    A[i * n + j] = t;
                }
            double tr1 = 0.0, tr2 = 0.0, tr11 = 0.0;
            for (int i = 0; i < n; ++i) tr1 = tr1 + A[i * n + i];
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) tr2 = tr2 + Ki[i * n + k] * K2[k * n + i];
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) tr11 = tr11 + A[i * n + k] * A[k * n + i];
            for (int i = 0; i < n; ++i) {                  /* u = K' alpha */
                double t = 0.0;
                for (int k = 0; k < n; ++k) t = t + K1[i * n + k] * al[k];
                u[i] = t;
            }
            double ak1a = 0.0, ak2a = 0.0, uku = 0.0;
            for (int i = 0; i < n; ++i) ak1a = ak1a + al[i] * u[i];
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) ak2a = ak2a + al[i] * K2[i * n + k] * al[k];
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) uku = uku + u[i] * Ki[i * n + k] * u[k];
            const double ps1 = -ak1a;
            const double ps2 = 2.0 * uku - ak2a;
            if (d1) *d1 = -0.5 * tr1 - hn * ps1 / psi;
            if (d2) *d2 = -0.5 * (tr2 - tr11) - hn * (ps2 / psi - (ps1 / psi) * (ps1 / psi));
        }
    } else {
        if (d1) *d1 = NAN;
        if (d2) *d2 = NAN;
    }
    free(D); free(K); free(Cm); free(Ci); free(Ki); free(K1); free(K2); free(A); free(al); free(u);
    return ll;
}

/* Safeguarded Newton maximisation of lagp_oracle_loglik over [tmin, tmax]
   (reading M3).  *iters (may be NULL) receives the iterations taken. */
double lagp_oracle_mle_theta(const double* S, const double* y, int n, int p, double theta0,
                             double g, double tmin, double tmax, double tol, int maxit,
                             int* iters)
{
    double a = tmin, b = tmax;
    double t = theta0 < a ? a : (theta0 > b ? b : theta0);
    int it = 0;
    while (it < maxit) {
        ++it;
        double d1 = 0.0, d2 = 0.0;
        const double ll = lagp_oracle_loglik(S, y, n, p, t, g, &d1, &d2);
        if (!(ll == ll) || !(d1 == d1)) break;
        if (d1 > 0.0) a = t; else b = t;
        if (b - a <= tol * t) break;
        double tn = t - d1 / d2;
        if (!(d2 < 0.0) || !(tn > a && tn < b)) tn = 0.5 * (a + b);
        const double step = tn - t;
        t = tn;
        if (fabs(step) <= tol * t) break;
    }
    if (iters) *iters = it;
    return t;
}

/* Resets a location to the empty design at lengthscale theta. */
static void reset_location(loc_t* L, double theta)
{
    L->theta = theta;
    if (L->gused)
        for (int i = 0; i < L->j; ++i) L->gused[L->gsel[i]] = 0;
    L->j = 0;
    memset(L->used, 0, (size_t)L->nc);
    for (int i = 0; i < L->n * L->n; ++i) L->Kinv[i] = 0.0;
}

/* Greedy design at L->theta from the empty design (as in one_location). */
static int build_design(loc_t* L, int search, int nrays)
{
    for (int r = 0; r < L->n0; ++r)
        if (!(add_point(L, r) > 0.0)) return ST_BAD_UPDATE;
    for (int j = L->n0; j < L->n; ++j) {
        double gap = 0.0;
        int ne = 0;
        if (greedy_step(L, search, nrays, &gap, &ne)) return ST_BAD_UPDATE;
    }
    return 0;
}

/*
 * One location with local inference for theta (readings M1-M4): stages
 * designs and estimates, then the predictive equations at the last estimate
 * on the last design.  K^{-1} at the estimate is rebuilt by the partitioned
 * update over the design in selection order (R12).
 */
static int one_location_mle(const double* X, const double* Y, int64_t N, int p,
                            const double* lo, const double* hi, const double* x, int n0, int n,
                            int nc, double theta0, double g, double tmin, double tmax,
                            int search, int nrays, int stages, double* mean, double* s2,
                            double* theta_out, int32_t* sel_out)
{
    int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
    loc_t L;
    loc_init(&L, X, N, p, lo, hi, x, n0, n, nc, theta0, g, cidx);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* orank = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* yS = (double*)malloc(sizeof(double) * (size_t)n);
    int status = 0;

    double theta = theta0;
    for (int s = 0; s < stages && !status; ++s) {
        reset_location(&L, theta);
        status = build_design(&L, search, nrays);
        if (status) break;
        for (int i = 0; i < n; ++i) yS[i] = Y[L.gsel[i]];
        theta = lagp_oracle_mle_theta(L.S, yS, n, p, theta, g, tmin, tmax, 1e-10, 200, NULL);
    }
    if (!status) {
        memcpy(order, L.gsel, sizeof(int32_t) * (size_t)n);
        memcpy(orank, L.sel, sizeof(int32_t) * (size_t)n);
        reset_location(&L, theta);
        for (int i = 0; i < n && !status; ++i)
            if (!(add_point_g(&L, order[i], orank[i]) > 0.0)) status = ST_BAD_UPDATE;
    }
    if (!status) {
        predict(&L, yS, mean, s2);
        *theta_out = theta;
        for (int i = 0; i < n; ++i) sel_out[i] = L.gsel[i];
    } else {
        *mean = NAN;
        *s2 = NAN;
        *theta_out = NAN;
        for (int i = 0; i < n; ++i) sel_out[i] = -1;
    }
    free(cidx); free(order); free(orank); free(yS);
    loc_free(&L);
    return status;
}

/* Batch driver of one_location_mle over M locations (OpenMP over locations
   when nthreads != 1); sel_out is [M][n].  Returns the threads used. */
int lagp_oracle_predict_mle(const double* X, const double* Y, int64_t N, int p,
                            const double* Xref, int64_t M, int n0, int n, int nc,
                            double theta0, double g, double tmin, double tmax, int search,
                            int nrays, int stages, double* mean, double* s2, double* theta_out,
                            int32_t* sel_out, int32_t* status_out, int nthreads)
{
    double* lo = (double*)malloc(sizeof(double) * (size_t)p);
    double* hi = (double*)malloc(sizeof(double) * (size_t)p);
    lagp_oracle_bbox(X, N, p, lo, hi);
    int used_threads = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t m = 0; m < M; ++m) {
#ifdef _OPENMP
        if (m == 0) used_threads = omp_get_num_threads();
#endif
        const int R = nrays > 0 ? nrays : p;
        status_out[m] = one_location_mle(X, Y, N, p, lo, hi, Xref + m * p, n0, n, nc, theta0,
                                         g, tmin, tmax, search, R, stages, mean + m, s2 + m,
                                         theta_out + m, sel_out + m * n);
    }
    (void)nthreads;
    free(lo);
    free(hi);
    return used_threads;
}
