/*
 * Plain, slow, FP64 CPU oracle of the epipolar consistency (ECC) hot path of
 * Preuhs, Manhart, Maier, "Fast Epipolar Consistency without the Need for Pseudo
 * Matrix Inverses" (arXiv 1806.02637).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - Eq. (4)/(5) projective algebra (meet, dual line matrix), source position
 *     from the rows of P, Eq. (13)/(14) line construction and, as the comparison
 *     path, the prior pseudo-inverse line l = P^{+T} E;
 *   - the Grangeat intermediate function S_lambda (Eq. 1) sampled on an
 *     (alpha, s) grid: cosine-weighted 2-D Radon transform of the projection by
 *     Joseph's method, half-step central difference in s, (D^2 + s^2)/D^2 weight;
 *   - the pair inconsistency d (Eq. 15), the Cauchy norm e (Eq. 16) and the sum
 *     over pairs (Eq. 17);
 *   - the gradient of that sum with respect to per-view rigid motion parameters,
 *     or to the entries of each view's projection matrix (geometric calibration,
 *     Introduction), by complex-step differentiation of the same code (no hand
 *     derivation).
 * Readings of the paper where it is silent are listed in the repository's design
 * notes; the ones that fix arithmetic are restated beside the code below.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no fast-math).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ real */
#define REAL double
#define SFX(name) name##_r
#define RE(x) (x)
#define R_SQRT(x) sqrt(x)
#define R_COS(x) cos(x)
#define R_SIN(x) sin(x)
#define R_ATAN2(y, x) atan2((y), (x))
#include "ecc_pair_generic.h"
#undef REAL
#undef SFX
#undef RE
#undef R_SQRT
#undef R_COS
#undef R_SIN
#undef R_ATAN2

/* --------------------------------------------------------------- complex */
static double complex catan2_step(double complex y, double complex x) {
    /* real part: atan2 of the real parts; imaginary part: first-order
     * derivative d atan2 = (x dy - y dx) / (x^2 + y^2) applied to the imaginary
     * parts (complex-step rule for a real-analytic function of two variables). */
    double xr = creal(x), yr = creal(y);
    double re = atan2(yr, xr);
    double im = (xr * cimag(y) - yr * cimag(x)) / (xr * xr + yr * yr);
    return re + I * im;
}
#define REAL double complex
#define SFX(name) name##_c
#define RE(x) creal(x)
#define R_SQRT(x) csqrt(x)
#define R_COS(x) ccos(x)
#define R_SIN(x) csin(x)
#define R_ATAN2(y, x) catan2_step((y), (x))
#include "ecc_pair_generic.h"
#undef REAL
#undef SFX
#undef RE
#undef R_SQRT
#undef R_COS
#undef R_SIN
#undef R_ATAN2

#define ORC_PI 3.14159265358979323846

/* ============================================================ exported algebra */

void orc_meet(const double a[4], const double b[4], double L[6]) { meet_r(a, b, L); }
void orc_dual(const double L[6], int corrected, double K[16]) { dual_r(L, corrected, K); }
void orc_source(const double P[12], double X[4]) { source_h_r(P, X); }
void orc_line_inf(const double P[12], const double E[4], double l[3]) { line_inf_r(P, E, l); }
int orc_line_pinv(const double P[12], const double E[4], double l[3]) { return line_pinv_r(P, E, l); }
void orc_apply_motion(const double P[12], const double th[6], double out[12]) { apply_motion_r(P, th, out); }

/* view record as 18 doubles: normalised P (12), C (3), up (3). */
int orc_view_setup(const double P[12], const double* theta, double out[18]) {
    double Pm[12];
    view_t_r v;
    if (theta) apply_motion_r(P, theta, Pm);
    else memcpy(Pm, P, sizeof Pm);
    if (view_setup_P_r(Pm, &v) != 0) return -1;
    memcpy(out, v.P, 12 * sizeof(double));
    memcpy(out + 12, v.C, 3 * sizeof(double));
    memcpy(out + 15, v.up, 3 * sizeof(double));
    return 0;
}

/* ================================================================ valid arcs */

/* Does the epipolar line of the pencil plane at kappa meet the detector of view vl? */
static int hits_at(const view_t_r* vl, const double w[3], const double v[3], const double Ca[3], double kappa,
                   int W, int H) {
    double E[4], l[3];
    plane_at_r(w, v, Ca, kappa, E);
    line_inf_r(vl->P, E, l);
    double cxd = 0.5 * (W - 1), cyd = 0.5 * (H - 1);
    double l3c = l[0] * cxd + l[1] * cyd + l[2];
    double h = sqrt(l[0] * l[0] + l[1] * l[1]);
    double s = -l3c / h;
    return fabs(s) <= 0.5 * W * fabs(l[0] / h) + 0.5 * H * fabs(l[1] / h);
}

/* The arc of pencil angles (mod pi) whose epipolar line meets the detector of
 * view vl, the other source being that of vo (N_kappa definition, Optimization
 * section).  Every line of the pencil passes through the epipole e = P_l C_o;
 * whether it meets the rectangle can only change where it passes a corner.  The
 * four corner planes P^T (e x x_c) give four angles; the arc between two
 * consecutive corner angles is tested at its midpoint; the valid set is the
 * complement of the one gap that misses (none: all of [-pi/2, pi/2)).
 * The lines through an epipole outside the rectangle that meet it form one
 * interval, so in exact arithmetic at most one gap misses.  A second miss can
 * only be a gap of (nearly) zero width: two corners on one line through the
 * epipole (an epipole at infinity along a detector edge, as for two sources on
 * one line parallel to the detector's columns).  That line meets the rectangle
 * along the edge (|s| equals the bound, a hit by reading R4), but its midpoint
 * test may round either way; so the widest missing gap is the one that misses.
 * Returns 0 and {lo, len}. */
static int arc_of_view(const view_t_r* vl, const view_t_r* vo, const double w[3], const double v[3],
                       const double Ca[3], int W, int H, double* lo, double* len) {
    double Xo[4] = {vo->C[0], vo->C[1], vo->C[2], 1.0};
    double e[3];
    for (int i = 0; i < 3; ++i)
        e[i] = vl->P[4 * i] * Xo[0] + vl->P[4 * i + 1] * Xo[1] + vl->P[4 * i + 2] * Xo[2] + vl->P[4 * i + 3];
    const double xs[4][3] = {{-0.5, -0.5, 1}, {W - 0.5, -0.5, 1}, {W - 0.5, H - 0.5, 1}, {-0.5, H - 0.5, 1}};
    double kap[4];
    for (int c = 0; c < 4; ++c) {
        double lc[3];
        cross3_r(e, xs[c], lc);
        double n[3];
        for (int j = 0; j < 3; ++j) n[j] = vl->P[j] * lc[0] + vl->P[4 + j] * lc[1] + vl->P[8 + j] * lc[2];
        double k = atan2(dot3_r(n, v), dot3_r(n, w));
        while (k >= 0.5 * ORC_PI) k -= ORC_PI;
        while (k < -0.5 * ORC_PI) k += ORC_PI;
        kap[c] = k;
    }
    for (int i = 1; i < 4; ++i) /* insertion sort */
        for (int j = i; j > 0 && kap[j] < kap[j - 1]; --j) {
            double t = kap[j];
            kap[j] = kap[j - 1];
            kap[j - 1] = t;
        }
    int miss = -1;
    double widest = -1.0;
    for (int g = 0; g < 4; ++g) {
        double a0 = kap[g], a1 = g < 3 ? kap[g + 1] : kap[0] + ORC_PI;
        if (!hits_at(vl, w, v, Ca, 0.5 * (a0 + a1), W, H) && a1 - a0 > widest) {
            widest = a1 - a0;
            miss = g;
        }
    }
    if (miss < 0) {
        *lo = -0.5 * ORC_PI;
        *len = ORC_PI;
        return 0;
    }
    double a0 = kap[miss], a1 = miss < 3 ? kap[miss + 1] : kap[0] + ORC_PI;
    double l0 = a1;
    while (l0 >= 0.5 * ORC_PI) l0 -= ORC_PI;
    *lo = l0;
    *len = ORC_PI - (a1 - a0);
    return 0;
}

/* Arcs of a pair: {sampled view (0 = a, 1 = b), lo_s, len_s, lo_o, len_o}.  The
 * shorter of the two views' arcs is sampled (ties: view a) and masked by the
 * other (reading of the kappa range; the paper gives K samples with step
 * Delta kappa and counts the planes that hit both detectors).  The two lengths
 * are equal in exact arithmetic for mirror-symmetric pairs (a circular trajectory,
 * also under shifts along its axis), so the tie is taken with a relative
 * tolerance of 1e-9 instead of being left to rounding. */
static int pair_arcs(const view_t_r* va, const view_t_r* vb, int W, int H, double arcs[5]) {
    double w[3], v[3], lo_a, len_a, lo_b, len_b;
    if (pair_frame_r(va, vb, w, v) != 0) return -1;
    if (arc_of_view(va, vb, w, v, va->C, W, H, &lo_a, &len_a) != 0) return -1;
    if (arc_of_view(vb, va, w, v, va->C, W, H, &lo_b, &len_b) != 0) return -1;
    if (len_a <= len_b + 1e-9 * fmax(len_a, len_b)) {
        arcs[0] = 0; arcs[1] = lo_a; arcs[2] = len_a; arcs[3] = lo_b; arcs[4] = len_b;
    } else {
        arcs[0] = 1; arcs[1] = lo_b; arcs[2] = len_b; arcs[3] = lo_a; arcs[4] = len_a;
    }
    return 0;
}

/* exported for tests: arcs of views (a, b) of a scan */
int orc_pair_arcs(const double Pa[12], const double Pb[12], const double* tha, const double* thb, int W, int H,
                  double arcs[5]) {
    view_t_r va, vb;
    double Pm[12];
    if (tha) apply_motion_r(Pa, tha, Pm); else memcpy(Pm, Pa, sizeof Pm);
    if (view_setup_P_r(Pm, &va) != 0) return -1;
    if (thb) apply_motion_r(Pb, thb, Pm); else memcpy(Pm, Pb, sizeof Pm);
    if (view_setup_P_r(Pm, &vb) != 0) return -1;
    return pair_arcs(&va, &vb, W, H, arcs);
}

/* exported for tests: look-up of one sinogram at one line. */
double orc_lookup(const double* sino, int n_alpha, int n_s, int W, int H, const double l[3], int* hit) {
    return lookup_r(sino, n_alpha, n_s, W, H, l, hit);
}

/* exported for tests: pencil frame of a pair */
int orc_pair_frame(const double Pa[12], const double Pb[12], double w[3], double v[3]) {
    view_t_r va, vb;
    if (view_setup_P_r(Pa, &va) != 0 || view_setup_P_r(Pb, &vb) != 0) return -1;
    return pair_frame_r(&va, &vb, w, v);
}

/* ========================================================== threading helper */

typedef struct {
    void (*fn)(void* ctx, long i);
    void* ctx;
    long begin, end;
} orc_job_t;

static void* orc_worker(void* p) {
    orc_job_t* j = (orc_job_t*)p;
    for (long i = j->begin; i < j->end; ++i) j->fn(j->ctx, i);
    return NULL;
}

/* Runs fn(ctx, i) for i in [0, n) on n_threads threads, contiguous chunks. */
static void orc_parallel_for(long n, int n_threads, void (*fn)(void*, long), void* ctx) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads > n) n_threads = (int)(n > 0 ? n : 1);
    pthread_t th[256];
    orc_job_t jobs[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].begin = n * t / n_threads;
        jobs[t].end = n * (t + 1) / n_threads;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    orc_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* =========================================================== dRadon/ds (K1) */

typedef struct {
    const double* P;
    const float* img;
    int W, H, n_alpha, n_s;
    double* out;
    double* gw; /* weighted images, n_views * H * W */
} radon_ctx_t;

/* Principal point (u0, v0) and source-detector distance D in pixels from the
 * normalised P = [M | t] (third row of M unit): u0 = m1.m3, v0 = m2.m3,
 * D = sqrt(|m1|^2 - u0^2) (square pixels, no skew). */
static void intrinsics(const double* Pn, double* u0, double* v0, double* D) {
    const double *m1 = Pn, *m2 = Pn + 4, *m3 = Pn + 8;
    *u0 = m1[0] * m3[0] + m1[1] * m3[1] + m1[2] * m3[2];
    *v0 = m2[0] * m3[0] + m2[1] * m3[1] + m2[2] * m3[2];
    *D = sqrt(m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2] - *u0 * *u0);
}

static void radon_weight_view(void* vctx, long lam) {
    radon_ctx_t* c = (radon_ctx_t*)vctx;
    view_t_r vw;
    if (view_setup_P_r(c->P + 12 * lam, &vw) != 0) return;
    double u0, v0, D;
    intrinsics(vw.P, &u0, &v0, &D);
    const float* g = c->img + (size_t)lam * c->H * c->W;
    double* gw = c->gw + (size_t)lam * c->H * c->W;
    for (int j = 0; j < c->H; ++j)
        for (int i = 0; i < c->W; ++i) {
            double du = i - u0, dv = j - v0;
            gw[(size_t)j * c->W + i] = (double)g[(size_t)j * c->W + i] * D / sqrt(D * D + du * du + dv * dv);
        }
}

/* Cosine-weighted projection, one row (fixed alpha) of the sinogram.
 * rho(alpha, sigma) = integral of the weighted projection along the line
 * (x - cx) cos(alpha) + (y - cy) sin(alpha) = sigma, by Joseph's method: for
 * |cos a| >= |sin a| step over the integer rows y and interpolate linearly in x,
 * with path length 1/|cos a| per row; otherwise step over the columns.  The
 * branch is decided on the integer m (4m <= n_alpha or 4m >= 3 n_alpha).
 * S(alpha, s_n) = [rho(s_n + ds/2) - rho(s_n - ds/2)] / ds * (D^2 + s_pp^2)/D^2,
 * s_pp the distance of the line from the principal point (Grangeat, Eq. 1). */
static void radon_row(void* vctx, long job) {
    radon_ctx_t* c = (radon_ctx_t*)vctx;
    long lam = job / c->n_alpha;
    int m = (int)(job % c->n_alpha);
    int W = c->W, H = c->H, n_s = c->n_s, n_alpha = c->n_alpha;
    view_t_r vw;
    if (view_setup_P_r(c->P + 12 * lam, &vw) != 0) return;
    double u0, v0, D;
    intrinsics(vw.P, &u0, &v0, &D);
    const double* gw = c->gw + (size_t)lam * H * W;
    double alpha = m * ORC_PI / n_alpha;
    double ca = cos(alpha), sa = sin(alpha);
    double cxd = 0.5 * (W - 1), cyd = 0.5 * (H - 1);
    double ds = sqrt((double)W * W + (double)H * H) / (n_s - 1);
    int rows_mode = (4 * m <= n_alpha) || (4 * m >= 3 * n_alpha);
    double* rho = (double*)malloc(sizeof(double) * (n_s + 1));
    for (int k = 0; k <= n_s; ++k) {
        double sigma = (k - 0.5 * n_s) * ds;
        double acc = 0.0;
        if (rows_mode) {
            for (int y = 0; y < H; ++y) {
                double x = cxd + (sigma - (y - cyd) * sa) / ca;
                double x0 = floor(x), f = x - x0;
                long i0 = (long)x0;
                double t0 = (i0 >= 0 && i0 < W) ? gw[(size_t)y * W + i0] : 0.0;
                double t1 = (i0 + 1 >= 0 && i0 + 1 < W) ? gw[(size_t)y * W + i0 + 1] : 0.0;
                acc += (1.0 - f) * t0 + f * t1;
            }
            acc /= fabs(ca);
        } else {
            for (int x = 0; x < W; ++x) {
                double y = cyd + (sigma - (x - cxd) * ca) / sa;
                double y0 = floor(y), f = y - y0;
                long j0 = (long)y0;
                double t0 = (j0 >= 0 && j0 < H) ? gw[(size_t)j0 * W + x] : 0.0;
                double t1 = (j0 + 1 >= 0 && j0 + 1 < H) ? gw[(size_t)(j0 + 1) * W + x] : 0.0;
                acc += (1.0 - f) * t0 + f * t1;
            }
            acc /= fabs(sa);
        }
        rho[k] = acc;
    }
    double* out = c->out + ((size_t)lam * n_alpha + m) * n_s;
    for (int n = 0; n < n_s; ++n) {
        double s_n = (n - 0.5 * (n_s - 1)) * ds;
        double spp = s_n - (u0 - cxd) * ca - (v0 - cyd) * sa;
        out[n] = (rho[n + 1] - rho[n]) / ds * (D * D + spp * spp) / (D * D);
    }
    free(rho);
}

/* S_lambda for all views: images [n_views][H][W] FP32, P [n_views][12] FP64,
 * output [n_views][n_alpha][n_s] FP64. */
int orc_radon_derivative(int n_views, const double* P, const float* images, int W, int H, int n_alpha, int n_s,
                         int n_threads, double* out) {
    if (n_views < 0 || W < 2 || H < 2 || n_alpha < 1 || n_s < 2) return -1;
    radon_ctx_t c = {P, images, W, H, n_alpha, n_s, out, NULL};
    c.gw = (double*)malloc(sizeof(double) * (size_t)n_views * W * H);
    if (!c.gw) return -2;
    orc_parallel_for(n_views, n_threads, radon_weight_view, &c);
    orc_parallel_for((long)n_views * n_alpha, n_threads, radon_row, &c);
    free(c.gw);
    return 0;
}

/* ================================================================ ECC (K2) */

typedef struct {
    int n_views;
    const double* P;
    const double* motion;
    const double* sino;
    int W, H, n_alpha, n_s, K;
    double c;
    const int* pairs;
    int construction;
    const double* arcs_in;
    double* arcs;
    double *d, *e;
    int* nk;
    int* mismatch;
    int* status;
    view_t_r* views;
    double* grad_pp; /* per pair 2 * npv partials (gradient mode) */
    int wrt_P;       /* gradient with respect to: 0 theta (npv = 6), 1 the entries of P (npv = 12) */
} ecc_ctx_t;

static void setup_view_job(void* vctx, long lam) {
    ecc_ctx_t* c = (ecc_ctx_t*)vctx;
    double Pm[12];
    if (c->motion) apply_motion_r(c->P + 12 * lam, c->motion + 6 * lam, Pm);
    else memcpy(Pm, c->P + 12 * lam, sizeof Pm);
    if (view_setup_P_r(Pm, &c->views[lam]) != 0) c->status[0] = -1;
}

/* Eq. (16): Cauchy norm; c <= 0 disables it. */
static double cauchy(double d, double c) { return c > 0 ? d / (1.0 + d / c) : d; }

static void pair_job(void* vctx, long p) {
    ecc_ctx_t* c = (ecc_ctx_t*)vctx;
    int a = c->pairs[2 * p], b = c->pairs[2 * p + 1];
    double* arcs = c->arcs + 5 * p;
    int mode = 0;
    if (c->arcs_in) {
        memcpy(arcs, c->arcs_in + 5 * p, 5 * sizeof(double));
        mode = 1;
    } else if (pair_arcs(&c->views[a], &c->views[b], c->W, c->H, arcs) != 0) {
        c->d[p] = 0; c->e[p] = 0; c->nk[p] = 0; c->status[p + 1] = -1;
        return;
    }
    size_t vs = (size_t)c->n_alpha * c->n_s;
    double sum;
    int nk, mm = 0;
    if (pair_sum_r(&c->views[a], &c->views[b], c->sino + vs * a, c->sino + vs * b, c->n_alpha, c->n_s, c->W, c->H,
                   c->K, arcs, c->construction, mode, &sum, &nk, &mm) != 0) {
        c->d[p] = 0; c->e[p] = 0; c->nk[p] = 0; c->status[p + 1] = -1;
        return;
    }
    double d = nk > 0 ? sum / nk : 0.0; /* Eq. (15) */
    c->d[p] = d;
    c->e[p] = cauchy(d, c->c);
    c->nk[p] = nk;
    c->mismatch[p] = mm;
}

static int* all_pairs(int n_views, int* n_pairs) {
    *n_pairs = n_views * (n_views - 1) / 2;
    int* pr = (int*)malloc(sizeof(int) * 2 * (size_t)(*n_pairs > 0 ? *n_pairs : 1));
    int q = 0;
    for (int a = 0; a < n_views; ++a)
        for (int b = a + 1; b < n_views; ++b) {
            pr[2 * q] = a;
            pr[2 * q + 1] = b;
            ++q;
        }
    return pr;
}

/* ECC over a list of pairs (NULL: all a < b in row-major order).
 *   P [n_views][12], motion [n_views][6] or NULL, sino [n_views][n_alpha][n_s] FP64.
 *   construction 0: Eq. (13)/(14); 1: pseudo-inverse.
 *   arcs_in [n_pairs][5] or NULL (NULL: computed, validity by the detector hit
 *   test; given: frozen arcs, validity by arc membership).
 *   Outputs per pair: d (Eq. 15), e (Eq. 16), N_kappa, arcs, and the number of
 *   samples where the two validity tests disagree; *total = sum of e in pair order
 *   (Eq. 17).  Returns 0, or the negated count of failed pairs. */
int orc_ecc(int n_views, const double* P, const double* motion, const double* sino, int W, int H, int n_alpha,
            int n_s, int K, double cauchy_c, const int* pairs, int n_pairs, int construction, const double* arcs_in,
            int n_threads, double* d, double* e, int* nk, double* arcs_out, int* mismatch, double* total) {
    int* own = NULL;
    if (!pairs) {
        own = all_pairs(n_views, &n_pairs);
        pairs = own;
    }
    ecc_ctx_t c;
    memset(&c, 0, sizeof c);
    c.n_views = n_views; c.P = P; c.motion = motion; c.sino = sino;
    c.W = W; c.H = H; c.n_alpha = n_alpha; c.n_s = n_s; c.K = K; c.c = cauchy_c;
    c.pairs = pairs; c.construction = construction; c.arcs_in = arcs_in;
    c.arcs = arcs_out; c.d = d; c.e = e; c.nk = nk; c.mismatch = mismatch;
    c.status = (int*)calloc((size_t)n_pairs + 1, sizeof(int));
    c.views = (view_t_r*)malloc(sizeof(view_t_r) * (size_t)(n_views > 0 ? n_views : 1));
    orc_parallel_for(n_views, n_threads, setup_view_job, &c);
    int bad = 0;
    if (c.status[0] != 0) bad = 1;
    else orc_parallel_for(n_pairs, n_threads, pair_job, &c);
    double t = 0.0;
    for (int p = 0; p < n_pairs && !bad; ++p) {
        t += e[p];
        if (c.status[p + 1] != 0) --bad;
    }
    *total = t;
    free(c.status);
    free(c.views);
    free(own);
    return bad > 0 ? -1 : bad;
}

/* ===================================================== gradient (complex step) */

static const double CSTEP = 1e-20;

static void to_complex_view(const view_t_r* r, view_t_c* z) {
    for (int i = 0; i < 12; ++i) z->P[i] = r->P[i];
    for (int i = 0; i < 3; ++i) { z->C[i] = r->C[i]; z->up[i] = r->up[i]; }
}

/* The first three rows of T(theta) = [R t; 0 1]: the motion model applied to P = [I | 0]. */
static void motion_rows(const double* th, double T[12]) {
    static const double I34[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    static const double zero[6] = {0, 0, 0, 0, 0, 0};
    apply_motion_r(I34, th ? th : zero, T);
}

/* Moved projection of a view whose parameter j is stepped by i*CSTEP: theta_j
 * (wrt_P = 0) or the entry P_j of the unmoved matrix (wrt_P = 1, P' = P T(theta)). */
static void stepped_projection(const ecc_ctx_t* c, int lam, int j, double complex Pm[12]) {
    const double* th = c->motion ? c->motion + 6 * lam : NULL;
    if (!c->wrt_P) {
        double complex tz[6];
        for (int i = 0; i < 6; ++i) tz[i] = th ? th[i] : 0.0;
        tz[j] += I * CSTEP;
        apply_motion_c(c->P + 12 * lam, tz, Pm);
        return;
    }
    double T[12];
    motion_rows(th, T);
    double complex Pz[12];
    for (int i = 0; i < 12; ++i) Pz[i] = c->P[12 * lam + i];
    Pz[j] += I * CSTEP;
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 4; ++col) {
            double complex acc = col == 3 ? Pz[4 * r + 3] : 0.0; /* row 4 of T is (0, 0, 0, 1) */
            for (int k = 0; k < 3; ++k) acc += Pz[4 * r + k] * T[4 * k + col];
            Pm[4 * r + col] = acc;
        }
}

static void grad_pair_job(void* vctx, long p) {
    ecc_ctx_t* c = (ecc_ctx_t*)vctx;
    const int npv = c->wrt_P ? 12 : 6;
    int ab[2] = {c->pairs[2 * p], c->pairs[2 * p + 1]};
    double* arcs = c->arcs + 5 * p;
    double* gp = c->grad_pp + 2 * npv * p;
    for (int i = 0; i < 2 * npv; ++i) gp[i] = 0.0;
    if (c->arcs_in) memcpy(arcs, c->arcs_in + 5 * p, 5 * sizeof(double));
    else if (pair_arcs(&c->views[ab[0]], &c->views[ab[1]], c->W, c->H, arcs) != 0) {
        c->status[p + 1] = -1;
        return;
    }
    size_t vs = (size_t)c->n_alpha * c->n_s;
    const double *sa = c->sino + vs * ab[0], *sb = c->sino + vs * ab[1];
    /* forward value (frozen-arc validity) */
    {
        double sum;
        int nk;
        if (pair_sum_r(&c->views[ab[0]], &c->views[ab[1]], sa, sb, c->n_alpha, c->n_s, c->W, c->H, c->K, arcs,
                       c->construction, 1, &sum, &nk, NULL) != 0) {
            c->status[p + 1] = -1;
            return;
        }
        double d = nk > 0 ? sum / nk : 0.0;
        c->d[p] = d;
        c->e[p] = cauchy(d, c->c);
        c->nk[p] = nk;
    }
    for (int side = 0; side < 2; ++side) {
        int lam = ab[side];
        for (int j = 0; j < npv; ++j) {
            view_t_c zv[2];
            double complex Pm[12];
            stepped_projection(c, lam, j, Pm);
            if (view_setup_P_c(Pm, &zv[side]) != 0) {
                c->status[p + 1] = -1;
                return;
            }
            to_complex_view(&c->views[ab[1 - side]], &zv[1 - side]);
            double complex sum;
            int nk;
            if (pair_sum_c(&zv[0], &zv[1], sa, sb, c->n_alpha, c->n_s, c->W, c->H, c->K, arcs, c->construction, 1,
                           &sum, &nk, NULL) != 0) {
                c->status[p + 1] = -1;
                return;
            }
            double complex d = nk > 0 ? sum / nk : 0.0;
            double complex e = c->c > 0 ? d / (1.0 + d / c->c) : d;
            gp[npv * side + j] = cimag(e) / CSTEP;
        }
    }
}

static int ecc_grad_impl(int n_views, const double* P, const double* motion, const double* sino, int W, int H,
                         int n_alpha, int n_s, int K, double cauchy_c, const int* pairs, int n_pairs,
                         int construction, const double* arcs_in, int n_threads, int wrt_P, double* d, double* e,
                         int* nk, double* arcs_out, double* total, double* grad) {
    const int npv = wrt_P ? 12 : 6;
    int* own = NULL;
    if (!pairs) {
        own = all_pairs(n_views, &n_pairs);
        pairs = own;
    }
    ecc_ctx_t c;
    memset(&c, 0, sizeof c);
    c.n_views = n_views; c.P = P; c.motion = motion; c.sino = sino;
    c.W = W; c.H = H; c.n_alpha = n_alpha; c.n_s = n_s; c.K = K; c.c = cauchy_c;
    c.pairs = pairs; c.construction = construction; c.arcs_in = arcs_in;
    c.arcs = arcs_out; c.d = d; c.e = e; c.nk = nk; c.wrt_P = wrt_P;
    c.status = (int*)calloc((size_t)n_pairs + 1, sizeof(int));
    c.views = (view_t_r*)malloc(sizeof(view_t_r) * (size_t)(n_views > 0 ? n_views : 1));
    c.grad_pp = (double*)malloc(sizeof(double) * 2 * npv * (size_t)(n_pairs > 0 ? n_pairs : 1));
    orc_parallel_for(n_views, n_threads, setup_view_job, &c);
    int bad = 0;
    if (c.status[0] != 0) bad = 1;
    else orc_parallel_for(n_pairs, n_threads, grad_pair_job, &c);
    memset(grad, 0, sizeof(double) * npv * (size_t)n_views);
    double t = 0.0;
    for (int p = 0; p < n_pairs && !bad; ++p) {
        if (c.status[p + 1] != 0) { --bad; continue; }
        t += e[p];
        for (int j = 0; j < npv; ++j) {
            grad[npv * pairs[2 * p] + j] += c.grad_pp[2 * npv * p + j];
            grad[npv * pairs[2 * p + 1] + j] += c.grad_pp[2 * npv * p + npv + j];
        }
    }
    *total = t;
    free(c.status);
    free(c.views);
    free(c.grad_pp);
    free(own);
    return bad > 0 ? -1 : bad;
}

/* Gradient of the total (Eq. 17) with respect to theta [n_views][6], with the
 * sampled arcs and the validity mask frozen at the evaluation point (or given in
 * arcs_in).  Also returns d, e, N_kappa per pair and the total. */
int orc_ecc_grad(int n_views, const double* P, const double* motion, const double* sino, int W, int H, int n_alpha,
                 int n_s, int K, double cauchy_c, const int* pairs, int n_pairs, int construction,
                 const double* arcs_in, int n_threads, double* d, double* e, int* nk, double* arcs_out, double* total,
                 double* grad) {
    return ecc_grad_impl(n_views, P, motion, sino, W, H, n_alpha, n_s, K, cauchy_c, pairs, n_pairs, construction,
                         arcs_in, n_threads, 0, d, e, nk, arcs_out, total, grad);
}

/* As orc_ecc_grad, with respect to the entries of each view's projection matrix:
 * grad_P [n_views][12] = d total / d P (the matrix before the view's motion; the
 * view uses P T(theta)).  Geometric calibration by the consistency (Introduction). */
int orc_ecc_grad_P(int n_views, const double* P, const double* motion, const double* sino, int W, int H,
                   int n_alpha, int n_s, int K, double cauchy_c, const int* pairs, int n_pairs, int construction,
                   const double* arcs_in, int n_threads, double* d, double* e, int* nk, double* arcs_out,
                   double* total, double* grad_P) {
    return ecc_grad_impl(n_views, P, motion, sino, W, H, n_alpha, n_s, K, cauchy_c, pairs, n_pairs, construction,
                         arcs_in, n_threads, 1, d, e, nk, arcs_out, total, grad_P);
}
