/*
 * Analytic cone-beam projector for seeded synthetic phantoms (input generation
 * only; it holds none of the consistency method's arithmetic).
 *
 * Each detector value is the line integral of the phantom along the ray from the
 * source through the pixel centre (the cone-beam model of the Grangeat section):
 *   Gaussian blob  A exp(-|x - mu|^2 / (2 sigma^2)):  A sqrt(2 pi) sigma exp(-dist^2 / (2 sigma^2)),
 *                  dist = distance of mu from the ray;
 *   uniform ellipsoid (density rho, centre c, rotation R, semi-axes a, b, c):
 *                  rho * chord length, from the quadratic in ellipsoid coordinates.
 *
 * Primitive record, 17 doubles: {type (0 blob, 1 ellipsoid), value (A or rho),
 * centre x y z, sigma or semi-axes a b c (3), rotation R row-major (9)}.
 * P [n_views][12] maps world mm to pixel coordinates (pixel centres on integers).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>

typedef struct {
    int n_views, W, H, n_prim;
    const double* P;
    const double* prim;
    float* out;
    int n_threads, tid;
} proj_ctx_t;

static int inv3(const double M[9], double R[9]) {
    double c0 = M[4] * M[8] - M[5] * M[7], c1 = M[5] * M[6] - M[3] * M[8], c2 = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * c0 + M[1] * c1 + M[2] * c2;
    if (det == 0.0) return -1;
    R[0] = c0 / det; R[1] = (M[2] * M[7] - M[1] * M[8]) / det; R[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    R[3] = c1 / det; R[4] = (M[0] * M[8] - M[2] * M[6]) / det; R[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    R[6] = c2 / det; R[7] = (M[1] * M[6] - M[0] * M[7]) / det; R[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    return 0;
}

static double ray_integral(const double src[3], const double dir[3], const double* prim, int n_prim) {
    double total = 0.0;
    for (int k = 0; k < n_prim; ++k) {
        const double* q = prim + 17 * k;
        double d[3] = {src[0] - q[2], src[1] - q[3], src[2] - q[4]};
        if (q[0] == 0.0) {
            double sig = q[5];
            double t = -(d[0] * dir[0] + d[1] * dir[1] + d[2] * dir[2]);
            double px = d[0] + t * dir[0], py = d[1] + t * dir[1], pz = d[2] + t * dir[2];
            double dist2 = px * px + py * py + pz * pz;
            total += q[1] * sqrt(2.0 * M_PI) * sig * exp(-dist2 / (2.0 * sig * sig));
        } else {
            /* a ray that misses the bounding sphere (radius: the largest semi-axis)
               misses the ellipsoid: skip the exact chord (same result, cheaper) */
            double rad = q[5] > q[6] ? q[5] : q[6];
            rad = rad > q[7] ? rad : q[7];
            double t = -(d[0] * dir[0] + d[1] * dir[1] + d[2] * dir[2]);
            double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (dd - t * t > rad * rad * (1.0 + 1e-9)) continue;
            const double* R = q + 8;
            double p[3], r[3];
            for (int i = 0; i < 3; ++i) {
                /* ellipsoid frame: R^T (x - c), then divide by the semi-axes */
                p[i] = (R[0 + i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2]) / q[5 + i];
                r[i] = (R[0 + i] * dir[0] + R[3 + i] * dir[1] + R[6 + i] * dir[2]) / q[5 + i];
            }
            double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double pr = p[0] * r[0] + p[1] * r[1] + p[2] * r[2];
            double pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
            double disc = pr * pr - rr * (pp - 1.0);
            if (disc > 0.0) total += q[1] * 2.0 * sqrt(disc) / rr;
        }
    }
    return total;
}

static void* proj_worker(void* arg) {
    proj_ctx_t* c = (proj_ctx_t*)arg;
    for (int lam = c->tid; lam < c->n_views; lam += c->n_threads) {
        const double* P = c->P + 12 * lam;
        double M[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]}, Mi[9];
        if (inv3(M, Mi) != 0) continue;
        double t[3] = {P[3], P[7], P[11]};
        double src[3];
        for (int i = 0; i < 3; ++i) src[i] = -(Mi[3 * i] * t[0] + Mi[3 * i + 1] * t[1] + Mi[3 * i + 2] * t[2]);
        float* img = c->out + (size_t)lam * c->W * c->H;
        for (int j = 0; j < c->H; ++j)
            for (int i = 0; i < c->W; ++i) {
                double dir[3];
                for (int k = 0; k < 3; ++k) dir[k] = Mi[3 * k] * i + Mi[3 * k + 1] * j + Mi[3 * k + 2];
                double nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
                for (int k = 0; k < 3; ++k) dir[k] /= nd;
                img[(size_t)j * c->W + i] = (float)ray_integral(src, dir, c->prim, c->n_prim);
            }
    }
    return NULL;
}

int synth_project(int n_views, const double* P, int W, int H, const double* prim, int n_prim, int n_threads,
                  float* out) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 128) n_threads = 128;
    pthread_t th[128];
    proj_ctx_t ctx[128];
    for (int t = 0; t < n_threads; ++t) {
        ctx[t] = (proj_ctx_t){n_views, W, H, n_prim, P, prim, out, n_threads, t};
        if (t > 0) pthread_create(&th[t], NULL, proj_worker, &ctx[t]);
    }
    proj_worker(&ctx[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Line integral at one continuous detector point (u, v) of one view (for tests). */
double synth_ray_value(const double* P, double u, double v, const double* prim, int n_prim) {
    double M[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]}, Mi[9];
    if (inv3(M, Mi) != 0) return NAN;
    double t[3] = {P[3], P[7], P[11]}, src[3], dir[3];
    for (int i = 0; i < 3; ++i) src[i] = -(Mi[3 * i] * t[0] + Mi[3 * i + 1] * t[1] + Mi[3 * i + 2] * t[2]);
    for (int k = 0; k < 3; ++k) dir[k] = Mi[3 * k] * u + Mi[3 * k + 1] * v + Mi[3 * k + 2];
    double nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int k = 0; k < 3; ++k) dir[k] /= nd;
    return ray_integral(src, dir, prim, n_prim);
}
