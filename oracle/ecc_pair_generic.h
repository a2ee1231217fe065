/*
 * Generic (scalar-type independent) part of the FP64 CPU oracle: the projective
 * algebra, the per-view set-up, the epipolar line construction, the sinogram
 * look-up and the per-pair consistency sum.
 *
 * TEST INFRASTRUCTURE ONLY (see ecc_oracle.c).  Included twice by ecc_oracle.c:
 * once with REAL = double (the plain forward evaluation) and once with
 * REAL = double complex (complex-step differentiation, used as the oracle of the
 * gradient).  Every branch decision (floor, fold, validity) is taken on real
 * parts, so the imaginary part carries exactly the derivative of the smooth
 * pieces while the decisions stay those of the real evaluation.
 *
 * Macros expected from the includer:
 *   REAL            scalar type
 *   SFX(name)       name mangling for this instantiation
 *   RE(x)           real part as double
 *   R_SQRT(x), R_COS(x), R_SIN(x)
 *   R_ATAN2(y, x)   two-argument arctangent
 */

typedef struct {
    REAL P[12];   /* projection matrix scaled so that the third row of M has unit norm and det M > 0 */
    REAL C[3];    /* source position (inhomogeneous world coordinates) */
    REAL up[3];   /* unit detector "up" axis: m3 x m1, normalised */
} SFX(view_t);

/* Eq. (4): meet of two planes a, b -> Pluecker coordinates (p,q,r,s,t,u). */
static void SFX(meet)(const REAL a[4], const REAL b[4], REAL L[6]) {
    L[0] = a[2] * b[3] - a[3] * b[2]; /* p */
    L[1] = a[1] * b[3] - a[3] * b[1]; /* q */
    L[2] = a[1] * b[2] - a[2] * b[1]; /* r */
    L[3] = a[0] * b[3] - a[3] * b[0]; /* s */
    L[4] = a[0] * b[2] - a[2] * b[0]; /* t */
    L[5] = a[0] * b[1] - a[1] * b[0]; /* u */
}

/* Eq. (5): dual line matrix L_K (row-major 4x4).  corrected = 1 applies the sign
 * reading of Eq. (5): the Pluecker coordinate p enters with the opposite sign,
 * which makes L_K annihilate both planes of the meet.  corrected = 0 is the
 * matrix exactly as printed (kept so that a test can show the printed form fails
 * the incidence identities). */
static void SFX(dual)(const REAL L[6], int corrected, REAL K[16]) {
    REAL p = corrected ? -L[0] : L[0];
    REAL q = L[1], r = L[2], s = L[3], t = L[4], u = L[5];
    K[0] = 0;   K[1] = -p;  K[2] = -q;  K[3] = r;
    K[4] = p;   K[5] = 0;   K[6] = s;   K[7] = -t;
    K[8] = q;   K[9] = -s;  K[10] = 0;  K[11] = u;
    K[12] = -r; K[13] = t;  K[14] = -u; K[15] = 0;
}

/* x = L_K p : the point common to the line and the plane p (Eq. 5). */
static void SFX(mat4_vec)(const REAL K[16], const REAL p[4], REAL x[4]) {
    for (int i = 0; i < 4; ++i)
        x[i] = K[4 * i + 0] * p[0] + K[4 * i + 1] * p[1] + K[4 * i + 2] * p[2] + K[4 * i + 3] * p[3];
}

/* Source position as the meet of the three rows of P, each a plane through the
 * source: x = L_K(meet(P1, P2)) P3 (Optimized Algorithm section, after Eq. 14).
 * Homogeneous 4-vector. */
static void SFX(source_h)(const REAL P[12], REAL X[4]) {
    REAL L[6], K[16];
    SFX(meet)(P + 0, P + 4, L);
    SFX(dual)(L, 1, K);
    SFX(mat4_vec)(K, P + 8, X);
}

/* Eq. (13) + Eq. (14): the epipolar line of plane E in the view with projection P,
 * through the line at infinity of E:  L = meet(E, pi_inf),  [l]_x = P L_K P^T,
 * l = (S12, S20, S01). */
static void SFX(line_inf)(const REAL P[12], const REAL E[4], REAL l[3]) {
    const REAL pinf[4] = {0, 0, 0, 1};
    REAL L[6], K[16], PK[12], S[9];
    SFX(meet)(E, pinf, L);
    SFX(dual)(L, 1, K);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 4; ++k) acc += P[4 * i + k] * K[4 * k + j];
            PK[4 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 4; ++k) acc += PK[4 * i + k] * P[4 * j + k];
            S[3 * i + j] = acc;
        }
    l[0] = S[1 * 3 + 2];
    l[1] = S[2 * 3 + 0];
    l[2] = S[0 * 3 + 1];
}

/* Prior method (Aichert et al., Optimized Algorithm section), kept as a comparison
 * path: l = P^{+T} E with the pseudo-inverse P^+ = P^T (P P^T)^{-1}, i.e.
 * l = (P P^T)^{-1} P E, with a 3x3 inverse by cofactors.  P must be normalised to
 * det M > 0 so that the line keeps the orientation of the infinity construction. */
static int SFX(line_pinv)(const REAL P[12], const REAL E[4], REAL l[3]) {
    REAL A[9], PE[3], inv[9];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 4; ++k) acc += P[4 * i + k] * P[4 * j + k];
            A[3 * i + j] = acc;
        }
        REAL acc = 0;
        for (int k = 0; k < 4; ++k) acc += P[4 * i + k] * E[k];
        PE[i] = acc;
    }
    inv[0] = A[4] * A[8] - A[5] * A[7];
    inv[1] = A[2] * A[7] - A[1] * A[8];
    inv[2] = A[1] * A[5] - A[2] * A[4];
    inv[3] = A[5] * A[6] - A[3] * A[8];
    inv[4] = A[0] * A[8] - A[2] * A[6];
    inv[5] = A[2] * A[3] - A[0] * A[5];
    inv[6] = A[3] * A[7] - A[4] * A[6];
    inv[7] = A[1] * A[6] - A[0] * A[7];
    inv[8] = A[0] * A[4] - A[1] * A[3];
    REAL det = A[0] * inv[0] + A[1] * inv[3] + A[2] * inv[6];
    if (RE(det) == 0.0) return -1;
    for (int i = 0; i < 3; ++i)
        l[i] = (inv[3 * i + 0] * PE[0] + inv[3 * i + 1] * PE[1] + inv[3 * i + 2] * PE[2]) / det;
    return 0;
}

/* Rigid motion of one view, P' = P T(theta) (the P_lambda T_lambda of the
 * Optimization section): T = [R t; 0 1], R = Rz(rz) Ry(ry) Rx(rx) about the world
 * origin, theta = (rx, ry, rz [rad], tx, ty, tz [mm]). */
static void SFX(apply_motion)(const double P[12], const REAL th[6], REAL out[12]) {
    REAL cx = R_COS(th[0]), sx = R_SIN(th[0]);
    REAL cy = R_COS(th[1]), sy = R_SIN(th[1]);
    REAL cz = R_COS(th[2]), sz = R_SIN(th[2]);
    REAL Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
    REAL Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
    REAL Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
    REAL Rzy[9], R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 3; ++k) acc += Rz[3 * i + k] * Ry[3 * k + j];
            Rzy[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 3; ++k) acc += Rzy[3 * i + k] * Rx[3 * k + j];
            R[3 * i + j] = acc;
        }
    REAL T[16] = {R[0], R[1], R[2], th[3], R[3], R[4], R[5], th[4], R[6], R[7], R[8], th[5], 0, 0, 0, 1};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) {
            REAL acc = 0;
            for (int k = 0; k < 4; ++k) acc += P[4 * i + k] * T[4 * k + j];
            out[4 * i + j] = acc;
        }
}

static void SFX(cross3)(const REAL a[3], const REAL b[3], REAL c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static REAL SFX(dot3)(const REAL a[3], const REAL b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Per-view set-up from an (already moved) projection matrix Pm: scale P so that
 * the third row of M has unit norm and det M > 0, source through the meet
 * construction, detector up axis m3 x m1.  Returns -1 for a degenerate P. */
static int SFX(view_setup_P)(const REAL Pm[12], SFX(view_t)* v) {
    REAL m1[3] = {Pm[0], Pm[1], Pm[2]}, m2[3] = {Pm[4], Pm[5], Pm[6]}, m3[3] = {Pm[8], Pm[9], Pm[10]};
    REAL c23[3];
    SFX(cross3)(m2, m3, c23);
    REAL detM = SFX(dot3)(m1, c23);
    REAL n3 = R_SQRT(SFX(dot3)(m3, m3));
    if (RE(n3) == 0.0 || RE(detM) == 0.0) return -1;
    REAL scale = (RE(detM) > 0 ? 1.0 : -1.0) / n3;
    for (int i = 0; i < 12; ++i) v->P[i] = Pm[i] * scale;
    REAL X[4];
    SFX(source_h)(v->P, X);
    if (RE(X[3]) == 0.0) return -1;
    for (int i = 0; i < 3; ++i) v->C[i] = X[i] / X[3];
    REAL a3[3] = {v->P[8], v->P[9], v->P[10]}, a1[3] = {v->P[0], v->P[1], v->P[2]}, up[3];
    SFX(cross3)(a3, a1, up);
    REAL nu = R_SQRT(SFX(dot3)(up, up));
    if (RE(nu) == 0.0) return -1;
    for (int i = 0; i < 3; ++i) v->up[i] = up[i] / nu;
    return 0;
}

/* Frame of the pencil of epipolar planes around the baseline C_a -> C_b:
 * u = baseline direction, w = (up_a + up_b) made orthogonal to u, v = w x u.
 * The plane at angle kappa has normal n = cos(kappa) w + sin(kappa) v.
 * If up_a + up_b is (nearly) parallel to u, the world axis least aligned with u
 * replaces it: the first axis whose |u_i| is within 1e-9 of the smallest, so that
 * axes tied in exact arithmetic (a baseline along the third axis: u_0 = u_1 = 0)
 * are not told apart by rounding.  Returns -1 if the two sources coincide. */
static int SFX(pair_frame)(const SFX(view_t)* va, const SFX(view_t)* vb, REAL w[3], REAL v[3]) {
    REAL d[3] = {vb->C[0] - va->C[0], vb->C[1] - va->C[1], vb->C[2] - va->C[2]};
    REAL nd = R_SQRT(SFX(dot3)(d, d));
    if (!(RE(nd) > 0.0)) return -1;
    REAL u[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
    REAL r[3] = {va->up[0] + vb->up[0], va->up[1] + vb->up[1], va->up[2] + vb->up[2]};
    REAL ru = SFX(dot3)(r, u);
    REAL wt[3] = {r[0] - ru * u[0], r[1] - ru * u[1], r[2] - ru * u[2]};
    REAL nw = R_SQRT(SFX(dot3)(wt, wt));
    if (RE(nw) < 1e-6) {
        double best = fabs(RE(u[0]));
        for (int i = 1; i < 3; ++i)
            if (fabs(RE(u[i])) < best) best = fabs(RE(u[i]));
        int ax = 0;
        while (fabs(RE(u[ax])) > best + 1e-9) ++ax;
        REAL ui = u[ax];
        for (int i = 0; i < 3; ++i) wt[i] = (i == ax ? 1.0 : 0.0) - ui * u[i];
        nw = R_SQRT(SFX(dot3)(wt, wt));
    }
    for (int i = 0; i < 3; ++i) w[i] = wt[i] / nw;
    SFX(cross3)(w, u, v);
    return 0;
}

/* The epipolar plane of the pencil at angle kappa: E = (n, -n.C_a). */
static void SFX(plane_at)(const REAL w[3], const REAL v[3], const REAL Ca[3], double kappa, REAL E[4]) {
    double ck = cos(kappa), sk = sin(kappa);
    for (int i = 0; i < 3; ++i) E[i] = ck * w[i] + sk * v[i];
    E[3] = -(E[0] * Ca[0] + E[1] * Ca[1] + E[2] * Ca[2]);
}

/* The epipolar line of plane E in a view, by the selected construction. */
static int SFX(line_of)(const REAL P[12], const REAL E[4], int construction, REAL l[3]) {
    if (construction == 0) {
        SFX(line_inf)(P, E, l);
        return 0;
    }
    return SFX(line_pinv)(P, E, l);
}

/* Look-up of S_lambda at detector line l (pixel coordinates, pixel centres on
 * integers): Eq. (3) indexing.  The line is written relative to the detector
 * centre ((W-1)/2, (H-1)/2) in normal form (cos a, sin a, -s); a is folded into
 * [0, pi) with S(a + pi, s) = -S(a, -s); S is bilinear in (a/da, s/ds + (n_s-1)/2)
 * with zero outside the s range; the row after the last wraps to row 0 at -s with
 * the opposite sign.  *hit = 1 when the line meets the detector rectangle
 * (pixel edges): |s| <= W/2 |cos a| + H/2 |sin a|. */
static REAL SFX(lookup)(const double* sino, int n_alpha, int n_s, int W, int H, const REAL l[3], int* hit) {
    const double pi = 3.14159265358979323846;
    double cxd = 0.5 * (W - 1), cyd = 0.5 * (H - 1);
    double ds = sqrt((double)W * W + (double)H * H) / (n_s - 1);
    REAL l3c = l[0] * cxd + l[1] * cyd + l[2];
    REAL h = R_SQRT(l[0] * l[0] + l[1] * l[1]);
    REAL ca = l[0] / h, sa = l[1] / h, s = -l3c / h;
    *hit = fabs(RE(s)) <= 0.5 * W * fabs(RE(ca)) + 0.5 * H * fabs(RE(sa));
    REAL alpha = R_ATAN2(l[1], l[0]);
    double sign = 1.0;
    if (RE(alpha) < 0.0) { alpha += pi; s = -s; sign = -sign; }
    if (RE(alpha) >= pi) { alpha -= pi; s = -s; sign = -sign; }
    REAL ia = alpha / (pi / n_alpha);
    REAL is = s / ds + 0.5 * (n_s - 1);
    double m0 = floor(RE(ia)), n0 = floor(RE(is));
    REAL fa = ia - m0, fs = is - n0;
    REAL rows[2];
    for (int dm = 0; dm < 2; ++dm) {
        long m = (long)m0 + dm;
        double t[2];
        for (int dn = 0; dn < 2; ++dn) {
            long n = (long)n0 + dn;
            if (m < n_alpha) {
                t[dn] = (n >= 0 && n < n_s) ? sino[(size_t)m * n_s + n] : 0.0;
            } else { /* row n_alpha is row 0 at -s, negated */
                long nm = (long)(n_s - 1) - n;
                t[dn] = (nm >= 0 && nm < n_s) ? -sino[nm] : 0.0;
            }
        }
        rows[dm] = (1.0 - fs) * t[0] + fs * t[1];
    }
    return sign * ((1.0 - fa) * rows[0] + fa * rows[1]);
}

/* Is kappa inside the arc [lo, lo + len) taken modulo pi? */
static int SFX(in_arc)(double kappa, double lo, double len) {
    const double pi = 3.14159265358979323846;
    double x = kappa - lo;
    x -= pi * floor(x / pi);
    return x <= len;
}

/* Eq. (15) for one pair, before the division by N_kappa: sum over the K sampled
 * planes of [S_a - S_b]^2 for the planes that hit both detectors.
 * arcs = {sampled view (0 = a, 1 = b), lo_s, len_s, lo_o, len_o}: planes
 * kappa_k = lo_s + (k + 1/2) len_s / K, k = 0..K-1, inside the sampled view's arc.
 * mode 0: validity = both lines meet their detector rectangle (the definition of
 *         N_kappa); *mismatch counts the samples where that differs from
 *         membership of kappa_k in the other view's arc.
 * mode 1: validity = membership in the other view's (frozen) arc. */
static int SFX(pair_sum)(const SFX(view_t)* va, const SFX(view_t)* vb, const double* sa, const double* sb,
                         int n_alpha, int n_s, int W, int H, int K, const double arcs[5], int construction,
                         int mode, REAL* sum_out, int* nk_out, int* mismatch) {
    REAL w[3], v[3];
    *sum_out = 0;
    *nk_out = 0;
    if (SFX(pair_frame)(va, vb, w, v) != 0) return -1;
    double lo = arcs[1], len = arcs[2], lo_o = arcs[3], len_o = arcs[4];
    REAL sum = 0;
    int nk = 0;
    for (int k = 0; k < K; ++k) {
        double kappa = lo + (k + 0.5) * len / K;
        REAL E[4], la[3], lb[3];
        SFX(plane_at)(w, v, va->C, kappa, E);
        if (SFX(line_of)(va->P, E, construction, la) != 0) return -1;
        if (SFX(line_of)(vb->P, E, construction, lb) != 0) return -1;
        int hit_a, hit_b;
        REAL Sa = SFX(lookup)(sa, n_alpha, n_s, W, H, la, &hit_a);
        REAL Sb = SFX(lookup)(sb, n_alpha, n_s, W, H, lb, &hit_b);
        int in_other = SFX(in_arc)(kappa, lo_o, len_o);
        int lit = hit_a && hit_b;
        if (mismatch && lit != in_other) ++*mismatch;
        int valid = mode == 0 ? lit : in_other;
        if (valid) {
            REAL dlt = Sa - Sb;
            sum += dlt * dlt;
            ++nk;
        }
    }
    *sum_out = sum;
    *nk_out = nk;
    return 0;
}
