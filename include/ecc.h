/*
 * ecc.h -- C ABI of the GB300 epipolar-consistency library (libecc.so).
 *
 * Computes the epipolar consistency metric of a cone-beam scan as defined in
 * Preuhs, Manhart, Maier, "Fast Epipolar Consistency without the Need for Pseudo
 * Matrix Inverses" (arXiv 1806.02637): the Grangeat intermediate function S of
 * every projection (Eq. 1), and for every pair of projections the mean squared
 * difference of S along the epipolar line pairs of the planes through both
 * sources (Eq. 15), with the Cauchy norm (Eq. 16), summed over pairs (Eq. 17).
 * Epipolar lines are built without any matrix inverse (Eq. 13/14).
 *
 * Conventions (all entry points)
 *   - Pointers marked "device" must be CUDA device memory of the context's device;
 *     "host" pointers are ordinary host memory.  The caller owns every buffer it
 *     passes; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Every call except ecc_create/ecc_destroy/ecc_last_error/
 *     ecc_status is asynchronous on that stream: outputs are valid once the
 *     stream has reached the end of the call.
 *   - Return value: ECC_OK (0) or a negative error code; on error a message is
 *     available from ecc_last_error(), no output has been written, and the
 *     context stays usable.  Errors that only the device can see do not fail the
 *     call: the affected pairs report N_kappa = 0, d = e = 0 (and no gradient),
 *     and a status bit is set that ecc_status() returns.  They are a degenerate
 *     projection matrix (rank below 3, det M = 0, or a NaN / Inf entry, the
 *     motion's included: ECC_STATUS_DEGENERATE_VIEW), coincident sources
 *     (ECC_STATUS_DEGENERATE_PAIR), and a pair whose sum of squared differences
 *     or gradient is not finite, i.e. a NaN / Inf sinogram value on its lines,
 *     from non-finite projection images (ECC_STATUS_NONFINITE_PAIR).
 *   - A context serves one host thread at a time; calls on one context must be
 *     issued on one stream (its scratch memory is reused across calls).
 *
 * Geometry
 *   P[n_views][12]: FP64, row-major 3x4 projection matrices mapping homogeneous
 *   world points [mm] to homogeneous detector pixels; pixel (i = column, j = row)
 *   has its centre at (i, j).  Any non-zero scale and sign of each P is accepted.
 *   Detectors are W columns x H rows, square pixels, no skew.
 *
 * Sinogram layout
 *   sino[n_views][n_alpha][n_s] of the element type `dtype`; row m holds
 *   alpha_m = m pi / n_alpha, column n holds s_n = (n - (n_s-1)/2) ds with
 *   ds = sqrt(W^2 + H^2) / (n_s - 1) pixels, s measured from the detector centre
 *   ((W-1)/2, (H-1)/2) along (cos alpha, sin alpha).
 */
#ifndef ECC_H_
#define ECC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecc_ctx ecc_ctx;

enum {
  ECC_OK = 0,
  ECC_EINVAL = -1,   /* invalid argument */
  ECC_ENOMEM = -2,   /* device allocation failed */
  ECC_ECUDA = -3,    /* CUDA runtime error */
  ECC_ETIMEOUT = -4, /* a bounded device wait gave up */
  ECC_EADMIT = -5,   /* request does not fit the memory budget */
  ECC_EPENDING = 1   /* result not ready yet */
};

enum { ECC_F32 = 0, ECC_F16 = 1, ECC_BF16 = 2 };

/* Device status bits returned by ecc_status() (and in ecc_result.flags). */
enum { ECC_STATUS_DEGENERATE_VIEW = 1, ECC_STATUS_DEGENERATE_PAIR = 2, ECC_STATUS_NONFINITE_PAIR = 4 };

/* Library version (major * 10000 + minor * 100 + patch). */
int ecc_version(void);

/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * scratch memory the context may hold (0 = no bound).  *out receives the
 * context.  Returns ECC_EINVAL for a bad device, ECC_ECUDA otherwise. */
int ecc_create(ecc_ctx** out, int device, size_t hbm_budget_bytes);

/* Frees the context and its scratch memory (waits for its work to finish). */
void ecc_destroy(ecc_ctx* ctx);

/* Message of the last error on this context (or of the last ecc_create failure
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* ecc_last_error(const ecc_ctx* ctx);

/* Waits for `stream`, then returns the device status bits accumulated by the
 * calls issued so far (ECC_STATUS_*) in *flags and clears them. */
int ecc_status(ecc_ctx* ctx, void* stream, int* flags);

/* Number of kernels this context has launched since it was created. */
long long ecc_kernel_launches(const ecc_ctx* ctx);

/* Per-kernel timing.  While enabled, every kernel launch of the context is
 * bracketed by two CUDA events recorded on its launch stream (adds two event
 * records per launch).  ecc_profile_read waits for `stream`, then writes up to
 * max_entries rows: names (32 bytes each, NUL-terminated, host memory), number
 * of launches and summed milliseconds per kernel name; *n_entries receives the
 * row count.  Reading clears the record. */
int ecc_profile_enable(ecc_ctx* ctx, int enable);
int ecc_profile_read(ecc_ctx* ctx, void* stream, int max_entries, char* names, long long* launches,
                     double* total_ms, int* n_entries);

/*
 * S_lambda for every view: the Grangeat intermediate function (Eq. 1), i.e. the
 * derivative with respect to the plane offset of the 3-D Radon transform on the
 * planes through the source, computed from the projection: the projection is
 * pre-weighted by D / sqrt(D^2 + u^2 + v^2) (u, v from the principal point, D
 * the source-detector distance, all in pixels, taken from P), integrated along
 * the detector lines of the (alpha, s) grid by Joseph's method (unit steps over
 * rows when |cos alpha| >= |sin alpha|, else over columns, linear interpolation,
 * zero outside the detector), differenced over a half step on either side of
 * s_n, and weighted by (D^2 + s_pp^2) / D^2 (s_pp: distance of the line from the
 * principal point).
 *
 *   P        device, FP64 [n_views][12]
 *   images   device, FP32 [n_views][H][W] line-integral projections
 *   sino_out device, [n_views][n_alpha][n_s] of dtype (ECC_F32, ECC_F16, ECC_BF16)
 *   scales_out device FP32 [n_views]: per-view scale factors of F16 storage,
 *            scale = max|S| / 2^14 over the view (1 for an all-zero view), stored
 *            value = S / scale rounded to FP16; required for ECC_F16, ignored
 *            otherwise.  F32 and BF16 store S itself (BF16 rounded to nearest).
 * Limits: 2 <= W, H <= 16384; 4 <= n_alpha <= 65535; 2 <= n_s <= 65535.
 */
int ecc_precompute_radon_derivative(ecc_ctx* ctx, int n_views, const double* P, const float* images, int W, int H,
                                    int n_alpha, int n_s, int dtype, void* sino_out, float* scales_out,
                                    void* stream);

/*
 * Epipolar consistency over a list of view pairs (Eq. 15-17).
 *
 * For each pair (a, b) the pencil of epipolar planes around the baseline C_a C_b
 * is parametrised by an angle kappa in a frame built from the baseline and the
 * two detectors' up axes; each plane's line in view lambda is l = cof(M) n
 * (Eq. 13/14; no inverse).  The arc of kappa whose lines meet view a's detector
 * and the arc for view b are found from the detector corners; the shorter arc is
 * sampled at n_kappa midpoints kappa_k = lo + (k + 1/2) len / n_kappa and a
 * sample counts if its plane meets both detectors (N_kappa of Eq. 15).  S_a and
 * S_b are bilinear look-ups in the (alpha, s) grid (alpha folded into [0, pi)
 * with S(alpha + pi, s) = -S(alpha, -s)).
 *   d_ab = (1/N_kappa) sum_k (S_a - S_b)^2   (0 if N_kappa = 0)
 *   e_ab = d_ab / (1 + d_ab / c)            (c = cauchy_c; c <= 0 gives e = d)
 *   total = sum over the pairs of e_ab       (FP64, fixed summation order)
 *
 *   P        device FP64 [n_views][12]
 *   motion   device FP64 [n_views][6] or NULL: per-view rigid motion theta =
 *            (rx, ry, rz [rad], tx, ty, tz [mm]); the view uses P T(theta) with
 *            T = [R t; 0 1], R = Rz(rz) Ry(ry) Rx(rx) (motion model of the
 *            Optimization section).  NULL = no motion.
 *   sino     device [n_views][n_alpha][n_s] of dtype; scales device FP32
 *            [n_views] for ECC_F16 (as written by the precompute), else NULL
 *   pairs    device int32 [n_pairs][2] or NULL = all a < b in row-major order
 *            (then n_pairs must equal n_views (n_views - 1) / 2)
 *   total    device FP64 [1]
 *   per_pair device FP64 [n_pairs][2] = {d, e} or NULL
 *   nkappa   device int32 [n_pairs] or NULL
 * Arithmetic: geometry per view in FP64; per pair (frame, maps, arcs, sample
 * ranges) and one line anchor per tile of 64 samples (of 32 when n_kappa < 96)
 * and view in double-float (about 48 bits); per-sample line offsets,
 * interpolation and accumulation in FP32.
 * Limits: 1 <= n_kappa <= 65536; 0 <= n_pairs <= 2^31 - 1.
 */
int ecc_evaluate(ecc_ctx* ctx, int n_views, const double* P, const double* motion, const void* sino,
                 const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa, double cauchy_c,
                 const int32_t* pairs, int n_pairs, double* total, double* per_pair, int32_t* nkappa, void* stream);

/*
 * As ecc_evaluate, plus the gradient of the total with respect to the per-view
 * motion parameters theta (motion model of the Optimization section; theta = 0
 * when motion is NULL), with the sampled planes (kappa arcs and validity) held at
 * the evaluation point:
 *   grad   device FP64 [n_views][6] = d total / d (rx, ry, rz, tx, ty, tz)
 * Per-sample derivatives of the bilinear look-ups are cell-wise constant (FP32);
 * the chain through the lines, the pencil frame, the sources and the cofactor
 * matrices to theta is FP64 (forward-mode tangents).  The paper's optimiser is
 * derivative-free; this gradient serves gradient-based motion estimation (the
 * argmin of Eq. 17).
 */
int ecc_evaluate_grad(ecc_ctx* ctx, int n_views, const double* P, const double* motion, const void* sino,
                      const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                      double cauchy_c, const int32_t* pairs, int n_pairs, double* total, double* per_pair,
                      int32_t* nkappa, double* grad, void* stream);

/*
 * Geometric calibration by the consistency (the Introduction names calibration as
 * a use of the epipolar consistency; Eq. 17 as the objective): as ecc_evaluate,
 * plus the gradient of the total with respect to the entries of each view's
 * projection matrix, with the sampled planes held at the evaluation point:
 *   grad_P device FP64 [n_views][12] = d total / d P, row-major like P.
 * It is the derivative with respect to the P passed in; with motion the view uses
 * P T(theta), so grad_P = (d total / d P') T(theta)^T.  The total is invariant
 * under P -> s P for each view, so sum_ij P_ij grad_P_ij = 0 per view (to
 * rounding); a step along grad_P changes the scale of P, which the evaluation
 * ignores.  The per-pair part reads the pair kernel's d e / d A, as
 * ecc_evaluate_grad; the chain through the pencil frame, the sources and the
 * cofactor matrices to P is FP64 (forward-mode tangents), summed per view in a
 * fixed order.  Errors as ecc_evaluate; ECC_EINVAL if grad_P is NULL.
 */
int ecc_evaluate_grad_projection(ecc_ctx* ctx, int n_views, const double* P, const double* motion, const void* sino,
                                 const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                                 double cauchy_c, const int32_t* pairs, int n_pairs, double* total,
                                 double* per_pair, int32_t* nkappa, double* grad_P, void* stream);

/*
 * As ecc_evaluate, but the planes of every pair (kappa arcs, step and validity
 * mask) are those sampled by the previous ecc_evaluate / ecc_evaluate_grad call on
 * this context; only the geometry (P, motion) may change.  The arguments n_views,
 * W, H, n_kappa, n_pairs and the pairs pointer must equal those of that call
 * (ECC_EINVAL otherwise).  This is the function the gradient differentiates, used
 * for finite-difference checks.
 */
int ecc_evaluate_frozen(ecc_ctx* ctx, int n_views, const double* P, const double* motion, const void* sino,
                        const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                        double cauchy_c, const int32_t* pairs, int n_pairs, double* total, double* per_pair,
                        int32_t* nkappa, void* stream);

/*
 * End-to-end evaluation from host buffers: copies P (host FP64 [n_views][12]) and
 * the projections (host FP32 [n_views][H][W], pinned memory recommended) to the
 * device, computes the sinograms (ECC_F32, kept in the context) and the total
 * over all pairs a < b, and copies the total back into *total_host.  Synchronous:
 * returns after the result is on the host.
 */
int ecc_scan_consistency_host(ecc_ctx* ctx, int n_views, const double* P_host, const float* images_host, int W,
                              int H, int n_alpha, int n_s, int n_kappa, double cauchy_c, double* total_host,
                              void* stream);

/*
 * Serving: motion-compensation jobs by continuous batching (not in the paper; the
 * paper's motion estimate minimises Eq. 17 over the per-view motion of the
 * Optimization section).  A job is one scan: its dRadon/ds precompute (as
 * ecc_precompute_radon_derivative), then n_iters gradient steps
 *   theta <- theta - step * d total / d theta   (as ecc_evaluate_grad, all a < b)
 * and a final evaluation at the last theta.  The context runs two threads: one
 * admits queued jobs in arrival order while the job's device memory fits the
 * serving budget (the context's hbm_budget_bytes, or 80 % of the device memory
 * free at the first ecc_submit when that is 0) and runs its precompute; the other
 * runs rounds in which every admitted job does one iteration.  A round's pair work
 * of all jobs is one persistent launch; jobs join and leave between rounds.  A
 * job's results do not depend on the other jobs in its rounds (every reduction has
 * a fixed order per job).
 *
 * The host arrays a job points to (P, motion0, images, motion_out, totals_out) must
 * stay valid until ecc_poll has returned something other than ECC_EPENDING for its
 * ticket.  Pinned host memory makes the input copies asynchronous.  While jobs are
 * served, the context may still be used for the other calls from its own thread.
 */
/* Motion models of a served job. */
enum { ECC_MOTION_PER_VIEW = 0, ECC_MOTION_AKIMA = 1 };

typedef struct ecc_job {
  int n_views;              /* >= 2 (<= 4096) */
  const double* P;          /* host FP64 [n_views][12] */
  const double* motion0;    /* host FP64 [n_views][6] initial theta, or NULL (zeros) */
  const float* images;      /* host FP32 [n_views][H][W] */
  int W, H, n_alpha, n_s;   /* detector and dRadon/ds grid (limits as the precompute) */
  int dtype;                /* sinogram storage: ECC_F32, ECC_F16 or ECC_BF16 */
  int n_kappa;              /* planes per pair (1 .. 65536) */
  double cauchy_c;          /* Eq. 16 (<= 0: none) */
  int n_iters;              /* gradient steps (>= 0) */
  double step;              /* step size */
  double* motion_out;       /* host FP64 [n_views][6] final theta, or NULL */
  double* totals_out;       /* host FP64 [n_iters + 1] total at theta_0 .. theta_n, or NULL */
  /* Motion model.  ECC_MOTION_PER_VIEW: the parameters of every view are the unknowns.
   * ECC_MOTION_AKIMA (the paper's model, Optimization section): each parameter is
   * motion0 plus an Akima spline (Akima 1970) over the view index with n_nodes nodes
   * at x_j = j (n_views - 1) / (n_nodes - 1); the node values (starting at 0) are the
   * unknowns and the step applies d total / d nodes (chain rule through the spline). */
  int motion_model;
  int n_nodes;              /* ECC_MOTION_AKIMA: 3 .. n_views */
  int param_mask;           /* bit k set: parameter k of (rx, ry, rz, tx, ty, tz) is estimated,
                               the others stay at motion0; 0 means all six */
  double* nodes_out;        /* host FP64 [n_nodes][6] final node values (ECC_MOTION_AKIMA), or NULL */
  const double* nodes0;     /* host FP64 [n_nodes][6] initial node values, or NULL (zeros).  Where all
                               slopes of a parameter are equal (e.g. all nodes 0) Akima's weights are
                               0/0 and the spline has kinks; the gradient there is that of the
                               equal-weights form t_j = (m_(j-1) + m_j) / 2. */
} ecc_job;

typedef struct ecc_result {
  int status;               /* ECC_OK or the error that ended the job */
  int iters;                /* gradient steps taken */
  double total_first;       /* total at theta_0 */
  double total_last;        /* total at the final theta */
  double queue_ms;          /* ecc_submit -> admission */
  double latency_ms;        /* ecc_submit -> results in host memory */
  size_t footprint_bytes;   /* device memory held while admitted (precompute peak) */
  long long line_pairs;     /* line-pair samples evaluated: pairs x n_kappa x (n_iters + 1) */
  int flags;                /* ECC_STATUS_* bits the job's device work raised (0: none); the
                               pairs they name were left out of its totals and gradients */
} ecc_result;

/* Device memory a job needs at admission (ECC_EINVAL for an invalid job). */
int ecc_job_footprint(const ecc_job* job, size_t* bytes);

/* Queues a job and returns its ticket.  ECC_EADMIT if the job can never fit the
 * serving budget; ECC_EINVAL for an invalid job, including a NaN / Inf entry in
 * P, motion0 or nodes0 (checked on the host; the images are checked on the
 * device, see ecc_result.flags). */
int ecc_submit(ecc_ctx* ctx, const ecc_job* job, uint64_t* ticket);

/* ECC_EPENDING while the job is queued or running.  Otherwise fills *out (if not
 * NULL), forgets the ticket and returns the job's status (ECC_OK, or the error that
 * ended it; the message is then in ecc_last_error).  ECC_EINVAL: unknown ticket. */
int ecc_poll(ecc_ctx* ctx, uint64_t ticket, ecc_result* out);

/* Serving counters since the first ecc_submit: rounds run, sum over rounds of the
 * jobs in them, the largest round, and the line-pair samples of completed jobs. */
int ecc_serve_stats(ecc_ctx* ctx, long long* rounds, long long* job_rounds, int* max_batch, long long* line_pairs);

/* Serving device time since the first ecc_submit, in milliseconds, from CUDA events
 * on the scheduler's streams: the admissions' input copies (host to device), their
 * dRadon/ds precomputes (with the view set-up), and the rounds (every launch of a
 * round, from its first copy to its last kernel).  A round is counted once it has
 * completed and the scheduler has seen it; with no job in flight the sums are complete.
 * Admissions run on their own stream and overlap the rounds, so the sums may exceed
 * the wall time. */
int ecc_serve_times(ecc_ctx* ctx, double* upload_ms, double* precompute_ms, double* round_ms);

/*
 * Allocation-free ecc_evaluate.  The paper has no counterpart: this is a service of
 * the library, not a step of the method.  It computes exactly what ecc_evaluate
 * computes, with the same arguments minus the context, for callers that must not
 * allocate device memory while running (an application that gives all free device
 * memory to its own pool at start-up, or a fixed-budget pipeline that cannot take
 * an allocation's implicit device synchronisation).  Its scratch lives in one
 * 5 MiB statically sized device array inside the library; it calls no allocator.
 *
 *   Device: the current CUDA device; all device pointers must be on it.  Every call
 *   looks up the scratch array's address in the current device's context
 *   (cudaGetSymbolAddress, a host-side lookup that allocates nothing); nothing is
 *   cached, so a cudaDeviceReset between calls leaves later calls valid.  The first
 *   call on a device may load the library's module: make it outside any stream
 *   capture.
 *   Limits of the static scratch (ECC_EINVAL with a message naming the limit
 *   otherwise): n_views <= 512, n_alpha <= 4096, n_pairs <= 8192 and
 *   n_pairs * ceil(n_kappa / 32) <= 131072; the other limits are ecc_evaluate's.
 *   Concurrency: every call on a device shares the one scratch array, so calls
 *   that overlap on the GPU race and give wrong results; serialise them (one
 *   stream, or wait for the previous call's stream).
 *   Device status bits are not reported (degenerate pairs still give
 *   N_kappa = 0 and d = e = 0).
 *   err: host buffer of err_len bytes receiving a NUL-terminated message on error
 *   (empty string on success), or NULL.
 */
int ecc_evaluate_noalloc(int n_views, const double* P, const double* motion, const void* sino, const float* scales,
                         int W, int H, int n_alpha, int n_s, int dtype, int n_kappa, double cauchy_c,
                         const int32_t* pairs, int n_pairs, double* total, double* per_pair, int32_t* nkappa,
                         void* stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* ECC_H_ */
