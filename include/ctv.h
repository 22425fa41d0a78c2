/*
 * ctv.h - C ABI of the GB300 complex constrained TV library.
 *
 * The library solves problem (1) of Gao & Cao, "A Complex Constrained Total
 * Variation Image Denoising Algorithm with Application to Phase Retrieval"
 * (arXiv 2109.05496):
 *
 *     min_{x in C}  1/2 ||x - b||_F^2 + lambda ||x||_TV                    (1)
 *
 * for complex images x, b, with the four complex TV seminorms of Eq. (7)-(10),
 * by the dual fast gradient projection of Algorithm 2 (Prop. 1, Eq. (16)-(20)),
 * and uses it as the proximal step of FISTA (Algorithm 1) for the TV-regularised
 * phase-retrieval problem (24).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller, unless a
 *   comment says "host". The library never frees them.
 * - Complex images are complex64, interleaved (re, im), row-major, m rows
 *   (index j) by n columns (index k), with a leading dimension ld >= n counted in
 *   complex elements. Pointers must be 8-byte aligned.
 * - The dual variable q = (r1, r2, s1, s2) of Prop. 1 is stored per pixel as a
 *   float4 (r1, s1, r2, s2) = (Re p1, Im p1, Re p2, Im p2) on a dense m x n grid
 *   (row stride n). p1 (vertical difference, Eq. (5)) is zero on row m-1 and p2
 *   (horizontal difference) is zero on column n-1: those slots do not exist in
 *   the paper and are kept at zero. Pointers must be 16-byte aligned.
 * - Every call is asynchronous and stream-ordered on `stream` unless it takes a
 *   host `stats` pointer, in which case it synchronises the stream before it
 *   returns so that the statistics can be filled in.
 * - Argument errors return CTV_EINVAL before anything is launched. A CUDA error
 *   raised while launching returns CTV_ECUDA. No entry point ever aborts the
 *   process.
 * - Workspaces are caller-owned device buffers of the size the matching
 *   *_workspace_size call returns, 256-byte aligned. The library allocates
 *   device memory only inside the *_create calls of plans.
 */
#ifndef CTV_H
#define CTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* ctv_stream;

typedef enum {
  CTV_OK = 0,
  CTV_EINVAL = 1,      /* invalid argument; nothing was launched */
  CTV_ENOMEM = 2,      /* a plan could not allocate its device memory */
  CTV_ECUDA = 3,       /* a CUDA runtime or cuFFT call failed */
  CTV_ETIMEOUT = 4,    /* unused: no kernel of this library waits on the device */
  CTV_ENONFINITE = 5,  /* a NaN or infinity in an input image (asynchronous, see below) */
  CTV_EUNSUPPORTED = 6, /* valid request that this build does not implement */
  CTV_ETOOBIG = 7       /* image larger than the fixed scratch of ctv_denoise_noalloc */
} ctv_status;

/* The four complex TV seminorms: Eq. (7) type-I isotropic, Eq. (8) type-I
 * anisotropic, Eq. (9) type-II isotropic, Eq. (10) type-II anisotropic. */
typedef enum {
  CTV_TV1_ISO = 0,
  CTV_TV1_ANISO = 1,
  CTV_TV2_ISO = 2,
  CTV_TV2_ANISO = 3
} ctv_tv_type;

/* The closed convex set C of problem (1), a product of per-pixel sets.
 * amp_bound != 0 adds |x| <= amp_max (Eq. (25) with amp_max = 1; projection
 * Eq. (26)). box != 0 instead bounds the parts: box_re[0] <= Re x <= box_re[1]
 * and box_im[0] <= Im x <= box_im[1] (amp_bound and box are exclusive: the
 * projection onto their intersection is not a composition of the two).
 * support_kind: 0 none; 1 rectangle rows [rect[0], rect[2]) x columns
 * [rect[1], rect[3]) (x = 0 outside); 2 mask: device uint8 array of m x n
 * bytes, row stride mask_ld, x = 0 where the byte is 0. */
typedef struct {
  int amp_bound;
  float amp_max;
  int support_kind;
  int rect[4];
  const uint8_t* mask;
  int mask_ld;
  int box;
  float box_re[2];
  float box_im[2];
} ctv_constraint;

/* Solver options.
 * max_iters   K, the number of iterations of Algorithm 2 (>= 0).
 * check_every evaluate primal, dual and gap every this many iterations (0: only
 *             at the end).
 * gap_tol     > 0 stops at the first check with gap <= gap_tol * max(primal, 1e-30);
 *             later passes become no-ops on the device (no host synchronisation).
 * alpha       the weight of Eq. (9)/(10), in [0, 1]; ignored by type I.
 * warm_start  nonzero: q_0 = r_1 = the q held in dual_state on entry (t_1 = 1).
 * config      kernel configuration index (see ctv_config_info); -1 picks one.
 * plain_gp    nonzero: the non-accelerated gradient projection of Eq. (21)
 *             (q_{k+1} = P_S(q_k - grad h(q_k) / (16 lam^2)), no extrapolation). */
typedef struct {
  int max_iters;
  int check_every;
  double gap_tol;
  float alpha;
  int warm_start;
  int config;
  int plain_gp;
} ctv_opts;

/* Result statistics of one image. iters: iterations actually run; stopped:
 * 1 if the gap test stopped the run; primal, dual, gap: P(x_K), the dual value
 * of App. A (Eq. (30) times lambda) at q_K, and their difference; status:
 * CTV_OK, CTV_ENONFINITE if b holds a NaN or an infinity (x and the values above
 * are then not meaningful), or CTV_EINVAL for a negative or NaN lambda read from
 * a device array. */
typedef struct {
  int iters;
  int stopped;
  double primal;
  double dual;
  double gap;
  int status;
} ctv_stats;

const char* ctv_status_string(int status);
int ctv_abi_version(void);

/* Asynchronous errors. Problem (1) and (24) are defined for finite data; a NaN
 * or an infinity in an input (b of a denoising call or plan, or z, sqrt_y or H
 * of phase retrieval) is only seen on the device, after the call has returned.
 * The kernels that read b (the finalize and the duality-gap evaluations of every
 * solve) and the residual kernel of phase retrieval test each value as they load
 * it and record CTV_ENONFINITE in a status word on the device; calls that return
 * statistics also report it in ctv_stats.status. ctv_get_last_error synchronises
 * `stream`, then returns the first error recorded on the current device since
 * the previous ctv_get_last_error (CTV_OK if none) and clears it. The word is
 * per device, shared by all streams: an error raised by work still running on
 * another stream may be reported by a later call instead. CTV_ECUDA if the
 * synchronisation or the read fails. */
int ctv_get_last_error(ctv_stream stream);

/* Kernel configurations of the fused FGP pass: iterations per pass (temporal
 * blocking depth) and the shared-memory region of one thread block. */
int ctv_num_configs(void);
int ctv_config_info(int config, int* iters_per_pass, int* region_w, int* region_h, int* threads);
/* The configuration that opts->config = -1 selects for an m x n image, K
 * iterations, a TV type and the set C (NULL: no constraint) in a solve without
 * gap checks - the autotuned choice when there is one. (With gap checks an
 * untuned choice of 8 iterations per pass moves to the same region with 6 where
 * that needs no more passes per check interval.) -1 if C is invalid. */
int ctv_default_config(int m, int n, int iters, int tv_type, const ctv_constraint* C);

/* Autotuner (no counterpart in the paper). ctv_autotune_denoise runs
 * ctv_denoise once per configuration plus `repeats` timed times on the caller's
 * data (same arguments as ctv_denoise, the options' config, stopping and warm
 * start ignored), writes x, synchronises `stream`, returns the fastest
 * configuration in *best_config (times_ms: NULL or ctv_num_configs() floats) and
 * records it for the image's size class and TV type, which then becomes the
 * choice of every call with opts->config = -1 on the same device. The size class
 * of an m x n image is floor(log2(m n)); ctv_tune_get / ctv_tune_set read and
 * write that table (-1: untuned) so that it can be saved and restored. There is
 * one table per device; every call uses the current device's. */
int ctv_size_class(int m, int n);
int ctv_tune_get(int size_class, int tv_type, int* config);
int ctv_tune_set(int size_class, int tv_type, int config);
int ctv_autotune_denoise(const void* b, void* x, int m, int n, int ld, float lambda,
                         const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                         void* workspace, size_t workspace_bytes, int repeats, int* best_config,
                         float* times_ms, ctv_stream stream);

/* --------------------------------------------------------------------------
 * Denoising, problem (1), by Algorithm 2.
 * b: input image(s); x: output x_K = P_C(b - lambda L^T(q_K)) (Eq. (18)).
 * dual_state: NULL, or q (float4 per pixel, m x n per image) - read on entry
 * when opts->warm_start is set, always overwritten with q_K on exit.
 * lambda = 0 gives x = P_C(b). m = 1 and/or n = 1 are valid.
 * -------------------------------------------------------------------------- */
size_t ctv_denoise_workspace_size(int batch, int m, int n);

/* Single-image solves that can stop early (check_every > 0 and gap_tol > 0,
 * at least two check intervals, m * n >= 512 * 512) are, from the second call with
 * identical arguments on, run as a cached CUDA graph whose check intervals are
 * conditional nodes, so that the intervals after the stop cost nothing; such a
 * call is still asynchronous on `stream`. Calls on a stream that is being
 * captured, and calls while ctv_profile_enable(1) is in force, always launch
 * their passes directly. */
int ctv_denoise(const void* b, void* x, int m, int n, int ld, float lambda,
                const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                void* dual_state, void* workspace, size_t workspace_bytes,
                ctv_stats* stats /* host, nullable */, ctv_stream stream);

/* A batch of equally sized images, image i at b + i * batch_stride (complex
 * elements, same for x), with per-image lambda in the DEVICE array lambdas
 * (batch floats, each >= 0). stats: host array of batch entries, or NULL. */
int ctv_denoise_batched(const void* b, void* x, int batch, int m, int n, int ld,
                        long long batch_stride, const float* lambdas,
                        const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                        void* dual_state, void* workspace, size_t workspace_bytes,
                        ctv_stats* stats, ctv_stream stream);

/* --------------------------------------------------------------------------
 * ctv_denoise without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory - programs
 * whose device memory all belongs to their own pool allocator, plugin hosts
 * whose callbacks must not allocate, latency-critical loops where a cudaMalloc
 * (which can synchronise the device) is not acceptable. It takes the same
 * arguments as ctv_denoise minus the dual state and the workspace: its scratch
 * (statistics record and FGP dual buffers) is a fixed device array inside the
 * library, sized for images of at most CTV_NOALLOC_MAX_PIXELS pixels (m * n;
 * 16 MiB, held on each device where the library's module has been loaded, until
 * that device's context is destroyed). Larger images return CTV_ETOOBIG;
 * opts->warm_start must be 0. It never calls cudaMalloc, cudaFree or any
 * allocating routine.
 * - Every call looks up the array's device address (cudaGetSymbolAddress) with
 *   the caller's device current. The first call on a device loads the module
 *   and places the array there; make that first call before any stream capture.
 * - Every call uses the same array, which keeps the previous call's contents
 *   (each call clears what must start at zero). Calls that overlap on the GPU -
 *   on two streams, or from two host threads - race on it and give wrong
 *   results: serialise them.
 * -------------------------------------------------------------------------- */
#define CTV_NOALLOC_MAX_PIXELS (512 * 512)

int ctv_denoise_noalloc(const void* b, void* x, int m, int n, int ld, float lambda,
                        const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                        ctv_stats* stats /* host, nullable */, ctv_stream stream);

/* --------------------------------------------------------------------------
 * Batched denoising of many images of uneven sizes (problem (1) per image).
 * Each image has its own shape, lambda, alpha, TV type and C; all share
 * opts->max_iters, check_every and gap_tol (warm_start must be 0; config -1
 * picks 5; plans support configurations 2, 5, 6, 7, 11, 14 and 18, others return
 * CTV_EUNSUPPORTED; CTV_CONFIG_AUTOTUNE makes ctv_plan_create build a plan in
 * each supported configuration in turn, time one execution of it after a
 * warm-up on the caller's images (writing their x, synchronising), and keep the fastest -
 * the autotuning of tile and T for this batch; no counterpart in the paper).
 * ctv_plan_create copies the descriptors, allocates the plan's
 * device memory (dual state 64 bytes per pixel plus work lists) and captures the
 * whole schedule - one launch per pass over the tiles of all images - into a
 * CUDA graph; ctv_plan_execute replays it on `stream` (asynchronous). The b and
 * x pointers of the descriptors must stay valid while the plan is used.
 * -------------------------------------------------------------------------- */
typedef struct {
  const void* b;      /* device complex64 input, row stride ld */
  void* x;            /* device complex64 output, row stride ld */
  int m, n, ld;
  float lambda;       /* >= 0 */
  float alpha;        /* type-II weight, [0, 1] */
  int tv_type;        /* ctv_tv_type */
  ctv_constraint C;
} ctv_image_desc;

#define CTV_CONFIG_AUTOTUNE (-2)
typedef struct ctv_plan ctv_plan;

int ctv_plan_create(const ctv_image_desc* descs, int count, const ctv_opts* opts, ctv_plan** out);
int ctv_plan_execute(ctv_plan* plan, ctv_stream stream);
/* Per-image statistics of the last execution (synchronises `stream`). */
int ctv_plan_stats(const ctv_plan* plan, ctv_stats* stats_host, ctv_stream stream);
/* Configuration used, kernel launches per execution, pixel-iterations per
 * execution and device bytes held; any pointer may be NULL. */
int ctv_plan_info(const ctv_plan* plan, int* config, int* launches_per_execute, double* pixel_iters,
                  size_t* device_bytes);
void ctv_plan_destroy(ctv_plan* plan);

/* --------------------------------------------------------------------------
 * Differentiation through K unrolled iterations of Algorithm 2 (no counterpart
 * in the paper; the forward map is exactly ctv_denoise_batched with stopping
 * off). A batch of `batch` dense m x n images (row stride n, image stride m n),
 * per-image lambda in the DEVICE array lambdas (> 0 for a meaningful lambda
 * gradient; lambda = 0 images get lambdabar = 0), opts->max_iters = K >= 1,
 * opts->alpha, opts->config (a configuration the recompute supports, else the
 * default); warm_start must be 0.
 * ctv_unrolled_forward writes x = x_K and keeps the state every ckpt_every
 * iterations in the workspace, together with every r_k of the last
 * checkpoint segment; ctv_unrolled_backward takes xbar = dL/dx and
 * returns bbar = dL/db (complex64, same layout as b) and lambdabar = dL/dlambda
 * (DEVICE float per image), recomputing each earlier checkpoint segment. The workspace
 * (ctv_unrolled_workspace_size bytes) must be the one the forward call used and
 * must not be touched in between.
 * -------------------------------------------------------------------------- */
size_t ctv_unrolled_workspace_size(int batch, int m, int n, int iters, int ckpt_every);
int ctv_unrolled_forward(const void* b, void* x, int batch, int m, int n, const float* lambdas,
                         const ctv_constraint* C, int tv_type, const ctv_opts* opts, int ckpt_every,
                         void* workspace, size_t workspace_bytes, ctv_stream stream);
int ctv_unrolled_backward(const void* b, const void* xbar, void* bbar, float* lambdabar, int batch,
                          int m, int n, const float* lambdas, const ctv_constraint* C, int tv_type,
                          const ctv_opts* opts, int ckpt_every, void* workspace,
                          size_t workspace_bytes, ctv_stream stream);

/* --------------------------------------------------------------------------
 * Phase retrieval, problem (24): min 1/2 || |A x| - sqrt(y) ||^2 + tau TV(x) + I_C(x),
 * with A = crop o IFFT2 o (H *) o FFT2 o pad on an M x N grid (Eq. (23) when
 * M = m and N = n; the object sits in the top-left m x n corner).
 * A plan owns the cuFFT plan and its device buffers (about 3 M N complex64
 * plus the FGP workspace); it is the only place the library allocates.
 * sqrt_y: m x n float32, dense (row stride n). H: M x N complex64 transfer
 * function (16-byte aligned). Images z, x, grad: m x n complex64, dense.
 * One plan must not be used by two streams at the same time.
 * -------------------------------------------------------------------------- */
typedef struct ctv_pr_plan ctv_pr_plan;

int ctv_pr_plan_create(int m, int n, int M, int N, ctv_pr_plan** out);
void ctv_pr_plan_destroy(ctv_pr_plan* plan);

/* grad = grad F(z) of Eq. (27) (A z / |A z| := 1 where A z = 0); loss: NULL or a
 * DEVICE double receiving F(z) of Eq. (24). */
int ctv_pr_gradient(ctv_pr_plan* plan, const void* z, const float* sqrt_y, const void* H,
                    void* grad, double* loss, ctv_stream stream);

/* Algorithm 1 (accelerate != 0; the gradient is taken at z_k) or ISTA, Eq. (14)
 * (accelerate == 0), outer_iters iterations with step gamma. Each prox step is
 * problem (15) with lambda = tau * gamma, solved by inner->max_iters iterations of
 * Algorithm 2 (inner->alpha, inner->config used; gap stopping allowed), its dual
 * warm-started from the previous outer iteration (t reset to 1).
 * x_io: x_0 on entry, x_K on exit. loss_hist: NULL or DEVICE array of
 * outer_iters doubles receiving F(z_k). */
int ctv_pr_solve(ctv_pr_plan* plan, const float* sqrt_y, const void* H, float tau, float gamma,
                 const ctv_constraint* C, int tv_type, const ctv_opts* inner, int outer_iters,
                 int accelerate, void* x_io, double* loss_hist, ctv_stream stream);

/* Algorithm 1 / Eq. (14) with the step chosen by backtracking (the paper selects
 * gamma "via a line search" without details; this is the sufficient-decrease
 * test of Beck and Teboulle's FISTA): at z_k, starting from the previous step
 * (gamma0 at k = 0), gamma is multiplied by eta in (0, 1) until
 * F(x) <= F(z_k) + <x - z_k, grad F(z_k)> + ||x - z_k||^2 / (2 gamma), x being
 * the prox step from z_k with that gamma (its FGP warm start restored for every
 * trial). Synchronises `stream` once per trial. gamma_hist: NULL or HOST array
 * of outer_iters floats receiving the accepted steps; loss_hist as above. */
int ctv_pr_solve_ls(ctv_pr_plan* plan, const float* sqrt_y, const void* H, float tau, float gamma0,
                    float eta, const ctv_constraint* C, int tv_type, const ctv_opts* inner,
                    int outer_iters, int accelerate, void* x_io, double* loss_hist,
                    float* gamma_hist, ctv_stream stream);

/* One proximal-gradient step for problem (2) with a caller-supplied gradient:
 * v = z - gamma * grad; x_out = prox_{gamma (tau TV + I_C)}(v) by Algorithm 2
 * (dual_state: NULL or the m x n float4 dual, warm start per inner->warm_start);
 * z_next = x_out + beta (x_out - x_prev)  (Alg. 1, step 5 with
 * beta = (t_k - 1)/t_{k+1}; beta = 0 gives ISTA, Eq. (14)).
 * workspace: ctv_prox_grad_workspace_size(m, n) bytes. */
size_t ctv_prox_grad_workspace_size(int m, int n);
int ctv_prox_grad_step(const void* z, const void* grad, float gamma, float tau,
                       const ctv_constraint* C, int tv_type, const ctv_opts* inner,
                       void* dual_state, const void* x_prev, void* x_out, void* z_next,
                       float beta, int m, int n, void* workspace, size_t workspace_bytes,
                       ctv_stream stream);

/* --------------------------------------------------------------------------
 * Measurement (no counterpart in the paper). ctv_profile_enable(on) resets the
 * counters; on = 1 brackets every following launch of the fused FGP pass kernel
 * with CUDA events on its stream, on = 2 brackets each run of consecutive pass
 * launches of a single-image or equally sized batch solve (a run ends at a gap
 * check or at the finalize), which leaves the overlap of back-to-back passes
 * intact; on = 0 stops timing. ctv_profile_read synchronises on those events
 * and returns the summed time in ms, the number of pass launches inside the
 * timed intervals, the pixel-iterations they processed, and the number of
 * kernel launches of the library since the last enable (counted whether or not
 * timing is on).
 * -------------------------------------------------------------------------- */
int ctv_profile_enable(int on);
int ctv_profile_read(double* pass_ms, long long* pass_launches, double* pass_pixel_iters,
                     long long* all_launches);

#ifdef __cplusplus
}
#endif
#endif /* CTV_H */
