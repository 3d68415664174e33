/*
 * admm_deconv.h -- C ABI of the GB300 (sm_103a) mask-decoupled ADMM solver for
 * image deconvolution with unknown boundaries.
 *
 * Method: M. S. C. Almeida, M. A. T. Figueiredo, "Deconvolving Images with
 * Unknown Boundaries Using the Alternating Direction Method of Multipliers".
 *   observation model   y = M A x + n                      (Sec. IV-A, eq. model_unknown_BC)
 *   TV-MD               Algorithm 3 with line 7 -> eq. new_line (Sec. IV-D)
 *   FA-MD               Algorithm 2, H1 = A, H2 = P, eqs. invAnalysis/invAnalysisp1,
 *                       prox eqs. prox_g_1_uBC and prox_g_2    (Sec. IV-C)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are row-major float32, H rows x W columns, on the FULL unknown
 *    domain (the observed region is a subset of it).
 *  - The blur A is periodic convolution on the full domain with the kernel
 *    centre at (0,0); its boundary condition is irrelevant on the observed
 *    pixels (Sec. IV-A). Kernels have odd sides, l = (side - 1) / 2 per axis.
 *  - TV uses forward periodic differences; the frame is the undecimated Haar
 *    frame (Parseval, P^T P = I) with `haar_levels` levels (3 L + 1 bands).
 *  - Every call is ordered on the CUDA stream passed as `stream` (a
 *    cudaStream_t, NULL = legacy default stream). Calls that run the solver
 *    return after the solve has finished on that stream.
 *  - Return values: ADMM_OK (0) or a negative ADMM_E* code; admm_strerror()
 *    names it. No call throws or aborts. A solve that reaches max_iters
 *    without meeting its tolerance is not an error (result.converged = 0).
 *  - Device pointers must be allocated with cudaMalloc (or equivalent) on the
 *    current device; host pointers may be pageable or pinned. The library
 *    never takes ownership of caller memory.
 *  - One library instance serialises its solve calls internally (a mutex).
 */
#ifndef ADMM_DECONV_H
#define ADMM_DECONV_H

#include <stdint.h>

#if defined(__GNUC__)
#define ADMM_API __attribute__((visibility("default")))
#else
#define ADMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define ADMM_OK                   0
#define ADMM_EINVAL              -1  /* bad argument (null, non-odd kernel, mu <= 0, ...) */
#define ADMM_ENOMEM              -2  /* device or host allocation failed                   */
#define ADMM_ECUDA               -3  /* a CUDA runtime call failed                         */
#define ADMM_EUNSUPPORTED_SIZE   -4  /* a side that is not m 2^k (m = 1, 3, 5), a multiple
                                        of 32 in 64..2048 (with fft_pad_policy
                                        ADMM_PAD_EXACT), or a side above 2048              */
#define ADMM_ENONFINITE          -5  /* an observed value or the iterate is NaN/Inf
                                        (divergence, Theorem 1)                            */
#define ADMM_ETIMEOUT            -6  /* a bounded device wait expired: the TV row phase
                                        (the bulk copies of its spectrum rows) and the frame
                                        synthesis tile (its TMA halo boxes) wait at most
                                        about a second; a problem whose wait ran out
                                        retires with this status (also in res->status)     */

/* ---- enums -------------------------------------------------------------- */
#define ADMM_REG_TV     0   /* isotropic TV, eq. unconstrained_TV_uBC            */
#define ADMM_REG_HAAR   1   /* l1 of undecimated Haar analysis coefficients,
                               eq. unconstrained_analysis_uBC                    */
/* Variants beyond the paper's two priors (same x-step; only the prox of the
   regulariser changes). */
#define ADMM_REG_TV_ANISO      2   /* anisotropic TV, lambda sum_i (|Dh x|_i + |Dv x|_i):
                                      eq. soft per difference component            */
#define ADMM_REG_HAAR_LL_FREE  3   /* frame prior with the last low-low band
                                      unpenalised (its prox is the identity)       */
#define ADMM_REG_HAAR_SYNTHESIS 4  /* FS-MD: the frame synthesis formulation,
                                      min 1/2 ||M(y - A W theta)||^2 + lambda ||theta||_1,
                                      x = W theta with W = P^T (Sec. IV-B, eq.
                                      unconstrained_synthesis_uBC); the
                                      duals d2 live on the coefficients theta. No
                                      warm start (admm_deconv_warm_start: EINVAL) */

/* Reeves-Sorel variants (Sec. IV-B/C/D, "Using the Reeves-Sorel technique"):
   the observation split is u1 = M A x with g1(u1) = 1/2 ||y - u1||^2 on the
   observed pixels, and the x-step's inverse (A^T M^T M A + gamma D^T D)^{-1}
   (TV) or (A^T M^T M A + gamma I)^{-1} (frame) is applied as
   C - C B^T (B C B^T - I)^{-1} B C (eqs. ReevesTV and reeves3), B the rows of
   A at the unobserved pixels, with one conjugate-gradient iteration per
   outer iteration warm-started from the previous one. */
#define ADMM_REG_TV_CG   5  /* TV-CG: the TV prior of eq. unconstrained_TV_uBC    */
#define ADMM_REG_HAAR_CG 6  /* FA-CG: the frame analysis prior of
                               eq. unconstrained_analysis_uBC
                               (both: no admm_deconv_warm_start, EINVAL; their
                               d1 is zero on unobserved pixels)                   */

#define ADMM_STOP_ITERS   0 /* run exactly max_iters iterations                  */
#define ADMM_STOP_REL_X   1 /* ||x_k - x_{k-1}|| / ||x_k|| < tol                 */
#define ADMM_STOP_REL_OBJ 2 /* |f_k - f_{k-1}| / |f_k| < tol (Sec. V's rule)     */

typedef struct admm_plan_s* admm_plan_t;   /* opaque; owned by the library */

/* Parameters of one problem (one image). */
typedef struct {
    int   H, W;            /* full unknown-image domain: sides m 2^k (m = 1, 3 or 5) that are
                              multiples of 32 in [64, 2048] (powers of two run the tuned
                              kernels, the others mixed-radix kernels on the exact domain;
                              the Reeves-Sorel variants take powers of two only), or any
                              size in [1, 2048] with fft_pad_policy = ADMM_PAD_NEXT          */
    int   psf_h, psf_w;    /* odd kernel sides, each <= the matching image side             */
    const float* psf;      /* HOST pointer, psf_h x psf_w row-major, centre at
                              (psf_h/2, psf_w/2); copied during admm_deconv_plan; the
                              DC gain sum(psf) must be nonzero (Sec. III-C proposition)     */
    float lambda;          /* regularisation weight lambda >= 0                             */
    float mu1, mu2;        /* ADMM penalties mu_1 (observation split), mu_2 (regulariser);
                              a value <= 0 selects the default rule: mu2 = 10 lambda
                              (Sec. V) and mu1 = min(1, 3 mu2) (Sec. V's mu1 rule is
                              garbled; penalties change only the speed, Theorem 1)          */
    int   reg;             /* ADMM_REG_TV, ADMM_REG_HAAR, ADMM_REG_TV_ANISO,
                              ADMM_REG_HAAR_LL_FREE, ADMM_REG_HAAR_SYNTHESIS,
                              ADMM_REG_TV_CG or ADMM_REG_HAAR_CG                            */
    int   haar_levels;     /* frame levels for the frame priors, 1..4 (0 = 4)              */
    int   stop;            /* ADMM_STOP_*                                                   */
    double tol;            /* tolerance of the stop rule                                    */
    int   max_iters;       /* iteration cap (> 0)                                           */
    int   check_every;     /* evaluate the rel-x rule every this many iterations (>= 1);
                              the rule always compares two consecutive iterates             */
    int   raw_mask;        /* 0: the observation mask is ANDed with the valid region
                              (pixels whose blurred value does not touch the unknown
                              boundary, Sec. IV-A); 1: use the mask exactly as given
                              (e.g. M = I for periodic deconvolution)                        */
    int   fft_pad_policy;  /* ADMM_PAD_EXACT (0): H and W must be sides the library
                              solves exactly (see H, W), else ADMM_EUNSUPPORTED_SIZE;
                              ADMM_PAD_NEXT (1): any H, W in 1..2048 -- a side that is not
                              solved exactly goes to the next one that is (300 -> 320;
                              the next power of two for the Reeves-Sorel variants), the
                              image in the domain's top-left corner and the added rows
                              and columns never observed (more unknown boundary, Sec.
                              IV-A: the domain only has to hold the image and the kernel
                              support); y, mask and x_out keep the caller's H x W      */
    const float* band_mu;  /* HOST pointer or NULL. ADMM_REG_HAAR and ADMM_REG_HAAR_LL_FREE
                              only: 3 L + 1 penalties, one per frame band, in the band order
                              of admm_deconv_get_state, replacing mu2 for that band. This is
                              Algorithm 2 with one function per band and the positive
                              diagonal Upsilon of eq. diagonal_penalty (Sec. II): the
                              x-step becomes (mu1 A^T A + sum_b mu_b P_b^T P_b)^{-1}
                              (mu1 A^T zeta1 + sum_b mu_b P_b^T zeta_b), still diagonal in
                              the DFT domain because each band is a convolution, and band b
                              is thresholded at lambda / mu_b. The minimiser is the same
                              (Theorem 1); only the speed changes. Each value finite and
                              > 0; copied during admm_deconv_plan. NULL: mu2 for every band */
} admm_params_t;

#define ADMM_PAD_EXACT 0
#define ADMM_PAD_NEXT  1

/* Per-problem outcome, written before a solve call returns. */
typedef struct {
    int    iters;          /* iterations run                                                */
    int    converged;      /* 1 if the stop rule was met before max_iters                  */
    int    status;         /* ADMM_OK or ADMM_ENONFINITE for this problem                  */
    int    reserved;
    double objective;      /* objective of eq. unconstrained_TV_uBC / _analysis_uBC at the
                              final iterate (FP32 data, compensated reduction)              */
    double rel_x;          /* last evaluated ||x_k - x_{k-1}|| / ||x_k||, or -1 if never    */
    double rel_obj;        /* last evaluated |f_k - f_{k-1}| / |f_k|, or -1 if never        */
    double t_start_ms;     /* device clock: from the call's set-up until the problem started
                              iterating (later than 0 when it waited for a free slot)       */
    double t_done_ms;      /* device clock: from the call's set-up until it retired        */
    double primal_res;     /* ||d_k - d_{k-1}|| over both splits, i.e. the norm of the
                              primal residual H z_k - u_k of Algorithm 2, at the last
                              iteration that evaluated the objective (FP32 data,
                              compensated reduction), or -1 if none did               */
} admm_result_t;

/*
 * admm_deconv_plan -- validate `p`, allocate the plan's device state and
 * precompute its spectra (a0 of the iteration: Lambda = DFT of the centred
 * kernel, and the diagonal of eq. fast_inversion for TV or eq. invAnalysisp1
 * for Haar, with the 1/(H W) of the inverse DFT folded in).
 *   out     [out] receives the plan handle (unchanged on error)
 *   p       [in]  parameters; p->psf is read before the call returns
 *   stream  [in]  cudaStream_t the precompute kernels are ordered on
 * Errors: ADMM_EINVAL, ADMM_EUNSUPPORTED_SIZE, ADMM_ENOMEM, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_plan(admm_plan_t* out, const admm_params_t* p, void* stream);

/*
 * admm_deconv_solve -- run the ADMM of the plan on one observation.
 *   y      [in]  H x W float32, observed values on observed pixels (other values
 *                are ignored); device or host memory
 *   mask   [in]  H x W uint8, nonzero = observed; NULL = the valid region only;
 *                device or host memory
 *   x_out  [out] H x W float32 estimate of the full image; device or host memory
 *   res    [out] host pointer, may be NULL
 * The solve starts from u0 = d0 = 0 (Algorithm 3 initialisation).
 * Errors: ADMM_EINVAL, ADMM_ECUDA, ADMM_ENONFINITE or ADMM_ETIMEOUT (also in
 * res->status).
 */
ADMM_API int admm_deconv_solve(admm_plan_t plan, const float* y, const uint8_t* mask, float* x_out,
                      admm_result_t* res, void* stream);

/*
 * admm_deconv_solve_batch -- solve `count` independent problems together.
 * Problems with the same (H, W, regulariser) advance in lock-step launches
 * (one launch per phase and iteration for the whole group); each problem
 * retires when its own stop rule is met. Arguments are arrays of `count`
 * entries with the meaning of admm_deconv_solve; masks may be NULL (then
 * every mask is the valid region) and any masks[i] may be NULL.
 * A plan may appear at most once per call.
 *   use_warmstart  0: every problem starts as admm_deconv_solve does (or from
 *                  its pending admm_deconv_warm_start / admm_deconv_set_state);
 *                  1: every ADMM_REG_TV problem without such a pending start
 *                  starts from the learned network loaded by
 *                  admm_warmstart_load (the network predicts x0 and the duals
 *                  d0 from [M^T y, mask] on the device, then the start of
 *                  admm_deconv_warm_start is used). One pass of the network
 *                  serves up to 16 problems of one size (no more than
 *                  16 x 512 x 512 pixels); each problem's start has the bits
 *                  of a pass over it alone. Other regularisers start cold.
 *                  ADMM_EINVAL if no network is loaded.
 * Errors: as admm_deconv_solve; the first failing problem's code is returned.
 */
ADMM_API int admm_deconv_solve_batch(const admm_plan_t* plans, int count, const float* const* y,
                            const uint8_t* const* masks, float* const* x_out,
                            admm_result_t* res, int use_warmstart, void* stream);

/*
 * admm_warmstart_load -- load the learned warm-start network (not in the
 * paper; see admm_warmstart.h) from a weights file into the library, for
 * admm_deconv_solve_batch(..., use_warmstart = 1, ...). The file is the
 * little-endian binary written by `python -m paper_1210_2687_gb300.warmstart
 * export`: 8 bytes "ADMMCNN1", int32 version (1), int32 reserved, int64
 * parameter count (admm_cnn_param_count()), float32 scales[4] (s0, s1, s2,
 * unused), float32 parameters in the layout of admm_cnn_set_params.
 * The network is created lazily on the device of the first solve that uses
 * it and grown to the largest image it meets. path = NULL unloads it.
 * Errors: ADMM_EINVAL (unreadable file, bad header or size), ADMM_ENOMEM.
 */
ADMM_API int admm_warmstart_load(const char* path);

/*
 * admm_deconv_state_size -- number of floats of the dual state d = (d1, d2)
 * of the plan: (1 + 2) H W for TV, (1 + 3 L + 1) H W for Haar.
 */
ADMM_API long long admm_deconv_state_size(admm_plan_t plan);

/*
 * admm_deconv_get_state -- copy the dual variables left by the last solve
 * into `d_out` (device or host, state_size floats). Layout: d1 (H x W, row-
 * major), then d2: TV -- H x W pairs (horizontal, vertical) interleaved per
 * pixel; Haar -- 3 L + 1 planes of H x W in band order.
 * Errors: ADMM_EINVAL, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_get_state(admm_plan_t plan, float* d_out, void* stream);

/*
 * admm_deconv_domain -- the domain the plan solves on: H x W as given, or the
 * padded size with fft_pad_policy = ADMM_PAD_NEXT. The state (admm_deconv_
 * get_state, get_full_state, set_state) and admm_deconv_warm_start's x0 and
 * d0 live on this domain, the image in its top-left corner.
 * Errors: ADMM_EINVAL (NULL arguments).
 */
ADMM_API int admm_deconv_domain(admm_plan_t plan, int* H, int* W);

/*
 * admm_deconv_full_state_size -- floats of the complete iteration state that
 * admm_deconv_get_full_state returns: the duals d (state_size floats), then
 * the row spectra of the next x-step's right-hand side, Hd x (Wd/2 + 1)
 * entries of four floats (Re, Im of zeta1's row DFT, Re, Im of w's row DFT;
 * Hd x Wd the plan's domain), and for ADMM_REG_HAAR_SYNTHESIS also the last
 * synthesis output w (Hd Wd floats) and zeta2 (3 L + 1 planes); for the
 * Reeves-Sorel variants also the conjugate-gradient iterate on the
 * unobserved pixels (Hd Wd floats, zero on observed ones).
 */
ADMM_API long long admm_deconv_full_state_size(admm_plan_t plan);

/*
 * admm_deconv_get_full_state -- copy the complete state left by the last
 * solve of the plan (device or host, full_state_size floats) and, if `iters`
 * is not NULL, the number of iterations that solve ran. Algorithm 2 carries
 * (u_k, d_k) from one iteration to the next; this library keeps d_k and, in
 * place of u_k, what the next x-step reads of zeta_k = u_k + d_k (the row
 * spectra of its right-hand side), so a solve started from this state with
 * admm_deconv_set_state continues the same iterate sequence bit for bit.
 * Errors: ADMM_EINVAL, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_get_full_state(admm_plan_t plan, float* state, int* iters, void* stream);

/*
 * admm_deconv_set_state -- make the next solve of the plan resume from a
 * state returned by admm_deconv_get_full_state (checkpoint / restart). The
 * next solve's first iteration is iteration k + 1 of the solve that produced
 * the state; its iterates (x, d) are bit-identical to those of one
 * uninterrupted solve. The stop rules restart their memory: the relative
 * changes are first evaluated at the second iteration after the restart,
 * and `iters` of the result counts from the restart. The state is consumed
 * by the next solve, like a warm start; it must come from a plan with the
 * same domain and regulariser (other parameters may differ, which then
 * changes the iteration from the restart on). Returns after the copies have
 * completed on `stream`, so `state` may be released then.
 * Errors: ADMM_EINVAL (NULL arguments, a plan made on another device), ADMM_ECUDA.
 */
ADMM_API int admm_deconv_set_state(admm_plan_t plan, const float* state, void* stream);

/*
 * admm_deconv_warm_start -- make the next solve of `plan` (admm_deconv_solve
 * or one entry of admm_deconv_solve_batch) start from a given point instead
 * of u0 = d0 = 0. Algorithm 2 converges from any (u0, d0) (Theorem 1); the
 * start used here is u0 = H x0 - d0, d0 given, with H = (A, D) for TV or
 * (A, P) for the frame prior, so that the first x-step returns x0 and the
 * first dual update starts from d0. The paper has no warm start: a learned
 * predictor (or an earlier solution) supplies x0 and d0.
 *   x0  H x W float32 starting image, device or host; NULL = zero image
 *   d0  state_size floats in the layout of admm_deconv_get_state, device or
 *       host; NULL = zero duals
 * The plan keeps the start until its next solve, which consumes it (later
 * solves start cold again). The stop rule compares consecutive iterates, so
 * it is first evaluated at the second iteration. Stream-ordered on `stream`;
 * returns after the copies have completed, so x0/d0 may be released then.
 * Errors: ADMM_EINVAL (NULL plan, plan made on another device), ADMM_ECUDA.
 */
ADMM_API int admm_deconv_warm_start(admm_plan_t plan, const float* x0, const float* d0, void* stream);

/* Options (admm_deconv_set_option); not in the paper. */
#define ADMM_OPT_MAX_SLOTS 1   /* value > 0: at most this many problems of a size class
                                  iterate at once in admm_deconv_solve_batch; the rest
                                  wait in a queue and start as problems retire.
                                  0 (default): chosen from the launch size            */
#define ADMM_OPT_FAIL_ALLOC 2  /* fault injection on the host, for testing the
                                  ADMM_ENOMEM paths: value n > 0 makes the n-th
                                  device or pinned-host allocation the library
                                  attempts from now on fail as if memory were
                                  exhausted (once); 0 (default) disarms it        */
#define ADMM_OPT_TEST_STALL 3  /* test hook for the bounded device waits: value 1
                                  makes the next solve's TV row phase (power-of-two
                                  domains) withhold one of its bulk copies in every
                                  CTA, so that the wait for it runs out (about a
                                  second) and each problem retires with
                                  ADMM_ETIMEOUT, the device staying usable; the
                                  option then resets to 0                         */

/*
 * admm_deconv_set_option -- set a library-wide option (see ADMM_OPT_*).
 * Errors: ADMM_EINVAL for an unknown option or a negative value.
 */
ADMM_API int admm_deconv_set_option(int option, long long value);

/* Device-time counters of the solver's launches (observability; not in the paper). */
typedef struct {
    double    col_ms;            /* summed device time of column-phase launches          */
    double    row_ms;            /* summed device time of the row-side launches of each
                                    iteration (one kernel for TV, four for the frame)   */
    long long col_launches;      /* column-phase launches timed                          */
    long long row_launches;      /* iterations whose row side was timed                  */
    long long kernel_launches;   /* every kernel the library launched (always counted)   */
} admm_profile_t;

/*
 * admm_deconv_profile -- read-and-reset the counters, then switch timing.
 *   enable  nonzero: following solves record a CUDA event on their stream
 *           between consecutive phase launches and add the elapsed times to
 *           the counters when the solve ends; zero: no events are recorded
 *   out     [out] if not NULL, receives the counters accumulated so far,
 *           which are then reset to zero
 * Timing is stream-ordered: a phase's time is the interval between the
 * events around it, so it includes any idle gap between launches.
 */
ADMM_API int admm_deconv_profile(int enable, admm_profile_t* out);

/*
 * admm_deconv_set_launch_overlap -- how the batch engine launches the
 * kernels of its iterations (not in the paper; a launch option only, the
 * arithmetic is the same either way).
 *   enable  nonzero (the default): each iteration kernel is launched with
 *           programmatic stream serialization, so it can be scheduled while
 *           its predecessor finishes and waits on the device for that
 *           predecessor's completion before reading its results; zero:
 *           plain stream-ordered launches
 * Library-global; takes effect at the next solve call. Returns ADMM_OK.
 * admm_deconv_get_launch_overlap returns the current setting (0 or 1).
 */
ADMM_API int admm_deconv_set_launch_overlap(int enable);
ADMM_API int admm_deconv_get_launch_overlap(void);

/* ---- launch configurations and the autotuner (not in the paper) ---------
 * The library compiles a few configurations of each phase per side length:
 * for the TV row phase (rows per strip, walk rows kept in flight, threads
 * per CTA) and for the column phase (spectrum columns per CTA). It also
 * chooses how many problems of a size class iterate at once, aiming for a
 * number of row-side CTAs per launch. A tuning table, one entry per
 * (device, H, W, regulariser, levels), says which configuration new plans of
 * that class use; untuned classes use index 0 of each list and 2400 CTAs.
 * Plans keep the configuration they were created with, and a batch groups
 * plans by shape AND configuration. The table is library-global. Entries are
 * per kernel family: plans of ADMM_REG_TV_ANISO use the ADMM_REG_TV entry,
 * plans of ADMM_REG_HAAR_LL_FREE and ADMM_REG_HAAR_SYNTHESIS the ADMM_REG_HAAR
 * entry. */
typedef struct {
    int    H, W;            /* [in] the size class ...                                        */
    int    reg;             /* [in] ... ADMM_REG_TV or ADMM_REG_HAAR ...                      */
    int    haar_levels;     /* [in] ... and levels (1..4 for Haar, 0 = 4; ignored for TV)     */
    int    row_variant;     /* index of the TV row-phase configuration of W (0 for Haar)     */
    int    col_variant;     /* index of the column-phase configuration of H                  */
    int    slot_ctas;       /* row-side CTAs per launch aimed for (0 = default 2400)         */
    int    lanes;           /* independent lanes (graph branches) the class's problems and
                               slots are split into, 1..4 (0 = default 2)                     */
    int    rows_per_strip;  /* [out] meaning of row_variant: rows per row-phase CTA, ...     */
    int    walk_depth;      /* [out] ... walk rows in flight (0 = read directly), ...        */
    int    row_threads;     /* [out] ... threads per row-phase CTA                           */
    int    col_block;       /* [out] meaning of col_variant: spectrum columns per CTA, ...   */
    int    col_min_ctas;    /* [out] ... the CTAs per SM its registers are sized for
                               (0 = the default for that block), ...                        */
    int    col_persistent;  /* [out] ... and 1 if its CTAs are persistent, walking the
                               launch's column blocks with a double-buffered tile          */
    double us_per_iter;     /* [out] autotuner: measured device time per problem-iteration
                               in microseconds (0 if the entry was not measured)             */
} admm_tuning_t;

/*
 * admm_deconv_variants -- number of compiled configurations of the class:
 * *n_row TV row-phase configurations of width W (1 for Haar, whose row side
 * has one), *n_col column-phase configurations of height H.
 * Errors: ADMM_EINVAL (NULL outputs, bad reg), ADMM_EUNSUPPORTED_SIZE.
 */
ADMM_API int admm_deconv_variants(int H, int W, int reg, int* n_row, int* n_col);

/*
 * admm_deconv_get_tuning -- the configuration new plans of the class get on
 * the current device. In: t->H, W, reg, haar_levels. Out: every other field
 * (indices 0 and us_per_iter 0 for an untuned class).
 * Errors: ADMM_EINVAL, ADMM_EUNSUPPORTED_SIZE, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_get_tuning(admm_tuning_t* t);

/*
 * admm_deconv_set_tuning -- install a configuration for the class on the
 * current device (e.g. one read back from a tuning cache). The [out] fields
 * are ignored; plans created afterwards use it.
 * Errors: ADMM_EINVAL (an index out of range, slot_ctas < 0),
 * ADMM_EUNSUPPORTED_SIZE, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_set_tuning(const admm_tuning_t* t);

/*
 * admm_deconv_autotune -- time every combination of the class's compiled
 * configurations and slot targets {default 2400, 1200, 4800} on the current
 * device, then 1 and 4 lanes for the fastest of those, and install the
 * fastest. Each trial creates `problems` plans of the
 * class on a synthetic observation (9 x 9 box blur, valid-region mask, rel-x
 * rule with tolerance 0 checked every 10 iterations, so no problem retires
 * early), runs `iters` iterations of all of them once to warm up and once
 * timed with CUDA events on `stream`, and frees them. The score is device
 * time per problem-iteration.
 *   problems    problems per trial (<= 0: enough to fill the largest slot
 *               target, at most 96)
 *   iters       iterations per solve (<= 0: 48)
 *   trials      [out] optional array of max_trials entries: every trial
 *   n_trials    [out] optional: number of trials run
 *   best        [out] optional: the configuration installed
 * Allocates device memory for the trials (problems plans at a time). Not
 * safe against plans of the same class being created concurrently from
 * other threads while it runs.
 * Errors: ADMM_EINVAL, ADMM_EUNSUPPORTED_SIZE, ADMM_ENOMEM, ADMM_ECUDA.
 */
ADMM_API int admm_deconv_autotune(int H, int W, int reg, int haar_levels, int problems, int iters,
                                  admm_tuning_t* trials, int max_trials, int* n_trials, admm_tuning_t* best,
                                  void* stream);

/*
 * admm_deconv_solve_noalloc -- one TV solve that allocates no memory.
 * The paper has no counterpart: this exists for callers that must not
 * allocate device memory while they run -- hosts whose own allocator already
 * owns the GPU's memory, fixed-budget or real-time loops where an allocation
 * could fail or stall, and plugins whose host application forbids libraries
 * from allocating. It needs no plan: every buffer it uses (spectra, duals,
 * descriptor, twiddles) lives in one fixed 4 MiB array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits. The call makes no cudaMalloc/cudaFree or other allocating call.
 *   p      [in]  parameters as for admm_deconv_plan; reg must be ADMM_REG_TV and
 *                H, W at most 256 (larger sizes return ADMM_EUNSUPPORTED_SIZE)
 *   y      [in]  H x W float32, DEVICE memory
 *   mask   [in]  H x W uint8, DEVICE memory, or NULL (valid region only)
 *   x_out  [out] H x W float32, DEVICE memory
 *   res    [out] host pointer, may be NULL
 * Every call resolves the array's device address on the current device with
 * that device current and rewrites the array's constant part (the twiddle
 * table), so it stays correct after a cudaDeviceReset. Under lazy module
 * loading (the CUDA default) the first call on a device loads the library's
 * device code there and with it the array: that first call may allocate, so
 * callers that must never allocate make one call during their initialisation.
 * Every call shares the array and clears what must start at zero; calls whose
 * device work overlaps (e.g. on two streams) race on it. The call holds the
 * library's lock for the whole solve, so other threads' library calls wait
 * meanwhile, and it synchronises `stream` (also when it fails after queueing
 * work), so it cannot be called while `stream` is being captured into a CUDA
 * graph. Returns after the solve has finished on `stream`.
 * Errors: ADMM_EINVAL (also for host pointers or a non-TV regulariser),
 * ADMM_EUNSUPPORTED_SIZE, ADMM_ECUDA, ADMM_ENONFINITE.
 */
ADMM_API int admm_deconv_solve_noalloc(const admm_params_t* p, const float* y, const uint8_t* mask,
                                       float* x_out, admm_result_t* res, void* stream);

/* admm_deconv_destroy -- free everything the plan owns (NULL is a no-op).
 * Synchronises the device first. */
ADMM_API void admm_deconv_destroy(admm_plan_t plan);

/* admm_strerror -- static string naming a status code. */
ADMM_API const char* admm_strerror(int code);

/* admm_deconv_version -- library version string. */
ADMM_API const char* admm_deconv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADMM_DECONV_H */
