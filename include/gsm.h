/*
 * gsm.h -- C interface of the GB300 library for free-space nonlocal potentials
 * u = U * rho by the Gaussian-sum method of L. Exl, N. J. Mauser and Y. Zhang,
 * "Accurate and efficient computation of nonlocal potentials based on
 * Gaussian-sum approximation" (arXiv:1501.04438).
 *
 * Problem (Sec. 1, Eq. ConvGen, Eq. kernelPhy): given a density rho sampled on
 * the uniform grid of Sec. 2.1 of the box [-L, L]^d (or a rectangular box,
 * gsm_options_t.box),
 *     x_j = -L + j h,  h = 2L/n,  j = 1..n    (array index i = j - 1),
 * compute u(x) = int U(x - y) rho(y) dy at the same points for
 *     3D Coulomb  U = 1/(4 pi |x|),   2D Coulomb U = 1/(2 pi |x|),
 *     2D Poisson  U = -ln|x| / (2 pi),
 *     3D dipolar  U of Eq. dipkerneld, evaluated as in Sec. 2.4:
 *                 u = -(n.m) rho - 3 U_Coulomb * (d_n d_m rho).
 * The method (Algorithm 1) splits u = I_1 + I_2: I_1 is the convolution with the
 * Gaussian-sum approximation U_GS of the kernel (Sec. 3), applied to the
 * zero-padded density as a Fourier multiplier (Eq. I1FFT, Eq. tensor, padding
 * to period 4 as in the remark that follows Eq. tensor); I_2 is the near-field
 * correction c0 rho + c2 Lap(rho) from the Taylor expansion of Sec. 2.3,
 * applied as part of the same multiplier with a spectral Laplacian.
 *
 * Arrays are C-ordered with x fastest: rho[z][y][x] (3D), rho[y][x] (2D).
 *
 * Conventions for every call:
 *  - All functions return a gsm_status_t; none aborts or throws.  After an
 *    error, gsm_last_error() returns a message for the calling thread.
 *  - Device pointers and the stream belong to the caller.  The library never
 *    frees caller memory.  Kernels run asynchronously on the given stream
 *    (a cudaStream_t passed as void*; NULL is the legacy default stream);
 *    errors raised by a running kernel surface at the caller's next
 *    synchronisation.
 *  - A plan owns its device memory (multiplier, twiddle tables, workspace)
 *    and is immutable once made.  One apply may be in flight per plan at a
 *    time, because the workspace is shared: applies on one plan must be
 *    ordered (same stream, or events).  Different plans are independent.
 *  - rho and u may be the same array (the first pass reads rho completely
 *    before the last pass writes u).
 */
#ifndef GSM_H
#define GSM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsm_plan_s *gsm_plan_t;
typedef struct gsm_batch_s *gsm_batch_t;

/* Kernels of Eq. kernelPhy, the dipolar kernel of Eq. dipkerneld, and the
 * Davey-Stewartson potential of Example 5, u = -(1/2 pi) ln|x| * (d_xx rho)
 * (the Poisson potential of d_xx rho, end of Sec. 2.4). */
typedef enum {
    GSM_COULOMB_3D = 0,
    GSM_COULOMB_2D = 1,
    GSM_POISSON_2D = 2,
    GSM_DIPOLAR_3D = 3,
    GSM_DAVEY_STEWARTSON_2D = 4,
    GSM_POWER_3D = 5,            /* U = |x|^-beta, 0 < beta < 3 (remark after Eq. sinc_quad) */
    GSM_POWER_2D = 6             /* U = |x|^-beta, 0 < beta < 2 */
} gsm_kernel_t;

/* Arithmetic of the FFT passes and of the multiplier product.
 *   GSM_FP64   : IEEE double.                  I/O: double.
 *   GSM_FP32   : IEEE single.                  I/O: float.
 *   GSM_FP32X2 : double-float (pairs of floats, about 48 significand bits),
 *                computed on the FP32 pipes.   I/O: double.
 * In every precision the Gaussian sum, the kernel tensor and the Taylor
 * coefficients are built in FP64 and rounded (FP32) or split (FP32X2) once. */
typedef enum {
    GSM_FP64 = 0,
    GSM_FP32 = 1,
    GSM_FP32X2 = 2
} gsm_precision_t;

typedef enum {
    GSM_OK = 0,
    GSM_ERR_INVALID_ARG = 1,      /* null pointer, bad kernel/dimension, L <= 0, ... */
    GSM_ERR_UNSUPPORTED_SIZE = 2, /* n odd, too small, or 2n not a product of 2, 3, 5 */
    GSM_ERR_OOM = 3,              /* device allocation failed */
    GSM_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    GSM_ERR_ACCURACY = 5,         /* no Gaussian sum with S <= 500 meets gs_eps */
    GSM_ERR_TIMEOUT = 6,          /* a bounded device wait ran out */
    GSM_ERR_BAD_PLAN = 7          /* null, destroyed or corrupted plan handle */
} gsm_status_t;

/* Options; gsm_default_options() fills the defaults listed here. */
typedef struct {
    double delta;               /* radius of the near-field ball B_delta in unit-box
                                   coordinates, Sec. 2.3 (default 1e-3) */
    int S;                      /* > 0: use this sinc-quadrature S; 0: the smallest
                                   S whose GS error on [delta, 2 |eta|] is <= gs_eps */
    gsm_precision_t precision;  /* default GSM_FP64 */
    double dip_n[3];            /* dipolar unit vectors n, m (default e_z, e_z); any */
    double dip_m[3];            /* directions (both along one axis: octant multiplier,
                                   otherwise a half-spectrum multiplier table) */
    int debug;                  /* 0; bit 0 set: FP32 plans use the shared-memory FFT engine
                                   in every pass even where the register-resident kernels
                                   apply (padded length 512); bit 1 set: 2D plans with a
                                   padded y (x) length >= 4096 transform each conv (x
                                   forward) line on one CTA instead of two half-length
                                   transforms on a CTA pair (for comparisons; same results
                                   to rounding) */
    double box[3];              /* rectangular box (Sec. 2.5, Eq. tensor_ani): if all
                                   d entries are > 0, axis a spans [-box[a], box[a]]
                                   and L is ignored; all 0 (default): [-L, L]^d.  The
                                   method is rescaled by the largest half-width; delta
                                   must be smaller than every box[a] / max box */
    double beta;                /* exponent of GSM_POWER_3D / GSM_POWER_2D, 0 < beta < d
                                   (default 1) */
    int host_zero_copy;         /* gsm_apply_host with page-locked host arrays: 1 (default)
                                   the passes read rho and write u in host memory over
                                   the host link; 0: staged copies */
} gsm_options_t;

/* Read-only facts about a plan. */
typedef struct {
    int kernel, d, n[3], M[3];  /* M = 2n: padded FFT lengths */
    double L, delta;
    int S, nterms;              /* sinc parameter and number of Gaussians */
    double gs_err;              /* achieved E_rel (1/r) or E_abs (ln r), Sec. 3 */
    double c0, c2;              /* Taylor coefficients of Sec. 2.3 (unit box) */
    int precision;
    size_t bytes_multiplier;    /* device bytes of the stored multiplier */
    size_t bytes_workspace;     /* device bytes of the FFT workspace */
    int npasses;                /* kernel launches of one apply (5 in 3D, 3 in 2D) */
    int launch_nl[5];           /* per pass: lines per CTA, */
    int launch_threads[5];      /*   threads per line, */
    int launch_emax[5];         /*   elements per thread (see gsm_plan_autotune) */
    double box[3];              /* half-width of each axis (L for a cube), x first */
    double beta;                /* exponent of the power kernels (1 otherwise) */
    int radix_fwd[3][12];       /* per axis: radices of the forward FFT in stage order,
                                   0 after the last (see gsm_plan_set_schedule) */
    int radix_inv[3][12];       /* the same for the inverse FFT */
} gsm_plan_info_t;

void gsm_default_options(gsm_options_t *opt);

/*
 * Make a plan (Algorithm 1, "Precomputation"): the Gaussian sum of 1/r, ln r or
 * r^-beta by sinc quadrature (Sec. 3.1-3.3; r^-beta through Eq. Gauss_int with
 * alpha = beta - 1 and the map tau = exp(s - e^-s)), the 1-D factors of Eq. tensor, the stored
 * tensor sum_q w_q G_k^q with the Taylor coefficients of Sec. 2.3 and the
 * rescaling constants of Sec. 2.1 folded in, and the twiddle tables.  All of it
 * is computed on the current CUDA device, in FP64, on `cuda_stream`; the call
 * synchronises that stream before it returns.
 *   out    : receives the handle (set to NULL on failure).
 *   kind   : kernel; d must be 3 for GSM_COULOMB_3D, GSM_DIPOLAR_3D and
 *            GSM_POWER_3D, 2 otherwise.  GSM_DAVEY_STEWARTSON_2D uses the Gaussian
 *            sum of ln r.  The power kernels take beta from opt (0 < beta < d).
 *   L      : half-width of the box [-L, L]^d, > 0.
 *   n      : d points per axis (x first), each even, >= 8, with 2n a product of
 *            2, 3 and 5 and 2n <= 8192.
 *   gs_eps : target accuracy of the Gaussian sum; <= 0 selects the default
 *            (2e-15 relative for 1/r and r^-beta, 1e-13 absolute for ln r), just above the
 *            rounding floors of the sums built in double (1/r: 0.9e-15 for
 *            delta = 1e-3, 1.2e-15 for delta = 1e-4; ln r: about 5e-14).
 *   opt    : NULL for defaults.
 * Errors: GSM_ERR_INVALID_ARG, GSM_ERR_UNSUPPORTED_SIZE, GSM_ERR_ACCURACY,
 *         GSM_ERR_OOM, GSM_ERR_CUDA.
 */
gsm_status_t gsm_plan(gsm_plan_t *out, gsm_kernel_t kind, int d, double L, const int *n,
                      double gs_eps, const gsm_options_t *opt, void *cuda_stream);

/*
 * Apply the plan (Algorithm 1, "Actual computation"): u = U * rho.
 *   rho, u : device arrays of prod(n) elements, double (FP64, FP32X2 plans) or
 *            float (FP32 plans), C-ordered, x fastest.  May alias.
 * Five passes in 3D (x forward, y forward, z forward-multiply-inverse,
 * y inverse, x inverse), three in 2D, launched on `cuda_stream`; no host
 * synchronisation.  Errors: GSM_ERR_BAD_PLAN, GSM_ERR_INVALID_ARG, GSM_ERR_CUDA.
 */
gsm_status_t gsm_apply(gsm_plan_t p, const void *rho, void *u, void *cuda_stream);

/*
 * One pass of gsm_apply, for timing passes separately: pass = 0..npasses-1,
 * in 3D x forward, y forward, z forward-multiply-inverse, y inverse, x
 * inverse; in 2D x forward, y forward-multiply-inverse, x inverse.  Pass 0
 * reads rho, the last pass writes u, the others use only the plan's
 * workspace.  Running passes 0..npasses-1 in order on one stream is exactly
 * gsm_apply.  Errors as gsm_apply, and GSM_ERR_INVALID_ARG for a bad pass.
 */
gsm_status_t gsm_apply_pass(gsm_plan_t p, int pass, const void *rho, void *u, void *cuda_stream);

/*
 * Choose the radix schedule and the launch shape of each pass by measurement
 * (no counterpart in the paper, whose FFTs come from a library).  For every
 * pass: first its radix schedule (the order of the radix-8, 4, 2, 5, 3 stages
 * of the pass's transform; for the conv pass the forward and the inverse
 * schedule together, including the pairs whose forward last and inverse
 * first stages share a radix and run fused with the multiplication), then its
 * launch shape (elements per thread, lines per CTA), each timed with CUDA
 * events on the plan's own workspace; the fastest is kept in the plan.  A
 * different schedule rounds differently, so results may change in the last
 * bits; the launch shape changes none.  Temporary input and output arrays are
 * allocated for the run; the stream is synchronised.  If the environment
 * variable GSM_AUTOTUNE_CACHE names a file, schedules and shapes found there
 * for this device, precision and grid are used without timing, and new
 * results are appended.  `report` (may be NULL) receives a text table of the
 * timings, truncated to report_len bytes.  Same plan rules as gsm_apply: no
 * apply may be in flight on the plan.
 */
gsm_status_t gsm_plan_autotune(gsm_plan_t p, void *cuda_stream, char *report, size_t report_len);

/*
 * Set the radix schedule of one transform of a plan (no counterpart in the
 * paper): axis 0..d-1, inverse 0 for the forward FFT along that axis, 1 for
 * the inverse; radices[0..count-1] in stage order, each 8, 4, 2, 5 or 3, their
 * product the padded length M of the axis, in the order the FFT engine runs
 * stages: all 8s, then 4s, 2s, 5s, 3s (so a forward schedule starts with an
 * even radix, as the pruned first stage of the zero-padded transform needs).
 * One exception: the inverse along the last axis (the conv pass) may start
 * with the last radix of that axis's forward schedule, followed by the rest in
 * engine order; those two stages then run fused with the multiplication
 * (e.g. forward 8 8 4, inverse 4 8 8).  A change that would leave the pair
 * invalid is refused: to move from such a pair to another forward schedule,
 * set the inverse to an engine-order schedule first.  The plan's twiddle
 * tables for that axis are rebuilt on
 * `cuda_stream` (synchronised when an old table is freed).  FP32 passes with
 * a padded length of 512 use register-resident kernels of fixed shape and
 * ignore the schedule.  Same plan rules as gsm_apply.  Errors:
 * GSM_ERR_BAD_PLAN, GSM_ERR_INVALID_ARG (bad axis or schedule), GSM_ERR_OOM.
 */
gsm_status_t gsm_plan_set_schedule(gsm_plan_t p, int axis, int inverse, const int *radices, int count,
                                   void *cuda_stream);

/*
 * Same as gsm_apply with HOST arrays, synchronising the stream before it
 * returns.  When both arrays are page-locked (cudaHostAlloc, cudaHostRegister,
 * torch pin_memory) and options.host_zero_copy is set, the first pass reads rho
 * and the last writes u directly in host memory through their mapped device
 * addresses: no copies.  Otherwise rho is copied to the device, applied, and u
 * copied back; staging buffers are allocated on the first such call and owned
 * by the plan.  In that case 3D plans overlap the
 * copies with the x passes: the copies run in 8 z-chunks on a stream the plan
 * creates on the first call, ordered against `cuda_stream` by events (work
 * queued before on `cuda_stream` completes first).  Copies overlap only from
 * page-locked (pinned) host memory; pageable arrays are copied synchronously
 * by the runtime, with the same result.  One host apply per plan at a time.
 */
gsm_status_t gsm_apply_host(gsm_plan_t p, const void *rho_host, void *u_host, void *cuda_stream);

/*
 * Apply `count` plans to their densities in one call: u[i] = U_i * rho[i].
 * (No counterpart in the paper, which treats one density at a time.)
 * Plans may differ in size, kernel and precision (each uses its own I/O type)
 * but must be distinct handles.  Plans whose padded lengths are all <= 512 go
 * through ONE kernel launch per precision and dimension (up to 48 instances
 * per launch) with a device work queue: each CTA of the launch takes the next
 * item (pass, instance, tile) from the queue, in pass-major order, when it
 * starts, and runs it once the instance's previous pass is complete, so the
 * passes of different instances overlap and no launch boundary separates
 * them.  Other plans, and FP32 plans with a
 * padded length of exactly 512 (which use register-resident kernels of their
 * own), are applied one by one on the stream.  The results are the same bits
 * as gsm_apply's.
 * Each wait of the queue kernel for a previous pass is bounded (10 s by
 * default): if one runs out, the kernel stops taking work, every CTA returns,
 * and the call reports GSM_ERR_TIMEOUT (the outputs are then not valid).  The
 * order in which work is taken guarantees that every wait ends, so the bound
 * is a safeguard, never reached in normal operation.
 * The call takes its queue state (about 1 KB per instance) from the stream-
 * ordered allocator, and synchronises `cuda_stream` before it returns, to read
 * the kernel's status.  Errors: as gsm_apply, GSM_ERR_OOM, GSM_ERR_TIMEOUT;
 * nothing is launched if any argument is invalid.
 */
gsm_status_t gsm_apply_batched(int count, const gsm_plan_t *plans, const void *const *rho,
                               void *const *u, void *cuda_stream);

/*
 * The same batched apply recorded once into a CUDA graph (a memset of the
 * queue state and the queue launches), so that every later run is a
 * single cudaGraphLaunch.  The graph holds the given rho[i] and u[i] pointers
 * and each plan's workspace: refill the same rho arrays between launches; the
 * plans must outlive the batch, and no other apply may be in flight on them
 * while the batch runs.  gsm_batch_create first runs the batch on
 * `cuda_stream` with 4 and with 8 lines per CTA, keeps the faster shape (so u
 * is written), then records the graph; it synchronises the stream and owns
 * the queue state (device memory) until gsm_batch_destroy.
 * gsm_batch_launch is asynchronous on its stream.  gsm_batch_wait synchronises
 * `cuda_stream` and reports the last launch's status: GSM_OK, or
 * GSM_ERR_TIMEOUT if a bounded wait ran out (see gsm_apply_batched).
 */
gsm_status_t gsm_batch_create(gsm_batch_t *out, int count, const gsm_plan_t *plans,
                              const void *const *rho, void *const *u, void *cuda_stream);
gsm_status_t gsm_batch_launch(gsm_batch_t b, void *cuda_stream);
gsm_status_t gsm_batch_wait(gsm_batch_t b, void *cuda_stream);
gsm_status_t gsm_batch_destroy(gsm_batch_t b);

/*
 * Hartree-type energy and its gradient (3D kernels), all on the device:
 *   rho = |psi|^2,  u = U * rho,  E = 1/2 h^3 sum rho u,
 *   grad = 2 h^3 u psi  (= dE/dRe psi + i dE/dIm psi; U is symmetric),
 * h^3 the volume of a grid cell.  psi and grad are interleaved complex
 * (re, im) arrays of prod(n) elements in the plan's I/O type; u has prod(n)
 * real elements; energy points to ONE element of the I/O type in device
 * memory.  grad may be NULL.  FP64 and FP32X2 plans only.
 */
gsm_status_t gsm_hartree(gsm_plan_t p, const void *psi, void *u, void *energy, void *grad,
                         void *cuda_stream);

gsm_status_t gsm_plan_info(gsm_plan_t p, gsm_plan_info_t *info);

/*
 * Saved plans (Sec. 2.2: the sum over q of w_q G_k^q does not depend on rho,
 * so it is computed once per discretisation and stored).
 *
 * gsm_plan_save writes into the HOST buffer `buf` (capacity bytes) the plan's
 * problem (kernel, d, n, box, delta, beta, dipolar n and m, requested accuracy), its
 * Gaussian sum (S, w_q, tau_q), Taylor coefficients c0, c2, the FP64 octant
 * kernel tensor ((n_x+1)(n_y+1)(n_z+1) doubles), the launch shape of every
 * pass and the radix schedules (as tuned by gsm_plan_autotune), followed by a
 * 64-bit FNV-1a checksum.
 * *bytes always receives the size needed; with buf == NULL nothing else
 * happens (size query).  A buffer smaller than that size:
 * GSM_ERR_INVALID_ARG.  Synchronous (device-to-host copies).
 *
 * gsm_plan_load creates a plan from such bytes without recomputing the
 * Gaussian sum, the Taylor coefficients or the tensor; the multiplier,
 * twiddles and workspace are rebuilt on `cuda_stream`.  precision < 0 keeps
 * the saved precision (and its launch shapes and schedules); GSM_FP64 /
 * GSM_FP32 / GSM_FP32X2 reuse the same FP64 tensor for another pass precision
 * with default launch shapes and schedules.  The result equals the saved plan bit for bit.  A
 * wrong magic, version, size or checksum: GSM_ERR_INVALID_ARG, *out = NULL.
 * The format is native little-endian; the caller owns buf.
 */
gsm_status_t gsm_plan_save(gsm_plan_t p, void *buf, size_t capacity, size_t *bytes);
gsm_status_t gsm_plan_load(gsm_plan_t *out, const void *buf, size_t bytes, int precision,
                           void *cuda_stream);

/* Free the plan's device memory (synchronises the device first). */
gsm_status_t gsm_plan_destroy(gsm_plan_t p);

const char *gsm_status_string(gsm_status_t s);
const char *gsm_last_error(void);

/* --- read-back of plan data (tests and diagnostics; synchronous) ------------- */

/* Gaussian-sum weights and exponents (w_q, tau_q), Eq. GS-Gene, in unit-box
 * coordinates.  Copies min(cap, nterms) terms; *nterms receives the count. */
gsm_status_t gsm_plan_gs_terms(gsm_plan_t p, double *w_host, double *tau_host, int cap, int *nterms);

/* The FP64 kernel tensor sum_q w_q G_k^q (Eq. tensor), WITHOUT the correction,
 * scaling and normalisation, on the octant k_a = 0..n_a, layout [kx][ky][kz]
 * with kz fastest (3D) or [kx][ky] (2D).  `count` must equal prod(n_a + 1). */
gsm_status_t gsm_plan_kernel_tensor(gsm_plan_t p, double *host_out, size_t count);

/* The 1-D factors g_q(k) = int_{-2}^{2} exp(-tau_q^2 y^2) cos(pi k y / 2) dy of
 * Eq. tensor for axis `axis`, layout [q][k], k = 0..n_axis; count must equal
 * nterms * (n_axis + 1). */
gsm_status_t gsm_plan_factors(gsm_plan_t p, int axis, double *host_out, size_t count);

/* --- FFT engine test hook ----------------------------------------------------
 * Unnormalised DFT of `nlines` contiguous lines of length M (device, interleaved
 * complex double), exp(sign 2 pi i jk/M), sign = -1 or +1, through the same
 * shared-memory Stockham engine the passes use, in `precision` arithmetic
 * (FP32 rounds the input to float and widens the output).  M a product of
 * 2, 3, 5, 8 <= M <= 8192.  Asynchronous on the stream. */
gsm_status_t gsm_fft_lines(int M, int nlines, int sign, gsm_precision_t precision,
                           const double *in_dev, double *out_dev, void *cuda_stream);

/* --- the same FFT without any device allocation ------------------------------
 * The paper has no counterpart to this entry point; it exists for callers.
 * gsm_fft_lines obtains its twiddle table with cudaMallocAsync and frees it on
 * every call.  Some callers cannot do that: code whose device memory is all
 * held by another allocator (a framework's caching pool), code on a latency-
 * critical path that must not take the allocator's locks or risk an
 * out-of-memory failure at call time, or a plug-in that is not allowed to own
 * device memory.  gsm_fft_lines_noalloc takes the same arguments and gives the
 * same bits as gsm_fft_lines (the same twiddle table and, in FP64, the same
 * FMA-form stage constants, so the same arithmetic), but keeps those tables in
 * a fixed 384 KiB scratch array that the library declares statically in device
 * memory:
 *   - it calls no cudaMalloc, cudaFree or other allocating routine;
 *   - the tables of every supported length fit (the largest, M = 8192 in FP64,
 *     take 339968 bytes); a length whose tables would not fit is rejected with
 *     GSM_ERR_UNSUPPORTED_SIZE, as is M > 8192;
 *   - every GPU that loads the library holds the 384 KiB until the process
 *     exits;
 *   - the first call on each device (more exactly, in each CUDA context: again
 *     after cudaDeviceReset) looks up the device address of the scratch, with
 *     the caller's device current; make that first call before any stream
 *     capture;
 *   - all calls share the one scratch array: calls that can overlap on the GPU
 *     (different streams, no ordering between them) race and may return wrong
 *     results; order them on one stream or with events.  Nothing in the
 *     scratch needs to start at zero: each call writes the whole table it reads.
 */
gsm_status_t gsm_fft_lines_noalloc(int M, int nlines, int sign, gsm_precision_t precision,
                                   const double *in_dev, double *out_dev, void *cuda_stream);

/* --- tensor-core DFT stage (measurement hook) ----------------------------------
 * No counterpart in the paper.  Unnormalised DFT of length 32 of `nvec`
 * contiguous vectors (device, interleaved complex double),
 * exp(sign 2 pi i jk/32), sign = -1 or +1, computed on the tensor cores
 * (tcgen05, bf16 operands, FP32 accumulation in tensor memory) with FP64-class
 * accuracy: each vector is scaled by a power of two and split into six 8-bit
 * digit planes, the DFT matrix likewise, and the 21 plane products that carry
 * 48 bits are accumulated exactly and recombined in 64-bit integer arithmetic
 * (the error-free splitting of Ozaki, Ogita, Oishi and Rump).  It exists to
 * measure whether tensor-core DFT stages pay for the FP64-class passes (they
 * do not replace any pass).  Allocates its 48 KB table and a status word from
 * the stream-ordered pool and synchronises `cuda_stream` before it returns;
 * GSM_ERR_TIMEOUT if the bounded wait for the tensor-core products ran out. */
gsm_status_t gsm_dft32_tc(int nvec, int sign, const double *in_dev, double *out_dev, void *cuda_stream);

/* --- failure-handling test hooks ----------------------------------------------
 * No counterpart in the paper.  Every device allocation the library makes goes
 * through one internal function that counts what is live.  These two calls let
 * a test check that each out-of-memory path releases what it had taken,
 * without exhausting a GPU.
 *
 * gsm_debug_fail_alloc(k): the k-th device allocation from now (k = 0: the
 * next one) fails as if the device were out of memory (the call that made it
 * returns GSM_ERR_OOM); later allocations succeed again.  k < 0 cancels a
 * pending failure.  Process-wide, for every thread and device.  Always GSM_OK.
 *
 * gsm_debug_alloc_stats(count, bytes): the number and the total size of the
 * library's live device allocations (plans, workspaces, staging buffers,
 * temporaries), process-wide.  GSM_ERR_INVALID_ARG if a pointer is NULL. */
gsm_status_t gsm_debug_fail_alloc(int k);
gsm_status_t gsm_debug_alloc_stats(size_t *count, size_t *bytes);

/* Test hook of the batch queue kernel (gsm_apply_batched,
 * gsm_batch_create), read when a batch is launched or recorded:
 * wait_ns > 0 bounds every wait by that many nanoseconds (<= 0: the default
 * 10 s); hold_instance >= 0 keeps the first pass of that instance (its index
 * among the grouped plans of the call, in order) from ever counting as
 * complete, so that the waits of its second pass run out and the call reports
 * GSM_ERR_TIMEOUT after wait_ns, with every CTA returning; -1 turns it off.
 * Nothing is left waiting after the call.  Process-wide.  Always GSM_OK. */
gsm_status_t gsm_debug_batch_wait(long long wait_ns, int hold_instance);

#ifdef __cplusplus
}
#endif
#endif /* GSM_H */
