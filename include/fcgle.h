/*
 * fcgle.h -- C ABI of the GB300 (sm_103a) FCGLE time-stepping library.
 *
 * The library advances the semidiscrete space-fractional complex
 * Ginzburg--Landau equation (paper Eq. FCGLE, Sec. 2)
 *
 *     u'(t) = K u(t) + g(t, u(t)),     (Eq. ODEs)
 *     K = A_d (+) ... (+) A_1,  A_mu = (nu + i eta) D_mu      (Eq. Ksum)
 *     g(t, u) = gamma u - (kappa + i zeta)|u|^2 u + s(t)      (Sec. 2)
 *
 * by applying f(theta K) directly through the eigendecompositions
 * D_mu = Q_mu Lam_mu Q_mu^T (Eq. diag): the Tucker form
 *     f(theta K) v = ((F o (V x_1 Q_1^T ... x_d Q_d^T)) x_1 Q_1 ... x_d Q_d)   (Eq. fKu_diag)
 * and, for f = exp, the Kronecker-product form
 *     exp(theta K) v = V x_1 exp(theta A_1) ... x_d exp(theta A_d)            (Eq. Neudeckerd).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tensors.  A solution tensor is N = n_1 * ... * n_d complex numbers,
 *   interleaved (re, im), in vec order with j_1 fastest (Eq. indexj):
 *   element (j_1, .., j_d) (0-based) is at j_1 + n_1 (j_2 + n_2 j_3).
 *   Element type: complex128 (two doubles) for FCGLE_FP64 handles,
 *   complex64 (two floats) for FCGLE_BF16X3 handles.  Pointers are DEVICE
 *   pointers unless the function name ends in _host.  The caller owns every
 *   tensor it passes; the library keeps no pointer to it after the call
 *   returns, except the source tensors, which are copied at set time.
 * Streams.  Every device entry point is asynchronous on the handle's CUDA
 *   stream (given at setup, changeable with fcgle_set_stream); the caller
 *   synchronises.  _host entry points synchronise before returning.
 *   The tensor-core mode-product kernels of FCGLE_BF16X3 handles are launched
 *   with programmatic dependent launch: each may start its prologue while the
 *   previous kernel of the stream drains and waits for that kernel's
 *   completion before touching global memory, so stream order is kept.  The
 *   environment variable FCGLE_PDL=0, read once per process, launches them
 *   plainly instead (same kernels, bitwise the same results).
 * Errors.  Every function returns an fcgle_status; nothing throws across the
 *   ABI.  On error, fcgle_last_error() returns a thread-local message.
 *   Failures that happen on the device while asynchronous work runs are kept
 *   in the handle's device error word and reported by the next call that
 *   synchronises (fcgle_sync, the _host entry points, fcgle_adjoint):
 *   FCGLE_ERR_TIMEOUT when a bounded wait inside a tensor-core kernel gave up,
 *   FCGLE_ERR_NUMERIC when a result tensor (the state written by fcgle_step,
 *   fcgle_integrate and fcgle_batch_integrate, the output of fcgle_apply_f,
 *   the gradient of fcgle_adjoint) holds a NaN or an Inf.  The check runs in
 *   the kernel that writes the result in the user layout (no extra pass); the
 *   result is still written.
 *   Invalid parameters (d not in 1..3, n_mu < 1, alpha_mu not in (1,2),
 *   nu <= 0, kappa <= 0, b_mu <= a_mu, fd_order not in {2,4}, unknown enum
 *   values, null pointers) give FCGLE_ERR_INVALID_ARG and leave the handle
 *   unchanged.  A CUDA failure gives FCGLE_ERR_CUDA; the handle must then be
 *   destroyed.
 * Memory.  fcgle_setup allocates every device buffer the handle needs for
 *   apply_f and the one-step schemes; the spectral scalar tensors of a given
 *   (scheme, tau) are allocated and filled once, on first use (outside any
 *   time loop), and cached on the handle until fcgle_destroy.
 */
#ifndef FCGLE_H
#define FCGLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FCGLE_OK = 0,
  FCGLE_ERR_INVALID_ARG = 1,
  FCGLE_ERR_NOMEM = 2,
  FCGLE_ERR_CUDA = 3,
  FCGLE_ERR_NUMERIC = 4,     /* eigendecomposition residual too large; non-finite result state */
  FCGLE_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  FCGLE_ERR_UNSUPPORTED = 6  /* valid request this build does not implement */
} fcgle_status;

/* Arithmetic of the mode products.  FCGLE_FP64: complex128 tensors, FP64
 * mode products.  FCGLE_BF16X3: complex64 tensors (FP32 storage), mode
 * products on the tcgen05 tensor cores with each FP32 operand split as
 * hi + lo (two bf16) and hi*hi + hi*lo + lo*hi accumulated in FP32; the
 * eigendecomposition is FP64 and the spectral scalars f(theta lam) are
 * formed from FP64 coefficients and evaluated in FP32.
 * FCGLE_TF32 (one-pass TF32 mode products) is not built: fcgle_setup returns
 * FCGLE_ERR_UNSUPPORTED for it.  It would read the same operand bytes as
 * FCGLE_BF16X3 (FP32 storage) at about 1e-3 relative error per mode product
 * (10-bit mantissa) instead of about 1e-5. */
typedef enum { FCGLE_FP64 = 0, FCGLE_TF32 = 1, FCGLE_BF16X3 = 2 } fcgle_precision;

/* f in f(theta K): (1 - z)^{-1}, e^z, phi_k(z) (Eq. phi). */
typedef enum { FCGLE_F_INV = 0, FCGLE_F_EXP = 1, FCGLE_F_PHI = 2 } fcgle_func;

/* Time integrators.  LIE: linearly-implicit Euler (Eq. lbdf2-v, first step).
 * LBDF2: linearised BDF2 (Eq. lbdf2-v).  KROGSTAD: Krogstad's exponential
 * RK4 (Eq. krogstad-v).  STRANG: Strang splitting with the exact nonlinear
 * flow (Eq. Strang; source ignored).  LAWSON_EULER, LAWSON_RK2 (Heun-based)
 * and ETD2RK (Cox-Matthews) are not in the paper; their definitions are the
 * ones of the oracle's scheme module. */
typedef enum {
  FCGLE_LIE = 0,
  FCGLE_LAWSON_EULER = 1,
  FCGLE_LAWSON_RK2 = 2,
  FCGLE_ETD2RK = 3,
  FCGLE_KROGSTAD = 4,
  FCGLE_LBDF2 = 5,
  FCGLE_STRANG = 6
} fcgle_scheme;

/* Problem statement (Eq. FCGLE, Sec. 2): d directions, n_mu interior points
 * on (a_mu, b_mu) with h_mu = (b_mu - a_mu)/(n_mu + 1), Riesz orders alpha_mu,
 * finite differences of order 2 (Eq. FD2) or 4 (Eq. FD4).  Entries mu >= d
 * are ignored. */
typedef struct {
  int d;
  int n[3];
  double a[3];
  double b[3];
  double alpha[3];
  double nu, eta, gamma, kappa, zeta;
  int fd_order;   /* 2 or 4 */
  int precision;  /* fcgle_precision */
} fcgle_params;

typedef struct fcgle_ctx* fcgle_handle;

/* Builds D_mu (Eq. Dnalpha / Eq. FD4), eigendecomposes each in FP64 on the
 * host (Householder tridiagonalisation + implicit QL with Wilkinson shifts),
 * checks ||D Q - Q Lam|| and ||Q^T Q - I|| (FCGLE_ERR_NUMERIC if above
 * 1e-11 relative), copies Q_mu and lam_mu to the device once (Sec. 4.2: the
 * only host-to-device transfer of the method) and allocates the work
 * buffers.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * For BF16X3 handles the setup also runs the kernel autotuner (see
 * fcgle_autotune_report) on that stream for problem shapes this process has
 * not tuned yet, and waits for it; do not call it during a stream capture.
 * On success *out owns everything; release it with fcgle_destroy. */
fcgle_status fcgle_setup(const fcgle_params* params, void* cuda_stream, fcgle_handle* out);

/* Replaces the handle's stream (cudaStream_t). */
fcgle_status fcgle_set_stream(fcgle_handle h, void* cuda_stream);

/* Source term s(t, x) = sum_k exp(sigma_k t) S_k(x), sigma_k complex
 * (sigma_reim[2k] + i sigma_reim[2k+1]).  S_dev[k] are device tensors in the
 * user layout; they are copied into the handle (the caller may free them
 * afterwards).  nterms = 0 removes the source.  At most 4 terms. */
fcgle_status fcgle_set_source(fcgle_handle h, int nterms, const double* sigma_reim,
                              const void* const* S_dev);

/* Replaces nu, eta, gamma, kappa, zeta of the handle (same validity rules as
 * fcgle_setup).  Cheap: D_mu and its eigendecomposition depend only on the
 * grid and alpha_mu; cached spectral tensors are dropped.  Synchronises the
 * handle's stream first (FP64 handles). */
fcgle_status fcgle_set_coefficients(fcgle_handle h, double nu, double eta, double gamma, double kappa,
                                    double zeta);

/* How e^{theta K} is applied (Sec. 3.1-3.2).  FCGLE_EXP_TUCKER: the Tucker
 * form Q diag(e^{theta lam}) Q^T (Eq. fKu_diag), 2d real mode products.
 * FCGLE_EXP_KRON: the Kronecker-product form V x_1 E_1 ... x_d E_d with
 * E_mu = exp(theta A_mu) = Q_mu diag(e^{theta (nu + i eta) lam_mu}) Q_mu^T
 * (Eqs. Neudecker, Neudeckerd), d complex mode products, half the tensor
 * traffic.  FP64 handles always use FCGLE_EXP_KRON for the exponential.
 * BF16X3 handles default to FCGLE_EXP_TUCKER; fcgle_set_exp_form switches
 * fcgle_apply_f with EXP / PHI k = 0 and the schemes whose only linear
 * operator is e^{tau K} (LAWSON_EULER, LAWSON_RK2, STRANG) to the Kronecker
 * form.  Those schemes then carry the physical state u, so the split-BF16
 * error of every product (about 1e-5 relative) enters the state each step
 * and accumulates with the step count, whereas the Tucker form carries the
 * spectral state and lets it enter only through tau-small increments: the
 * Kronecker form trades accuracy at T for bytes.  E_mu is built in FP64 on
 * the host once per theta (O(n_mu^3)) and cached until the coefficients
 * change; batches run the Kronecker form with per-instance launches.  The
 * adjoint always uses the Tucker form. */
typedef enum { FCGLE_EXP_TUCKER = 0, FCGLE_EXP_KRON = 1 } fcgle_exp_form;
fcgle_status fcgle_set_exp_form(fcgle_handle h, int form);

/* How a Tucker operator X x_1 M_1 x_2 M_2 x_3 M_3 (Eq. fKu_diag, Sec. 3.2)
 * of a 3D BF16X3 handle is run.  FCGLE_TUCKER_ROTATING: three mode products,
 * each reading the tensor with its contracted index fastest and writing the
 * new index slowest (16 bytes of HBM traffic per element and product).
 * FCGLE_TUCKER_SLAB: the mode-1 and mode-2 products fused per j_3 slab (the
 * intermediate stays in tensor memory; 16 bytes per element for the two),
 * then the mode-3 product reading the natural order with j_3 slowest; needs
 * p_2 <= 256, else FCGLE_ERR_UNSUPPORTED.  FCGLE_TUCKER_AUTO (the default):
 * the form the autotuner found faster for the handle's extents (see
 * fcgle_autotune_report).  The two forms round differently (both at the
 * split-BF16 level); the first and last Tucker operators of a time
 * integration (the precise split-TF32 transforms) and the grouped launches of
 * a batch always use the rotating form; fcgle_batch_create sets its instance
 * handles to FCGLE_TUCKER_ROTATING as well, so that every path of a batch
 * rounds alike (fcgle_set_tucker_form on an instance changes its own
 * per-instance launches only).  Other handles (FP64, d != 3) accept FCGLE_TUCKER_AUTO and
 * FCGLE_TUCKER_ROTATING and run their only form; FCGLE_TUCKER_SLAB gives
 * FCGLE_ERR_UNSUPPORTED there.  Any other value: FCGLE_ERR_INVALID_ARG. */
typedef enum { FCGLE_TUCKER_AUTO = 0, FCGLE_TUCKER_ROTATING = 1, FCGLE_TUCKER_SLAB = 2 } fcgle_tucker_form;
fcgle_status fcgle_set_tucker_form(fcgle_handle h, int form);

/* out = f(theta K) v with f = 1/(1-z) (func INV), e^z (EXP, Eq. Neudeckerd)
 * or phi_k (PHI, k in 0..4).  v and out are device tensors in the user layout
 * and may alias. */
fcgle_status fcgle_apply_f(fcgle_handle h, int func, int k, double theta,
                           const void* v, void* out);

/* The spectral scalars f(theta lam) (Sec. 3.2 after Eq. fKu_diag: the entries
 * of diag(f(Lam_1 (+) ... (+) Lam_d)); Eq. phi for phi_k) evaluated on the
 * device with exactly the arithmetic this handle's kernels use, for a host
 * list of real eigenvalue sums s_j (lam_j = (nu + i eta) s_j, s_j being a sum
 * of eigenvalues of the D_mu in the kernels):
 *     out_host[2 j] + i out_host[2 j + 1] = f(theta (nu + i eta) s_j),
 * f as in fcgle_apply_f (INV, EXP, PHI with k in 0..4).  FP64 handles evaluate
 * in FP64 (power series for |z| < 1, the recurrence of Eq. phi otherwise);
 * BF16X3 handles in FP32 as the tensor-core epilogues do: flags = 0 is the
 * generic evaluator of fcgle_apply_f's epilogue, flags = 1 (PHI, k in 1..3)
 * the per-launch polynomial in s along the ray theta (nu + i eta) that the
 * scheme epilogues use.  For inspection and testing of the reduced-precision
 * scalars; count entries, synchronises the stream, allocates two small
 * temporary device buffers. */
fcgle_status fcgle_spectral_scalars(fcgle_handle h, int func, int k, double theta, int count, const double* s_host,
                                    double* out_host, int flags);

/* One step of a one-step scheme (every scheme except LBDF2), in place:
 * u <- step(t, u) with step size tau > 0. */
fcgle_status fcgle_step(fcgle_handle h, int scheme, double tau, double t, void* u);

/* nsteps >= 0 constant steps of size tau from (t0, u0); the result goes to
 * uT (u0 and uT may alias).  LBDF2 starts with one LIE step (Eq. lbdf2-v). */
fcgle_status fcgle_integrate(fcgle_handle h, int scheme, double tau, int nsteps, double t0,
                             const void* u0, void* uT);

/* As fcgle_integrate with HOST buffers: copies u0 host -> device, integrates,
 * copies the result device -> host and synchronises the stream. */
fcgle_status fcgle_integrate_host(fcgle_handle h, int scheme, double tau, int nsteps, double t0,
                                  const void* u0_host, void* uT_host);

/* Gradient of the final-time misfit J = 1/2 sum_j |u_j(T) - u_target,j|^2
 * (T = t0 + nsteps tau, no cell volume) with respect to the initial state and
 * the parameters, by the discrete adjoint of the scheme (only
 * FCGLE_LAWSON_RK2; others give FCGLE_ERR_UNSUPPORTED).  Gradients are in the
 * real sense: grad_u0 = dJ/dRe u0 + i dJ/dIm u0 (device tensor, user layout);
 * grad_params[5] (host) = dJ/d(nu, eta, gamma, kappa, zeta); *loss (host) = J.
 * States are checkpointed every ckpt_every steps (0: one segment) and each
 * segment is recomputed once, so the cost is about three forward runs and
 * the extra device memory (5 ckpt_every + nsteps / ckpt_every + 9) tensors.
 * Synchronises the stream and reports device-side failures as fcgle_sync does;
 * a non-finite loss or parameter gradient gives FCGLE_ERR_NUMERIC.  The
 * exponential is applied in the Tucker form (Eq. fKu_diag with f = exp). */
fcgle_status fcgle_adjoint(fcgle_handle h, int scheme, double tau, int nsteps, double t0, const void* u0,
                           const void* u_target, int ckpt_every, void* grad_u0, double* grad_params,
                           double* loss);

/* Discrete L2 norm (prod_mu h_mu sum_j |u_j|^2)^{1/2} (Sec. 4) of a device
 * tensor, written to *out_host (synchronises the stream). */
fcgle_status fcgle_norm(fcgle_handle h, const void* u, double* out_host);

/* The same discrete L2 norm without a handle and without allocating device
 * memory.  The paper has no counterpart: this is a library convenience.
 *
 * Who needs it: fcgle_norm needs a handle, and fcgle_setup allocates about
 * fifteen state-sized work tensors; a caller that only wants the norm of a
 * tensor it already holds cannot always afford that, e.g. a monitor running
 * beside a solve that has already committed the device memory to its own
 * tensors, or code that must not call cudaMalloc/cudaFree (which synchronise
 * the device) while other work is in flight.
 *
 * p:   only d, n[], a[], b[] and precision are read (the cell volume is
 *      prod_mu (b_mu - a_mu) / (n_mu + 1), as in fcgle_norm); the other fields
 *      are ignored.
 * u:   device tensor in the user layout, complex128 (FCGLE_FP64) or complex64
 *      (FCGLE_BF16X3), caller-owned; read in place.
 * cuda_stream: the stream the two reduction kernels run on (NULL: the legacy
 *      default stream); the call synchronises it before returning.
 * out_host: the norm, sqrt(cell * sum_j |u_j|^2), accumulated in FP64.
 *
 * Scratch: a fixed array of 32769 doubles (256 KB) in the library's static
 * device memory holds one partial sum per chunk of 8192 entries, so at most
 * 268435456 (2^28) complex entries are accepted; larger tensors are rejected
 * with FCGLE_ERR_INVALID_ARG before anything runs on the device.  Every scratch
 * slot is written before it is read: nothing has to start at zero.  The fixed
 * chunking makes the result bitwise reproducible.
 *
 * Setup: the first call on each device (with that device current) looks up the
 * scratch array's device address once; make that first call before any stream
 * capture begins.  Nothing is promised about capturing calls into a graph.
 *
 * Concurrency: there is one scratch array per device and process, so calls
 * that overlapped on one device would race on it; the library serialises them
 * with a host lock held until the call returns. */
fcgle_status fcgle_norm_static(const fcgle_params* p, const void* u, void* cuda_stream, double* out_host);

/* Synchronises the handle's stream and reports device-side failures of the
 * work enqueued so far: FCGLE_ERR_TIMEOUT if a bounded wait inside a
 * tensor-core kernel gave up (its output is then invalid), FCGLE_ERR_NUMERIC
 * if a result tensor held a NaN or an Inf, FCGLE_ERR_CUDA on an asynchronous
 * CUDA error.  The first failure recorded since the last report wins; the
 * word is cleared when it is reported. */
fcgle_status fcgle_sync(fcgle_handle h);

/* Self-test of the bounded device-side waits (a library facility, not a step
 * of the method).  Every mbarrier wait of the tensor-core kernels is bounded
 * by a 2 s wall-clock limit, after which the kernel records a code in a device
 * error word and returns, so that the context stays usable and the host can
 * report FCGLE_ERR_TIMEOUT (see fcgle_sync).  This call runs that same wait on
 * an mbarrier that nothing ever completes (one warp, no data), then a second
 * kernel on the same stream, and synchronises the stream; it takes about 2 s.
 *
 * cuda_stream: a cudaStream_t (NULL: the legacy default stream).
 * code_out:    receives the code the wait recorded (99 for this wait).
 *
 * Returns FCGLE_ERR_TIMEOUT with *code_out = 99 when the wait gave up at its
 * limit, reported it, and the follow-up kernel ran: the expected outcome.
 * Any other status means the mechanism failed (FCGLE_ERR_CUDA if the wait
 * completed or the follow-up did not run); NULL code_out gives
 * FCGLE_ERR_INVALID_ARG before anything runs. */
fcgle_status fcgle_selftest_bounded_wait(void* cuda_stream, int* code_out);

/* Sizes: N (complex elements of a user tensor) and the bytes of one user
 * tensor. */
fcgle_status fcgle_sizes(fcgle_handle h, size_t* n_elems, size_t* n_bytes);

/* Internal layout size: P = p_1 * ... * p_d, p_mu = n_mu rounded up to a
 * multiple of 4 (FP64 handles) or 8 (BF16X3 handles).  An internal tensor is two planes (re, im) of P reals
 * (double for FP64 handles, float for BF16X3 handles), each plane in vec
 * order on the padded extents, padding exactly zero. */
fcgle_status fcgle_internal_elems(fcgle_handle h, size_t* P);

/* One raw mu-mode product (Sec. 3.2) on internal-layout device buffers, for
 * kernel-level testing and timing:
 *   Y[c][i][r] = sum_k M[i][k] X[c][r][k],   M = Q_mu^T (flags bit 0 set) or Q_mu,
 * where X is read with direction mu as its fastest index (r = every other
 * index, in order) and Y gets direction mu as its slowest index.  By default
 * X and Y hold 2 P reals each (double / float).  flags bit 1 (BF16X3 handles
 * only): X and Y are in the split form the tensor-core kernel reads and
 * writes, 4 P bf16 = the hi planes (re, im) followed by the lo planes, each
 * value being hi + lo.  flags bit 2 (BF16X3 handles only, not with bit 1):
 * the precise product used for the first and last Tucker operators of a time
 * integration, FP32 in and out: split-TF32 (x = hi + lo, both TF32, three
 * tensor-core products hi.hi + hi.lo + lo.hi, about 2^-21 relative) when
 * d >= 2, R is a multiple of 8 and p_mu <= 256 (the tensor core's FP32
 * accumulation error grows with the contracted length), FP32 on the CUDA
 * cores otherwise.  flags bit 3 (BF16X3 handles, d = 3, p_2 <= 256, with
 * bit 1, direction 0): the slab-fused mode-1 and mode-2 products in the
 * natural order, Y[c][j3][i2][i1] = sum M_2[i2][j2] M_1[i1][j1]
 * X[c][j3][j2][j1] with M_mu = Q_mu^T (bit 0) or Q_mu.  flags bit 4 (BF16X3
 * handles, d >= 2, R % 8 == 0, with bit 1, direction d-1): the product above
 * with X read in the natural order, X[c][k][r] (direction mu slowest); Y as
 * above.  Other flag bits or combinations give FCGLE_ERR_INVALID_ARG.  X and
 * Y must not overlap.  direction in 0..d-1. */
fcgle_status fcgle_mode_product(fcgle_handle h, int direction, int flags, const void* X, void* Y);

/* The kernel autotuner (a library facility, not a step of the method).  The
 * split-BF16 plain mode product has several tile and shared-memory ring
 * configurations (X ring 4 / 3 / 2 deep with the M ring taking the rest, the
 * block of M resident in shared memory for p <= 256, or wide tiles of 128 r
 * per plane); the best one depends on the contracted extent p and on the
 * number of units per SM.  fcgle_setup and fcgle_batch_create time every
 * eligible configuration once per process for each new (p, R) a handle runs
 * the plain product on, on the handle's work buffers (synchronously, a few
 * kernel launches each), and the fastest is used from then on.  For 3D
 * handles fcgle_setup also times one Tucker operator in the rotating and in
 * the slab-fused form (fcgle_set_tucker_form) once per process per extents
 * (p_1, p_2, p_3).  The environment variable FCGLE_PLAIN_CFG=<id> (0..5,
 * read once) forces one configuration where it is eligible.
 * This call writes a text report, one line per tuned shape with the time of
 * every eligible configuration and the choice, into buf (size bytes,
 * NUL-terminated, truncated if short) and the full length + 1 into *needed
 * (either pointer may be NULL). */
fcgle_status fcgle_autotune_report(char* buf, size_t size, size_t* needed);

/* Number of kernel launches this handle has issued since setup (all
 * entry points; used to report launch counts). */
fcgle_status fcgle_launch_count(fcgle_handle h, long long* count);

fcgle_status fcgle_destroy(fcgle_handle h);

/* ---------------------------------------------------------------- batches
 * Many independent instances (uneven sizes and parameters) advanced together.
 * The instances are spread over nstreams internal streams (longest processing
 * time first on the mode-product work; nstreams <= 0: min(count, 16)) and set
 * up in parallel host threads.  fcgle_batch_integrate with use_graph != 0
 * captures one time step of all instances (fork/join over the streams) into a
 * CUDA graph, cached per (scheme, tau), and launches it once per step; with
 * sources present (time-dependent steps) it enqueues the kernels directly. */
typedef struct fcgle_batch_ctx* fcgle_batch;

/* Creates the instances (in parallel host threads), then synchronises the
 * device and runs the autotuner for each instance in turn, so that no other
 * work overlaps its timing launches. */
fcgle_status fcgle_batch_create(int count, const fcgle_params* params, void* cuda_stream, int nstreams,
                                fcgle_batch* out);

/* Handle of instance i, owned by the batch (use it for set_source /
 * set_coefficients / apply_f / sync; do not destroy it or change its stream).
 * Calls on it run on one of the batch's internal non-blocking streams, which
 * are not ordered after work on the caller's stream: make their inputs ready
 * first (e.g. synchronise the device). */
fcgle_status fcgle_batch_instance(fcgle_batch b, int i, fcgle_handle* h);

/* nsteps steps of every instance i from u0[i] into uT[i] (device tensors in
 * each instance's user layout and precision).  Asynchronous on the batch's
 * stream (the stream given at creation), joined back to it at the end.
 * use_graph: 0 enqueues every instance's kernels directly (one launch per mode
 * product); 1 captures one step of all instances into a CUDA graph and replays
 * it; 2 (grouped) additionally merges the instances: each phase of a step
 * (the k-th mode product of a Tucker operator of every instance) becomes one
 * persistent launch over a device table of all instances' tensor maps, sizes
 * and epilogue parameters, so a step of the batch is a few launches whatever
 * the number of instances; the phases are captured into a graph per
 * (scheme, tau) and rebuilt when fcgle_set_coefficients or fcgle_set_source
 * changed an instance since the capture.  Grouped needs BF16X3 instances with
 * d >= 2 and falls back to 1 otherwise.  Steps with a source term run with
 * direct launches.  The call is asynchronous and reports no device-side
 * failure itself: call fcgle_sync on the instance handles to collect them (a
 * timeout inside a grouped launch is recorded on instance 0's handle, a
 * non-finite result on the instance's own handle). */
fcgle_status fcgle_batch_integrate(fcgle_batch b, int scheme, double tau, int nsteps, double t0,
                                   const void* const* u0, void* const* uT, int use_graph);

/* Kernel launches issued by all instances so far and graph launches so far. */
fcgle_status fcgle_batch_launch_count(fcgle_batch b, long long* kernels, long long* graph_launches);

fcgle_status fcgle_batch_destroy(fcgle_batch b);

const char* fcgle_status_string(fcgle_status s);

/* Thread-local description of the last error on this thread ("" if none). */
const char* fcgle_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FCGLE_H */
