/*
 * qrctm.h -- C ABI of the B300 (sm_103a) QR-CTMRG library.
 *
 * The library contracts a C4v-symmetric infinite PEPS made of one real
 * rank-5 tensor A[s,u,l,d,r] (physical dimension d, bond dimension D) with
 * the corner transfer matrix renormalisation group in which the isometry
 * comes from an unpivoted QR decomposition of the reduced corner
 * ct = C T (Zhang, Yang, Corboz, arXiv 2505.00494: QR-CTMRG paragraph and
 * Fig. 1(e,f)), and evaluates the Heisenberg / J1-J2 energy per site and its
 * gradient with respect to A (Results paragraphs; Automatic differentiation
 * paragraph; fixed-point differentiation as in the Discussion).
 *
 * Conventions (all arrays row-major, FP64, on the device unless stated):
 *   A   [d][D][D][D][D]       legs (s, up, left, down, right)
 *   C   [chi][chi]            corner, symmetric, unit Frobenius norm
 *   T   [chi][D*D][chi]       edge, T[a][k][b] = T[b][k][a], unit norm;
 *                             inner leg k = x*D + x' (ket-major)
 * Every call returns a qrctm_status.  No exception or abort crosses the ABI.
 * All device work is queued on the stream given in the configuration; calls
 * that return host scalars synchronise that stream.  The caller owns every
 * pointer it passes; the library never frees them.  The library allocates no
 * device memory for data: all scratch lives in the caller's workspace (the
 * only driver objects a context creates are the stream and CUDA graph that
 * qrctm_step replays, released by qrctm_destroy).
 */
#ifndef QRCTM_H
#define QRCTM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QRCTM_OK = 0,
  QRCTM_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported option   */
  QRCTM_ERR_CUDA = 2,          /* a CUDA runtime call failed (see last_error)  */
  QRCTM_ERR_NOT_CONVERGED = 3, /* max_iter reached; the context stays usable   */
  QRCTM_ERR_NUMERIC = 4,       /* NaN/Inf or a zero norm met in a kernel       */
  QRCTM_ERR_NOT_SYMMETRIC = 5, /* A is not C4v symmetric (rel. tol 1e-12)      */
  QRCTM_ERR_WORKSPACE = 6,     /* workspace smaller than required              */
  QRCTM_ERR_TIMEOUT = 7,       /* a bounded device-side wait ran out           */
  QRCTM_ERR_STATE = 8          /* call out of order (e.g. step before init)    */
} qrctm_status;

typedef enum { QRCTM_FP64 = 0, QRCTM_SPLIT = 1 } qrctm_precision;
typedef enum {
  QRCTM_LAYERS_AUTO = 0,
  QRCTM_LAYERS_DOUBLE = 1,
  QRCTM_LAYERS_SPLIT = 2,
  /* a classical network tensor a[u,l,d,r] is given directly (Discussion:
     classical partition functions); D is its bond, T's inner leg has D (not
     D^2) values, d must be 1, precision FP64, with_nnn = with_grad = 0 */
  QRCTM_LAYERS_NETWORK = 3
} qrctm_layers;
typedef enum { QRCTM_GRAD_IMPLICIT = 0, QRCTM_GRAD_UNROLL = 1 } qrctm_grad_mode;
typedef enum { QRCTM_METHOD_QR = 0, QRCTM_METHOD_EIGEN = 1 } qrctm_method;

typedef struct {
  int d;              /* physical dimension (>= 1)                               */
  int D;              /* virtual bond dimension (>= 1)                           */
  int chi;            /* environment bond dimension (D*D .. 1024)                */
  int precision;      /* qrctm_precision: FP64 everywhere, or split TF32x3
                         contractions on the tensor cores with FP64 QR panels,
                         normalisation, spectrum and energy traces               */
  int layers;         /* qrctm_layers: AUTO picks SPLIT (ket and bra layers
                         absorbed one after the other) when 2*d < D*D            */
  int warmup_steps;   /* standard-CTMRG steps in qrctm_init_env (0 = automatic:
                         max(2, steps needed to grow chi from D^2); -1 = none,
                         i.e. keep the bulk-initialised boundary, chi = D^2)     */
  int check_every;    /* convergence test every this many steps (>= 1)          */
  double tol;         /* default convergence tolerance on the corner spectrum   */
  int max_iter;       /* default iteration cap                                  */
  int grad_max_iter;  /* cap on applications of J^T in the adjoint solve (0 = 200) */
  double grad_tol;    /* relative residual target of the adjoint solve (0 = 1e-12) */
  int with_nnn;       /* 1: reserve workspace for the J2 (2x2 patch) energy term */
  int with_grad;      /* 1: reserve workspace for qrctm_energy_grad              */
  void* stream;       /* cudaStream_t; NULL = legacy default stream             */
  int method;         /* qrctm_method: QR (QR-CTMRG, QR-CTMRG paragraph) or EIGEN
                         (standard C4v CTMRG with a full eigendecomposition of the
                         enlarged corner, Standard CTMRG paragraph; FP64 only, the
                         comparison method; cuSOLVER's handle keeps a small device
                         state of its own)                                      */
  int opt_history;    /* > 0: reserve workspace for qrctm_optimize keeping up to this
                         many L-BFGS pairs (1..32; needs with_grad)             */
  int grad_store;     /* 0..32 (needs with_grad): reserve workspace for the tapes of
                         this many steps.  An unrolled gradient of k <= grad_store
                         steps then records each step's tape once on the way
                         forward and reads it on the way back; otherwise (0, or
                         k larger) it keeps only each step's (C, T) and re-runs
                         the step's forward pass before its reverse pass.  The
                         result is the same derivative either way.  Costs
                         grad_store x (the bytes of one tape, about 4 (chi D^2)^2
                         doubles) of workspace.                                  */
} qrctm_config;

typedef struct {
  double J1;          /* nearest-neighbour coupling                              */
  double J2;          /* next-nearest-neighbour coupling (plain bond)            */
  int sublattice_rotation;  /* 1: the NN bond is taken with one sublattice rotated
                         by exp(i pi sigma^y / 2) (Results, Heisenberg paragraph),
                         h~ = (-XX + YY - ZZ)/4, so that the Neel state is the
                         uniform C4v state; 0: the plain bond (XX + YY + ZZ)/4 on
                         NN pairs too.  NNN pairs share a sublattice: plain bond. */
} qrctm_model;

typedef struct qrctm_ctx qrctm_ctx;

/* Phases of the iteration timed by qrctm_phase_times (kernels K1..K9 of the
 * step: reduced corner, QR, the three contractions of T', corner update,
 * symmetrise/normalise, spectrum), plus the energy and gradient calls. */
enum {
  QRCTM_PH_CT = 0,        /* ct = C T                       (Fig. 1(e))        */
  QRCTM_PH_QR = 1,        /* ct = Q R                       (QR-CTMRG para.)   */
  QRCTM_PH_X1 = 2,        /* X1 = Q^T T                                          */
  QRCTM_PH_ABSORB = 3,    /* ket and bra layers of A absorbed                    */
  QRCTM_PH_PROJECT = 4,   /* T' = X2 Q                                           */
  QRCTM_PH_CORNER = 5,    /* C' from T', R, Q               (Fig. 1(f))        */
  QRCTM_PH_SYMNORM = 6,   /* symmetrise and normalise C', T'                     */
  QRCTM_PH_SPECTRUM = 7,  /* |eig(C)| and its change                             */
  QRCTM_PH_ENERGY = 8,    /* reduced density matrices and energy                 */
  QRCTM_PH_GRAD = 9,      /* adjoint (gradient) passes                           */
  QRCTM_PH_WARMUP = 10,   /* standard warm-up steps                              */
  QRCTM_PH_QR_PANEL = 11, /* the FP64 panel factorisations inside QR (nested)     */
  QRCTM_NUM_PHASES = 12
};

/* Bytes of device workspace needed for `cfg` (0 if cfg is invalid).  Host
 * only; no CUDA call. */
size_t qrctm_workspace_bytes(const qrctm_config* cfg);

/* Create a context over a caller-owned device workspace of `bytes` bytes
 * (256-byte aligned).  The workspace must stay valid until qrctm_destroy.
 * Errors: INVALID_ARG (bad cfg, null or misaligned pointer), WORKSPACE (too
 * small; both checked before any CUDA call). */
qrctm_status qrctm_create(const qrctm_config* cfg, void* workspace, size_t bytes,
                          qrctm_ctx** out);
void qrctm_destroy(qrctm_ctx* ctx);

/* Set the iPEPS tensor and initialise the environment (QR-CTMRG paragraph:
 * a few standard steps first, growing chi to the target).
 * A: device, d*D^4 doubles, must be C4v symmetric (checked, NOT_SYMMETRIC
 *    otherwise); copied into the workspace.
 * C0, T0: optional device environment (chi*chi and chi*D^2*chi).  If both are
 *    given they are symmetrised, normalised and used as is (no warm-up).  If
 *    both are NULL the boundary is built from A (contracting the ket and bra
 *    legs on the open boundary, footnote of the Standard CTMRG paragraph) and
 *    grown to chi by `warmup_steps` standard steps whose isometry spans the
 *    dominant-|eigenvalue| subspace of the enlarged corner (block subspace
 *    iteration, Fig. 1(d)). */
qrctm_status qrctm_init_env(qrctm_ctx* ctx, const double* A, const double* C0, const double* T0);

/* qrctm_init_env from host memory: A (d*D^4 doubles) and the optional C0, T0
 * (both or neither) are host arrays, copied to the device on the context's
 * stream inside this call (pinned memory makes the copies asynchronous
 * DMA).  A is staged in a per-step scratch region of the workspace, C0 and
 * T0 in the raw environment buffers; the call then proceeds as
 * qrctm_init_env.  Same errors; the caller keeps ownership of its arrays. */
qrctm_status qrctm_init_env_host(qrctm_ctx* ctx, const double* A_host, const double* C0_host,
                                 const double* T0_host);

/* Run n_steps QR-CTMRG steps (Fig. 1(e,f)).  If delta_out is non-NULL the
 * corner spectrum change since the previous test is computed and returned
 * (host double; synchronises).  The first step at a given environment bond
 * captures the step's launches into a CUDA graph (on a stream the context
 * creates) that later steps replay on the configured stream; with profiling
 * on, or where capture fails, the launches are issued one by one. */
qrctm_status qrctm_step(qrctm_ctx* ctx, int n_steps, double* delta_out);

/* Step until the change of the sorted, normalised |eig(C)| between two
 * tests (every check_every steps) is below tol, or max_iter steps ("repeated
 * until convergence", Standard CTMRG paragraph).  iters_out / delta_out:
 * host, may be NULL.  Returns NOT_CONVERGED at max_iter (environment kept). */
qrctm_status qrctm_run_to_convergence(qrctm_ctx* ctx, double tol, int max_iter, int* iters_out,
                                      double* delta_out);

/* Energy per site 2 J1 <h~>_nn + 2 J2 <h>_nnn of the current environment
 * (Results paragraphs: Heisenberg bond with the sublattice rotation
 * exp(i pi sigma^y / 2) on one sublattice for nearest neighbours; plain
 * bond for next-nearest neighbours).  d must be 2; J2 != 0 needs with_nnn.
 * e_out: host. */
qrctm_status qrctm_energy(qrctm_ctx* ctx, const qrctm_model* model, double* e_out);

/* Energy and its gradient with respect to A at the converged environment
 * (Automatic differentiation paragraph; fixed-point AD, Discussion).
 * mode IMPLICIT: adjoint fixed point of two QR-CTMRG steps at the current
 * environment (the map's fixed point up to the sign gauge it alternates);
 * mode UNROLL: backpropagation through k_unroll steps started from the
 * current (detached) environment (1 <= k_unroll <= 32).  grad: device,
 * d*D^4 doubles, the C4v-projected gradient.  e_out: host, the energy at the
 * current environment (implicit) or after the k steps (unroll).  Needs
 * with_grad (and with_nnn when J2 != 0), d = 2, D >= 2.  All reverse passes
 * run in FP64 for an FP64 context; a split-precision context runs every
 * contraction of the taped steps, of the energy and of the reverse passes on
 * the TF32x3 tensor-core engine and factors ct with the step's own split QR
 * (FP32-class, e_out included; the QR panels, the QR adjoint's product with
 * R^-T, normalisations and traces stay FP64).  Unroll mode keeps the k tapes
 * in the workspace when grad_store >= k, else re-runs each step's forward
 * pass before its reverse pass (same result).  Implicit mode solves
 * (I - J^T) xbar = dE/d(env), J the
 * Jacobian of the two steps, by restarted GMRES(40); it stops when the
 * relative residual falls below grad_tol or after grad_max_iter
 * applications of J^T (each one reverse pass through both steps). */
qrctm_status qrctm_energy_grad(qrctm_ctx* ctx, const qrctm_model* model, int mode, int k_unroll,
                               double* grad, double* e_out);

/* ----- classical networks (layers = QRCTM_LAYERS_NETWORK) ----------------- */

/* Set the network tensor and the boundary (Discussion: QR-CTMRG applies to
 * classical partition functions).  a: device, D^4 doubles, a[u,l,d,r]
 * row-major, C4v symmetric (checked to 1e-12 relative, else
 * QRCTM_ERR_NOT_SYMMETRIC); copied into the workspace.  v: device, D
 * doubles, or NULL for all ones: the legs pointing out of the system are
 * contracted with v,
 *   C0[d,r] = sum_{u,l} v[u] v[l] a[u,l,d,r],  T0[u,r,d] = sum_l v[l] a[u,l,d,r],
 * (a fixed-spin vector selects one ordered state), then the warm-up steps
 * grow chi as in qrctm_init_env.  C0, T0: optional device environment
 * (chi*chi and chi*D*chi doubles, both or neither); when given they are
 * symmetrised, normalised and used as is (v ignored, no warm-up), e.g. the
 * converged environment of a neighbouring coupling.  QRCTM_ERR_INVALID_ARG
 * on a context that is not in network mode. */
qrctm_status qrctm_init_env_network(qrctm_ctx* ctx, const double* a, const double* v,
                                    const double* C0, const double* T0);

/* Partition function per site and a one-site expectation value at the
 * current environment: kappa = Z11 Z00 / Z10^2 with Z00 = Tr C^4, Z10 the
 * 2x1 ring (C T C)(C T C), Z11 the 3x3 patch (four C, four T, one a), so
 * -beta f = ln kappa; obs = Z11(a_obs) / Z11(a).  a_obs: device, D^4
 * doubles (a with the observable inserted at the site), or NULL (obs_out
 * untouched).  ln_kappa_out, obs_out: host (either may be NULL).
 * QRCTM_ERR_NUMERIC when kappa <= 0 or a trace is not finite.  Runs on the
 * context's stream and synchronises it. */
qrctm_status qrctm_network_observables(qrctm_ctx* ctx, const double* a_obs, double* ln_kappa_out,
                                       double* obs_out);

/* ----- variational optimisation ------------------------------------------ */

/* Options of qrctm_optimize (Automatic differentiation paragraph).  Zero
 * fields take the defaults in brackets. */
typedef struct {
  int history;        /* L-BFGS pairs kept [the config's opt_history]           */
  int nograd_steps;   /* QR-CTMRG steps without gradient tracking per
                         evaluation (the paper takes 2; 0 is allowed)           */
  int k_unroll;       /* tracked steps of the unrolled gradient, 1..32 [10]     */
  int max_ls;         /* points tried per line search [10]                      */
  double c1;          /* Armijo constant [1e-4]                                 */
  double step0;       /* length of the first step along -g [0.1]                */
  double env_tol;     /* spectrum tolerance of a fresh environment [config tol] */
  int env_max_iter;   /* iteration cap of a fresh environment [config max_iter] */
} qrctm_lbfgs_options;

/* Minimise the energy per site over the C4v tensor A by L-BFGS (Automatic
 * differentiation paragraph).  Every evaluation at a point A' runs
 * opt->nograd_steps QR-CTMRG steps, then the energy and its gradient
 * through opt->k_unroll tracked steps (qrctm_energy_grad, UNROLL mode); it
 * starts from the environment the previous accepted point ended with, except
 * the start and the second and later points of a line search, which build a
 * fresh environment (qrctm_init_env, then qrctm_run_to_convergence to
 * env_tol).  Steps: p = -H g by the two-loop recursion (H0 = s.y/y.y), the
 * first step of length step0 along -g, later ones from alpha = 1, halved
 * until E' <= E + c1 alpha g.p (at most max_ls points); pairs with
 * s.y <= 1e-10 |s||y| are skipped; a non-descent direction resets the
 * history.  The two-loop recursion, trial points and pair updates run in
 * device kernels.
 * A: device, d*D^4 doubles, C4v symmetric; the start on entry, the last
 * accepted point on return.  energies: host, n_steps + 1 doubles (E at the
 * start and after each accepted step) or NULL.  steps_out, evaluations_out:
 * host, accepted steps and energy+gradient evaluations (either may be NULL).
 * Needs opt_history > 0 and with_grad (and with_nnn when J2 != 0).
 * Returns QRCTM_ERR_NOT_CONVERGED when a line search finds no decrease (A
 * holds the last accepted point); the loop also ends early at a zero
 * gradient. */
qrctm_status qrctm_optimize(qrctm_ctx* ctx, const qrctm_model* model,
                            const qrctm_lbfgs_options* opt, int n_steps, double* A,
                            double* energies, int* steps_out, int* evaluations_out);

/* Copy the environment out: C (chi*chi), T (chi*D^2*chi) on the device (may be
 * NULL); spectrum_host: chi doubles, sorted |eig(C)| (may be NULL). */
qrctm_status qrctm_get_env(qrctm_ctx* ctx, double* C, double* T, double* spectrum_host);

/* qrctm_get_env into host memory: C_host (chi*chi) and T_host (chi*D^2*chi)
 * (either may be NULL) are copied device-to-host on the context's stream;
 * the call returns after the copies are complete. */
qrctm_status qrctm_get_env_host(qrctm_ctx* ctx, double* C_host, double* T_host,
                                double* spectrum_host);

/* Phase timing.  With profiling on, the library records a pair of CUDA
 * events on the context's stream around every phase and opens an NVTX range
 * named "qrctm:<phase>" (ct, qr, x1, absorb, project, corner, symnorm,
 * spectrum, energy, grad, warmup, qr_panel) around its launches, which run
 * eagerly instead of from the step's CUDA graph; qrctm_phase_times
 * synchronises the stream, writes the accumulated milliseconds and the number
 * of timed occurrences of each phase since the previous call
 * (QRCTM_NUM_PHASES entries each, host arrays, either may be NULL) and resets
 * the accumulators.  Events are created on first use and reused. */
qrctm_status qrctm_set_profiling(qrctm_ctx* ctx, int enable);
qrctm_status qrctm_phase_times(qrctm_ctx* ctx, double* ms_out, long long* count_out);

/* Number of kernels this library has launched in this process so far. */
unsigned long long qrctm_kernel_launches(void);

/* Applications of J^T (implicit mode) or unrolled steps used by the last
 * qrctm_energy_grad call. */
int qrctm_grad_iterations(const qrctm_ctx* ctx);

/* Relative residual ||b - (I - J^T) xbar|| / ||b|| of the last implicit
 * adjoint solve, as estimated by GMRES (0 after an unrolled gradient).  This
 * call has no counterpart in the paper; it reports solver convergence. */
double qrctm_grad_residual(const qrctm_ctx* ctx);

/* Elementwise distance of the environment x = (C, T) from a fixed point of
 * two QR-CTMRG steps, ||G(x) - x|| / ||x|| with G = F o F, measured by the
 * last implicit qrctm_energy_grad call (0 after an unrolled one).  The
 * implicit adjoint assumes G(x) = x (Discussion: fixed-point differentiation).
 * The spectrum test that ends qrctm_run_to_convergence is gauge invariant
 * and can be met while the environment still rotates slowly within
 * near-degenerate parts of the corner spectrum; the implicit gradient's
 * error then grows with this residual, and the unrolled mode (which assumes
 * no fixed point) is the safer choice.  No counterpart in the paper. */
double qrctm_grad_fixed_point_residual(const qrctm_ctx* ctx);

/* Steps run since qrctm_init_env. */
int qrctm_iterations(const qrctm_ctx* ctx);

/* Text of the last error on this context ("" if none). */
const char* qrctm_last_error(const qrctm_ctx* ctx);

/* ----- standalone operations (no context) --------------------------------- */

/* Y = sym(X), the mean over the 8 C4v operations on the virtual legs (iPEPS
 * paragraph; n(D) free parameters per its footnote); if normalize,
 * Y /= ||Y||_F.  X, Y: device, d*D^4 doubles, distinct.  workspace:
 * qrctm_c4v_symmetrize_workspace_bytes() device bytes (only for normalize).
 * stream: cudaStream_t or NULL.  Synchronises when normalize is set. */
size_t qrctm_c4v_symmetrize_workspace_bytes(void);
qrctm_status qrctm_c4v_symmetrize(int d, int D, const double* X, double* Y, int normalize,
                                  void* workspace, size_t bytes, void* stream);

/* Unpivoted Householder QR with diag(R) >= 0 (QR-CTMRG paragraph) of a
 * column-major m x n device matrix M (m >= n >= 1, n <= 2048; otherwise
 * QRCTM_ERR_INVALID_ARG and a workspace size of 0).  Q: m x n column-major,
 * R: n x n row-major (upper triangular).  workspace: 256-byte aligned,
 * qrctm_qr_workspace_bytes(m, n) bytes, zero-filled before its first use
 * (the call leaves its control words zero again).  Synchronises. */
size_t qrctm_qr_workspace_bytes(int m, int n);
qrctm_status qrctm_householder_qr(int m, int n, const double* M, double* Q, double* R,
                                  void* workspace, size_t bytes, void* stream);

/* qrctm_householder_qr with the bound of the panel kernel's device waits made
 * explicit (the paper has no counterpart; this is the library's failure
 * detection).  Each panel column ends with a grid-wide exchange: every CTA
 * adds its partial sums and arrives on a counter, and the CTAs wait until all
 * have arrived.  A wait gives up after wait_spins polls (0 = the default,
 * 2^25, about a second) and the call returns QRCTM_ERR_TIMEOUT instead of
 * hanging; Q and R are then undefined.  extra_arrivals (>= 0) raises the
 * number of arrivals every wait expects above the CTAs launched, so that no
 * wait can be satisfied: a value above 0 exists only to exercise the timeout
 * path, from a test, without a fault.  Either way the call leaves its
 * workspace's control words zero, so the next call runs normally.
 * Synchronises `stream`. */
qrctm_status qrctm_householder_qr_bounded(int m, int n, const double* M, double* Q, double* R,
                                          void* workspace, size_t bytes, void* stream,
                                          long long wait_spins, int extra_arrivals);

/* Split-precision matrix product on the tensor cores (the contraction engine
 * of the QR-CTMRG split path):  C[m*ldc + n] = sum_k A[m*lda + k] B[n*ldb + k]
 * for 0 <= m < M, 0 <= n < N, with A, B FP32 (device, K contiguous, lda and
 * ldb multiples of 4, 16-byte aligned) and C FP64 (device, row-major).  Each
 * operand is split into a TF32 head and an FP32 tail; the three products
 * head*head + head*tail + tail*head accumulate in FP32 (about 2^-21 relative
 * error per product).  work: optional device scratch of work_elems floats; with
 * it, K is cut into chunks of at most 512 (and more chunks when the M x N
 * grid is small) whose FP32 partial sums are added in FP64; NULL = one pass
 * over K.  err_word: device int (required) that the kernel sets
 * if one of its bounded waits runs out; it is cleared first and read back, and
 * a set word is returned as QRCTM_ERR_TIMEOUT.  Synchronises `stream`. */
qrctm_status qrctm_gemm_tf32x3(int M, int N, int K, const float* A, long long lda, const float* B,
                               long long ldb, double* C, long long ldc, float* work,
                               long long work_elems, int* err_word, void* stream);

/* The same product with pre-split operands: A (optional) and B are given as
 * TF32 head planes (A, B) and tail planes (A_lo, B_lo) of the same layout,
 * as qrctm_tf32_split leaves them, so the kernel splits nothing (an operand
 * that many output tiles share is split once instead of once per tile).
 * B_lo is required; A_lo = NULL means A is plain FP32 and split in the kernel.
 * A pre-split A with a plain B is QRCTM_ERR_INVALID_ARG.  Same result
 * bits as qrctm_gemm_tf32x3 on the unsplit operands.  Synchronises. */
qrctm_status qrctm_gemm_tf32x3_presplit(int M, int N, int K, const float* A, const float* A_lo,
                                        long long lda, const float* B, const float* B_lo,
                                        long long ldb, double* C, long long ldc, float* work,
                                        long long work_elems, int* err_word, void* stream);

/* In-place split of the FP32 device matrix x (rows x cols, row stride ld >=
 * cols, rows * cols < 2^32) for the TF32x3 product: x[r*ld + c] becomes its
 * TF32 head (nearest, ties away from zero) and lo[r*ld + c] (device, same
 * layout) the TF32 tail of the remainder; a NaN stays in the head.  Elements
 * between cols and ld are left alone.  Synchronises `stream`. */
qrctm_status qrctm_tf32_split(long long rows, int cols, float* x, long long ld, float* lo,
                              void* stream);

/* Householder QR that allocates nothing: the same result as
 * qrctm_householder_qr, for callers that cannot obtain device memory of their
 * own (a plug-in handed only input/output pointers by a host application that
 * owns the device memory, a process whose device memory is already reserved
 * by another runtime, code that must not enter the CUDA allocator).  The paper
 * has no counterpart; this is a convenience of the library.  The scratch is
 * one 48 MiB array inside the library that every device loading the library
 * keeps until exit.  Limits: n <= 1024 and m * n <= 1048576 (for example
 * 5184 x 144); larger sizes return QRCTM_ERR_WORKSPACE without touching the
 * device.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, so cudaDeviceReset (which unloads the module and may move the
 * array) is not supported between calls.  All calls share the array and each clears the
 * words that must start at zero, so calls whose GPU work overlaps (other
 * streams, other host threads) race and must be serialised by the caller.
 * Synchronises `stream`. */
qrctm_status qrctm_householder_qr_noalloc(int m, int n, const double* M, double* Q, double* R,
                                          void* stream);

/* Library version string. */
const char* qrctm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QRCTM_H */
