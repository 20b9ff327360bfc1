// Library context: configuration, workspace carving and the per-step
// device buffers of the QR-CTMRG iteration.
#pragma once

#include <string>
#include <vector>

#include "qrctm.h"
#include "qrctm_internal.cuh"

struct qrctm_ctx {
  qrctm_config cfg;
  cudaStream_t st;
  int d, D, D2, chi;   // chi = target environment bond
  int chi_cur;         // current bond (< chi only if the warm-up could not grow it)
  bool split_layers;
  bool split_prec;
  bool network;        // a classical network tensor is given directly (bond D2 = D)
  // workspace
  char* ws;
  size_t ws_bytes;
  // state
  double *A, *C, *T, *Cn, *Tn, *Craw, *Traw;
  // step intermediates
  double *Mcm, *Q, *R, *X1, *Z, *X2, *Y2;
  // warm-up
  double *Xs, *Yw;
  // spectrum
  double *spec_work, *s_cur, *s_prev, *delta_d;
  // corner of a fresh environment whose spectrum is still to be taken: the
  // first convergence test reduces it beside the current corner
  double *C_init, *spec_work2;
  int chi_init;
  bool spec_pending;
  double* partials;
  double* tmpA;
  double* a;           // double layer (only with DOUBLE layers)
  // energy
  double *E1, *E2, *E3, *rho, *e_d;
  // split precision: FP32 operand copies (rows padded to 4 floats) and the
  // tensor-core split-K partial sums
  float *T32, *C32, *Qt32, *Qc32, *Ts32, *Rt32, *Aket32, *Abra32, *tc_part, *qr32;
  // TF32 tails of the pre-split operands (T32, C32, Qt32, Qc32 then hold the heads)
  float *T32lo, *C32lo, *Qt32lo, *Qc32lo, *Rt32lo;
  long long tc_part_elems;
  // gradient
  char* G;             // gradient region base (carved by grad.cu)
  size_t G_bytes;
  qrctm::QrWork qrw;
  int* err;
  int iters;
  int grad_iters;
  double grad_resid;
  double grad_fp_resid;   // ||G(x) - x|| / ||x|| at the last implicit gradient
  bool nn_plain;          // plain NN bond (model->sublattice_rotation == 0)
  cudaEvent_t panel_ev;   // open panel-phase event (profiling)
  // standard (eigendecomposition) method
  void* solver;            // cusolverDnHandle_t, created on first use
  double* eig_E;           // dense symmetric enlarged corner, then its eigenvectors
  double* eig_w;           // eigenvalues
  double* eig_work;        // solver workspace
  size_t eig_work_doubles;
  int* eig_info;
  int* eig_idx;            // kept eigenvalue indices, by rank
  // L-BFGS optimisation (qrctm_optimize): pair ring S, Y (opt_hist x n),
  // accepted / trial points and gradients, direction, scratch, the
  // environments of the accepted point and of the last evaluation
  int opt_hist;
  double *opt_S, *opt_Y, *opt_x, *opt_xt, *opt_g, *opt_gt, *opt_p, *opt_q, *opt_out;
  double *opt_Cp, *opt_Tp, *opt_Cc, *opt_Tc;
  bool grad_keep_env;      // an unrolled gradient leaves (C, T) after its k steps
  char* tape_store;        // tapes of up to tape_store_k steps (unrolled gradient)
  int tape_store_k;
  // split-precision contractions of the energy and adjoint passes
  bool mm_split;
  float* mm32;
  size_t mm32_floats;
  double last_delta;
  bool have_env;
  bool spec_valid;
  std::string last_error;
  // one QR-CTMRG step as a CUDA graph (captured on g_stream, replayed on st)
  cudaGraphExec_t g_exec;
  cudaStream_t g_stream;
  int g_chi;                       // environment bond the graph was captured for
  unsigned long long g_launches;   // kernels in the graph
  bool graph_off;                  // capture failed once: eager launches
  // phase timing (qrctm_set_profiling)
  bool prof;
  struct PhaseRec { int ph; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<PhaseRec> recs;
  double ph_ms[QRCTM_NUM_PHASES];
  long long ph_n[QRCTM_NUM_PHASES];
};

namespace qrctm {

// Records a pair of CUDA events around a phase when profiling is on.
struct PhaseScope {
  qrctm_ctx* c;
  int ph;
  cudaEvent_t a;
  PhaseScope(qrctm_ctx* c_, int ph_);
  ~PhaseScope();
};

// A contraction descriptor that may use the context's split-K scratch.
inline Gemm gemm_ctx(qrctm_ctx* c) {
  Gemm g = gemm_init();
  g.part = c->qrw.splitk;
  g.part_elems = kSplitKElems;
  return g;
}

// Contraction of the energy / adjoint passes: split precision (TF32x3 on the
// tensor cores from gathered FP32 operands) when c->mm_split, else FP64.
cudaError_t gemm_run(qrctm_ctx* c, const Gemm& g);
// gemm_run with K cut into chunks of at most kchunk (a multiple of 4; 0 = one
// pass) on the tensor-core engine, the chunk results summed in FP64.
cudaError_t gemm_run_kchunked(qrctm_ctx* c, const Gemm& g, long long kchunk);
size_t mm_split_floats(const Gemm& g);

// Workspace plan (api.cu); 256-byte aligned regions.
size_t make_plan(const qrctm_config& cfg, bool carve, qrctm_ctx* ctx);

// Steps (ctmrg.cu)
cudaError_t reduced_corner(qrctm_ctx* c, const double* C, const double* T, int chi_in,
                           double* Mcm);
cudaError_t renorm_edge(qrctm_ctx* c, const double* P, int chi_out, const double* T,
                        int chi_in, double* Tout);
cudaError_t qr_step(qrctm_ctx* c);
cudaError_t warmup_step(qrctm_ctx* c, int chi_in, int chi_out);
cudaError_t spectrum_check(qrctm_ctx* c);

// Split-precision step (split_step.cu)
cudaError_t split_prepare_A(qrctm_ctx* c);
cudaError_t qr_step_split(qrctm_ctx* c);
// One QR-CTMRG step of the context's precision, in place on (C, T), replayed
// from the context's CUDA graph (api.cu)
cudaError_t qr_step_graph(qrctm_ctx* c);
// Standard step with a full eigendecomposition (eigen_step.cu)
cudaError_t eigen_step(qrctm_ctx* c, int ci, int co);
size_t eigen_work_doubles(long long m);
void eigen_release(qrctm_ctx* c);
// fused ket + bra absorption (FP32), see absorb.cu
// tensor-core absorption of both layers (d = 2, D = 6; absorb_tc.cu)
bool absorb_tc_ok(int d, int D);
cudaError_t absorb_tc(const float* X1, const float* Ak, const float* Ab, float* X2, int ch,
                      long long D2p, long long dD2p, long long mp, int* err, cudaStream_t s);
bool absorb_fused_ok(int d, int D);
// FP64 ket + bra in one kernel (FP64 path, d = 2, D = 4, 6): X1 slice-contiguous
// [(mu,b)][(u_b,k_b)][(u_k,k_k)], X2 [(mu,b)][(d_k,j_k)][(d_b,j_b)], ngroups slices.
bool absorb64_ok(int d, int D);
cudaError_t absorb64(const double* X1, const double* A, double* X2, long long ngroups, int d, int D,
                     int* err, cudaStream_t s);
cudaError_t absorb_fused(const float* X1, const float* Ak, const float* Ab, float* X2, int ch,
                         int D, int d, long long D2p, long long dD2p, long long mp, int* err,
                         cudaStream_t s);

// Classical networks (network.cu)
cudaError_t network_boundary(int b, const double* a, const double* v, double* C0, double* T0,
                             cudaStream_t s);
cudaError_t network_traces(qrctm_ctx* c, const double* a_obs);

// L-BFGS device helpers (optimize.cu), one block each
cudaError_t lbfgs_direction(int n, int cnt, int head, int hist, const double* S, const double* Y,
                            const double* g, double* q, double* p, double* out, cudaStream_t s);
cudaError_t lbfgs_trial(int n, const double* x, double a, const double* p, double* xt,
                        cudaStream_t s);
cudaError_t lbfgs_pair(int n, const double* xt, const double* x, const double* gt,
                       const double* g, double* s_out, double* y_out, double* out,
                       cudaStream_t s);

// Layout of the double-layer intermediate X2 and the enlarged corner read from
// it.  An iPEPS double layer keeps X2[m][b][d_k][j_k][d_b][j_b] (the ket and
// bra halves of the d and j legs apart, the order the split-layer absorption
// produces); a network tensor has no halves and X2 is X2[m][b][d][j].
//   store_n: column (d, j) of the absorption output -> offset in an X2 row
//   ct_row:  (b, l) -> offset (row of Ct, contraction index of the projection)
//   ct_col:  (r, j) -> offset (column of Ct, row of the projection output)
struct X2Maps { IdxMap store_n, ct_row, ct_col; };
inline X2Maps x2_maps(const qrctm_ctx* c, int ci) {
  const int D = c->D, D2 = c->D2;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  X2Maps x;
  if (c->network) {
    x.store_n = im1(1);
    x.ct_row = im2(D2, D2, D4);
    x.ct_col = im2(D2, 1, (long long)ci * D4);
  } else {
    x.store_n = im4(D, D, D, 1, D2, D, D3);
    x.ct_row = im3(D, D, D, D3, D4);
    x.ct_col = im3(D, D, 1, D2, (long long)ci * D4);
  }
  return x;
}

// Energy (energy.cu)
cudaError_t energy_fp64(qrctm_ctx* c, double J1, double J2);
// FP64 traces Tr(P_p P_q) of nb <= 4 matrices (m x m at P + p m^2) and their
// cotangent Pb_p = sum_q (rhob + rhob^T)[p][q] P_q^T; part: kTraceParts * 16
// doubles of scratch (the context's partials).
constexpr int kTraceParts = 1184;
bool trace_pairs_ok(int nb);
cudaError_t trace_pairs(const double* P, int nb, long long m, double* part, double* rho,
                        cudaStream_t s);
cudaError_t trace_pairs_vjp(const double* P, int nb, long long m, const double* rhob, double* Pb,
                            cudaStream_t s);

// Gradient (grad.cu)
size_t grad_bytes(int d, int D, int chi);

}  // namespace qrctm
