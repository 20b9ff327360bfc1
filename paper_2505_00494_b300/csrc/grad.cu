// Energy gradient dE/dA through the QR-CTMRG fixed point (Automatic
// differentiation paragraph; fixed-point differentiation, Discussion).
//
// E(A) = e(A, x*(A)) with x* = (C*, T*) a fixed point of the iteration.  The
// QR map F alternates a sign gauge between steps, so the fixed-point equation
// is written for two steps G = F o F, x* = G(x*, A):
//   dE/dA = de/dA + xbar^T dG/dA,   (I - J_G^T) xbar = ebar,
// with ebar = de/dx and J_G = dG/dx.  xbar = sum_n (J_G^T)^n ebar formally;
// the series converges as slowly as the CTMRG iteration itself (the ratio of
// the leading transfer-matrix eigenvalues), so the linear system is solved by
// restarted GMRES instead, one application of J_G^T being two reverse steps.
// Unrolled mode instead backpropagates through k recorded steps started from
// the current environment (held fixed): their tapes are recorded into the
// workspace's tape store on the way forward and read on the way back, or,
// without room for k tapes, a forward sweep of plain steps keeps their (C, T)
// checkpoints and each step's tape is recomputed from its checkpoint on the
// way back.  The gradient is projected onto the C4v
// subspace at the end (the function is only defined there).  The passes take
// the context's precision: FP64, or in a split context the TF32x3 engine with
// the step's own split QR (thin-output contractions, the traces and the QR
// adjoint's product with R^-T in FP64).
#include <algorithm>
#include <cmath>
#include <vector>

#include "grad.cuh"

namespace qrctm {

namespace {

constexpr int kMaxUnroll = kGradMaxUnroll;
constexpr int kGmresM = 40;   // GMRES restart length
inline size_t al8(size_t n) { return ((n * 8) + 255) & ~size_t(255); }

struct GradLayout {
  StepTape tape[2];
  AdjWork adj;
  double *ebC, *ebT, *yC, *yT, *y2C, *y2T, *xbC, *xbT, *Abar, *gsym;
  // energy reverse pass
  double *ctb, *L1b, *Wb, *Z1b, *Z2b, *HLb, *rhob, *Ctb, *Pb;
  double *ckC, *ckT;   // unroll checkpoints
  double* red;         // reductions
  double* kry;         // GMRES basis: (kGmresM + 1) env-sized vectors [C (chi^2), T]
  double *ev0, *ev1, *evx;   // env-sized vectors: right-hand side, work, solution
};

// Lay one step's tape out from base (base = nullptr: only count bytes).
size_t tape_layout(int d, int D, int chi, char* base, StepTape* T) {
  const size_t D2 = (size_t)D * D, m = (size_t)chi * D2, mm = m * m, c2 = (size_t)chi * chi,
               mc = m * chi;
  size_t off = 0;
  auto take = [&](double** p, size_t n) {
    if (base && p) *p = reinterpret_cast<double*>(base + off);
    off += al8(n > 0 ? n : 1);
  };
  take(T ? &T->Cin : nullptr, c2);
  take(T ? &T->Tin : nullptr, mc);
  take(T ? &T->ct : nullptr, mc);
  take(T ? &T->Q : nullptr, mc);
  take(T ? &T->R : nullptr, c2);
  take(T ? &T->Rinv : nullptr, c2);
  take(T ? &T->X1 : nullptr, mm);
  take(T ? &T->Z : nullptr, mm * d);
  take(T ? &T->X2 : nullptr, mm);
  take(T ? &T->Traw : nullptr, mc);
  take(T ? &T->Ts : nullptr, mc);
  take(T ? &T->Y2 : nullptr, mc);
  take(T ? &T->Craw : nullptr, c2);
  take(T ? &T->Cout : nullptr, c2);
  take(T ? &T->Tout : nullptr, mc);
  take(T ? &T->parts : nullptr, 512);
  return off;
}

// Lay the gradient region out (carve = false: only count bytes).
size_t layout(int d, int D, int chi, bool nnn, char* base, GradLayout* L) {
  const size_t D2 = (size_t)D * D, m = (size_t)chi * D2, mm = m * m, c2 = (size_t)chi * chi,
               mc = m * chi;
  size_t off = 0;
  auto take = [&](double** p, size_t n) {
    if (base && p) *p = reinterpret_cast<double*>(base + off);
    off += al8(n > 0 ? n : 1);
  };
  for (int t = 0; t < 2; ++t)
    off += tape_layout(d, D, chi, base ? base + off : nullptr, L ? &L->tape[t] : nullptr);
  AdjWork* A = L ? &L->adj : nullptr;
  take(A ? &A->Cs : nullptr, c2);
  take(A ? &A->Craw : nullptr, c2);
  take(A ? &A->Tnorm : nullptr, mc);
  take(A ? &A->Ts : nullptr, mc);
  take(A ? &A->Traw : nullptr, mc);
  take(A ? &A->Y2 : nullptr, mc);
  take(A ? &A->Q : nullptr, mc);
  take(A ? &A->R : nullptr, c2);
  take(A ? &A->X2 : nullptr, mm);
  take(A ? &A->Z : nullptr, mm * d);
  take(A ? &A->X1 : nullptr, mm);
  take(A ? &A->ct : nullptr, mc);
  take(A ? &A->Ms : nullptr, c2);
  take(A ? &A->Ss : nullptr, c2);
  take(A ? &A->Bs : nullptr, mc);
  take(A ? &A->scr : nullptr, 1024);
  take(L ? &L->ebC : nullptr, c2);
  take(L ? &L->ebT : nullptr, mc);
  take(L ? &L->yC : nullptr, c2);
  take(L ? &L->yT : nullptr, mc);
  take(L ? &L->y2C : nullptr, c2);
  take(L ? &L->y2T : nullptr, mc);
  take(L ? &L->xbC : nullptr, c2);
  take(L ? &L->xbT : nullptr, mc);
  take(L ? &L->Abar : nullptr, (size_t)d * D2 * D2);
  take(L ? &L->gsym : nullptr, (size_t)d * D2 * D2);
  take(L ? &L->ctb : nullptr, mc);
  take(L ? &L->L1b : nullptr, mc);
  take(L ? &L->Wb : nullptr, mm);
  take(L ? &L->Z1b : nullptr, mm * d);
  take(L ? &L->Z2b : nullptr, mm * d * d);
  take(L ? &L->HLb : nullptr, mc * d * d);
  take(L ? &L->rhob : nullptr, 64);
  take(L ? &L->Ctb : nullptr, nnn ? mm : 1);
  take(L ? &L->Pb : nullptr, nnn ? mm * d * d : 1);
  take(L ? &L->ckC : nullptr, c2 * (kMaxUnroll + 1));
  take(L ? &L->ckT : nullptr, mc * (kMaxUnroll + 1));
  take(L ? &L->red : nullptr, 1024);
  take(L ? &L->kry : nullptr, (c2 + mc) * (kGmresM + 1));
  take(L ? &L->ev0 : nullptr, c2 + mc);
  take(L ? &L->ev1 : nullptr, c2 + mc);
  take(L ? &L->evx : nullptr, c2 + mc);
  return off;
}

inline unsigned nb256(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 8192); }


__global__ void add_diag_phys_k(double* Co_bar, const double* Ct_bar, int d, long long mm) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm;
       e += (long long)gridDim.x * blockDim.x)
    for (int s = 0; s < d; ++s) Co_bar[((long long)s * d + s) * mm + e] += Ct_bar[e];
}

__constant__ double g_h[16] = {0.25, 0, 0, 0, 0, -0.25, 0.5, 0, 0, 0.5, -0.25, 0, 0, 0, 0, 0.25};
__constant__ double g_hr[16] = {-0.25, 0, 0, -0.5, 0, 0.25, 0, 0, 0, 0, 0.25, 0, -0.5, 0, 0, -0.25};

// rhobar[s1][t1][s2][t2] = scale * (h[(t1 t2),(s1 s2)] - E delta_{s1 t1} delta_{s2 t2}) / Tr rho,
// the cotangent of scale * Tr(rho h) / Tr(rho); plain = 0: rotated bond h~.
__global__ void rho_bar_k(const double* rho, int plain, double scale, double* rhob) {
  const double* h = plain ? g_h : g_hr;
  const int e = threadIdx.x;
  __shared__ double num, den;
  if (e == 0) {
    double n_ = 0.0, d_ = 0.0;
    for (int s1 = 0; s1 < 2; ++s1)
      for (int t1 = 0; t1 < 2; ++t1)
        for (int s2 = 0; s2 < 2; ++s2)
          for (int t2 = 0; t2 < 2; ++t2) {
            const double r = rho[((s1 * 2 + t1) * 2 + s2) * 2 + t2];
            n_ += r * h[(t1 * 2 + t2) * 4 + (s1 * 2 + s2)];
            if (s1 == t1 && s2 == t2) d_ += r;
          }
    num = n_;
    den = d_;
  }
  __syncthreads();
  if (e < 16) {
    const int t2 = e & 1, s2 = (e >> 1) & 1, t1 = (e >> 2) & 1, s1 = (e >> 3) & 1;
    const double E = num / den;
    double v = h[(t1 * 2 + t2) * 4 + (s1 * 2 + s2)];
    if (s1 == t1 && s2 == t2) v -= E;
    rhob[e] = scale * v / den;
  }
}

// Q[c m + i] = Q32[c mp + i]: the split QR's FP32 columns widened for the tape.
__global__ void q32_to_f64_k(const float* __restrict__ Q32, long long mp, double* __restrict__ Q,
                             long long m, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long col = e / m;
    Q[e] = static_cast<double>(Q32[col * mp + (e - col * m)]);
  }
}

__global__ void trace_phys2_k(const double* __restrict__ Co, double* __restrict__ Ct, int d,
                              long long mm) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < d; ++s) acc += Co[((long long)s * d + s) * mm + e];
    Ct[e] = acc;
  }
}

__global__ void energy2_k(const double* rho_nn, const double* rho_nnn, double J1, double J2,
                          int nn_plain, double* e_out) {
  auto be = [](const double* rho4, const double* h) {
    double num = 0.0, den = 0.0;
    for (int s1 = 0; s1 < 2; ++s1)
      for (int t1 = 0; t1 < 2; ++t1)
        for (int s2 = 0; s2 < 2; ++s2)
          for (int t2 = 0; t2 < 2; ++t2) {
            const double r = rho4[((s1 * 2 + t1) * 2 + s2) * 2 + t2];
            num += r * h[(t1 * 2 + t2) * 4 + (s1 * 2 + s2)];
            if (s1 == t1 && s2 == t2) den += r;
          }
    return num / den;
  };
  double e = 2.0 * J1 * be(rho_nn, nn_plain ? g_h : g_hr);
  if (rho_nnn) e += 2.0 * J2 * be(rho_nnn, g_h);
  e_out[0] = e;
}

}  // namespace

size_t grad_bytes(int d, int D, int chi) { return layout(d, D, chi, true, nullptr, nullptr); }
size_t tape_bytes(int d, int D, int chi) { return tape_layout(d, D, chi, nullptr, nullptr); }

// ---------------------------------------------------------------------------
// Forward step with tape, and its reverse pass
// ---------------------------------------------------------------------------
// In a split context the tape keeps X1, Z and X2 and their cotangents in
// FP32: they feed only TF32x3 products, whose FP32 operand copies the gathers
// would make anyway, and the FP64 values the engine would write are FP32 sums
// widened exactly.  Half the bytes for the largest tensors of the step.
static Gemm tape32(const qrctm_ctx* c, Gemm g, bool a, bool b, bool cc) {
  if (c->mm_split) {
    g.a_f32 = a;
    g.b_f32 = b;
    g.c_f32 = cc;
  }
  return g;
}

// The tape's four contractions through X1, Z, X2 (FP32 in a split context).
static Gemm x1_t(qrctm_ctx* c, const Dims& k, const StepTape& t) {
  return tape32(c, g_x1(c, k, t.Q, t.Tin, t.X1), false, false, true);
}
static Gemm ket_t(qrctm_ctx* c, const Dims& k, const StepTape& t) {
  return tape32(c, g_ket(c, k, t.X1, c->A, t.Z), true, false, true);
}
static Gemm bra_t(qrctm_ctx* c, const Dims& k, const StepTape& t) {
  return tape32(c, g_bra(c, k, t.Z, c->A, t.X2), true, false, true);
}
static Gemm proj_t(qrctm_ctx* c, const Dims& k, const StepTape& t) {
  return tape32(c, g_proj(c, k, t.X2, t.Q, t.Traw), true, false, false);
}

static cudaError_t step_fwd_tape(qrctm_ctx* c, const double* Cin, const double* Tin,
                                 StepTape& t) {
  const Dims k(c);
  cudaStream_t s = c->st;
  cudaError_t e;
  if (Cin != t.Cin &&
      (e = cudaMemcpyAsync(t.Cin, Cin, sizeof(double) * k.ch * k.ch, cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess)
    return e;
  if (Tin != t.Tin &&
      (e = cudaMemcpyAsync(t.Tin, Tin, sizeof(double) * k.m * k.ch, cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess)
    return e;
  if ((e = gemm_run(c, g_ct(c, k, t.Cin, t.Tin, t.ct))) != cudaSuccess) return e;
  if (c->split_prec) {
    // the QR the split step itself runs: FP64 panels, TF32x3 blocked updates
    const long long mp = (k.m + 3) & ~3ll;
    if ((e = householder_qr_split((int)k.m, k.ch, t.ct, t.R, c->qrw, c->qr32, c->Qc32, false,
                                  c->tc_part, c->tc_part_elems, s)) != cudaSuccess)
      return e;
    q32_to_f64_k<<<nb256(k.m * k.ch), 256, 0, s>>>(c->Qc32, mp, t.Q, k.m, k.ch);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if ((e = householder_qr_f64((int)k.m, k.ch, t.ct, t.Q, t.R, c->qrw, s)) != cudaSuccess) {
    return e;
  }
  if ((e = triu_inverse(t.R, t.Rinv, k.ch, c->err, s)) != cudaSuccess) return e;
  if ((e = gemm_run(c, x1_t(c, k, t))) != cudaSuccess) return e;
  if ((e = gemm_run(c, ket_t(c, k, t))) != cudaSuccess) return e;
  if ((e = gemm_run(c, bra_t(c, k, t))) != cudaSuccess) return e;
  if ((e = gemm_run(c, proj_t(c, k, t))) != cudaSuccess) return e;
  if ((e = sym_edge(t.Traw, t.Ts, k.ch, k.D2, s)) != cudaSuccess) return e;
  if ((e = gemm_run(c, g_y2(c, k, t.Ts, t.R, t.Y2))) != cudaSuccess) return e;
  if ((e = gemm_run(c, g_craw(c, k, t.Y2, t.Q, t.Craw))) != cudaSuccess) return e;
  return sym_norm_env(t.Craw, t.Ts, t.Cout, t.Tout, k.ch, k.D2, t.parts, c->err, s);
}

// (Cbar_out, Tbar_out) -> (Cbar_in, Tbar_in); Abar accumulated when non-null.
static cudaError_t step_vjp(qrctm_ctx* c, const StepTape& t, const AdjWork& a,
                            const double* Cbo, const double* Tbo, double* Cbi, double* Tbi,
                            double* Abar) {
  const Dims k(c);
  cudaStream_t s = c->st;
  cudaError_t e;
  const long long c2 = (long long)k.ch * k.ch, mc = k.m * k.ch;
  // normalisation and symmetrisation of the outputs
  if ((e = norm_vjp(t.Cout, Cbo, a.Cs, c2, t.parts, 256, a.scr, false, s)) != cudaSuccess) return e;
  if ((e = sym_corner_vjp(a.Cs, a.Craw, k.ch, false, s)) != cudaSuccess) return e;
  if ((e = norm_vjp(t.Tout, Tbo, a.Tnorm, mc, t.parts + 256, 256, a.scr + 256, false, s)) !=
      cudaSuccess)
    return e;
  if ((e = sym_edge(a.Tnorm, a.Ts, k.ch, k.D2, s)) != cudaSuccess) return e;
  // C' = Y2 Q ; Y2 = Ts R
  if ((e = gemm_vjp(c, g_craw(c, k, t.Y2, t.Q, t.Craw), a.Craw, a.Y2, a.Q, false, false)) !=
      cudaSuccess)
    return e;
  if ((e = gemm_vjp(c, g_y2(c, k, t.Ts, t.R, t.Y2), a.Y2, a.Ts, a.R, true, false)) != cudaSuccess)
    return e;
  // Ts = sym(Traw)
  if ((e = sym_edge(a.Ts, a.Traw, k.ch, k.D2, s)) != cudaSuccess) return e;
  // Traw = X2 Q ; bra ; ket ; X1 = Q^T T
  if ((e = gemm_vjp(c, proj_t(c, k, t), a.Traw, a.X2, a.Q, false, true)) !=
      cudaSuccess)
    return e;
  if ((e = gemm_vjp(c, bra_t(c, k, t), a.X2, a.Z, Abar, false, true)) != cudaSuccess)
    return e;
  if ((e = gemm_vjp(c, ket_t(c, k, t), a.Z, a.X1, Abar, false, true)) != cudaSuccess)
    return e;
  if ((e = gemm_vjp(c, x1_t(c, k, t), a.X1, a.Q, Tbi, true, false)) != cudaSuccess)
    return e;
  // QR
  if ((e = qr_vjp(c, (int)k.m, k.ch, t.Q, t.R, t.Rinv, a.Q, a.R, a.ct, a.Ms, a.Ss, a.Bs)) !=
      cudaSuccess)
    return e;
  // ct = C T
  return gemm_vjp(c, g_ct(c, k, t.Cin, t.Tin, t.ct), a.ct, Cbi, Tbi, false, true);
}

// ---------------------------------------------------------------------------
// Energy with its reverse pass: (Cbar, Tbar) overwritten, Abar overwritten.
// ---------------------------------------------------------------------------
static cudaError_t energy_vjp(qrctm_ctx* c, const GradLayout& L, const double* C, const double* T,
                              double J1, double J2, double* Cb, double* Tb, double* Ab,
                              double* e_out_dev) {
  const Dims k(c);
  cudaStream_t s = c->st;
  cudaError_t e;
  const int D = k.D, D2 = k.D2, d = k.d, ch = k.ch;
  const long long m = k.m, mm = m * m, dD2 = k.dD2, D3 = k.D3, D4 = k.D4;
  const long long Sq = (long long)ch * D2 * ch, D2c = (long long)D2 * ch, D4c = D4 * ch;
  const long long c2 = (long long)ch * ch, mc = m * ch;
  double* ct = c->Mcm;
  double* L1 = c->Y2;
  double* W = c->X1;
  double* Z1 = c->Z;
  double* Z2 = c->E1;
  double* HL = c->E2;
  double* rho = c->rho;
  if ((e = cudaMemsetAsync(Cb, 0, sizeof(double) * c2, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Tb, 0, sizeof(double) * mc, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Ab, 0, sizeof(double) * d * D4, s)) != cudaSuccess) return e;
  // ---- forward (2x1 patch) ----
  const Gemm f_ct = g_ct(c, k, C, T, ct);
  Gemm f_l1 = gemm_ctx(c);
  f_l1.M = m; f_l1.N = ch; f_l1.K = ch;
  f_l1.A = ct; f_l1.a_m = im1(1); f_l1.a_k = im1(m);
  f_l1.B = C; f_l1.b_k = im1(ch); f_l1.b_n = im1(1);
  f_l1.C = L1; f_l1.c_m = im1(ch); f_l1.c_n = im1(1);
  Gemm f_w = gemm_ctx(c);
  f_w.M = m; f_w.N = m; f_w.K = ch;
  f_w.A = L1; f_w.a_m = im1(1); f_w.a_k = im1(m);
  f_w.B = T; f_w.b_k = im1(m); f_w.b_n = im1(1);
  f_w.C = W; f_w.c_m = im1(m); f_w.c_n = im1(1);
  Gemm f_ket = gemm_ctx(c);
  f_ket.M = (long long)ch * ch * D2; f_ket.N = dD2; f_ket.K = D2;
  f_ket.A = W; f_ket.a_m = im4(D, D, ch, ch, Sq, 1, m); f_ket.a_k = im2(D, D * Sq, (long long)D * ch);
  f_ket.B = c->A; f_ket.b_k = im2(D, D2, D3); f_ket.b_n = im3(D, D, 1, D, D4);
  f_ket.C = Z1; f_ket.c_m = im1(dD2); f_ket.c_n = im1(1);
  Gemm f_bra = gemm_ctx(c);
  f_bra.M = (long long)ch * ch * dD2; f_bra.N = dD2; f_bra.K = D2;
  f_bra.A = Z1; f_bra.a_m = im4(D, D, d, 1, D, D2, D2 * dD2); f_bra.a_k = im2(D, dD2, D * dD2);
  f_bra.B = c->A; f_bra.b_k = im2(D, D3, D2); f_bra.b_n = im3(D, D, 1, D, D4);
  f_bra.C = Z2;
  f_bra.c_m = im5(D, D, d, ch, (long long)D * D2c, D, (long long)d * D4c, (long long)d * d * D4c,
                  D2);
  f_bra.c_n = im3(D, D, D2c, 1, D4c);
  Gemm f_hl = gemm_ctx(c);
  f_hl.M = (long long)ch * d * d * D2; f_hl.N = ch; f_hl.K = m;
  f_hl.A = Z2; f_hl.a_m = im1(m); f_hl.a_k = im1(1);
  f_hl.B = T; f_hl.b_k = im1(ch); f_hl.b_n = im1(1);
  f_hl.C = HL; f_hl.c_m = im1(ch); f_hl.c_n = im1(1);
  Gemm f_rho = gemm_ctx(c);
  f_rho.M = d * d; f_rho.N = d * d; f_rho.K = (long long)ch * D2 * ch;
  f_rho.A = HL; f_rho.a_m = im1(D2c); f_rho.a_k = im3(ch, D2, 1, ch, (long long)d * d * D2c);
  f_rho.B = HL; f_rho.b_k = im3(ch, D2, 1, ch, (long long)d * d * D2c); f_rho.b_n = im1(D2c);
  f_rho.C = rho; f_rho.c_m = im1(d * d); f_rho.c_n = im1(1);
  const Gemm* fwd[] = {&f_ct, &f_l1, &f_w, &f_ket, &f_bra, &f_hl, &f_rho};
  for (const Gemm* g : fwd)
    if ((e = gemm_run(c, *g)) != cudaSuccess) return e;
  // ---- reverse (2x1 patch): E_nn = 2 J1 Tr(rho h~)/Tr(rho) ----
  double* ctb = L.ctb;
  rho_bar_k<<<1, 32, 0, s>>>(rho, c->nn_plain ? 1 : 0, 2.0 * J1, L.rhob);
  note_launch();
  if ((e = gemm_vjp(c, f_rho, L.rhob, L.HLb, nullptr, false, false)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_rho, L.rhob, nullptr, L.HLb, false, true)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_hl, L.HLb, L.Z2b, Tb, false, true)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_bra, L.Z2b, L.Z1b, Ab, false, true)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_ket, L.Z1b, L.Wb, Ab, false, true)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_w, L.Wb, L.L1b, Tb, false, true)) != cudaSuccess) return e;
  if ((e = gemm_vjp(c, f_l1, L.L1b, ctb, Cb, false, true)) != cudaSuccess) return e;
  double* rho_nnn = nullptr;
  if (J2 != 0.0) {
    // ---- forward (2x2 patch): rho = Tr(Co Ct Co Ct) ----
    rho_nnn = c->rho + 16;
    double* X = c->X1;
    double* Zo = c->Z;
    double* Co = c->E1;
    double* Ct = c->X2;
    double* P = c->E3;
    const Gemm f_x = g_x1(c, k, ct, T, X);
    const Gemm f_keto = g_ket(c, k, X, c->A, Zo);
    Gemm f_brao = gemm_ctx(c);
    f_brao.M = (long long)ch * ch * dD2; f_brao.N = dD2; f_brao.K = D2;
    f_brao.A = Zo; f_brao.a_m = im4(D, D, d, 1, D, D2, D2 * dD2); f_brao.a_k = im2(D, dD2, D * dD2);
    f_brao.B = c->A; f_brao.b_k = im2(D, D2, D3); f_brao.b_n = im3(D, D, 1, D, D4);
    f_brao.C = Co;
    f_brao.c_m = im5(D, D, d, ch, D, D * m, (long long)d * mm, (long long)D2 * m, D2);
    f_brao.c_n = im3(D, D, 1, m, mm);
    Gemm f_P = gemm_ctx(c);
    f_P.M = m; f_P.N = m; f_P.K = m; f_P.batch = d * d;
    f_P.A = Co; f_P.a_m = im1(m); f_P.a_k = im1(1); f_P.a_b = im1(mm);
    f_P.B = Ct; f_P.b_k = im1(m); f_P.b_n = im1(1); f_P.b_b = im0();
    f_P.C = P; f_P.c_m = im1(m); f_P.c_n = im1(1); f_P.c_b = im1(mm);
    Gemm f_rn = gemm_ctx(c);
    f_rn.M = d * d; f_rn.N = d * d; f_rn.K = mm;
    f_rn.A = P; f_rn.a_m = im1(mm); f_rn.a_k = im1(1);
    f_rn.B = P; f_rn.b_k = im2((int)m, m, 1); f_rn.b_n = im1(mm);
    f_rn.C = rho_nnn; f_rn.c_m = im1(d * d); f_rn.c_n = im1(1);
    if ((e = gemm_run(c, f_x)) != cudaSuccess) return e;
    if ((e = gemm_run(c, f_keto)) != cudaSuccess) return e;
    if ((e = gemm_run(c, f_brao)) != cudaSuccess) return e;
    trace_phys2_k<<<1184, 256, 0, s>>>(Co, Ct, d, mm);
    note_launch();
    if ((e = gemm_run(c, f_P)) != cudaSuccess) return e;
    const bool tr = trace_pairs_ok(d * d);
    if (tr) {
      if ((e = trace_pairs(P, d * d, m, c->partials, rho_nnn, s)) != cudaSuccess) return e;
    } else if ((e = gemm_run(c, f_rn)) != cudaSuccess) {
      return e;
    }
    // ---- reverse (2x2 patch) ----
    rho_bar_k<<<1, 32, 0, s>>>(rho_nnn, 1, 2.0 * J2, L.rhob + 16);
    note_launch();
    if (tr) {
      if ((e = trace_pairs_vjp(P, d * d, m, L.rhob + 16, L.Pb, s)) != cudaSuccess) return e;
    } else {
      if ((e = gemm_vjp(c, f_rn, L.rhob + 16, L.Pb, nullptr, false, false)) != cudaSuccess) return e;
      if ((e = gemm_vjp(c, f_rn, L.rhob + 16, nullptr, L.Pb, false, true)) != cudaSuccess) return e;
    }
    // Co and Ct cotangents; Ct = sum_s Co[s][s]
    if ((e = gemm_vjp(c, f_P, L.Pb, L.Z2b, L.Ctb, false, false)) != cudaSuccess) return e;
    add_diag_phys_k<<<1184, 256, 0, s>>>(L.Z2b, L.Ctb, d, mm);
    note_launch();
    if ((e = gemm_vjp(c, f_brao, L.Z2b, L.Z1b, Ab, false, true)) != cudaSuccess) return e;
    if ((e = gemm_vjp(c, f_keto, L.Z1b, L.Wb, Ab, false, true)) != cudaSuccess) return e;
    if ((e = gemm_vjp(c, f_x, L.Wb, ctb, Tb, true, true)) != cudaSuccess) return e;
  }
  // ct = C T
  if ((e = gemm_vjp(c, f_ct, ctb, Cb, Tb, true, true)) != cudaSuccess) return e;
  energy2_k<<<1, 1, 0, s>>>(rho, rho_nnn, J1, J2, c->nn_plain ? 1 : 0, e_out_dev);
  note_launch();
  (void)c2; (void)mc;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Drivers
// ---------------------------------------------------------------------------
static cudaError_t dot_host(qrctm_ctx* c, const double* x, const double* y, long long n,
                           double* red, double* out) {
  cudaError_t e = dot_partials(x, y, n, red, 64, c->st);
  if (e != cudaSuccess) return e;
  double h[64];
  if ((e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, c->st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return e;
  double acc = 0.0;
  for (int i = 0; i < 64; ++i) acc += h[i];
  *out = acc;
  return cudaSuccess;
}

// w = v - J_G^T v for an env-sized vector v = [C (chi^2), T (chi^2 D^2)]
static cudaError_t adjoint_operator(qrctm_ctx* c, GradLayout& L, const double* v, double* w) {
  const Dims k(c);
  const long long c2 = (long long)k.ch * k.ch, n = c2 + k.m * k.ch;
  cudaError_t e;
  if ((e = step_vjp(c, L.tape[1], L.adj, v, v + c2, L.y2C, L.y2T, nullptr)) != cudaSuccess)
    return e;
  if ((e = step_vjp(c, L.tape[0], L.adj, L.y2C, L.y2T, w, w + c2, nullptr)) != cudaSuccess)
    return e;
  // w <- v - w
  axpby(w, v, 1.0, -1.0, n, c->st);
  return cudaGetLastError();
}

// Restarted GMRES for (I - J_G^T) x = b (b = L.ev0, x -> L.evx); returns the
// number of operator applications.
static cudaError_t adjoint_gmres(qrctm_ctx* c, GradLayout& L, double tol, int max_apply,
                                 int* applies, double* rel_resid) {
  const Dims k(c);
  const long long n = (long long)k.ch * k.ch + k.m * k.ch;
  const int M = kGmresM;
  cudaStream_t s = c->st;
  cudaError_t e;
  double bnorm2;
  if ((e = dot_host(c, L.ev0, L.ev0, n, L.red, &bnorm2)) != cudaSuccess) return e;
  const double bnorm = std::sqrt(bnorm2);
  if ((e = fill_zero(L.evx, n, s)) != cudaSuccess) return e;
  *applies = 0;
  *rel_resid = 0.0;
  if (!(bnorm > 0.0)) return cudaSuccess;
  std::vector<double> H((M + 1) * M), cs(M), sn(M), g(M + 1), y(M);
  auto Vj = [&](int j) { return L.kry + (long long)j * n; };
  double resid = bnorm;
  while (*applies < max_apply && resid > tol * bnorm) {
    // r = b - A x  (x = 0 on the first cycle)
    if (*applies == 0) {
      cudaMemcpyAsync(Vj(0), L.ev0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    } else {
      if ((e = adjoint_operator(c, L, L.evx, L.ev1)) != cudaSuccess) return e;
      ++*applies;
      cudaMemcpyAsync(Vj(0), L.ev0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
      axpby(Vj(0), L.ev1, -1.0, 1.0, n, s);
    }
    double beta2;
    if ((e = dot_host(c, Vj(0), Vj(0), n, L.red, &beta2)) != cudaSuccess) return e;
    const double beta = std::sqrt(beta2);
    if (!(beta > tol * bnorm)) { resid = beta; break; }
    axpby(Vj(0), Vj(0), 0.0, 1.0 / beta, n, s);   // v0 <- r / beta
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < M && *applies < max_apply; ++j) {
      if ((e = adjoint_operator(c, L, Vj(j), Vj(j + 1))) != cudaSuccess) return e;
      ++*applies;
      for (int i = 0; i <= j; ++i) {   // modified Gram-Schmidt
        double h;
        if ((e = dot_host(c, Vj(j + 1), Vj(i), n, L.red, &h)) != cudaSuccess) return e;
        H[i * M + j] = h;
        axpby(Vj(j + 1), Vj(i), -h, 1.0, n, s);
      }
      double hn2;
      if ((e = dot_host(c, Vj(j + 1), Vj(j + 1), n, L.red, &hn2)) != cudaSuccess) return e;
      const double hn = std::sqrt(hn2);
      H[(j + 1) * M + j] = hn;
      if (hn > 0.0) axpby(Vj(j + 1), Vj(j + 1), 0.0, 1.0 / hn, n, s);
      // Givens rotations on column j
      for (int i = 0; i < j; ++i) {
        const double a = H[i * M + j], b = H[(i + 1) * M + j];
        H[i * M + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * M + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[j * M + j], b = H[(j + 1) * M + j];
      const double r = std::hypot(a, b);
      cs[j] = (r > 0) ? a / r : 1.0;
      sn[j] = (r > 0) ? b / r : 0.0;
      H[j * M + j] = r;
      H[(j + 1) * M + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      resid = std::fabs(g[j + 1]);
      if (!(resid > tol * bnorm) || hn == 0.0) { ++j; break; }
    }
    // y = H^{-1} g (upper triangular j x j), x += V y
    for (int i = j - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < j; ++l) acc -= H[i * M + l] * y[l];
      y[i] = acc / H[i * M + i];
    }
    for (int i = 0; i < j; ++i) axpby(L.evx, Vj(i), y[i], 1.0, n, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  *rel_resid = resid / bnorm;
  return cudaSuccess;
}

cudaError_t energy_grad_run(qrctm_ctx* c, double J1, double J2, int mode, int k_unroll,
                            double* grad, double* e_out, int* iters_out, double* resid_out,
                            double* fp_resid_out) {
  if (!c->G) return cudaErrorInvalidValue;
  if (mode != 0 && (k_unroll < 1 || k_unroll > kMaxUnroll)) return cudaErrorInvalidValue;
  GradLayout L;
  layout(c->d, c->D, c->chi, true, c->G, &L);
  cudaError_t e;
  const Dims k(c);
  cudaStream_t s = c->st;
  const long long c2 = (long long)k.ch * k.ch, mc = k.m * k.ch, nA = (long long)k.d * k.D4;
  double* e_dev = c->e_d;
  int iters = 0;
  double resid = 0.0;
  if (mode == 0) {
    // implicit: tapes of two steps at the current environment
    if ((e = step_fwd_tape(c, c->C, c->T, L.tape[0])) != cudaSuccess) return e;
    if ((e = step_fwd_tape(c, L.tape[0].Cout, L.tape[0].Tout, L.tape[1])) != cudaSuccess) return e;
    // how far the current environment is from a fixed point of the two-step
    // map, elementwise: ||G(x) - x|| / ||x|| with x = (C, T), each of unit
    // norm.  The adjoint equation holds at G(x) = x; the spectrum test that
    // ends the forward iteration is gauge invariant and can be met long
    // before the environment stops moving elementwise.
    {
      const long long n = c2 + mc;
      cudaMemcpyAsync(L.ev1, L.tape[1].Cout, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(L.ev1 + c2, L.tape[1].Tout, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
      axpby(L.ev1, c->C, -1.0, 1.0, c2, s);
      axpby(L.ev1 + c2, c->T, -1.0, 1.0, mc, s);
      double d2 = 0.0;
      if ((e = dot_host(c, L.ev1, L.ev1, n, L.red, &d2)) != cudaSuccess) return e;
      if (fp_resid_out) *fp_resid_out = std::sqrt(d2 / 2.0);
    }
    if ((e = energy_vjp(c, L, c->C, c->T, J1, J2, L.ebC, L.ebT, L.Abar, e_dev)) != cudaSuccess)
      return e;
    // xbar solves (I - J_G^T) xbar = ebar   (restarted GMRES)
    cudaMemcpyAsync(L.ev0, L.ebC, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(L.ev0 + c2, L.ebT, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
    if ((e = adjoint_gmres(c, L, c->cfg.grad_tol, c->cfg.grad_max_iter, &iters, &resid)) !=
        cudaSuccess)
      return e;
    cudaMemcpyAsync(L.xbC, L.evx, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(L.xbT, L.evx + c2, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
    // A-part: xbar through both steps
    if ((e = step_vjp(c, L.tape[1], L.adj, L.xbC, L.xbT, L.y2C, L.y2T, L.Abar)) != cudaSuccess)
      return e;
    if ((e = step_vjp(c, L.tape[0], L.adj, L.y2C, L.y2T, L.yC, L.yT, L.Abar)) != cudaSuccess)
      return e;
  } else {
    // unrolled: k steps from the current (detached) environment
    const int K = k_unroll;
    cudaMemcpyAsync(L.ckC, c->C, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(L.ckT, c->T, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
    if (c->tape_store && K <= c->tape_store_k) {
      // every step's tape recorded once on the way forward, read on the way back
      const size_t tb = tape_bytes(c->d, c->D, c->chi);
      std::vector<StepTape> tp(K);
      for (int i = 0; i < K; ++i)
        tape_layout(c->d, c->D, c->chi, c->tape_store + (size_t)i * tb, &tp[i]);
      for (int i = 0; i < K; ++i) {
        const double* Cin = i == 0 ? L.ckC : tp[i - 1].Cout;
        const double* Tin = i == 0 ? L.ckT : tp[i - 1].Tout;
        if ((e = step_fwd_tape(c, Cin, Tin, tp[i])) != cudaSuccess) return e;
      }
      if ((e = energy_vjp(c, L, tp[K - 1].Cout, tp[K - 1].Tout, J1, J2, L.yC, L.yT, L.Abar,
                          e_dev)) != cudaSuccess)
        return e;
      for (int i = K - 1; i >= 0; --i) {
        if ((e = step_vjp(c, tp[i], L.adj, L.yC, L.yT, L.y2C, L.y2T, L.Abar)) != cudaSuccess)
          return e;
        std::swap(L.yC, L.y2C);
        std::swap(L.yT, L.y2T);
      }
      iters = K;
      if (fp_resid_out) *fp_resid_out = 0.0;
      if (c->grad_keep_env) {
        // the optimiser continues from the environment after the k steps
        cudaMemcpyAsync(c->C, tp[K - 1].Cout, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(c->T, tp[K - 1].Tout, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
        c->iters += K;
        c->spec_valid = false;
        c->spec_pending = false;
      }
    } else {
      // the forward sweep keeps only the checkpoints, so it runs the plain step
      // (the same map, without the tape's stored intermediates) in place on
      // the context's environment
      for (int i = 1; i <= K; ++i) {
        if ((e = qr_step_graph(c)) != cudaSuccess) return e;
        cudaMemcpyAsync(L.ckC + i * c2, c->C, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(L.ckT + i * mc, c->T, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
      }
      if (c->grad_keep_env) {
        // the optimiser continues from the environment after the k steps
        c->spec_valid = false;
        c->spec_pending = false;
      } else {
        cudaMemcpyAsync(c->C, L.ckC, sizeof(double) * c2, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(c->T, L.ckT, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s);
        c->iters -= K;
      }
      if ((e = energy_vjp(c, L, L.ckC + K * c2, L.ckT + K * mc, J1, J2, L.yC, L.yT, L.Abar,
                          e_dev)) != cudaSuccess)
        return e;
      for (int i = K; i >= 1; --i) {
        if ((e = step_fwd_tape(c, L.ckC + (i - 1) * c2, L.ckT + (i - 1) * mc, L.tape[0])) !=
            cudaSuccess)
          return e;
        if ((e = step_vjp(c, L.tape[0], L.adj, L.yC, L.yT, L.y2C, L.y2T, L.Abar)) != cudaSuccess)
          return e;
        std::swap(L.yC, L.y2C);
        std::swap(L.yT, L.y2T);
      }
      iters = K;
      if (fp_resid_out) *fp_resid_out = 0.0;
    }
  }
  // project onto the C4v subspace
  if ((e = c4v_symmetrize(k.d, k.D, L.Abar, grad, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(e_out, e_dev, sizeof(double), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (iters_out) *iters_out = iters;
  if (resid_out) *resid_out = resid;
  (void)nA;
  return cudaSuccess;
}

}  // namespace qrctm
