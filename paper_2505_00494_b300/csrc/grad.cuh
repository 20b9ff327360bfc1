// Adjoint (gradient) machinery: contraction descriptors of the FP64 step and
// energy, shared by the taped forward passes and their reverse passes.
#pragma once

#include "ctx.cuh"

namespace qrctm {

IdxMap concat_map(const IdxMap& x, long long xrange, const IdxMap& y);
cudaError_t gemm_vjp(qrctm_ctx* c, const Gemm& f, const double* Dbar, double* Abar, double* Bbar,
                     bool accA, bool accB);
cudaError_t dot_partials(const double* x, const double* y, long long n, double* partials,
                         int nparts, cudaStream_t s);
cudaError_t triu_inverse(const double* R, double* X, int n, int* err, cudaStream_t s);
cudaError_t sym_corner_vjp(const double* X, double* Y, int chi, bool acc, cudaStream_t s);
cudaError_t norm_vjp(const double* y, const double* ybar, double* xbar, long long n,
                     const double* nrm_parts, int nparts, double* scratch, bool acc,
                     cudaStream_t s);
cudaError_t qr_vjp(qrctm_ctx* c, int m, int n, const double* Q, const double* R,
                   const double* Rinv, const double* Qbar, const double* Rbar, double* Mbar,
                   double* Ms, double* Ss, double* Bs);

// Shape constants of the current context.
struct Dims {
  int d, D, D2, ch;
  long long D3, D4, m, dD2, Su, Smu, Sk;
  explicit Dims(const qrctm_ctx* c)
      : d(c->d), D(c->D), D2(c->D2), ch(c->chi_cur) {
    D3 = (long long)D2 * D;
    D4 = (long long)D2 * D2;
    m = (long long)ch * D2;
    dD2 = (long long)d * D2;
    Su = (long long)ch * D2 * ch;
    Smu = (long long)D2 * ch;
    Sk = ch;
  }
};

// ---- the FP64 QR-CTMRG step (split layers), as contraction descriptors ----
// ct[(a,i),b] = sum_g C[a,g] T[g,i,b]            (column-major (chi D2) x chi)
inline Gemm g_ct(qrctm_ctx* c, const Dims& k, const double* C, const double* T, double* ct) {
  Gemm g = gemm_ctx(c);
  g.M = k.ch; g.N = k.ch; g.K = k.ch; g.batch = k.D2;
  g.A = C; g.a_m = im1(k.ch); g.a_k = im1(1); g.a_b = im0();
  g.B = T; g.b_k = im1(k.m); g.b_n = im1(1); g.b_b = im1(k.ch);
  g.C = ct; g.c_m = im1(k.D2); g.c_n = im1(k.m); g.c_b = im1(1);
  return g;
}
// X1[(u,m),(k,b)] = sum_a Q[(a,u),m] T[a,(k,b)]
inline Gemm g_x1(qrctm_ctx* c, const Dims& k, const double* Q, const double* T, double* X1) {
  Gemm g = gemm_ctx(c);
  g.M = k.m; g.N = k.m; g.K = k.ch;
  g.A = Q; g.a_m = im2(k.ch, k.m, 1); g.a_k = im1(k.D2);
  g.B = T; g.b_k = im1(k.m); g.b_n = im1(1);
  g.C = X1; g.c_m = im1(k.m); g.c_n = im1(1);
  return g;
}
// ket: Z[(m,b,u_b,k_b),(s,d_k,j_k)] = sum_{u_k,k_k} X1 A[s,u_k,k_k,d_k,j_k]
inline Gemm g_ket(qrctm_ctx* c, const Dims& k, const double* X1, const double* A, double* Z) {
  Gemm g = gemm_ctx(c);
  g.M = (long long)k.ch * k.ch * k.D2; g.N = k.dD2; g.K = k.D2;
  g.A = X1; g.a_m = im4(k.D, k.D, k.ch, k.Sk, k.Su, 1, k.Smu);
  g.a_k = im2(k.D, k.D * k.Sk, k.D * k.Su);
  g.B = A; g.b_k = im2(k.D, k.D2, k.D3); g.b_n = im3(k.D, k.D, 1, k.D, k.D4);
  g.C = Z; g.c_m = im1(k.dD2); g.c_n = im1(1);
  return g;
}
// bra: X2[(m,b,d_k,j_k),(d_b,j_b)] = sum_{s,u_b,k_b} Z A[s,u_b,k_b,d_b,j_b]
inline Gemm g_bra(qrctm_ctx* c, const Dims& k, const double* Z, const double* A, double* X2) {
  Gemm g = gemm_ctx(c);
  g.M = (long long)k.ch * k.ch * k.D2; g.N = k.D2; g.K = k.dD2;
  g.A = Z; g.a_m = im3(k.D, k.D, 1, k.D, k.D2 * k.dD2);
  g.a_k = im3(k.D, k.D, k.dD2, k.D * k.dD2, k.D2);
  g.B = A; g.b_k = im3(k.D, k.D, k.D2, k.D3, k.D4); g.b_n = im1(1);
  g.C = X2; g.c_m = im1(k.D2); g.c_n = im1(1);
  return g;
}
// T'[(m,j),n] = sum_{(b,d)} X2[m,b,d_k,j_k,d_b,j_b] Q[(b,d),n]
inline Gemm g_proj(qrctm_ctx* c, const Dims& k, const double* X2, const double* Q, double* Tr) {
  Gemm g = gemm_ctx(c);
  g.M = k.m; g.N = k.ch; g.K = k.m;
  g.A = X2; g.a_m = im3(k.D, k.D, 1, k.D2, (long long)k.ch * k.D4);
  g.a_k = im3(k.D, k.D, k.D, k.D3, k.D4);
  g.B = Q; g.b_k = im1(1); g.b_n = im1(k.m);
  g.C = Tr; g.c_m = im1(k.ch); g.c_n = im1(1);
  return g;
}
// Y2[n,(g,j)] = sum_m Ts[n,j,m] R[m,g]   (batched over j)
inline Gemm g_y2(qrctm_ctx* c, const Dims& k, const double* Ts, const double* R, double* Y2) {
  Gemm g = gemm_ctx(c);
  g.M = k.ch; g.N = k.ch; g.K = k.ch; g.batch = k.D2;
  g.A = Ts; g.a_m = im1(k.m); g.a_k = im1(1); g.a_b = im1(k.ch);
  g.B = R; g.b_k = im1(k.ch); g.b_n = im1(1); g.b_b = im0();
  g.C = Y2; g.c_m = im1(k.m); g.c_n = im1(k.D2); g.c_b = im1(1);
  return g;
}
// C'[n,p] = sum_{(g,j)} Y2[n,(g,j)] Q[(g,j),p]
inline Gemm g_craw(qrctm_ctx* c, const Dims& k, const double* Y2, const double* Q, double* Cr) {
  Gemm g = gemm_ctx(c);
  g.M = k.ch; g.N = k.ch; g.K = k.m;
  g.A = Y2; g.a_m = im1(k.m); g.a_k = im1(1);
  g.B = Q; g.b_k = im1(1); g.b_n = im1(k.m);
  g.C = Cr; g.c_m = im1(k.ch); g.c_n = im1(1);
  return g;
}

// Intermediates of one step kept for its reverse pass.
struct StepTape {
  double *Cin, *Tin, *ct, *Q, *R, *Rinv, *X1, *Z, *X2, *Traw, *Ts, *Y2, *Craw, *Cout, *Tout;
  double* parts;   // 512: ||sym C'||^2 partial sums [0,256), ||T'||^2 [256,512)
};

// Cotangent scratch of a reverse step.
struct AdjWork {
  double *Cs, *Craw, *Tnorm, *Ts, *Traw, *Y2, *Q, *R, *X2, *Z, *X1, *ct, *Ms, *Ss, *Bs, *scr;
};

size_t grad_bytes(int d, int D, int chi);
// Bytes of one step's tape (each 256-byte aligned piece of a StepTape).
size_t tape_bytes(int d, int D, int chi);
constexpr int kGradMaxUnroll = 32;
cudaError_t energy_grad_run(qrctm_ctx* c, double J1, double J2, int mode, int k_unroll,
                            double* grad, double* e_out, int* iters_out, double* resid_out,
                            double* fp_resid_out);

}  // namespace qrctm
