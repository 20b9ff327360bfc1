// Blocked Householder QR of the reduced corner for the split-precision path
// (QR-CTMRG paragraph: unpivoted QR, diag(R) >= 0).
//
// The panels are factored exactly as in the FP64 path (cooperative FP64
// panel kernel, FP64 reflector norms, Parlett's form of v_0).  The compact-WY
// products that dominate the flop count -- the trailing updates
// W2 <- (I - V T V^T)^T W2, the Gram matrices V^T V of the T factors and the
// formation of Q = H_1 ... H_n [I; 0] -- run on the TF32x3 tensor-core engine
// from FP32 copies of V and of the blocks they act on, reading and writing
// the FP64 matrices (FP32-class accuracy, the precision of the rest of the
// split path).
#include "qrctm_internal.cuh"
#include "tc_gemm.cuh"

#include <algorithm>

namespace qrctm {

namespace {
inline long long pad4(long long x) { return (x + 3) & ~3ll; }
}  // namespace

size_t qr_split_floats(int m, int n) {
  const long long mp = pad4(m), npan = (n + kQrPanel - 1) / kQrPanel;
  return (size_t)(2 * n * mp + npan * (long long)m * kQrPanel + (long long)n * kQrPanel + 1024);
}

cudaError_t householder_qr_split(int m, int n, const double* M, double* Q, double* R,
                                 const QrWork& w, float* f32, float* part, long long part_elems,
                                 cudaStream_t s) {
  if (m < n || n <= 0) return cudaErrorInvalidValue;
  const int NB = kQrPanel;
  const long long mp = pad4(m);
  const int npan = (n + NB - 1) / NB;
  float* V32 = f32;                                  // [q][i]   n x mp   (reflector q, row i)
  float* X32 = V32 + (long long)n * mp;              // [c][i]   n x mp   (W2 or Q block copy)
  float* Vr32 = X32 + (long long)n * mp;             // [p][i][q] npan x m x NB
  float* Yt32 = Vr32 + (long long)npan * m * NB;     // [c][q]   n x NB
  auto tc = [&](TcGemm g) {
    g.err = w.err;
    g.part = part;
    g.part_elems = part_elems;
    return gemm_tc(g, s);
  };
  cudaError_t e = cudaMemcpyAsync(w.W, M, sizeof(double) * (size_t)m * n,
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  for (int p = 0; p < npan; ++p) {
    const int j0 = p * NB, nbj = std::min(NB, n - j0), mr = m - j0, n2 = n - j0 - nbj;
    double *G, *tau;
    if ((e = qr_panel_step(m, j0, nbj, w, s, &G, &tau)) != cudaSuccess) return e;
    double* Tp = w.Tf + (size_t)p * NB * NB;
    // FP32 copies of this panel's reflectors: V32[j0+q][j0+i], Vr32[p][j0+i][q]
    float* Vp = V32 + (long long)j0 * mp + j0;
    if ((e = gather_f32(w.V + (size_t)j0 * m + j0, Vp, nbj, mr, mp, im1(m), im1(1), s)) !=
        cudaSuccess)
      return e;
    float* Vrp = Vr32 + (long long)p * m * NB + (long long)j0 * NB;
    if ((e = gather_f32(w.V + (size_t)j0 * m + j0, Vrp, mr, nbj, NB, im1(1), im1(m), s)) !=
        cudaSuccess)
      return e;
    {
      // G = V_p^T V_p (row stride NB), then T
      TcGemm g{};
      g.A = TcOperand{Vp, nbj, mr, mp, 1, 0};
      g.B = TcOperand{Vp, nbj, mr, mp, 1, 0};
      g.M = nbj; g.N = nbj; g.K = mr; g.batch = 1;
      g.C = G; g.c_fp64 = true; g.c_m = im1(NB); g.c_n = im1(1); g.c_b = im0();
      g.alpha = 1.0; g.beta = 0.0;
      if ((e = tc(g)) != cudaSuccess) return e;
      if ((e = qr_tfactor(G, tau, Tp, nbj, s)) != cudaSuccess) return e;
    }
    if (n2 > 0) {
      // X32[c][i] = W2[i, c];   Y^T[c][q] = sum_i W2[i,c] V[i,q]  -> w.Y[q][c]
      float* Xp = X32 + j0;
      if ((e = gather_f32(w.W + (size_t)(j0 + nbj) * m + j0, Xp, n2, mr, mp, im1(m), im1(1), s)) !=
          cudaSuccess)
        return e;
      TcGemm g{};
      g.A = TcOperand{Xp, n2, mr, mp, 1, 0};
      g.B = TcOperand{Vp, nbj, mr, mp, 1, 0};
      g.M = n2; g.N = nbj; g.K = mr; g.batch = 1;
      g.C = w.Y; g.c_fp64 = true; g.c_m = im1(1); g.c_n = im1(n2); g.c_b = im0();
      g.alpha = 1.0; g.beta = 0.0;
      if ((e = tc(g)) != cudaSuccess) return e;
      // Y2 = T^T Y  (FP64, nbj x n2)
      Gemm h = gemm_init();
      h.M = nbj; h.N = n2; h.K = nbj;
      h.A = Tp; h.a_m = im1(1); h.a_k = im1(NB);
      h.B = w.Y; h.b_k = im1(n2); h.b_n = im1(1);
      h.C = w.Y2; h.c_m = im1(n2); h.c_n = im1(1);
      if ((e = gemm_f64(h, s)) != cudaSuccess) return e;
      // Yt32[c][q] = Y2[q][c];  W2[i,c] -= sum_q V[i,q] Y2[q,c]
      if ((e = gather_f32(w.Y2, Yt32, n2, nbj, NB, im1(1), im1(n2), s)) != cudaSuccess) return e;
      g = TcGemm{};
      g.A = TcOperand{Vrp, mr, nbj, NB, 1, 0};
      g.B = TcOperand{Yt32, n2, nbj, NB, 1, 0};
      g.M = mr; g.N = n2; g.K = nbj; g.batch = 1;
      g.C = w.W + (size_t)(j0 + nbj) * m + j0; g.c_fp64 = true;
      g.c_m = im1(1); g.c_n = im1(m); g.c_b = im0();
      g.alpha = -1.0; g.beta = 1.0;
      if ((e = tc(g)) != cudaSuccess) return e;
    }
  }
  if ((e = qr_extract_r(w.W, R, m, n, s)) != cudaSuccess) return e;
  // Q = H_1 ... H_n [I; 0], panels in reverse order
  if ((e = set_identity_cols(Q, m, n, s)) != cudaSuccess) return e;
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * NB, nbj = std::min(NB, n - j0), mr = m - j0, nq = n - j0;
    const double* Tp = w.Tf + (size_t)p * NB * NB;
    const float* Vp = V32 + (long long)j0 * mp + j0;
    const float* Vrp = Vr32 + (long long)p * m * NB + (long long)j0 * NB;
    float* Xp = X32 + j0;
    // X32[c][i] = Q[j0+i, j0+c];  Y^T = Qs^T V  -> w.Y[q][c]
    if ((e = gather_f32(Q + (size_t)j0 * m + j0, Xp, nq, mr, mp, im1(m), im1(1), s)) !=
        cudaSuccess)
      return e;
    TcGemm g{};
    g.A = TcOperand{Xp, nq, mr, mp, 1, 0};
    g.B = TcOperand{Vp, nbj, mr, mp, 1, 0};
    g.M = nq; g.N = nbj; g.K = mr; g.batch = 1;
    g.C = w.Y; g.c_fp64 = true; g.c_m = im1(1); g.c_n = im1(nq); g.c_b = im0();
    g.alpha = 1.0; g.beta = 0.0;
    if ((e = tc(g)) != cudaSuccess) return e;
    // Y2 = T Y
    Gemm h = gemm_init();
    h.M = nbj; h.N = nq; h.K = nbj;
    h.A = Tp; h.a_m = im1(NB); h.a_k = im1(1);
    h.B = w.Y; h.b_k = im1(nq); h.b_n = im1(1);
    h.C = w.Y2; h.c_m = im1(nq); h.c_n = im1(1);
    if ((e = gemm_f64(h, s)) != cudaSuccess) return e;
    if ((e = gather_f32(w.Y2, Yt32, nq, nbj, NB, im1(1), im1(nq), s)) != cudaSuccess) return e;
    // Qs -= V Y2
    g = TcGemm{};
    g.A = TcOperand{Vrp, mr, nbj, NB, 1, 0};
    g.B = TcOperand{Yt32, nq, nbj, NB, 1, 0};
    g.M = mr; g.N = nq; g.K = nbj; g.batch = 1;
    g.C = Q + (size_t)j0 * m + j0; g.c_fp64 = true;
    g.c_m = im1(1); g.c_n = im1(m); g.c_b = im0();
    g.alpha = -1.0; g.beta = 1.0;
    if ((e = tc(g)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qrctm
