// The QR-CTMRG step in split precision (QR-CTMRG paragraph, Fig. 1(e,f)).
//
// The environment (C, T), the QR of the reduced corner, the symmetrisation
// and the Frobenius normalisation stay in FP64.  The contractions run on the
// tensor cores in TF32x3 (see tc_gemm.cu) on FP32 copies of their operands:
//
//   ct[(a,i),b]  = sum_g C[a,g] T[b,i,g]                  (FP64 out, to the QR)
//   X1[m,b,ub,kb,uk,kk] = sum_a Q[(a,u),m] T[b,k,a]        (FP32)
//   Z [m,b,dk,jk,s,ub,kb] = sum_{uk,kk} X1 A[s,uk,kk,dk,jk]  (ket layer, FP32)
//   X2[m,jk,jb,b,dk,db]  = sum_{s,ub,kb} Z A[s,ub,kb,db,jb]  (bra layer, FP32)
//     (at D = 6 both layers run in one tensor-core kernel with Z on chip;
//      for other even D in one fused FP32 kernel; otherwise as two
//      tensor-core contractions through Z in HBM)
//   T'[m,j,n]    = sum_{b,d} X2[m,j,(b,d)] Q[(b,d),n]      (FP64 out)
//   Y2[n,g,j]    = sum_m T's[n,j,m] R[m,g]                 (FP32, batched over j)
//   C'[n,p]      = sum_{(g,j)} Y2[n,(g,j)] Q[(g,j),p]      (FP64 out)
//
// Every FP32 operand is stored K-contiguous with its row length padded to a
// multiple of 4 floats (16 bytes, the TMA stride rule); the padding is never
// read (TMA reads the true K extent and fills beyond it with zeros).  The
// operands that many output tiles share (T, C, both layouts of Q, R^T) are split
// into TF32 head and tail planes once, when they are formed, instead of in
// every tile of the contraction.
#include "ctx.cuh"
#include "tc_gemm.cuh"

namespace qrctm {

namespace {

inline long long pad4(long long x) { return (x + 3) & ~3ll; }

TcOperand op(const float* p, long long rows, long long K, long long stride, int batch = 1,
             long long bstride = 0, const float* lo = nullptr) {
  return TcOperand{p, rows, K, stride, batch, bstride, lo};
}

TcGemm tc0(qrctm_ctx* c) {
  TcGemm g{};
  g.batch = 1;
  g.c_b = im0();
  g.alpha = 1.0;
  g.beta = 0.0;
  g.err = c->err;
  g.part = c->tc_part;
  g.part_elems = c->tc_part_elems;
  return g;
}

}  // namespace

// FP32 copies of A for the ket and bra contractions (once per qrctm_init_env):
//   Aket[(s,d,r)][(u,l)]  and  Abra[(d,r)][(s,u,l)],  rows padded to 4 floats.
cudaError_t split_prepare_A(qrctm_ctx* c) {
  const int D = c->D, D2 = c->D2, d = c->d;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long D2p = pad4(D2), dD2p = pad4((long long)d * D2);
  cudaError_t e;
  // Aket row (s,d,r) = s*D2 + d*D + r -> A offset s*D4 + d*D + r; col (u,l) -> u*D3 + l*D2
  if ((e = gather_f32(c->A, c->Aket32, (long long)d * D2, D2, D2p, im3(D, D, 1, D, D4),
                      im2(D, D2, D3), c->st)) != cudaSuccess)
    return e;
  // Abra row (d,r) -> d*D + r; col (s,u,l) = s*D2 + u*D + l -> s*D4 + u*D3 + l*D2
  if ((e = gather_f32(c->A, c->Abra32, D2, (int)((long long)d * D2), dD2p, im2(D, 1, D),
                      im3(D, D, D2, D3, D4), c->st)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

cudaError_t qr_step_split(qrctm_ctx* c) {
  const int ch = c->chi_cur, D = c->D, D2 = c->D2, d = c->d;
  const long long m = (long long)ch * D2, D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long chp = pad4(ch), D2p = pad4(D2), dD2 = (long long)d * D2, dD2p = pad4(dD2);
  const long long mp = pad4(m);
  cudaStream_t st = c->st;
  cudaError_t e;
  // heads; the tails sit in the *lo planes of the same layout
  float* T32 = c->T32;      // [(b,k_b,k_k)][a]   rows chi*D2, stride chp (k = k_k D + k_b)
  float* C32 = c->C32;      // [a][g]       stride chp
  float* Qt32 = c->Qt32;    // [(m,u)][a]   rows chi*D2, stride chp
  float* Qc32 = c->Qc32;    // [n][(b,d)]   rows chi, stride mp (FP32 Q, split after use)
  float* X1 = reinterpret_cast<float*>(c->X1);
  float* Zf = reinterpret_cast<float*>(c->Z);
  float* X2 = reinterpret_cast<float*>(c->X2);
  {
    PhaseScope ps(c, QRCTM_PH_CT);
    // rows (b, k_b, k_k) with k_k fastest: the X1 product then writes runs
    // along its lowest output digit
    if ((e = gather_f32(c->T, T32, m, ch, chp, im3(D, D, (long long)D * ch, ch, (long long)D2 * ch),
                        im1(1), st, c->T32lo)) != cudaSuccess)
      return e;
    if ((e = gather_f32(c->C, C32, ch, ch, chp, im1(ch), im1(1), st, c->C32lo)) != cudaSuccess)
      return e;
    // ct(a, (b,i)) = sum_g C[a,g] T[b,i,g]  ->  Mcm[b*m + a*D2 + i]
    // (column n = (b, i_b, i_k), i = i_k D + i_b)
    TcGemm g = tc0(c);
    g.A = op(C32, ch, ch, chp, 1, 0, c->C32lo);
    g.B = op(T32, m, ch, chp, 1, 0, c->T32lo);
    g.M = ch; g.N = m; g.K = ch;
    g.C = c->Mcm; g.c_fp64 = true;
    g.c_m = im1(D2); g.c_n = im3(D, D, D, 1, m);
    // FP32 copy for the QR's tensor-core products: row b, K index (a, i)
    g.C32 = qr_split_x32(c->qr32);
    g.c32_m = im1(D2); g.c32_n = im3(D, D, D, 1, mp);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_QR);
    // R in FP64; Q as its FP32 rows Qc32[n][(b,d)] = Q[(b,d),n]
    if ((e = householder_qr_split((int)m, ch, c->Mcm, c->R, c->qrw, c->qr32, Qc32, true,
                                  c->tc_part, c->tc_part_elems, st)) != cudaSuccess)
      return e;
    // Qt32[(mu,u)][a] = Q[(a,u),mu]
    if ((e = gather_f32f(Qc32, Qt32, m, ch, chp, im2(D2, 1, mp), im1(D2), st, c->Qt32lo)) !=
        cudaSuccess)
      return e;
    if ((e = split_f32(Qc32, c->Qc32lo, ch, (int)m, mp, st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_X1);
    // X1 stored [m][b][u_b][k_b] x (u_k,k_k) with rows padded to D2p
    TcGemm g = tc0(c);
    g.A = op(Qt32, m, ch, chp, 1, 0, c->Qt32lo);
    g.B = op(T32, m, ch, chp, 1, 0, c->T32lo);
    g.M = m; g.N = m; g.K = ch;
    g.C = X1; g.c_fp64 = false;
    // row (mu,u): u = u_k*D + u_b ; col (b,k_b,k_k), k = k_k*D + k_b
    // offset = ((mu*chi + b)*D2 + u_b*D + k_b)*D2p + u_k*D + k_k
    g.c_m = im3(D, D, D * D2p, D, (long long)ch * D2 * D2p);
    g.c_n = im3(D, D, 1, D2p, D2 * D2p);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_ABSORB);
    if (absorb_tc_ok(d, D)) {
      // both layers on the tensor cores in one kernel, Z kept on chip
      if ((e = absorb_tc(X1, c->Aket32, c->Abra32, X2, ch, D2p, dD2p, mp, c->err, st)) !=
          cudaSuccess)
        return e;
    } else if (absorb_fused_ok(d, D)) {
      // ket and bra in one pass, Z kept on chip
      if ((e = absorb_fused(X1, c->Aket32, c->Abra32, X2, ch, D, d, D2p, dD2p, mp, c->err, st)) !=
          cudaSuccess)
        return e;
    } else {
    // ket: Z[(mu,b,u_b,k_b)][(s,d_k,j_k)] stored [(mu,b)][d_k][j_k] x (s,u_b,k_b) padded dD2p
    TcGemm g = tc0(c);
    g.A = op(X1, (long long)ch * ch * D2, D2, D2p);
    g.B = op(c->Aket32, dD2, D2, D2p);
    g.M = (long long)ch * ch * D2; g.N = dD2; g.K = D2;
    g.C = Zf; g.c_fp64 = false;
    g.c_m = im3(D, D, 1, D, D2 * dD2p);
    g.c_n = im3(D, D, dD2p, D * dD2p, D2);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
    // bra: X2[(mu,b,d_k,j_k)][(d_b,j_b)] stored [mu][j_k][j_b] x (b,d_k,d_b) padded mp
    g = tc0(c);
    g.A = op(Zf, (long long)ch * ch * D2, dD2, dD2p);
    g.B = op(c->Abra32, D2, dD2, dD2p);
    g.M = (long long)ch * ch * D2; g.N = D2; g.K = dD2;
    g.C = X2; g.c_fp64 = false;
    g.c_m = im4(D, D, ch, D * mp, D, D2, D2 * mp);
    g.c_n = im2(D, mp, 1);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
    }
  }
  {
    PhaseScope ps(c, QRCTM_PH_PROJECT);
    // T'[(mu,j)][n] = sum_{(b,d)} X2[(mu,j)][(b,d)] Q[(b,d),n]
    TcGemm g = tc0(c);
    g.A = op(X2, m, m, mp);
    g.B = op(Qc32, ch, m, mp, 1, 0, c->Qc32lo);
    g.M = m; g.N = ch; g.K = m;
    g.C = c->Traw; g.c_fp64 = true;
    g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_CORNER);
    if ((e = sym_edge(c->Traw, c->Tn, ch, D2, st)) != cudaSuccess) return e;
    // Ts32[n][j][mu] (mu padded), Rt32[g][mu] = R[mu][g]
    if ((e = gather_f32(c->Tn, c->Ts32, m, ch, chp, im1(ch), im1(1), st)) != cudaSuccess)
      return e;
    // R^T is shared by every batch entry and row block: split once
    if ((e = gather_f32(c->R, c->Rt32, ch, ch, chp, im1(1), im1(ch), st, c->Rt32lo)) !=
        cudaSuccess)
      return e;
    // Y2[n][(g,j)] = sum_mu Ts[n,j,mu] R[mu,g], batch j; stored [n] x (g,j) padded mp
    float* Y2f = reinterpret_cast<float*>(c->Y2);
    TcGemm g = tc0(c);
    g.A = op(c->Ts32, ch, ch, (long long)D2 * chp, D2, chp);
    g.B = op(c->Rt32, ch, ch, chp, 1, 0, c->Rt32lo);
    g.M = ch; g.N = ch; g.K = ch; g.batch = D2;
    g.C = Y2f; g.c_fp64 = false;
    g.c_m = im1(mp); g.c_n = im1(D2); g.c_b = im1(1);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
    // C'[n][p] = sum_{(g,j)} Y2[n][(g,j)] Q[(g,j),p]
    g = tc0(c);
    g.A = op(Y2f, ch, m, mp);
    g.B = op(Qc32, ch, m, mp, 1, 0, c->Qc32lo);
    g.M = ch; g.N = ch; g.K = m;
    g.C = c->Craw; g.c_fp64 = true;
    g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_tc(g, st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_SYMNORM);
    if ((e = sym_norm_env(c->Craw, c->Tn, c->C, c->T, ch, D2, c->partials, c->err, st)) !=
        cudaSuccess)
      return e;
  }
  c->iters += 1;
  return cudaSuccess;
}

}  // namespace qrctm
