// One QR-CTMRG step and the standard warm-up step (QR-CTMRG and Standard
// CTMRG paragraphs, Fig. 1(d)-(f)), FP64 path.
//
// Layouts (row-major unless stated):
//   C[a][b], T[a][k][b]                       environment
//   Mcm  column-major (chi*D2) x chi         reduced corner ct[(g,i),r]
//   Q    column-major (chi*D2) x chi, R row-major chi x chi
//   X1[u][m][k][b]                           sum_a P[(a,u),m] T[a,k,b]
//   Z [m][b][u_b][k_b][s][d_k][j_k]          ket layer absorbed
//   X2[m][b][d_k][j_k][d_b][j_b]             both layers absorbed
//   T'[m][j][n], Y2[n][g][j]
// The reshapes and permutations between them are folded into the index maps
// of the contraction engine, so no separate permute pass runs.
#include "ctx.cuh"

namespace qrctm {

// ct[(g,i),r] = sum_h C[g,h] T[h,i,r], batched over i; written column-major.
cudaError_t reduced_corner(qrctm_ctx* c, const double* C, const double* T, int ci, double* Mcm) {
  const int D2 = c->D2;
  const long long mi = (long long)ci * D2;
  Gemm g = gemm_ctx(c);
  g.M = ci; g.N = ci; g.K = ci; g.batch = D2;
  g.A = C; g.a_m = im1(ci); g.a_k = im1(1); g.a_b = im0();
  g.B = T; g.b_k = im1((long long)D2 * ci); g.b_n = im1(1); g.b_b = im1(ci);
  g.C = Mcm; g.c_m = im1(D2); g.c_n = im1(mi); g.c_b = im1(1);
  return gemm_f64(g, c->st);
}

// X1 = P^T T (over the chi leg), absorb A (ket then bra, or the double layer
// a), then project the other side with P:
//   T'[m,j,n] = sum P[(a,u),m] T[a,k,b] a[u,k,d,j] P[(b,d),n]
// P: column-major (ci*D2) x co.  X2 stays in c->X2; Tout == nullptr skips
// the last projection (the warm-up uses X2 as the enlarged corner).
cudaError_t renorm_edge(qrctm_ctx* c, const double* P, int co, const double* T, int ci,
                        double* Tout) {
  const int D = c->D, D2 = c->D2, d = c->d;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long mi = (long long)ci * D2;
  const long long Su = (long long)co * D2 * ci, Smu = (long long)D2 * ci, Sk = ci;
  cudaError_t e;
  // X1[(u,m),(k,b)] = sum_a P[(a,u),m] T[a,(k,b)], u = (u_k,u_b), k = (k_k,k_b);
  // for the fused FP64 absorption stored slice by slice instead,
  // X1[(m,b)][(u_b,k_b)][(u_k,k_k)]
  const bool fused64 = c->split_layers && absorb64_ok(d, D);
  {
    PhaseScope ps(c, QRCTM_PH_X1);
    Gemm g = gemm_ctx(c);
    g.M = (long long)D2 * co; g.N = (long long)D2 * ci; g.K = ci;
    g.A = P; g.a_m = im2(co, mi, 1); g.a_k = im1(D2);
    g.B = T; g.b_k = im1((long long)D2 * ci); g.b_n = im1(1);
    g.C = c->X1; g.c_m = im1(g.N); g.c_n = im1(1);
    if (fused64) {
      g.c_m = im3(co, D, (long long)ci * D4, D3, D);
      g.c_n = im3(ci, D, D4, D2, 1);
    }
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  }
  {
  PhaseScope ps_abs(c, QRCTM_PH_ABSORB);
  if (fused64) {
    // both layers in one FP64 kernel, Z on chip; X2 as the bra GEMM writes it
    if ((e = absorb64(c->X1, c->A, c->X2, (long long)co * ci, d, D, c->err, c->st)) != cudaSuccess)
      return e;
  } else if (c->split_layers) {
    const long long dD2 = (long long)d * D2;
    // ket: Z[(m,b,u_b,k_b),(s,d_k,j_k)] = sum_{u_k,k_k} X1 A[s,u_k,k_k,d_k,j_k]
    Gemm g = gemm_ctx(c);
    g.M = (long long)co * ci * D2; g.N = dD2; g.K = D2;
    g.A = c->X1; g.a_m = im4(D, D, ci, Sk, Su, 1, Smu); g.a_k = im2(D, D * Sk, D * Su);
    g.B = c->A; g.b_k = im2(D, D2, D3); g.b_n = im3(D, D, 1, D, D4);
    g.C = c->Z; g.c_m = im1(dD2); g.c_n = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
    // bra: X2[(m,b,d_k,j_k),(d_b,j_b)] = sum_{s,u_b,k_b} Z A[s,u_b,k_b,d_b,j_b]
    g = gemm_ctx(c);
    g.M = (long long)co * ci * D2; g.N = D2; g.K = dD2;
    g.A = c->Z; g.a_m = im3(D, D, 1, D, D2 * dD2); g.a_k = im3(D, D, dD2, D * dD2, D2);
    g.B = c->A; g.b_k = im3(D, D, D2, D3, D4); g.b_n = im1(1);
    g.C = c->X2; g.c_m = im1(D2); g.c_n = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  } else {
    // X2[(m,b),(d,j)] = sum_{(u,k)} X1 a[(u,k),(d,j)], stored [m,b,d_k,j_k,d_b,j_b]
    Gemm g = gemm_ctx(c);
    g.M = (long long)co * ci; g.N = D4; g.K = D4;
    g.A = c->X1; g.a_m = im2(ci, 1, Smu); g.a_k = im2(D2, Sk, Su);
    g.B = c->a; g.b_k = im1(D4); g.b_n = im1(1);
    g.C = c->X2; g.c_m = im1(D4); g.c_n = x2_maps(c, ci).store_n;
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  }
  }
  if (Tout == nullptr) return cudaSuccess;
  // T'[(m,j),n] = sum_{(b,d)} X2[m,b,d_k,j_k,d_b,j_b] P[(b,d),n]
  {
    PhaseScope ps(c, QRCTM_PH_PROJECT);
    Gemm g = gemm_ctx(c);
    g.M = (long long)co * D2; g.N = co; g.K = mi;
    const X2Maps xm = x2_maps(c, ci);
    g.A = c->X2; g.a_m = xm.ct_col; g.a_k = xm.ct_row;
    g.B = P; g.b_k = im1(1); g.b_n = im1(mi);
    g.C = Tout; g.c_m = im1(co); g.c_n = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One QR-CTMRG step at bond chi_cur:
//   ct = C T, ct = Q R, T' = Q^T (T a) Q, T's = sym(T'),
//   C'[n,p] = sum_{m,g,j} T's[m,j,n] R[m,g] Q[(g,j),p]   (Fig. 1(f)),
//   (C, T) <- normalise(sym(C'), T's).
cudaError_t qr_step(qrctm_ctx* c) {
  const int ch = c->chi_cur, D2 = c->D2;
  const long long m = (long long)ch * D2;
  cudaError_t e;
  {
    PhaseScope ps(c, QRCTM_PH_CT);
    if ((e = reduced_corner(c, c->C, c->T, ch, c->Mcm)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_QR);
    if ((e = householder_qr_f64((int)m, ch, c->Mcm, c->Q, c->R, c->qrw, c->st)) != cudaSuccess)
      return e;
  }
  if ((e = renorm_edge(c, c->Q, ch, c->T, ch, c->Traw)) != cudaSuccess) return e;
  {
    PhaseScope ps(c, QRCTM_PH_CORNER);
    if ((e = sym_edge(c->Traw, c->Tn, ch, D2, c->st)) != cudaSuccess) return e;
    // Y2[n,(g,j)] = sum_m T's[n,j,m] R[m,g]   (batched over j; T's symmetric)
    Gemm g = gemm_ctx(c);
    g.M = ch; g.N = ch; g.K = ch; g.batch = D2;
    g.A = c->Tn; g.a_m = im1((long long)D2 * ch); g.a_k = im1(1); g.a_b = im1(ch);
    g.B = c->R; g.b_k = im1(ch); g.b_n = im1(1); g.b_b = im0();
    g.C = c->Y2; g.c_m = im1((long long)ch * D2); g.c_n = im1(D2); g.c_b = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
    // C'[n,p] = sum_{(g,j)} Y2[n,(g,j)] Q[(g,j),p]
    g = gemm_ctx(c);
    g.M = ch; g.N = ch; g.K = m;
    g.A = c->Y2; g.a_m = im1(m); g.a_k = im1(1);
    g.B = c->Q; g.b_k = im1(1); g.b_n = im1(m);
    g.C = c->Craw; g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  }
  {
    PhaseScope ps(c, QRCTM_PH_SYMNORM);
    if ((e = sym_norm_env(c->Craw, c->Tn, c->C, c->T, ch, D2, c->partials, c->err, c->st)) !=
        cudaSuccess)
      return e;
  }
  c->iters += 1;
  return cudaSuccess;
}

// Standard step growing chi_in -> chi_out with an isometry U spanning the
// dominant |eigenvalue| subspace of the enlarged corner Ct (Fig. 1(d)),
// obtained by block subspace iteration Q <- qr(Ct Q) from the first chi_out
// columns of Ct.  C' = U^T Ct U, T' = U^T (T a) U.
cudaError_t warmup_step(qrctm_ctx* c, int ci, int co) {
  const int D = c->D, D2 = c->D2;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long mi = (long long)ci * D2;
  cudaError_t e;
  if ((e = reduced_corner(c, c->C, c->T, ci, c->Mcm)) != cudaSuccess) return e;
  // X2 <- enlarged corner: the first half of renorm_edge with P = ct
  if ((e = renorm_edge(c, c->Mcm, ci, c->T, ci, nullptr)) != cudaSuccess) return e;
  // Ct((b,l),(r,j)) = X2[r,b,l,j]
  const X2Maps xm = x2_maps(c, ci);
  const IdxMap ct_row = xm.ct_row, ct_col = xm.ct_col;
  // (every use of Ct comes before the final renorm_edge overwrites X2)
  auto apply_ct = [&](const double* X, double* Y, int ncol) -> cudaError_t {
    Gemm g = gemm_ctx(c);
    g.M = mi; g.N = ncol; g.K = mi;
    g.A = c->X2; g.a_m = ct_row; g.a_k = ct_col;
    g.B = X; g.b_k = im1(1); g.b_n = im1(mi);
    g.C = Y; g.c_m = im1(1); g.c_n = im1(mi);
    return gemm_f64(g, c->st);
  };
  // start block: first co columns of Ct
  if ((e = set_identity_cols(c->Q, (int)mi, co, c->st)) != cudaSuccess) return e;
  if ((e = apply_ct(c->Q, c->Xs, co)) != cudaSuccess) return e;
  const int sweeps = 4;
  for (int it = 0; it < sweeps; ++it) {
    if ((e = householder_qr_f64((int)mi, co, c->Xs, c->Q, c->R, c->qrw, c->st)) != cudaSuccess)
      return e;
    if ((e = apply_ct(c->Q, c->Xs, co)) != cudaSuccess) return e;
  }
  if ((e = householder_qr_f64((int)mi, co, c->Xs, c->Q, c->R, c->qrw, c->st)) != cudaSuccess)
    return e;
  // C' = U^T (Ct U)
  if ((e = apply_ct(c->Q, c->Yw, co)) != cudaSuccess) return e;
  {
    Gemm g = gemm_ctx(c);
    g.M = co; g.N = co; g.K = mi;
    g.A = c->Q; g.a_m = im1(mi); g.a_k = im1(1);
    g.B = c->Yw; g.b_k = im1(1); g.b_n = im1(mi);
    g.C = c->Craw; g.c_m = im1(co); g.c_n = im1(1);
    if ((e = gemm_f64(g, c->st)) != cudaSuccess) return e;
  }
  if ((e = renorm_edge(c, c->Q, co, c->T, ci, c->Traw)) != cudaSuccess) return e;
  if ((e = sym_norm_env(c->Craw, c->Traw, c->C, c->T, co, D2, c->partials, c->err, c->st)) !=
      cudaSuccess)
    return e;
  c->chi_cur = co;
  return cudaSuccess;
}

cudaError_t spectrum_check(qrctm_ctx* c) {
  PhaseScope ps(c, QRCTM_PH_SPECTRUM);
  if (c->spec_pending) {
    // first test after an initialisation: s_prev <- |eig(C_init)| and
    // s_cur <- |eig(C)| in one set of launches
    c->spec_pending = false;
    return corner_spectrum_pair(c->C_init, c->chi_init, c->spec_work2, c->s_prev, c->C,
                                c->chi_cur, c->spec_work, c->s_cur, c->delta_d, c->err, c->st);
  }
  // s_prev <- s_cur, then s_cur <- |eig(C)|, delta <- ||s_cur - s_prev||
  cudaError_t e = cudaMemcpyAsync(c->s_prev, c->s_cur, sizeof(double) * c->chi,
                                  cudaMemcpyDeviceToDevice, c->st);
  if (e != cudaSuccess) return e;
  return corner_spectrum(c->C, c->chi_cur, c->spec_work, c->s_cur,
                         c->spec_valid ? c->s_prev : nullptr, c->chi_cur, c->delta_d, c->err,
                         c->st);
}

}  // namespace qrctm
