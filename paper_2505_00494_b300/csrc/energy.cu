// Energy per site from reduced density matrices (Results paragraphs:
// Heisenberg model with the sublattice rotation exp(i pi sigma^y / 2), and
// the J1-J2 model).
//
// rho_nn : two horizontally adjacent sites of a 2x1 patch (4 C, 6 T).  The
//          left half HL[X,h,Z,s,t] contracts the left column C T C, the top
//          and bottom edges above/below the site and the site itself (ket,
//          then bra with its physical index left open); by the C4v symmetry
//          of A the right half equals HL, so rho = sum_{X,h,Z} HL (x) HL.
// rho_nnn: two diagonal sites of a 2x2 patch (4 C, 8 T).  The four quadrants
//          are one enlarged corner; with its physical legs open (Ct_open) on
//          the diagonal sites, rho = Tr(Ct_open Ct Ct_open Ct).
// The traces and the energy are reduced in FP64 on the device.  In a
// split-precision context the one O((chi D^2)^3) product of the energy,
// P(s,t) = Ct_open(s,t) Ct (d^2 products of (chi D^2)-square matrices, ~90%
// of the J2 term's work), runs on the TF32x3 tensor-core engine in K chunks
// of 512 whose FP32 results are summed in FP64 (one FP32 pass over the whole
// K = chi D^2 moved the d2 D6 chi144 energy by 2.3e-7); every other
// contraction and every trace stay FP64.
#include "ctx.cuh"

namespace qrctm {

namespace {

// Ct[e] = sum_s Ct_open[s][s][e]
__global__ void trace_phys_k(const double* __restrict__ Co, double* __restrict__ Ct, int d,
                             long long mm) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < d; ++s) acc += Co[((long long)s * d + s) * mm + e];
    Ct[e] = acc;
  }
}

// Bond operators on (s1 s2),(t1 t2) for spin 1/2 (basis up = 0, down = 1):
//   h  = S.S = (XX + YY + ZZ)/4,
//   h~ = (1 x U)^dag h (1 x U), U = exp(i pi sigma^y/2) = i sigma^y,
//      = (-XX + YY - ZZ)/4.
__constant__ double c_h[16] = {0.25, 0, 0, 0,  0, -0.25, 0.5, 0,  0, 0.5, -0.25, 0,  0, 0, 0, 0.25};
__constant__ double c_hr[16] = {-0.25, 0, 0, -0.5,  0, 0.25, 0, 0,  0, 0, 0.25, 0,  -0.5, 0, 0, -0.25};

// rho4[s1][t1][s2][t2] -> <h> = Tr(rho h) / Tr(rho), rho[(s1 s2),(t1 t2)]
__device__ double bond_expect(const double* rho4, const double* h) {
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
}

__global__ void energy_k(const double* rho_nn, const double* rho_nnn, double J1, double J2,
                         int nn_plain, double* e_out, int* err) {
  const double enn = bond_expect(rho_nn, nn_plain ? c_h : c_hr);
  double e = 2.0 * J1 * enn;
  double ennn = 0.0;
  if (rho_nnn != nullptr) {
    ennn = bond_expect(rho_nnn, c_h);
    e += 2.0 * J2 * ennn;
  }
  if (!(e == e) || isinf(e)) atomicOr(err, ERRF_NUMERIC);
  e_out[0] = e;
  e_out[1] = enn;
  e_out[2] = ennn;
}

// Traces of pairs of the nb = d^2 matrices P_p (m x m, row-major, P_p at
// P + p mm): rho[p][q] = sum_{i,j} P_p[i][j] P_q[j][i] = Tr(P_p P_q), and the
// adjoint Pb_p[i][j] = sum_q W[p][q] P_q[j][i], W = rhob + rhob^T.  A
// contraction with a d^2 x d^2 output over (chi D^2)^2 terms reads P once (and
// once transposed) and is bound by the FP64 pipe at a few d^4 FMA per
// element; as a general GEMM its 64 x 48 tiles were ~99% idle.  One CTA works
// on 32 x 32 tiles (I, J): its own block P_p[I,J] in registers, the partner
// block P_q[J,I] through shared memory read transposed.  The trace's per-CTA
// partial sums are added in a fixed order by a second kernel.
constexpr int kTrT = 32;          // tile edge
constexpr int kTrThreads = 256;   // 32 x 8: four rows of a tile per thread
constexpr int kTrMaxNb = 4;

__global__ void __launch_bounds__(kTrThreads) trace_pairs_k(const double* __restrict__ P, int nb,
                                                            long long m, double* __restrict__ part) {
  __shared__ double Bt[kTrMaxNb][kTrT][kTrT + 1];
  __shared__ double red[kTrThreads / 32][kTrMaxNb * kTrMaxNb];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // column b, rows ty + 8 r
  const long long mm = m * m;
  const long long nt = (m + kTrT - 1) / kTrT;
  double acc[kTrMaxNb * kTrMaxNb];
#pragma unroll
  for (int u = 0; u < kTrMaxNb * kTrMaxNb; ++u) acc[u] = 0.0;
  for (long long t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const long long I = t / nt, J = t % nt;
    __syncthreads();
    // partner block P_q[J rows][I cols], coalesced along I, kept as Bt[q][row j][col i]
    for (int r = ty; r < kTrT; r += 8) {
      const long long gj = J * kTrT + r, gi = I * kTrT + tx;
#pragma unroll
      for (int q = 0; q < kTrMaxNb; ++q)
        Bt[q][r][tx] = (q < nb && gj < m && gi < m) ? P[q * mm + gj * m + gi] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < kTrT; r += 8) {
      const long long gi = I * kTrT + r, gj = J * kTrT + tx;   // own element (i, j)
      if (gi >= m || gj >= m) continue;
      double a[kTrMaxNb];
#pragma unroll
      for (int p = 0; p < kTrMaxNb; ++p) a[p] = (p < nb) ? P[p * mm + gi * m + gj] : 0.0;
#pragma unroll
      for (int q = 0; q < kTrMaxNb; ++q) {
        const double bq = Bt[q][tx][r];                          // P_q[j][i]
#pragma unroll
        for (int p = 0; p < kTrMaxNb; ++p) acc[p * kTrMaxNb + q] = fma(a[p], bq, acc[p * kTrMaxNb + q]);
      }
    }
  }
  // block reduction: warp shuffles, then the 8 warps in a fixed order
#pragma unroll
  for (int u = 0; u < kTrMaxNb * kTrMaxNb; ++u) {
    double v = acc[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (tx == 0) red[ty][u] = v;
  }
  __syncthreads();
  if (threadIdx.x < kTrMaxNb * kTrMaxNb) {
    double v = 0.0;
    for (int w = 0; w < kTrThreads / 32; ++w) v += red[w][threadIdx.x];
    part[(long long)blockIdx.x * kTrMaxNb * kTrMaxNb + threadIdx.x] = v;
  }
}

__global__ void trace_pairs_sum_k(const double* __restrict__ part, int nparts, int nb,
                                  double* __restrict__ rho) {
  // one warp per (p, q): lanes stride over the CTA partials, then a fixed
  // shuffle tree
  const int u = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (u >= nb * nb) return;
  const int p = u / nb, q = u % nb;
  double v = 0.0;
  for (int b = lane; b < nparts; b += 32) v += part[(long long)b * kTrMaxNb * kTrMaxNb + p * kTrMaxNb + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) rho[p * nb + q] = v;
}

__global__ void __launch_bounds__(kTrThreads) trace_pairs_vjp_k(const double* __restrict__ P, int nb,
                                                                long long m,
                                                                const double* __restrict__ rhob,
                                                                double* __restrict__ Pb) {
  __shared__ double Bt[kTrMaxNb][kTrT][kTrT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long mm = m * m;
  const long long nt = (m + kTrT - 1) / kTrT;
  double w[kTrMaxNb][kTrMaxNb];
#pragma unroll
  for (int p = 0; p < kTrMaxNb; ++p)
#pragma unroll
    for (int q = 0; q < kTrMaxNb; ++q)
      w[p][q] = (p < nb && q < nb) ? rhob[p * nb + q] + rhob[q * nb + p] : 0.0;
  for (long long t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const long long I = t / nt, J = t % nt;
    __syncthreads();
    for (int r = ty; r < kTrT; r += 8) {
      const long long gj = J * kTrT + r, gi = I * kTrT + tx;
#pragma unroll
      for (int q = 0; q < kTrMaxNb; ++q)
        Bt[q][r][tx] = (q < nb && gj < m && gi < m) ? P[q * mm + gj * m + gi] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < kTrT; r += 8) {
      const long long gi = I * kTrT + r, gj = J * kTrT + tx;
      if (gi >= m || gj >= m) continue;
      double b[kTrMaxNb];
#pragma unroll
      for (int q = 0; q < kTrMaxNb; ++q) b[q] = Bt[q][tx][r];       // P_q[j][i]
#pragma unroll
      for (int p = 0; p < kTrMaxNb; ++p) {
        if (p >= nb) break;
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < kTrMaxNb; ++q) v = fma(w[p][q], b[q], v);
        Pb[p * mm + gi * m + gj] = v;
      }
    }
  }
}

}  // namespace

// Uses c->Mcm (ct), c->Y2 (L1), c->X1 (W / X), c->Z (ket), c->X2 (Ct),
// c->E1 (bra / Ct_open), c->E2 (HL), c->E3 (P), c->rho, c->e_d.
bool trace_pairs_ok(int nb) { return nb >= 1 && nb <= kTrMaxNb; }

// rho[p][q] = Tr(P_p P_q) for the nb matrices P_p (m x m) at P + p m^2;
// part: scratch of at least kTraceParts * 16 doubles.
cudaError_t trace_pairs(const double* P, int nb, long long m, double* part, double* rho,
                        cudaStream_t s) {
  if (!trace_pairs_ok(nb)) return cudaErrorInvalidValue;
  const long long nt = (m + kTrT - 1) / kTrT;
  const int grid = (int)std::min<long long>(nt * nt, kTraceParts);
  trace_pairs_k<<<grid, kTrThreads, 0, s>>>(P, nb, m, part);
  note_launch();
  trace_pairs_sum_k<<<1, 32 * kTrMaxNb * kTrMaxNb, 0, s>>>(part, grid, nb, rho);
  note_launch();
  return cudaGetLastError();
}

// Pb_p = sum_q (rhob[p][q] + rhob[q][p]) P_q^T: the cotangent of every P_p
// for rho = Tr(P_p P_q) (overwrites Pb).
cudaError_t trace_pairs_vjp(const double* P, int nb, long long m, const double* rhob, double* Pb,
                            cudaStream_t s) {
  if (!trace_pairs_ok(nb)) return cudaErrorInvalidValue;
  const long long nt = (m + kTrT - 1) / kTrT;
  const int grid = (int)std::min<long long>(nt * nt, 8ll * device_sm_count());
  trace_pairs_vjp_k<<<grid, kTrThreads, 0, s>>>(P, nb, m, rhob, Pb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t energy_fp64(qrctm_ctx* c, double J1, double J2) {
  const int D = c->D, D2 = c->D2, d = c->d, ch = c->chi_cur;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long m = (long long)ch * D2, dD2 = (long long)d * D2;
  const long long Sq = (long long)ch * D2 * ch;
  cudaError_t e;
  cudaStream_t st = c->st;
  // ct = C T
  if ((e = reduced_corner(c, c->C, c->T, ch, c->Mcm)) != cudaSuccess) return e;
  // L1[(x1,q),z1] = sum_y ct[(x1,q),y] C[y,z1]
  {
    Gemm g = gemm_ctx(c);
    g.M = m; g.N = ch; g.K = ch;
    g.A = c->Mcm; g.a_m = im1(1); g.a_k = im1(m);
    g.B = c->C; g.b_k = im1(ch); g.b_n = im1(1);
    g.C = c->Y2; g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // W[(q,z1),(p,X)] = sum_x1 L1[x1,q,z1] T[x1,p,X]
  {
    Gemm g = gemm_ctx(c);
    g.M = m; g.N = m; g.K = ch;
    g.A = c->Y2; g.a_m = im1(1); g.a_k = im1(m);
    g.B = c->T; g.b_k = im1(m); g.b_n = im1(1);
    g.C = c->X1; g.c_m = im1(m); g.c_n = im1(1);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // ket: Z1[(z1,X,q_b,p_b),(s,d_k,h_k)] = sum_{p_k,q_k} W A[s,p_k,q_k,d_k,h_k]
  {
    Gemm g = gemm_ctx(c);
    g.M = (long long)ch * ch * D2; g.N = dD2; g.K = D2;
    g.A = c->X1; g.a_m = im4(D, D, ch, ch, Sq, 1, m); g.a_k = im2(D, D * Sq, (long long)D * ch);
    g.B = c->A; g.b_k = im2(D, D2, D3); g.b_n = im3(D, D, 1, D, D4);
    g.C = c->Z; g.c_m = im1(dD2); g.c_n = im1(1);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // bra (physical index t open): Z2 stored [X][s][t][h_k][h_b][z1][d_k][d_b]
  {
    const long long D2c = (long long)D2 * ch, D4c = D4 * ch;
    Gemm g = gemm_ctx(c);
    g.M = (long long)ch * ch * dD2; g.N = dD2; g.K = D2;
    g.A = c->Z; g.a_m = im4(D, D, d, 1, D, D2, D2 * dD2); g.a_k = im2(D, dD2, D * dD2);
    g.B = c->A; g.b_k = im2(D, D3, D2); g.b_n = im3(D, D, 1, D, D4);
    g.C = c->E1;
    g.c_m = im5(D, D, d, ch, (long long)D * D2c, D, (long long)d * D4c,
                (long long)d * d * D4c, D2);
    g.c_n = im3(D, D, D2c, 1, D4c);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // HL[(X,s,t,h),Z] = sum_{(z1,d)} Z2[X,s,t,h,(z1,d)] T[(z1,d),Z]
  {
    Gemm g = gemm_ctx(c);
    g.M = (long long)ch * d * d * D2; g.N = ch; g.K = m;
    g.A = c->E1; g.a_m = im1(m); g.a_k = im1(1);
    g.B = c->T; g.b_k = im1(ch); g.b_n = im1(1);
    g.C = c->E2; g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // rho_nn[(s1,t1),(s2,t2)] = sum_{X,h,Z} HL[X,s1,t1,h,Z] HL[X,s2,t2,h,Z]
  {
    const long long st_str = (long long)D2 * ch;
    Gemm g = gemm_ctx(c);
    g.M = d * d; g.N = d * d; g.K = (long long)ch * D2 * ch;
    g.A = c->E2; g.a_m = im1(st_str); g.a_k = im3(ch, D2, 1, ch, (long long)d * d * D2 * ch);
    g.B = c->E2; g.b_k = im3(ch, D2, 1, ch, (long long)d * d * D2 * ch); g.b_n = im1(st_str);
    g.C = c->rho; g.c_m = im1(d * d); g.c_n = im1(1);
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  double* rho_nnn = nullptr;
  if (J2 != 0.0) {
    if (c->E3 == nullptr) return cudaErrorInvalidValue;
    rho_nnn = c->rho + 16;
    // X[(i,r),(k,b)] = sum_g ct[(g,i),r] T[g,(k,b)] and the ket layer -> c->Z
    const long long Su = (long long)ch * D2 * ch, Smu = (long long)D2 * ch, Sk = ch;
    {
      Gemm g = gemm_ctx(c);
      g.M = m; g.N = m; g.K = ch;
      g.A = c->Mcm; g.a_m = im2(ch, m, 1); g.a_k = im1(D2);
      g.B = c->T; g.b_k = im1(m); g.b_n = im1(1);
      g.C = c->X1; g.c_m = im1(m); g.c_n = im1(1);
      if ((e = gemm_run(c, g)) != cudaSuccess) return e;
      g = gemm_ctx(c);
      g.M = (long long)ch * ch * D2; g.N = dD2; g.K = D2;
      g.A = c->X1; g.a_m = im4(D, D, ch, Sk, Su, 1, Smu); g.a_k = im2(D, D * Sk, D * Su);
      g.B = c->A; g.b_k = im2(D, D2, D3); g.b_n = im3(D, D, 1, D, D4);
      g.C = c->Z; g.c_m = im1(dD2); g.c_n = im1(1);
      if ((e = gemm_run(c, g)) != cudaSuccess) return e;
    }
    // bra with t open: Ct_open stored [s][t][b][l_k][l_b][r][j_k][j_b]
    {
      const long long mm = m * m;
      Gemm g = gemm_ctx(c);
      g.M = (long long)ch * ch * dD2; g.N = dD2; g.K = D2;
      g.A = c->Z; g.a_m = im4(D, D, d, 1, D, D2, D2 * dD2); g.a_k = im2(D, dD2, D * dD2);
      g.B = c->A; g.b_k = im2(D, D2, D3); g.b_n = im3(D, D, 1, D, D4);
      g.C = c->E1;
      g.c_m = im5(D, D, d, ch, D, D * m, (long long)d * mm, (long long)D2 * m, D2);
      g.c_n = im3(D, D, 1, m, mm);
      if ((e = gemm_run(c, g)) != cudaSuccess) return e;
      trace_phys_k<<<1184, 256, 0, st>>>(c->E1, c->X2, d, mm);
      note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // P(s,t) = Ct_open(s,t) Ct  (tensor cores in a split-precision context)
      g = gemm_ctx(c);
      g.M = m; g.N = m; g.K = m; g.batch = d * d;
      g.A = c->E1; g.a_m = im1(m); g.a_k = im1(1); g.a_b = im1(mm);
      g.B = c->X2; g.b_k = im1(m); g.b_n = im1(1); g.b_b = im0();
      g.C = c->E3; g.c_m = im1(m); g.c_n = im1(1); g.c_b = im1(mm);
      const bool was = c->mm_split;
      c->mm_split = c->split_prec && c->mm32 != nullptr;
      e = gemm_run_kchunked(c, g, 512);
      c->mm_split = was;
      if (e != cudaSuccess) return e;
      // rho_nnn[(s1,t1),(s4,t4)] = sum_{a,c} P(s1,t1)[a,c] P(s4,t4)[c,a]
      if (trace_pairs_ok(d * d)) {
        if ((e = trace_pairs(c->E3, d * d, m, c->partials, rho_nnn, st)) != cudaSuccess) return e;
      } else {
        g = gemm_ctx(c);
        g.M = d * d; g.N = d * d; g.K = mm;
        g.A = c->E3; g.a_m = im1(mm); g.a_k = im1(1);
        g.B = c->E3; g.b_k = im2((int)m, m, 1); g.b_n = im1(mm);
        g.C = rho_nnn; g.c_m = im1(d * d); g.c_n = im1(1);
        if ((e = gemm_run(c, g)) != cudaSuccess) return e;
      }
    }
  }
  energy_k<<<1, 1, 0, st>>>(c->rho, rho_nnn, J1, J2, c->nn_plain ? 1 : 0, c->e_d, c->err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
