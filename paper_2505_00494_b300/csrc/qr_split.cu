// Blocked Householder QR of the reduced corner for the split-precision path
// (QR-CTMRG paragraph: unpivoted QR, diag(R) >= 0).
//
// The panels are factored exactly as in the FP64 path (cooperative FP64
// panel kernel, FP64 reflector norms, Parlett's form of v_0).  The
// compact-WY products that dominate the flop count run on the TF32x3
// tensor-core engine from FP32 copies of V and of the blocks they act on,
// reading and writing the FP64 matrices (FP32-class accuracy, the precision
// of the rest of the split path).  Per panel of nb reflectors:
//
//   1. panel kernel: V (FP64) and its FP32 copies (K-contiguous rows of X32,
//      and Vr32 rows for the update);
//   2. one tensor-core product  S = V^T [V | W2]  left as K-chunk partials;
//   3. wy_prep: sums the partials (compensated FP32 summation), builds T in
//      FP64 from G = V^T V and tau (T_12 = -T_11 G_12 T_22 by recursive
//      doubling) and forms Y2 = T^T (V^T W2) as FP32 rows for the update;
//   4. W2 <- W2 - V Y2 on the tensor cores.
// After a TF32x3 product the trailing matrix is FP32-class accurate, so it is
// kept in FP32 only (X32, rows = columns of ct): each panel converts its 32
// columns to FP64 when it loads them (the first panel reads ct itself in
// FP64), and the entries of R above a panel's diagonal block come from X32.
// Q = H_1 ... H_n [I; 0] comes from the aggregated compact-WY form of all n
// reflectors, I - V T V^T with T^-1 = diag(1/tau) + striu(V^T V):
//   Q = [I; 0] - V W,   W = T V_top^T  (V_top = the first n rows of V),
// i.e. one tensor-core Gram product V^T V, a triangular solve U W = V_top^T
// (U = T^-1; one warp per column of W, FP32 -- Q is FP32 in this path) and
// one tensor-core product V W.  Its rows Q32[c][i] (= column c of Q) are
// what the rest of the step consumes.
#include "qrctm_internal.cuh"
#include "tc_gemm.cuh"

#include <algorithm>

namespace qrctm {

namespace {

// Compensated FP32 sum (TwoSum per term, Knuth) of ksplit partials
// p[z * stride], z = 0, 1, ...: the loads of up to sixteen partials are
// issued before they are added (in the same order), so the L2 round trips
// overlap instead of following the summation chain.  Returns (sum, tail).
__device__ __forceinline__ float2 sum_partials(const float* __restrict__ p, long long stride,
                                               int ksplit) {
  float sh = 0.f, se = 0.f;
  auto add = [&](float x) {
    const float t = sh + x;
    const float bp = t - sh;
    se += (sh - (t - bp)) + (x - bp);
    sh = t;
  };
  int z = 0;
  for (; z + 16 <= ksplit; z += 16) {
    float x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = p[(long long)(z + u) * stride];
#pragma unroll
    for (int u = 0; u < 16; ++u) add(x[u]);
  }
  if (z < ksplit) {
    // the remaining (< 16) partials, loaded together before they are added
    float x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = (z + u < ksplit) ? p[(long long)(z + u) * stride] : 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (z + u < ksplit) add(x[u]);
    z = ksplit;
  }
  for (; z < ksplit; ++z) add(p[(long long)z * stride]);
  return make_float2(sh, se);
}

constexpr int NB = kQrPanel;
constexpr int kWyThreads = 1024;   // two partial sums per thread for a 32 x 32 block
constexpr int kQrMaxKsplit = 48;   // K chunks of the V^T [.] products (M = 32: more CTAs)

inline long long pad4(long long x) { return (x + 3) & ~3ll; }

// part: K-chunk partials [ksplit][nb][N] of S = V^T B.
// mode 0 (factorisation): G = S[:, 0:nb] -> T (Tp <- T by CTA 0),
//   Yt[c][q] = (T^T S[:, ycol0 + c])[q];
// mode 1 (formation of Q): T = Tp, Yt[c][q] = (T S[:, ycol0 + c])[q].
// CTA b handles columns c in [32 b, 32 b + 32) of the ncol Y columns.
// T and Y2 are formed in FP32, the precision of the tensor-core update that
// consumes them (and of G, whose entries are compensated FP32 sums of
// TF32x3 products): the recursion's dependent chains then cost FP32
// latencies instead of B300's 64-clock FP64 ones.  T's diagonal (tau) is
// kept in FP64 in Tp for the formation of Q.
__global__ void __launch_bounds__(kWyThreads) wy_prep_kernel(const float* __restrict__ part,
                                                             int ksplit, int nb, long long N,
                                                             int ycol0, int ncol,
                                                             const double* __restrict__ tau,
                                                             double* __restrict__ Tp,
                                                             float* __restrict__ Yt, int mode) {
  __shared__ float Ts[NB][NB + 1];
  __shared__ float Gs[NB][NB + 1];
  __shared__ float Ws[NB][NB + 1];
  __shared__ float Yf[NB][NB + 1];
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * NB;
  const long long MN = (long long)nb * N;
  // sum of the K-chunk partials by compensated FP32 summation (Knuth's
  // TwoSum: s + e carries the sum up to the final rounding)
  auto psum = [&](int q, long long col) {
    const float2 r = sum_partials(part + (long long)q * N + col, MN, ksplit);
    return r.x + r.y;
  };
  for (int e = tid; e < NB * NB; e += kWyThreads) {
    const int q = e / NB, c = e % NB;
    Yf[q][c] = (q < nb && c0 + c < ncol) ? psum(q, ycol0 + c0 + c) : 0.f;
    if (mode == 0) {
      Gs[q][c] = (q < nb && c < nb) ? psum(q, c) : 0.f;
      Ts[q][c] = (q == c && q < nb) ? static_cast<float>(tau[q]) : 0.f;
    } else {
      Ts[q][c] = static_cast<float>(Tp[q * NB + c]);
    }
  }
  __syncthreads();
  if (mode == 0) {
    // recursive doubling over diagonal blocks of size s:
    //   W = G_12 T_22,  T_12 = -T_11 W   (both factors upper triangular)
    for (int s = 1; s < NB; s <<= 1) {
      const int cnt = (NB / (2 * s)) * s * s;
      for (int e = tid; e < cnt; e += kWyThreads) {
        const int k = e / (s * s), i = (e / s) % s, j = e % s, b0 = 2 * s * k;
        float acc = 0.f;
        for (int l = 0; l <= j; ++l) acc = fmaf(Gs[b0 + i][b0 + s + l], Ts[b0 + s + l][b0 + s + j], acc);
        Ws[b0 + i][b0 + s + j] = acc;
      }
      __syncthreads();
      for (int e = tid; e < cnt; e += kWyThreads) {
        const int k = e / (s * s), i = (e / s) % s, j = e % s, b0 = 2 * s * k;
        float acc = 0.f;
        for (int l = i; l < s; ++l) acc = fmaf(Ts[b0 + i][b0 + l], Ws[b0 + l][b0 + s + j], acc);
        Ts[b0 + i][b0 + s + j] = -acc;
      }
      __syncthreads();
    }
    if (blockIdx.x == 0)
      for (int e = tid; e < NB * NB; e += kWyThreads) {
        const int q = e / NB, c = e % NB;
        Tp[e] = (q == c && q < nb) ? tau[q] : static_cast<double>(Ts[q][c]);
      }
  }
  // Y2 = T^T Y (mode 0) or T Y (mode 1), written transposed
  for (int e = tid; e < NB * NB; e += kWyThreads) {
    const int c = e / NB, q = e % NB;
    if (c0 + c >= ncol) continue;
    float acc = 0.f;
    if (mode == 0) {
      for (int l = 0; l <= q; ++l) acc = fmaf(Ts[l][q], Yf[l][c], acc);
    } else {
      for (int l = q; l < NB; ++l) acc = fmaf(Ts[q][l], Yf[l][c], acc);
    }
    Yt[(long long)(c0 + c) * NB + q] = acc;
  }
}

// UT[i][l] = U[l][i] for the aggregated compact-WY factor U = T^-1:
// U[l][i] = (V^T V)[l][i] for l < i, 1/tau_i for l = i, 0 below; G = V^T V
// from its K-chunk partials [ksplit][n][n] (compensated FP32 summation), tau
// from the diagonals of the per-panel T factors (Tf, stride NB x NB per panel).
__global__ void build_ut_kernel(const float* __restrict__ part, int ksplit, int n,
                                const double* __restrict__ Tf, float* __restrict__ UT,
                                long long ldu) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), l = (int)(e % n);
  float v = 0.f;
  if (l < i) {
    const long long nn = (long long)n * n;
    const float2 r = sum_partials(part + (long long)l * n + i, nn, ksplit);
    v = r.x + r.y;
  } else if (l == i) {
    const double tau = Tf[(size_t)(i / NB) * NB * NB + (i % NB) * NB + (i % NB)];
    v = static_cast<float>(1.0 / tau);
  }
  UT[(long long)i * ldu + l] = v;
}

// Wt[k][i] = W[i][k] with U W = V_top^T, one warp per column k: b_i =
// V[k][i] (zero for i > k), back substitution in axpy form from i = k down:
// x_i = b_i tau_i (= b_i / U_ii), then b_l -= U[l][i] x_i for l < i.  The
// rows of U^T and tau are staged in shared memory (all eight warps of a CTA
// use them) when they fit, else each row is loaded one step ahead.
// MAXQ values per lane: n <= 32 MAXQ (16 up to n = 512, 32 up to 1024).
constexpr int kSolveMaxPerLane = 32;   // n <= 1024
constexpr int kSolveSmemMaxN = 200;    // U^T staged in shared memory up to n = 200
// STAGED (n <= kSolveSmemMaxN) is a template parameter so that the row loads
// of U^T compile to shared-memory loads, not generic ones.
template <int MAXQ, bool STAGED>
__global__ void __launch_bounds__(256) q_solve_kernel(const float* __restrict__ UT, long long ldu,
                                                      const float* __restrict__ Vt,
                                                      long long ldv, const double* __restrict__ Tf,
                                                      int n, float* __restrict__ Wt) {
  extern __shared__ float qs[];
  constexpr bool staged = STAGED;
  float* taus = qs;                       // [n]
  float* us = qs + ((n + 3) & ~3);        // [n][n] when staged
  for (int e = threadIdx.x; e < n; e += blockDim.x)
    taus[e] = static_cast<float>(Tf[(size_t)(e / NB) * NB * NB + (e % NB) * NB + (e % NB)]);
  if (staged) {
    // rows of U^T by warps, lanes along the row (no per-element division);
    // 16-byte copies when rows are 16-byte aligned in both places
    const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
    if ((n & 3) == 0 && (ldu & 3) == 0) {
      const int n4 = n >> 2;
      for (int row = wid; row < n; row += nw) {
        const float4* src = reinterpret_cast<const float4*>(UT + (long long)row * ldu);
        float4* dst = reinterpret_cast<float4*>(us + (long long)row * n);
        for (int c = ln; c < n4; c += 32) dst[c] = src[c];
      }
    } else {
      for (int row = wid; row < n; row += nw)
        for (int c = ln; c < n; c += 32) us[(long long)row * n + c] = UT[(long long)row * ldu + c];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= n) return;
  float b[MAXQ];   // b[q] holds entry i = lane + 32 q
#pragma unroll
  for (int qq = 0; qq < MAXQ; ++qq) {
    const int i = lane + 32 * qq;
    b[qq] = (i <= k && i < n) ? Vt[(long long)k * ldv + i] : 0.f;
  }
  float* out = Wt + (long long)k * ldv;
  for (int i = lane; i < n; i += 32) out[i] = 0.f;
  __syncwarp();
  const int nq = (k + 32) / 32;           // slots that can hold l < i <= k
  float u[MAXQ], un[MAXQ];
  auto load_row = [&](int i, float* dst) {
    const float* src = staged ? us + (long long)i * n : UT + (long long)i * ldu;
#pragma unroll
    for (int qq = 0; qq < MAXQ; ++qq) {
      const int l = lane + 32 * qq;
      dst[qq] = (qq < nq && l < i) ? src[l] : 0.f;
    }
  };
  load_row(k, un);
  for (int i = k; i >= 0; --i) {
#pragma unroll
    for (int qq = 0; qq < MAXQ; ++qq) u[qq] = un[qq];
    if (i > 0) load_row(i - 1, un);       // next row while this one is applied
    const int owner = i & 31, slot = i >> 5;
    float bi = 0.f;
#pragma unroll
    for (int qq = 0; qq < MAXQ; ++qq)
      if (qq == slot) bi = b[qq];
    const float xi = __shfl_sync(0xffffffffu, bi, owner) * taus[i];
    if (lane == 0) out[i] = xi;
#pragma unroll
    for (int qq = 0; qq < MAXQ; ++qq) b[qq] = fmaf(-u[qq], xi, b[qq]);
  }
}

// Q32[c][i] = delta_ci (the FP32 rows of Q = [I; 0]), row stride ldq
// one CTA row per column c (blockIdx.y), threads along the rows i
__global__ void init_q32_kernel(float* Q32, int m, int n, long long ldq) {
  const int c = blockIdx.y;
  float* col = Q32 + (long long)c * ldq;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    col[i] = (i == c) ? 1.f : 0.f;
}

// R (row-major n x n): R[i][j] for i <= j from the FP64 panel output W when
// row i lies in column j's panel, else from the FP32 trailing rows X32[j][i]
__global__ void extract_r_split_kernel(const double* __restrict__ W, const float* __restrict__ X32,
                                       double* __restrict__ R, int m, int n, long long ldx) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const int p0 = (j / NB) * NB;
  R[e] = (i > j) ? 0.0
                 : (i >= p0 ? W[(long long)j * m + i]
                            : static_cast<double>(X32[(long long)j * ldx + i]));
}

}  // namespace

size_t qr_split_floats(int m, int n) {
  const long long mp = pad4(m), ldv = pad4(n);
  return (size_t)(2 * n * mp + (long long)m * ldv + (long long)n * NB + 2 * (long long)n * ldv +
                  1024);
}

float* qr_split_x32(float* f32) { return f32; }

cudaError_t householder_qr_split(int m, int n, const double* M, double* R, const QrWork& w,
                                 float* f32, float* Q32, bool x32_ready, float* part,
                                 long long part_elems, cudaStream_t s) {
  if (m < n || n <= 0) return cudaErrorInvalidValue;
  if (n > 32 * kSolveMaxPerLane) return cudaErrorInvalidValue;
  const long long mp = pad4(m), ldv = pad4(n);
  const int npan = (n + NB - 1) / NB;
  float* X32 = f32;                                  // [c][i]   n x mp  (W, then V rows)
  float* V32 = X32 + (long long)n * mp;              // [c][i]   n x mp  (V, zero above)
  float* Vt32 = V32 + (long long)n * mp;             // [i][c]   m x ldv (V, zero above)
  float* Yt32 = Vt32 + (long long)m * ldv;           // [c][q]   n x NB
  float* UT = Yt32 + (long long)n * NB;              // [i][l]   n x ldv
  float* Wt = UT + (long long)n * ldv;               // [k][i]   n x ldv
  // the first panel reads ct in FP64 through w.W
  cudaError_t e = cudaMemcpyAsync(w.W, M, sizeof(double) * (size_t)m * std::min(n, NB),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  // reflector copies are written from their diagonal down; clear the rest
  if ((e = cudaMemsetAsync(V32, 0, sizeof(float) * (size_t)(n * mp + m * ldv), s)) != cudaSuccess)
    return e;
  if (!x32_ready &&
      (e = gather_f32(M, X32, n, m, mp, im1(m), im1(1), s)) != cudaSuccess)
    return e;
  // S = V^T B over rows j0.. (K-chunk partials), then wy_prep
  auto vt_times = [&](const float* Vrows, int nbj, const float* Brows, int nrows, int mr,
                      int* ksplit) {
    TcGemm g{};
    g.A = TcOperand{Vrows, nbj, mr, mp, 1, 0};
    g.B = TcOperand{Brows, nrows, mr, mp, 1, 0};
    g.M = nbj; g.N = nrows; g.K = mr; g.batch = 1;
    g.c_b = im0();
    g.err = w.err;
    g.part = part; g.part_elems = part_elems;
    g.partials_only = true;
    g.ksplit_out = ksplit;
    g.max_ksplit = kQrMaxKsplit;
    return gemm_tc(g, s);
  };
  // panels with two columns per grid-wide exchange (FP32-class accuracy is
  // all the rest of this path keeps)
  QrWork wp = w;
  wp.pair_rounds = true;
  for (int p = 0; p < npan; ++p) {
    const int j0 = p * NB, nbj = std::min(NB, n - j0), mr = m - j0, n2 = n - j0 - nbj;
    double *G, *tau;
    if ((e = qr_panel_step(m, j0, nbj, wp, s, &G, &tau, X32, mp, Vt32, p == 0 ? nullptr : X32, V32,
                           ldv)) != cudaSuccess)
      return e;
    const float* Vrows = X32 + (long long)j0 * mp + j0;
    int ksplit = 1;
    if ((e = vt_times(Vrows, nbj, Vrows, n - j0, mr, &ksplit)) != cudaSuccess) return e;
    double* Tp = w.Tf + (size_t)p * NB * NB;
    const unsigned grid = (unsigned)std::max(1, (n2 + NB - 1) / NB);
    wy_prep_kernel<<<grid, kWyThreads, 0, s>>>(part, ksplit, nbj, n - j0, nbj, n2, tau, Tp, Yt32,
                                                0);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n2 > 0) {
      // FP32 trailing rows X[c][i] -= V Y2
      TcGemm g{};
      g.A = TcOperand{Vt32 + (long long)j0 * ldv + j0, mr, nbj, ldv, 1, 0};
      g.B = TcOperand{Yt32, n2, nbj, NB, 1, 0};
      g.M = mr; g.N = n2; g.K = nbj; g.batch = 1;
      g.C = X32 + (long long)(j0 + nbj) * mp + j0; g.c_fp64 = false;
      g.c_m = im1(1); g.c_n = im1(mp); g.c_b = im0();
      g.alpha = -1.0; g.beta = 1.0;
      g.err = w.err;
      if ((e = gemm_tc(g, s)) != cudaSuccess) return e;
    }
  }
  {
    const long long tot = (long long)n * n;
    extract_r_split_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w.W, X32, R, m, n, mp);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // Q = [I; 0] - V W with U W = V_top^T
  int ksplit = 1;
  if ((e = vt_times(V32, n, V32, n, m, &ksplit)) != cudaSuccess) return e;   // G = V^T V
  {
    const long long tot = (long long)n * n;
    build_ut_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, ksplit, n, w.Tf, UT, ldv);
    note_launch();
    const size_t qsm = sizeof(float) * (((n + 3) & ~3) + (n <= kSolveSmemMaxN ? (size_t)n * n : 0));
    // the fewest values per lane that hold a column (32 MAXQ >= n); U^T
    // staged in shared memory up to n = kSolveSmemMaxN
    // shared-memory limits are per-device attributes of the kernels
    device_once((const void*)q_solve_kernel<4, true>, [] {
      const int mx = (int)(sizeof(float) * (kSolveSmemMaxN * kSolveSmemMaxN + 32 * 8));
      cudaError_t r = cudaFuncSetAttribute(q_solve_kernel<4, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(q_solve_kernel<5, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(q_solve_kernel<8, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      return r;
    });
    const unsigned qg = (unsigned)((n + 7) / 8);
    const bool stg = n <= kSolveSmemMaxN;
    if (n <= 128 && stg)
      q_solve_kernel<4, true><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    else if (n <= 160 && stg)
      q_solve_kernel<5, true><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    else if (n <= 256 && stg)
      q_solve_kernel<8, true><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    else if (n <= 256)
      q_solve_kernel<8, false><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    else if (n <= 512)
      q_solve_kernel<16, false><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    else
      q_solve_kernel<32, false><<<qg, 256, qsm, s>>>(UT, ldv, Vt32, ldv, w.Tf, n, Wt);
    note_launch();
    init_q32_kernel<<<dim3((unsigned)std::min(((long long)m + 255) / 256, 64ll), (unsigned)n), 256,
                      0, s>>>(Q32, m, n, mp);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  TcGemm g{};
  g.A = TcOperand{Vt32, m, n, ldv, 1, 0};
  g.B = TcOperand{Wt, n, n, ldv, 1, 0};
  g.M = m; g.N = n; g.K = n; g.batch = 1;
  g.C = Q32; g.c_fp64 = false; g.c_m = im1(1); g.c_n = im1(mp); g.c_b = im0();
  g.alpha = -1.0; g.beta = 1.0;
  g.err = w.err;
  return gemm_tc(g, s);
}

}  // namespace qrctm
