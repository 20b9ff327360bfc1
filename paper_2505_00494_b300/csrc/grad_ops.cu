// Building blocks of the hand-written adjoint (Automatic differentiation
// paragraph; fixed-point differentiation named in the Discussion).
//
// * gemm_vjp: the two cotangent contractions of a forward contraction (each
//   cotangent stored like its primal: FP64, or FP32 where the descriptor
//   says so)
//     D[b](m,n) = alpha sum_k A[b](m,k) B[b](k,n)
//   Abar[b](m,k) (+)= alpha sum_n Dbar[b](m,n) B[b](k,n),
//   Bbar[b](k,n) (+)= alpha sum_m A[b](m,k) Dbar[b](m,n),
//   addressed through the same index maps as the forward.  An operand shared
//   by every batch entry (zero batch stride) gets its cotangent summed over
//   the batch by folding the batch digit into the contraction index.
// * QR adjoint for M = Q R (m >= n, diag R > 0):
//     S = copyutl(Rbar R^T - Q^T Qbar)  (upper triangle mirrored downwards)
//     Mbar = (Qbar + Q S) R^{-T}
//   (differentiate Q^T Q = I and the triangularity of R: dQ = Q Omega +
//   (I - Q Q^T) dM R^{-1} with Omega antisymmetric; its strictly lower part is
//   that of Q^T dM R^{-1}).
// * normalisation y = x / ||x||:  xbar = (ybar - y <y, ybar>) / ||x||.
// * reflection symmetrisation: self-adjoint, its adjoint is itself.
#include "grad.cuh"

namespace qrctm {

namespace {

bool zero_map(const IdxMap& m) {
  for (int t = 0; t < m.nd; ++t)
    if (m.str[t] != 0) return false;
  return true;
}

}  // namespace

IdxMap concat_map(const IdxMap& x, long long xrange, const IdxMap& y) {
  IdxMap r = x;
  long long prod = 1;
  for (int t = 0; t < x.nd - 1; ++t) prod *= x.rad[t];
  r.rad[x.nd - 1] = (int)(xrange / prod);
  for (int t = 0; t < y.nd; ++t) {
    r.rad[x.nd + t] = y.rad[t];
    r.str[x.nd + t] = y.str[t];
  }
  r.nd = x.nd + y.nd;
  return r;
}

cudaError_t gemm_vjp(qrctm_ctx* c, const Gemm& f, const double* Dbar, double* Abar, double* Bbar,
                     bool accA, bool accB) {
  cudaError_t e;
  if (Abar) {
    Gemm g = gemm_ctx(c);
    if (f.batch > 1 && zero_map(f.a_b)) {
      if (f.c_n.nd + f.c_b.nd > kMaxDigits || f.b_n.nd + f.b_b.nd > kMaxDigits)
        return cudaErrorInvalidValue;
      g.M = f.M; g.N = f.K; g.K = f.N * f.batch; g.batch = 1;
      g.A = Dbar; g.a_m = f.c_m; g.a_k = concat_map(f.c_n, f.N, f.c_b);
      g.B = f.B; g.b_k = concat_map(f.b_n, f.N, f.b_b); g.b_n = f.b_k;
      g.C = Abar; g.c_m = f.a_m; g.c_n = f.a_k;
    } else {
      g.M = f.M; g.N = f.K; g.K = f.N; g.batch = f.batch;
      g.A = Dbar; g.a_m = f.c_m; g.a_k = f.c_n; g.a_b = f.c_b;
      g.B = f.B; g.b_k = f.b_n; g.b_n = f.b_k; g.b_b = f.b_b;
      g.C = Abar; g.c_m = f.a_m; g.c_n = f.a_k; g.c_b = f.a_b;
    }
    // Dbar is stored like D, Abar like A
    g.a_f32 = f.c_f32; g.b_f32 = f.b_f32; g.c_f32 = f.a_f32;
    g.alpha = f.alpha;
    g.beta = accA ? 1.0 : 0.0;
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  if (Bbar) {
    Gemm g = gemm_ctx(c);
    if (f.batch > 1 && zero_map(f.b_b)) {
      if (f.a_m.nd + f.a_b.nd > kMaxDigits || f.c_m.nd + f.c_b.nd > kMaxDigits)
        return cudaErrorInvalidValue;
      g.M = f.K; g.N = f.N; g.K = f.M * f.batch; g.batch = 1;
      g.A = f.A; g.a_m = f.a_k; g.a_k = concat_map(f.a_m, f.M, f.a_b);
      g.B = Dbar; g.b_k = concat_map(f.c_m, f.M, f.c_b); g.b_n = f.c_n;
      g.C = Bbar; g.c_m = f.b_k; g.c_n = f.b_n;
    } else {
      g.M = f.K; g.N = f.N; g.K = f.M; g.batch = f.batch;
      g.A = f.A; g.a_m = f.a_k; g.a_k = f.a_m; g.a_b = f.a_b;
      g.B = Dbar; g.b_k = f.c_m; g.b_n = f.c_n; g.b_b = f.c_b;
      g.C = Bbar; g.c_m = f.b_k; g.c_n = f.b_n; g.c_b = f.b_b;
    }
    // Bbar is stored like B
    g.a_f32 = f.a_f32; g.b_f32 = f.c_f32; g.c_f32 = f.b_f32;
    g.alpha = f.alpha;
    g.beta = accB ? 1.0 : 0.0;
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

// X = R^{-1} for upper-triangular R (n x n, row-major): one warp per column
// j, back substitution X[i][j] = -(sum_{l=i+1..j} R[i][l] X[l][j]) / R[i][i].
__global__ void triu_inverse_k(const double* __restrict__ R, double* __restrict__ X, int n,
                               int* err) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  for (int i = lane; i < n; i += 32) X[(long long)i * n + j] = 0.0;
  __syncwarp();
  const double rjj = R[(long long)j * n + j];
  if (!(rjj != 0.0) && lane == 0) atomicOr(err, ERRF_NUMERIC);
  if (lane == 0) X[(long long)j * n + j] = 1.0 / rjj;
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    double s = 0.0;
    for (int l = i + 1 + lane; l <= j; l += 32) s = fma(R[(long long)i * n + l], X[(long long)l * n + j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) X[(long long)i * n + j] = -s / R[(long long)i * n + i];
    __syncwarp();
  }
}

// The same inverse for n <= kTriuSmemMaxN: the block's part of R (rows and
// columns up to its last column) is staged column-major in shared memory with
// the reciprocals of its diagonal, and each warp solves R x = e_j by columns:
// x_l = -p_l / R[l][l] for l = j, j-1, ..., 0, then p_i += R[i][l] x_l for
// every i < l, lanes over i.  A step costs one FP64 instruction per 32 rows
// and no reduction, where the row form above waits on global loads and a
// shuffle tree at every step.
constexpr int kTriuSmemMaxN = 160, kTriuNT = (kTriuSmemMaxN + 31) / 32;

__global__ void triu_inverse_smem_k(const double* __restrict__ R, double* __restrict__ X, int n,
                                    int* err) {
  extern __shared__ double tri_sm[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * warps, jmax = min(n - 1, j0 + warps - 1), ld = jmax + 1;
  double* sRt = tri_sm;               // [l][i] = R[i][l], i <= l <= jmax
  double* invd = tri_sm + ld * ld;    // 1 / R[l][l]
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    const int i = e / ld, l = e - i * ld;
    if (l >= i) sRt[l * ld + i] = R[(long long)i * n + l];
  }
  for (int l = threadIdx.x; l < ld; l += blockDim.x) {
    const double r = R[(long long)l * n + l];
    if (!(r != 0.0)) atomicOr(err, ERRF_NUMERIC);
    invd[l] = 1.0 / r;
  }
  __syncthreads();
  const int j = j0 + warp;
  if (j >= n) return;
  for (int i = j + 1 + lane; i < n; i += 32) X[(long long)i * n + j] = 0.0;
  double p[kTriuNT];
#pragma unroll
  for (int t = 0; t < kTriuNT; ++t) p[t] = 0.0;
  for (int l = j; l >= 0; --l) {
    const int slot = l >> 5;
    double own = 0.0;
#pragma unroll
    for (int t = 0; t < kTriuNT; ++t)
      if (t == slot) own = p[t];
    const double xv = (l == j) ? invd[j] : -own * invd[l];
    const double xl = __shfl_sync(0xffffffffu, xv, l & 31);
    if (lane == 0) X[(long long)l * n + j] = xl;
#pragma unroll
    for (int t = 0; t < kTriuNT; ++t) {
      if (32 * t < l) {
        const int i = lane + 32 * t;
        if (i < l) p[t] = fma(sRt[l * ld + i], xl, p[t]);
      }
    }
  }
}

// S[i][j] = M[i][j] (i <= j), M[j][i] (i > j)
__global__ void copyutl_k(const double* __restrict__ M, double* __restrict__ S, int n) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  S[e] = (i <= j) ? M[e] : M[(long long)j * n + i];
}

// partial dot products of (x, y) per block (fixed order)
__global__ void dot_partials_k(const double* __restrict__ x, const double* __restrict__ y,
                               long long n, double* partials) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// xbar = (ybar - y <y,ybar>) / nrm, with <y,ybar> and nrm^2 from partial sums
__global__ void norm_vjp_k(const double* __restrict__ y, const double* __restrict__ ybar,
                           double* __restrict__ xbar, long long n, const double* dot_parts,
                           const double* nrm_parts, int nparts, bool acc) {
  __shared__ double sdot, sinv;
  if (threadIdx.x < 32) {
    // one warp, the same fixed order in every block
    double d = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) {
      d += dot_parts[i];
      q += nrm_parts[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (threadIdx.x == 0) {
      sdot = d;
      sinv = 1.0 / sqrt(q);
    }
  }
  __syncthreads();
  const double dt = sdot, inv = sinv;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (ybar[i] - y[i] * dt) * inv;
    xbar[i] = acc ? xbar[i] + v : v;
  }
}

__global__ void sym_corner_acc_k(const double* __restrict__ X, double* __restrict__ Y, int chi,
                                 bool acc) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)chi * chi) return;
  const int i = (int)(e / chi), j = (int)(e % chi);
  const double v = 0.5 * (X[e] + X[(long long)j * chi + i]);
  Y[e] = acc ? Y[e] + v : v;
}

inline unsigned nb256(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 8192); }

}  // namespace

cudaError_t dot_partials(const double* x, const double* y, long long n, double* partials,
                         int nparts, cudaStream_t s) {
  dot_partials_k<<<nparts, 256, 0, s>>>(x, y, n, partials);
  note_launch();
  return cudaGetLastError();
}

cudaError_t triu_inverse(const double* R, double* X, int n, int* err, cudaStream_t s) {
  if (n <= kTriuSmemMaxN) {
    const size_t smem = sizeof(double) * ((size_t)n * n + n);
    cudaError_t e = device_once((const void*)triu_inverse_smem_k, [] {
      return cudaFuncSetAttribute(
          triu_inverse_smem_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
          (int)(sizeof(double) * (kTriuSmemMaxN * kTriuSmemMaxN + kTriuSmemMaxN)));
    });
    if (e != cudaSuccess) return e;
    triu_inverse_smem_k<<<(n + 3) / 4, 128, smem, s>>>(R, X, n, err);
  } else {
    triu_inverse_k<<<(n + 3) / 4, 128, 0, s>>>(R, X, n, err);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t sym_corner_vjp(const double* X, double* Y, int chi, bool acc, cudaStream_t s) {
  sym_corner_acc_k<<<nb256((long long)chi * chi), 256, 0, s>>>(X, Y, chi, acc);
  note_launch();
  return cudaGetLastError();
}

// xbar (+)= (ybar - y <y,ybar>) / ||x||, where ||x||^2 is given by nrm_parts.
cudaError_t norm_vjp(const double* y, const double* ybar, double* xbar, long long n,
                     const double* nrm_parts, int nparts, double* scratch, bool acc,
                     cudaStream_t s) {
  dot_partials_k<<<256, 256, 0, s>>>(y, ybar, n, scratch);
  note_launch();
  norm_vjp_k<<<nb256(n), 256, 0, s>>>(y, ybar, xbar, n, scratch, nrm_parts, nparts, acc);
  note_launch();
  return cudaGetLastError();
}

// Mbar = (Qbar + Q copyutl(Rbar R^T - Q^T Qbar)) R^{-T}
// Q column-major m x n; Qbar column-major m x n; R, Rbar, Rinv row-major n x n.
cudaError_t qr_vjp(qrctm_ctx* c, int m, int n, const double* Q, const double* R,
                   const double* Rinv, const double* Qbar, const double* Rbar, double* Mbar,
                   double* Ms, double* Ss, double* Bs) {
  cudaError_t e;
  cudaStream_t s = c->st;
  {
    // Ms = Rbar R^T
    Gemm g = gemm_ctx(c);
    g.M = n; g.N = n; g.K = n;
    g.A = Rbar; g.a_m = im1(n); g.a_k = im1(1);
    g.B = R; g.b_k = im1(1); g.b_n = im1(n);
    g.C = Ms; g.c_m = im1(n); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    // Ms -= Q^T Qbar (on the TF32x3 engine in a split context: Q has
    // orthonormal columns, so this product adds no more than the rounding
    // its operands already carry)
    g = gemm_ctx(c);
    g.M = n; g.N = n; g.K = m;
    g.A = Q; g.a_m = im1(m); g.a_k = im1(1);
    g.B = Qbar; g.b_k = im1(1); g.b_n = im1(m);
    g.C = Ms; g.c_m = im1(n); g.c_n = im1(1);
    g.alpha = -1.0; g.beta = 1.0;
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  copyutl_k<<<nb256((long long)n * n), 256, 0, s>>>(Ms, Ss, n);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Bs = Qbar + Q Ss   (column-major m x n; TF32x3 in a split context, as
  // above; the product with R^{-T} below stays FP64, where the conditioning
  // of R would amplify rounding)
  if ((e = cudaMemcpyAsync(Bs, Qbar, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess)
    return e;
  {
    Gemm g = gemm_ctx(c);
    g.M = m; g.N = n; g.K = n;
    g.A = Q; g.a_m = im1(1); g.a_k = im1(m);
    g.B = Ss; g.b_k = im1(n); g.b_n = im1(1);
    g.C = Bs; g.c_m = im1(1); g.c_n = im1(m);
    g.beta = 1.0;
    if ((e = gemm_run(c, g)) != cudaSuccess) return e;
  }
  // Mbar[i][j] = sum_l Bs[i][l] Rinv[j][l]   (column-major m x n)
  {
    Gemm g = gemm_ctx(c);
    g.M = m; g.N = n; g.K = n;
    g.A = Bs; g.a_m = im1(1); g.a_k = im1(m);
    g.B = Rinv; g.b_k = im1(1); g.b_n = im1(n);
    g.C = Mbar; g.c_m = im1(1); g.c_n = im1(m);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qrctm
