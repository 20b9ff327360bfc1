// Environment set-up, symmetrisation/normalisation and the convergence test.
//
// * C4v projector of the iPEPS tensor (iPEPS paragraph).
// * Boundary initialisation from the bulk tensor (footnote of the Standard
//   CTMRG paragraph): ket and bra legs that point out of the system traced.
// * Reflection symmetrisation and FP64 Frobenius normalisation of C and T
//   after every step (a step the paper leaves implicit).
// * Corner spectrum |eig(C)| in FP64 for the convergence test ("repeated
//   until convergence"): Householder tridiagonalisation followed by Sturm
//   bisection, one CTA.
#include "qrctm_internal.cuh"

#include <algorithm>

namespace qrctm {

namespace {

__constant__ int c_perm[8][4] = {
    {0, 1, 2, 3}, {1, 2, 3, 0}, {2, 3, 0, 1}, {3, 0, 1, 2},
    {0, 3, 2, 1}, {1, 0, 3, 2}, {2, 1, 0, 3}, {3, 2, 1, 0},
};

__global__ void c4v_sym_kernel(int d, int D, const double* __restrict__ X, double* __restrict__ Y) {
  const long long D4 = (long long)D * D * D * D;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * D4) return;
  const long long s = e / D4;
  long long r = e % D4;
  int v[4];
  for (int k = 3; k >= 0; --k) { v[k] = (int)(r % D); r /= D; }
  double acc = 0.0;
  for (int g = 0; g < 8; ++g) {
    int w[4];
    for (int k = 0; k < 4; ++k) w[c_perm[g][k]] = v[k];
    acc += X[s * D4 + (((long long)w[0] * D + w[1]) * D + w[2]) * D + w[3]];
  }
  Y[e] = acc * 0.125;
}

__global__ void sumsq_kernel(const double* __restrict__ x, long long n, double* partials) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(x[i], x[i], acc);
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

__global__ void scale_kernel(const double* __restrict__ x, double* __restrict__ y, long long n,
                             const double* __restrict__ partials, int nparts, int* err) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += partials[q];
    double nrm = sqrt(s);
    if (!(nrm > 0.0) || isinf(nrm)) {
      if (blockIdx.x == 0) atomicOr(err, ERRF_NUMERIC);
      inv = 0.0;
    } else {
      inv = 1.0 / nrm;
    }
  }
  __syncthreads();
  const double f = inv;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

__global__ void sym_corner_kernel(const double* __restrict__ C, double* __restrict__ Co, int chi) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)chi * chi) return;
  int i = (int)(e / chi), j = (int)(e % chi);
  Co[e] = 0.5 * (C[e] + C[(long long)j * chi + i]);
}

__global__ void sym_edge_kernel(const double* __restrict__ T, double* __restrict__ To, int chi,
                                int D2) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)chi * D2 * chi;
  if (e >= tot) return;
  long long a = e / ((long long)D2 * chi);
  long long r = e % ((long long)D2 * chi);
  long long k = r / chi, b = r % chi;
  To[e] = 0.5 * (T[e] + T[(b * D2 + k) * chi + a]);
}

// C0[(d d'),(r r')] = sum_{s,u,l} A[s,u,l,d,r] A[s,u,l,d',r']
// T0[(u u'),(r r'),(d d')] = sum_{s,l} A[s,u,l,d,r] A[s,u',l,d',r']
__global__ void init_env_k(int d, int D, const double* __restrict__ A, double* __restrict__ C0,
                           double* __restrict__ T0) {
  const long long D2 = (long long)D * D, D4 = D2 * D2;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  auto Aat = [&](int s, int u, int l, int dd, int r) {
    return A[(((((long long)s * D + u) * D + l) * D + dd) * D) + r];
  };
  if (e < D4) {
    int rp = (int)(e % D), r = (int)((e / D) % D), dp = (int)((e / D2) % D), dd = (int)(e / (D2 * D));
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int u = 0; u < D; ++u)
        for (int l = 0; l < D; ++l) acc = fma(Aat(s, u, l, dd, r), Aat(s, u, l, dp, rp), acc);
    C0[e] = acc;
  }
  const long long D6 = D4 * D2;
  if (e < D6) {
    // e = ((u D + u') D2 + (r D + r')) D2 + (d D + d')
    long long t = e;
    int dp = (int)(t % D); t /= D;
    int dd = (int)(t % D); t /= D;
    int rp = (int)(t % D); t /= D;
    int r = (int)(t % D); t /= D;
    int up = (int)(t % D); t /= D;
    int u = (int)t;
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int l = 0; l < D; ++l) acc = fma(Aat(s, u, l, dd, r), Aat(s, up, l, dp, rp), acc);
    T0[e] = acc;
  }
}

// a[(u u'),(l l'),(d d'),(r r')] = sum_s A[s,u,l,d,r] A[s,u',l',d',r']
__global__ void double_layer_k(int d, int D, const double* __restrict__ A, double* __restrict__ a) {
  const long long D4 = (long long)D * D * D * D;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D4 * D4) return;
  long long t = e;
  int rp = (int)(t % D); t /= D;
  int r = (int)(t % D); t /= D;
  int dp = (int)(t % D); t /= D;
  int dd = (int)(t % D); t /= D;
  int lp = (int)(t % D); t /= D;
  int l = (int)(t % D); t /= D;
  int up = (int)(t % D); t /= D;
  int u = (int)t;
  const long long ket = (((long long)u * D + l) * D + dd) * D + r;
  const long long bra = (((long long)up * D + lp) * D + dp) * D + rp;
  double acc = 0.0;
  for (int s = 0; s < d; ++s) acc = fma(A[s * D4 + ket], A[s * D4 + bra], acc);
  a[e] = acc;
}

__global__ void fill_zero_k(double* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

__global__ void axpby_k(double* y, const double* x, double a, double b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// ---------------------------------------------------------------------------
// Corner spectrum: one CTA of 1024 threads.
// work: chi*chi (matrix) + 5*chi doubles.
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Number of eigenvalues of the symmetric tridiagonal (dg, e2 = offdiag^2)
// below x: sign changes of the leading-minor sequence
//   p_0 = 1, p_1 = d_0 - x, p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2},
// i.e. negative pivots of T - x I (Sylvester's inertia).  No divisions: the
// pair (p_{i-1}, p_i) is rescaled by an exact power of two when it leaves
// [2^-400, 2^400]; an exact zero p_i is replaced by -pivmin * p_{i-1}.
__device__ int sturm_count(const double* dg, const double* e2, int n, double x, double pivmin) {
  int cnt = 0;
  double pm = 1.0, pc = dg[0] - x;
  if (pc == 0.0) pc = -pivmin;
  cnt += (pc < 0.0);
  for (int i = 1; i < n; ++i) {
    double pn = fma(dg[i] - x, pc, -e2[i - 1] * pm);
    if (pn == 0.0) pn = -pivmin * pc;
    cnt += ((pn < 0.0) != (pc < 0.0));
    pm = pc;
    pc = pn;
    const double a = fabs(pc);
    if (a > 0x1p400) { pc *= 0x1p-400; pm *= 0x1p-400; }
    else if (a < 0x1p-400) { pc *= 0x1p400; pm *= 0x1p400; }
  }
  return cnt;
}

// Householder tridiagonalisation of (C + C^T)/2.  The matrix lives in shared
// memory when it fits (n <= kSmemSpecMax), else in `work`.
constexpr int kSmemSpecMax = 160;

__global__ void __launch_bounds__(1024) spectrum_kernel(const double* __restrict__ C, int n,
                                                        double* work, double* s_new,
                                                        const double* s_old, int n_old,
                                                        double* delta, int* err) {
  __shared__ double red[32];
  __shared__ double sc[2];
  extern __shared__ double spec_smem[];
  double* Am = (n <= kSmemSpecMax) ? spec_smem : work;   // n x n
  double* dg = work + (size_t)n * n; // n
  double* of = dg + n;               // n (off-diagonal)
  double* ev = of + n;               // n
  double* v = ev + n;                // n (squared off-diagonal, after the loop)
  double* p = v + n;                 // n (bracket, after the loop)
  __shared__ double sv[1024], sp[1024];   // Householder vector and A v during the loop
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long e = tid; e < (long long)n * n; e += nt) {
    int i = (int)(e / n), j = (int)(e % n);
    Am[e] = 0.5 * (C[e] + C[(long long)j * n + i]);
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    double xi = (tid < L) ? Am[(long long)(k + 1 + tid) * n + k] : 0.0;
    double nrm2 = block_sum(xi * xi, red);
    if (tid == 0) {
      double x0 = Am[(long long)(k + 1) * n + k];
      double alpha = sqrt(nrm2);
      double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
      sc[0] = x0 + sgn * alpha;         // v_0 (v_i = x_i for i > 0)
      of[k] = -sgn * alpha;
      dg[k] = Am[(long long)k * n + k];
    }
    __syncthreads();
    if (nrm2 == 0.0) {
      if (tid == 0) of[k] = 0.0;
      __syncthreads();
      continue;
    }
    if (tid < L) sv[tid] = (tid == 0) ? sc[0] : xi;
    __syncthreads();
    double vv = block_sum((tid < L) ? sv[tid] * sv[tid] : 0.0, red);
    const double beta = 2.0 / vv;
    // p = beta * A22 v  (A22 symmetric: read columns; four independent sums)
    if (tid < L) {
      const double* col = Am + (long long)(k + 1) * n + k + 1 + tid;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = 0;
      for (; j + 4 <= L; j += 4) {
        a0 = fma(col[(long long)j * n], sv[j], a0);
        a1 = fma(col[(long long)(j + 1) * n], sv[j + 1], a1);
        a2 = fma(col[(long long)(j + 2) * n], sv[j + 2], a2);
        a3 = fma(col[(long long)(j + 3) * n], sv[j + 3], a3);
      }
      for (; j < L; ++j) a0 = fma(col[(long long)j * n], sv[j], a0);
      sp[tid] = beta * ((a0 + a1) + (a2 + a3));
    }
    __syncthreads();
    double pv = block_sum((tid < L) ? sp[tid] * sv[tid] : 0.0, red);
    const double K = 0.5 * beta * pv;
    if (tid < L) sp[tid] = sp[tid] - K * sv[tid];      // w
    __syncthreads();
    for (int i = tid >> 5; i < L; i += nt >> 5) {
      const double vi = sv[i], pi = sp[i];
      double* row = Am + (long long)(k + 1 + i) * n + k + 1;
      for (int j = tid & 31; j < L; j += 32) row[j] -= vi * sp[j] + pi * sv[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = Am[(long long)(n - 2) * n + n - 2];
      of[n - 2] = Am[(long long)(n - 1) * n + n - 2];
    }
    dg[n - 1] = Am[(long long)(n - 1) * n + n - 1];
  }
  __syncthreads();
  // squared off-diagonals into v, Gershgorin interval into p[0..2]
  double lo_l = 1e300, hi_l = -1e300, amax = 0.0;
  for (int i = tid; i < n; i += nt) {
    double r = (i > 0 ? fabs(of[i - 1]) : 0.0) + (i + 1 < n ? fabs(of[i]) : 0.0);
    lo_l = fmin(lo_l, dg[i] - r);
    hi_l = fmax(hi_l, dg[i] + r);
    amax = fmax(amax, fmax(fabs(dg[i]), r));
    if (i + 1 < n) v[i] = of[i] * of[i];
  }
  __shared__ double mn[32], mx[32], am[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo_l = fmin(lo_l, __shfl_xor_sync(0xffffffffu, lo_l, o));
    hi_l = fmax(hi_l, __shfl_xor_sync(0xffffffffu, hi_l, o));
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  if ((tid & 31) == 0) { mn[tid >> 5] = lo_l; mx[tid >> 5] = hi_l; am[tid >> 5] = amax; }
  __syncthreads();
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, big = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) { lo = fmin(lo, mn[w]); hi = fmax(hi, mx[w]); big = fmax(big, am[w]); }
    if (!(big == big) || isinf(big)) atomicOr(err, ERRF_NUMERIC);
    p[0] = lo - 1e-14 * fabs(lo) - 1e-300;
    p[1] = hi + 1e-14 * fabs(hi) + 1e-300;
    p[2] = fmax(1e-300, big * 1e-300);       // pivot floor of the Sturm recurrence
  }
  (void)s_new; (void)s_old; (void)n_old; (void)delta;
}

// Eigenvalue i of the tridiagonal (dg, e^2) by multisection: one warp per
// eigenvalue, the 32 lanes evaluate Sturm counts at 32 interior points of the
// current bracket, which shrinks 33-fold per round until it stops shrinking.
__global__ void bisect_kernel(const double* work, int n, double* ev_out) {
  const double* dg = work + (size_t)n * n;
  const double* v = dg + 3 * (size_t)n;       // e^2
  const double* p = v + n;                    // lo, hi, pivmin
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double a = p[0], b = p[1];
  const double pivmin = p[2];
  for (int round = 0; round < 64; ++round) {
    const double h = (b - a) / 33.0;
    const double x = a + h * (lane + 1);
    const bool above = (x > a && x < b) ? (sturm_count(dg, v, n, x, pivmin) > i) : (x >= b);
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    // first lane whose point lies above eigenvalue i bounds it from above
    const int first = mask ? __ffs(mask) - 1 : 32;
    const double na = (first == 0) ? a : a + h * first;
    const double nb = (first == 32) ? b : a + h * (first + 1);
    if (!(nb < b || na > a)) break;          // no progress: bracket at resolution
    a = na;
    b = nb;
    if (b - a <= 4e-16 * fmax(fabs(a), fabs(b))) break;
  }
  if (lane == 0) ev_out[i] = 0.5 * (a + b);
}

// sorted |lambda| (descending, ties by index) and the change to the previous
__global__ void spectrum_finish_kernel(const double* ev, int n, double* s_new, const double* s_old,
                                       int n_old, double* delta) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) {
    double ai = fabs(ev[i]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double aj = fabs(ev[j]);
      rank += (aj > ai) || (aj == ai && j < i);
    }
    s_new[rank] = ai;
  }
  __syncthreads();
  const int nm = n > n_old ? n : n_old;
  double acc = 0.0;
  for (int i = tid; i < nm; i += nt) {
    double x = (i < n) ? s_new[i] : 0.0;
    double y = (s_old != nullptr && i < n_old) ? s_old[i] : 0.0;
    acc += (x - y) * (x - y);
  }
  double tot = block_sum(acc, red);
  if (tid == 0) *delta = sqrt(tot);
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__global__ void gather_f32_k(const double* __restrict__ in, float* __restrict__ out,
                             long long nrows, int ncols, long long stride, IdxMap rmap,
                             IdxMap cmap) {
  const long long tot = nrows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ncols, c = e % ncols;
    out[r * stride + c] = static_cast<float>(in[map_off(rmap, r) + map_off(cmap, c)]);
  }
}

}  // namespace

cudaError_t gather_f32(const double* in, float* out, long long nrows, int ncols, long long stride,
                       IdxMap rmap, IdxMap cmap, cudaStream_t s) {
  const long long tot = nrows * ncols;
  if (tot <= 0) return cudaSuccess;
  gather_f32_k<<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, s>>>(
      in, out, nrows, ncols, stride, rmap, cmap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t c4v_symmetrize(int d, int D, const double* X, double* Y, cudaStream_t s) {
  long long n = (long long)d * D * D * D * D;
  c4v_sym_kernel<<<nblk(n), 256, 0, s>>>(d, D, X, Y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sum_squares_partials(const double* x, long long n, double* partials, int nparts,
                                 cudaStream_t s) {
  sumsq_kernel<<<nparts, 256, 0, s>>>(x, n, partials);
  note_launch();
  return cudaGetLastError();
}

cudaError_t scale_by_inv_norm(const double* x, double* y, long long n, const double* partials,
                              int nparts, int* err, cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 1184) nb = 1184;
  if (nb < 1) nb = 1;
  scale_kernel<<<(unsigned)nb, 256, 0, s>>>(x, y, n, partials, nparts, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sym_edge(const double* Tin, double* Tout, int chi, int D2, cudaStream_t s) {
  long long n = (long long)chi * D2 * chi;
  sym_edge_kernel<<<nblk(n), 256, 0, s>>>(Tin, Tout, chi, D2);
  note_launch();
  return cudaGetLastError();
}

// partials must hold 2 * 256 doubles
cudaError_t sym_norm_env(const double* Cin, const double* Tin, double* Cout, double* Tout,
                         int chi, int D2, double* partials, int* err, cudaStream_t s) {
  const int NP = 256;
  long long nC = (long long)chi * chi, nT = (long long)chi * D2 * chi;
  sym_corner_kernel<<<nblk(nC), 256, 0, s>>>(Cin, Cout, chi);
  note_launch();
  sym_edge_kernel<<<nblk(nT), 256, 0, s>>>(Tin, Tout, chi, D2);
  note_launch();
  sumsq_kernel<<<NP, 256, 0, s>>>(Cout, nC, partials);
  note_launch();
  sumsq_kernel<<<NP, 256, 0, s>>>(Tout, nT, partials + NP);
  note_launch();
  cudaError_t e = scale_by_inv_norm(Cout, Cout, nC, partials, NP, err, s);
  if (e != cudaSuccess) return e;
  return scale_by_inv_norm(Tout, Tout, nT, partials + NP, NP, err, s);
}

cudaError_t init_env_kernel(int d, int D, const double* A, double* C0, double* T0,
                            cudaStream_t s) {
  long long n = (long long)D * D * D * D * D * D;
  init_env_k<<<nblk(n), 256, 0, s>>>(d, D, A, C0, T0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t double_layer_kernel(int d, int D, const double* A, double* a, cudaStream_t s) {
  long long n = (long long)D * D * D * D;
  n = n * n;
  double_layer_k<<<nblk(n), 256, 0, s>>>(d, D, A, a);
  note_launch();
  return cudaGetLastError();
}

// work: chi*chi + 8*chi + 16 doubles: matrix, diagonal, off-diagonal, (unused),
// squared off-diagonal, Gershgorin bracket + pivot floor, eigenvalues
cudaError_t corner_spectrum(const double* C, int chi, double* work, double* s_new,
                            const double* s_old, int chi_old, double* delta, int* err,
                            cudaStream_t s) {
  if (chi < 1 || chi > 1024) return cudaErrorInvalidValue;
  const size_t smem = (chi <= kSmemSpecMax) ? sizeof(double) * chi * chi : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(spectrum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(double) * kSmemSpecMax * kSmemSpecMax));
    attr = true;
  }
  spectrum_kernel<<<1, 1024, smem, s>>>(C, chi, work, s_new, s_old, chi_old, delta, err);
  note_launch();
  double* ev = work + (size_t)chi * chi + 5 * (size_t)chi + 8;
  bisect_kernel<<<(chi + 3) / 4, 128, 0, s>>>(work, chi, ev);
  note_launch();
  spectrum_finish_kernel<<<1, 256, 0, s>>>(ev, chi, s_new, s_old, chi_old, delta);
  note_launch();
  return cudaGetLastError();
}

cudaError_t fill_zero(double* p, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  fill_zero_k<<<(unsigned)nb, 256, 0, s>>>(p, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  axpby_k<<<(unsigned)nb, 256, 0, s>>>(y, x, a, b, n);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
