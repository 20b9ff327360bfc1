// Environment set-up, symmetrisation/normalisation and the convergence test.
//
// * C4v projector of the iPEPS tensor (iPEPS paragraph).
// * Boundary initialisation from the bulk tensor (footnote of the Standard
//   CTMRG paragraph): ket and bra legs that point out of the system traced.
// * Reflection symmetrisation and FP64 Frobenius normalisation of C and T
//   after every step (a step the paper leaves implicit).
// * Corner spectrum |eig(C)| in FP64 for the convergence test ("repeated
//   until convergence"): Householder tridiagonalisation (one thread-block
//   cluster) followed by Sturm multisection, one CTA per eigenvalue (FP32
//   rounds narrow the bracket, FP64 rounds finish it).
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
  if (threadIdx.x < 32) {
    // the block's copy of the norm: lanes take every 32nd partial, then a
    // shuffle tree (a short dependent chain; the order is fixed)
    double s = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32) s += partials[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(s);
      if (!(nrm > 0.0) || isinf(nrm)) {
        if (blockIdx.x == 0) atomicOr(err, ERRF_NUMERIC);
        inv = 0.0;
      } else {
        inv = 1.0 / nrm;
      }
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

// I: index type (32-bit when chi D2 chi fits: 32-bit divisions)
template <typename I>
__global__ void sym_edge_kernel(const double* __restrict__ T, double* __restrict__ To, int chi,
                                int D2) {
  const I e = static_cast<I>(blockIdx.x) * blockDim.x + threadIdx.x;
  const I tot = static_cast<I>(chi) * D2 * chi;
  if (e >= tot) return;
  const I dc = static_cast<I>(D2) * chi;
  const I a = e / dc, r = e - a * dc;
  const I k = r / chi, b = r - k * chi;
  To[e] = 0.5 * (T[e] + T[(static_cast<long long>(b) * D2 + k) * chi + a]);
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
// Corner spectrum: Householder tridiagonalisation in one CTA of 1024 threads,
// eigenvalues by multisection on Sturm counts, then |lambda| sorted.
//
// Double precision runs on a narrow pipe on this part (a warp-wide FP64
// instruction costs tens of cycles of the SM), so every reduction folds the
// per-warp partials in warp 0 only, the rank-2 update touches the lower
// triangle only, and the Sturm recurrence tests signs and exponents with
// integer instructions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block (fixed order).  `red` holds 32 slots, `out` one.
__device__ double block_sum(double v, double* red, double* out) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s;
  }
  __syncthreads();
  return *out;
}

// Number of eigenvalues of the symmetric tridiagonal (dg, e2 = offdiag^2)
// below x: sign changes of the leading-minor sequence
//   p_0 = 1, p_1 = d_0 - x, p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2},
// i.e. negative pivots of T - x I (Sylvester's inertia).  No divisions: the
// pair (p_{i-1}, p_i) is rescaled by an exact power of two when the exponent
// of p_i leaves [-400, 400], tested every fourth step (four steps raise the
// exponent by at most 4 log2(3 ||T||): under 8 for the unit-norm corner), so
// that the dependent chain of a step is one FMA; an exact zero p_i is
// replaced by -pivmin p_{i-1}.
__device__ __forceinline__ void sturm_step(double dx, double me2, double& pc, double& pm,
                                           double pivmin, int& cnt) {
  double pn = fma(dx, pc, me2 * pm);
  if (((__double2hiint(pn) & 0x7fffffff) | __double2loint(pn)) == 0) pn = -pivmin * pc;
  cnt += ((__double2hiint(pn) ^ __double2hiint(pc)) < 0);
  pm = pc;
  pc = pn;
}

__device__ __forceinline__ void sturm_rescale(double& pc, double& pm) {
  const int ex = (int)((__double_as_longlong(pc) >> 52) & 0x7ff) - 1023;
  if (ex > 400) { pc *= 0x1p-400; pm *= 0x1p-400; }
  else if (ex < -400) { pc *= 0x1p400; pm *= 0x1p400; }
}

__device__ int sturm_count(const double* dg, const double* e2, int n, double x, double pivmin) {
  double pm = 1.0, pc = dg[0] - x;
  if ((__double_as_longlong(pc) << 1) == 0) pc = -pivmin;
  int cnt = (__double_as_longlong(pc) < 0);
  int i = 1;
  for (; i + 4 <= n; i += 4) {
    double dx[4], me2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      dx[u] = dg[i + u] - x;
      me2[u] = -e2[i + u - 1];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sturm_step(dx[u], me2[u], pc, pm, pivmin, cnt);
    sturm_rescale(pc, pm);
  }
  for (; i < n; ++i) {
    sturm_step(dg[i] - x, -e2[i - 1], pc, pm, pivmin, cnt);
    sturm_rescale(pc, pm);
  }
  return cnt;
}

// The matrix lives in shared memory when it fits (n <= kSmemSpecMax, leading
// dimension n + 1), else in `work` (leading dimension n).
constexpr int kSmemSpecMax = 160;

__global__ void __launch_bounds__(1024) spectrum_kernel(const double* __restrict__ C, int n,
                                                        double* work, int* err) {
  __shared__ double red[32];
  __shared__ double sc[4];
  extern __shared__ double spec_smem[];
  const bool in_smem = (n <= kSmemSpecMax);
  const long long ld = in_smem ? n + 1 : n;
  double* Am = in_smem ? spec_smem : work;   // lower triangle of (C + C^T)/2
  double* dg = work + (size_t)n * n; // n
  double* of = dg + n;               // n (off-diagonal)
  double* v = of + 2 * n;            // n (squared off-diagonal, after the loop)
  double* p = v + n;                 // lo, hi, pivmin
  __shared__ double sv[1024], sp[1024];   // Householder vector and A v during the loop
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wrp = tid >> 5;
  for (long long e = tid; e < (long long)n * n; e += nt) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (j <= i) Am[i * ld + j] = 0.5 * (C[e] + C[(long long)j * n + i]);
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    double* base = Am + (k + 1) * ld + (k + 1);          // A22[i][j] = base[i*ld + j], j <= i
    const double xi = (tid < L) ? Am[(k + 1 + tid) * ld + k] : 0.0;
    const double nrm2 = block_sum(xi * xi, red, &sc[3]);
    if (tid == 0) {
      const double x0 = Am[(k + 1) * ld + k];
      dg[k] = Am[k * ld + k];
      if (nrm2 == 0.0) {
        of[k] = 0.0;
        sc[1] = 0.0;
      } else {
        const double alpha = sqrt(nrm2);
        const double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
        sc[0] = x0 + sgn * alpha;                        // v_0 (v_i = x_i for i > 0)
        sc[1] = 1.0 / (alpha * (alpha + fabs(x0)));      // beta = 2 / ||v||^2
        of[k] = -sgn * alpha;
      }
    }
    __syncthreads();
    const double beta = sc[1];
    if (beta == 0.0) continue;                           // column already reduced
    if (tid < L) sv[tid] = (tid == 0) ? sc[0] : xi;
    __syncthreads();
    // p = beta A22 v from the lower triangle: row tid up to the diagonal,
    // then column tid below it
    double pt = 0.0;
    if (tid < L) {
      const double* row = base + tid * ld;
      double a0 = 0.0, a1 = 0.0;
      int j = 0;
      for (; j + 1 <= tid; j += 2) {
        a0 = fma(row[j], sv[j], a0);
        a1 = fma(row[j + 1], sv[j + 1], a1);
      }
      if (j <= tid) a0 = fma(row[j], sv[j], a0);
      j = tid + 1;
      for (; j + 1 < L; j += 2) {
        a0 = fma(base[j * ld + tid], sv[j], a0);
        a1 = fma(base[(j + 1) * ld + tid], sv[j + 1], a1);
      }
      if (j < L) a0 = fma(base[j * ld + tid], sv[j], a0);
      pt = beta * (a0 + a1);
      sp[tid] = pt;
    }
    const double pv = block_sum((tid < L) ? pt * sv[tid] : 0.0, red, &sc[3]);
    const double K = 0.5 * beta * pv;
    if (tid < L) sp[tid] = fma(-K, sv[tid], pt);          // w = p - K v
    __syncthreads();
    // A22 -= v w^T + w v^T on the lower triangle
    for (int i = wrp; i < L; i += (nt >> 5)) {
      const double vi = sv[i], wi = sp[i];
      double* row = base + i * ld;
      for (int j = lane; j <= i; j += 32) row[j] = fma(-vi, sp[j], fma(-wi, sv[j], row[j]));
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = Am[(n - 2) * ld + n - 2];
      of[n - 2] = Am[(n - 1) * ld + n - 2];
    }
    dg[n - 1] = Am[(n - 1) * ld + n - 1];
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
  if (lane == 0) { mn[wrp] = lo_l; mx[wrp] = hi_l; am[wrp] = amax; }
  __syncthreads();
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, big = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) { lo = fmin(lo, mn[w]); hi = fmax(hi, mx[w]); big = fmax(big, am[w]); }
    if (!(big == big) || isinf(big)) atomicOr(err, ERRF_NUMERIC);
    p[0] = lo - 1e-14 * fabs(lo) - 1e-300;
    p[1] = hi + 1e-14 * fabs(hi) + 1e-300;
    p[2] = fmax(1e-300, big * 1e-300);       // pivot floor of the Sturm recurrence
  }
}

// Cluster variant of the tridiagonalisation: CS CTAs (8, or 16 for larger
// chi) share the work.  CTA r of the cluster owns the rows i = r (mod CS) of the
// full symmetric matrix in its shared memory.  Per column k:
//   (a) owners publish x_i = A[i][k] (i > k); after a cluster barrier every
//       CTA gathers x over distributed shared memory and forms v, beta
//       redundantly (same data, same order, same result);
//   (b) owners publish p_i = beta (A v)_i and their partial v.p; after the
//       second barrier every CTA forms K = beta v.p / 2 and w = p - K v,
//       then updates its own rows, A -= v w^T + w v^T.
constexpr int kSpecClusterMaxN8 = 360;    // 8-CTA cluster (portable size)
constexpr int kSpecCluster16From = 97;    // 16 CTAs preferred from here (half the FP64 work per SM)
// 16-CTA cluster (non-portable size): ceil(n/16) rows of n doubles plus 4 n
// doubles per CTA fit the 227 KB of shared memory up to n = 640
constexpr int kSpecClusterMaxN16 = 640;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ double ld_dsmem(const double* local_addr, unsigned rank) {
  unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(local_addr)), ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

// GMEM: the rows of the symmetrised matrix stay in the work buffer (row i at
// work + i n, n^2 doubles; L2-resident) instead of shared memory, for n
// above what the CTAs' shared memory holds.  Each CTA touches only its own
// rows, so the choice changes no synchronisation.
// FP64 reductions priced for B300, which issues one FP64 instruction at a time
// per SM sub-partition: work is spread over the four sub-partitions (warps
// 0-3 of the block) and the trees are as shallow as the data allows.

// Sum over warps 0-3 (128 threads, fixed order); the result in thread 0.
// red: 4 slots.  Named barrier 1 among the four warps.
__device__ __forceinline__ double quad_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  asm volatile("bar.sync 1, 128;" ::: "memory");
  return (red[0] + red[1]) + (red[2] + red[3]);
}

// Four per-lane partial sums (rows 0..3) reduced across the warp at once:
// after the two exchange levels each lane carries one row (row 2 b4 + b3 of
// its lane bits), the last three levels finish it; 6 FP64 adds for four rows
// (5 per row one at a time).  Every lane returns the total of its row.
__device__ __forceinline__ double warp_sum4(double a0, double a1, double a2, double a3) {
  const int lane = threadIdx.x & 31;
  const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
  // level 16: keep rows {0,1} (lanes < 16) or {2,3}, send the other pair
  const double s0 = hi16 ? a0 : a2, s1 = hi16 ? a1 : a3;
  const double r0 = __shfl_xor_sync(0xffffffffu, s0, 16);
  const double r1 = __shfl_xor_sync(0xffffffffu, s1, 16);
  const double c0 = (hi16 ? a2 : a0) + r0, c1 = (hi16 ? a3 : a1) + r1;
  // level 8: keep one row of the pair
  const double r2 = __shfl_xor_sync(0xffffffffu, hi8 ? c0 : c1, 8);
  double v = (hi8 ? c1 : c0) + r2;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// njobs = 2: a second cluster reduces (C1, work1), same n, in the same launch.
template <int CS, bool GMEM>
__global__ void __launch_bounds__(256) spectrum_cluster_kernel(const double* __restrict__ C0, int n,
                                                               double* work0,
                                                               const double* __restrict__ C1,
                                                               double* work1, int njobs,
                                                               int* err) {
  extern __shared__ double csm[];
  __shared__ double red[32];
  __shared__ double sc[6];
  __shared__ double pvp[2];
  // the row distribution needs exactly CS CTAs per cluster, one cluster per job
  if (cluster_size() != (unsigned)CS || (njobs != 1 && njobs != 2) ||
      gridDim.x != (unsigned)(CS * njobs)) {
    if (threadIdx.x == 0) atomicOr(err, ERRF_BOUNDS);
    return;
  }
  const bool second = blockIdx.x >= (unsigned)CS;
  const double* __restrict__ C = second ? C1 : C0;
  double* work = second ? work1 : work0;
  const unsigned r = cluster_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wrp = tid >> 5;
  const int nloc = (n - (int)r + CS - 1) / CS;          // rows r, r + CS, ...
  const int nloc_max = (n + CS - 1) / CS;
  // own row li (global row r + li CS)
  auto rowp = [&](int li) -> double* {
    return GMEM ? work + (size_t)((int)r + li * CS) * n : csm + (size_t)li * n;
  };
  // published (read by the other CTAs), by column parity: p of own rows by
  // local index, and the pivot row (its owner's copy before the update)
  double* psb = GMEM ? csm : csm + (size_t)nloc_max * n;   // [2][nloc_max]
  double* rpb = psb + 2 * (size_t)nloc_max;                // [2][n]
  // local: x of the current column (turned into v in place) and of the next
  double* xb = rpb + 2 * (size_t)n;                        // [2][n]
  double* ww = xb + 2 * (size_t)n;                         // [n]  w
  double* qrow = ww + n;                                   // [nloc_max]  (A x) of own rows
  double* dg = work + (size_t)n * n;
  double* of = dg + n;
  double* v2 = of + 2 * n;
  double* pb = v2 + n;
  for (int e = tid; e < nloc * n; e += nt) {
    const int li = e / n, j = e % n, i = (int)r + li * CS;
    rowp(li)[j] = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
  }
  // x of column 0 (rows 1..n-1), in every CTA
  for (int t = tid; t + 1 < n; t += nt) xb[t] = 0.5 * (C[(size_t)(t + 1) * n] + C[t + 1]);
  if (tid == 0 && r == 0) dg[0] = C[0];
  __syncthreads();
  // Column k, with x = A[k+1.., k] already in every CTA: v and beta from x;
  // p = beta A v on own rows (published); the owner of row k + 1 publishes
  // that row; one cluster barrier; every CTA gathers p and the pivot row,
  // forms w = p - (beta p^T v / 2) v and, by symmetry, the next column
  // x' = A[k+2.., k+1] - v_{k+1} w - w_{k+1} v from the pivot row; own rows
  // take the rank-2 update.  Published buffers alternate with the column's
  // parity: a CTA overwrites a parity only after the next barrier, which
  // every CTA passes only after its reads of that parity.
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1, par = k & 1;
    double* vv = xb + (size_t)par * n;                     // x, then v
    double* xn = xb + (size_t)(par ^ 1) * n;               // next column's x
    // own rows i > k: first local row index with i > k
    const int li0 = (k + 1 - (int)r + CS - 1 < 0) ? 0 : (k + 1 - (int)r + CS - 1) / CS;
    // Warps 0-3 (one per SM sub-partition): ||x||^2, then the reflector
    // scalars in thread 0.  At the same time warps 5-7 (sub-partitions 1-3)
    // form q = A x on own rows i > k with the unmodified x: v differs from x
    // only in its first entry (v_0 = x_0 + sgn(x_0) alpha), so
    // A v = q + sgn(x_0) alpha A[., k+1].  Warp 4 of the pivot row's owner
    // publishes that row (entries k+1..n-1, before this column's update).
    double* psw = psb + (size_t)par * nloc_max;
    if (wrp < 4) {
      double sq = 0.0;
      for (int t = tid; t < L; t += 128) sq = fma(vv[t], vv[t], sq);
      const double nrm2 = quad_sum(sq, red);
      if (tid == 0) {
        const double x0 = vv[0];
        const int x0h = __double2hiint(x0), x0l = __double2loint(x0);
        if (((__double2hiint(nrm2) & 0x7fffffff) | __double2loint(nrm2)) == 0) {
          // x = 0: the reflector is the identity (beta = 0: p = w = 0)
          sc[0] = x0;
          sc[1] = 0.0;
          sc[2] = 0.0;
          sc[4] = 0.0;
          if (r == 0) of[k] = 0.0;
        } else {
          // Newton reciprocal square root and reciprocal from FP32 seeds: the
          // IEEE FP64 sqrt and divide are long chains on B300's FP64 pipe
          const double alpha = nrm2 * rsqrt_nr(nrm2);
          const double salpha =                          // sgn(x0) alpha
              __hiloint2double(__double2hiint(alpha) ^ (x0h & (int)0x80000000),
                               __double2loint(alpha));
          const double ax0 = __hiloint2double(x0h & 0x7fffffff, x0l);
          sc[0] = x0 + salpha;
          sc[4] = salpha;
          const double beta = rcp_nr(alpha * (alpha + ax0));
          sc[1] = beta;
          // beta / 2: exact, by the exponent, for a normal beta
          const int bh = __double2hiint(beta), be = (bh >> 20) & 0x7ff;
          sc[2] = (be > 1 && be < 0x7ff) ? __hiloint2double(bh - (1 << 20), __double2loint(beta))
                                         : 0.5 * beta;
          if (r == 0)
            of[k] = __hiloint2double(__double2hiint(salpha) ^ (int)0x80000000,
                                     __double2loint(salpha));
        }
      }
    } else if (wrp >= 5) {
      // rows li0 + g + 3 q (q < 4) per warp g = wrp - 5, then the next 12
      const int g = wrp - 5;
      for (int g0 = li0 + g; g0 < nloc; g0 += 12) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int li = g0 + 3 * q;
          if (li < nloc) {
            const double* row = rowp(li) + k + 1;
            double acc = 0.0;
            for (int t = lane; t < L; t += 32) acc = fma(row[t], vv[t], acc);
            a[q] = acc;
          }
        }
        const double tot = warp_sum4(a[0], a[1], a[2], a[3]);
        const int q = ((lane >> 4) << 1) | ((lane >> 3) & 1);   // row slot of this lane
        const int li = g0 + 3 * q;
        if ((lane & 7) == 0 && li < nloc) qrow[li] = tot;
      }
    } else if ((int)((k + 1) % CS) == (int)r) {
      const double* row = rowp((k + 1) / CS);
      double* rp = rpb + (size_t)par * n;
      for (int j = k + 1 + lane; j < n; j += 32) rp[j] = row[j];
    }
    __syncthreads();
    const double beta = sc[1];
    // p_i = beta (q_i + sgn(x_0) alpha A[i][k+1]) on own rows; the CTA's
    // share of p^T v (v_i = x_i below row k + 1, v_{k+1} = x_0 + sgn alpha)
    if (wrp == 0) {
      const double salpha = sc[4], v0 = sc[0];
      double pv = 0.0;
      for (int li = li0 + lane; li < nloc; li += 32) {
        const int i = (int)r + li * CS;
        const double pi = beta * fma(salpha, rowp(li)[k + 1], qrow[li]);
        psw[li] = pi;
        pv = fma(pi, (i == k + 1) ? v0 : vv[i - k - 1], pv);
      }
      pv = warp_sum(pv);
      if (lane == 0) {
        pvp[par] = pv;
        vv[0] = v0;
      }
    }
    cluster_sync_all();
    // gather: p (own entries of every CTA), the pivot row (one CTA), the p^T v parts
    const unsigned piv = (unsigned)((k + 1) % CS);
    const double* rpr = rpb + (size_t)par * n;
    double rowv[4], pvv[4];                          // entries k+1+t, t = tid + nt m
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int t = tid + nt * m;
      const int i = k + 1 + t;
      rowv[m] = (t < L) ? ld_dsmem(rpr + i, piv) : 0.0;
      pvv[m] = (t < L) ? ld_dsmem(psw + i / CS, (unsigned)(i % CS)) : 0.0;
    }
    double p0 = ld_dsmem(psw + (k + 1) / CS, piv);   // p_{k+1}, in every thread
    double pvs = (lane < CS) ? ld_dsmem(&pvp[par], (unsigned)lane) : 0.0;
#pragma unroll
    for (int o = CS / 2; o > 0; o >>= 1) pvs += __shfl_xor_sync(0xffffffffu, pvs, o);
    pvs = __shfl_sync(0xffffffffu, pvs, 0);          // lanes >= CS hold no part
    // K = beta p^T v / 2 (every warp has the same sum); w = p - K v; the next
    // column x'[t'] = A'[k+2+t', k+1] = a - v_{k+1} w_i - w_{k+1} v_i from the
    // pivot-row entry a, and the diagonal A'[k+1][k+1]
    const double K = sc[2] * pvs;
    const double v1 = vv[0], w1 = fma(-K, v1, p0);   // vv[0] = v0 since before the barrier
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int t = tid + nt * m;
      if (t < L) {
        const double wt = fma(-K, vv[t], pvv[m]);
        ww[t] = wt;
        const double a = fma(-v1, wt, fma(-w1, vv[t], rowv[m]));
        if (t == 0) {
          if (r == 0) dg[k + 1] = a;
        } else {
          xn[t - 1] = a;
        }
      }
    }
    for (int t = tid + nt * 4; t < L; t += nt) {      // n > 4 nt only (not reached: n <= 1024)
      const int i = k + 1 + t;
      const double wt = fma(-K, vv[t], ld_dsmem(psw + i / CS, (unsigned)(i % CS)));
      ww[t] = wt;
      xn[t - 1] = fma(-v1, wt, fma(-w1, vv[t], ld_dsmem(rpr + i, piv)));
    }
    __syncthreads();
    // own rows: A[i][j] -= v_i w_j + w_i v_j  (j > k)
    const int rows_left = nloc - li0;
    for (int e = tid; e < rows_left * L; e += nt) {
      const int li = li0 + e / L, t = e % L, i = (int)r + li * CS, ti = i - k - 1;
      double* a = rowp(li) + k + 1 + t;
      *a = fma(-vv[ti], ww[t], fma(-ww[ti], vv[t], *a));
    }
    __syncthreads();
  }
  // the last 2 x 2 block
  if (tid == 0) {
    for (int i = n - 2; i < n; ++i)
      if (i >= 0 && (i % CS) == (int)r) {
        const double* row = rowp(i / CS);
        dg[i] = row[i];
        if (i == n - 1 && n >= 2) of[n - 2] = row[n - 2];
      }
  }
  cluster_sync_all();
  if (r != 0) return;
  // squared off-diagonals, Gershgorin interval and pivot floor (CTA 0)
  double lo_l = 1e300, hi_l = -1e300, amax = 0.0;
  for (int i = tid; i < n; i += nt) {
    double rr = (i > 0 ? fabs(of[i - 1]) : 0.0) + (i + 1 < n ? fabs(of[i]) : 0.0);
    lo_l = fmin(lo_l, dg[i] - rr);
    hi_l = fmax(hi_l, dg[i] + rr);
    amax = fmax(amax, fmax(fabs(dg[i]), rr));
    if (i + 1 < n) v2[i] = of[i] * of[i];
  }
  __shared__ double mn[32], mx[32], am[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo_l = fmin(lo_l, __shfl_xor_sync(0xffffffffu, lo_l, o));
    hi_l = fmax(hi_l, __shfl_xor_sync(0xffffffffu, hi_l, o));
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  if (lane == 0) { mn[wrp] = lo_l; mx[wrp] = hi_l; am[wrp] = amax; }
  __syncthreads();
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, big = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) { lo = fmin(lo, mn[w]); hi = fmax(hi, mx[w]); big = fmax(big, am[w]); }
    if (!(big == big) || isinf(big)) atomicOr(err, ERRF_NUMERIC);
    pb[0] = lo - 1e-14 * fabs(lo) - 1e-300;
    pb[1] = hi + 1e-14 * fabs(hi) + 1e-300;
    pb[2] = fmax(1e-300, big * 1e-300);
  }
}

// Eigenvalues of the tridiagonal (dg, e^2) by multisection, one CTA of four
// warps per eigenvalue (one per SM sub-partition), down to the absolute
// resolution 4 eps max(|lo|, |hi|) of the Gershgorin interval (the accuracy
// a backward-stable method attains).
constexpr int kBisectMaxN = 1024;
constexpr int kBisectThreads = 128;

// Fast Sturm counts on T scaled by a power of two so that ||T|| <= 1
// (|d_i - x| <= 2, e2_i <= 1): the leading-minor recurrence of sturm_count
// with one FMA per step on the dependent chain.  Every four steps the pair
// (p_{i-1}, p_i) may be rescaled by a power of two; the decision comes from
// the value four steps older (four steps change the exponent by at most
// log2(3^4) < 7), and the factor is folded into the step's inputs: with
// q = S p, a new factor s at step k gives q_k = (s dx_k) q_{k-1} + (s me2_k)
// q_{k-2} and q_{k+1} = dx_{k+1} q_k + (s me2_{k+1}) q_{k-1}.  Sign changes
// and exact zeros are tested off the chain; a count that met an exact zero
// is flagged (the caller redoes it with the safe recurrence).  me2 = -e2.
template <typename F>
struct SturmLimits;
template <>
struct SturmLimits<double> {
  static constexpr int kBits = 11, kBias = 1023, kThr = 400;
  __device__ static double scale(int up) { return up ? 0x1p400 : 0x1p-400; }
  __device__ static int hi(double x) { return __double2hiint(x); }
  // on the 32-bit halves: a 64-bit shift test costs twice as much on B300
  __device__ static bool zero(double x) {
    return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) == 0;
  }
};
template <>
struct SturmLimits<float> {
  static constexpr int kBits = 8, kBias = 127, kThr = 60;
  __device__ static float scale(int up) { return up ? 0x1p60f : 0x1p-60f; }
  __device__ static int hi(float x) { return __float_as_int(x); }
  __device__ static bool zero(float x) { return (__float_as_int(x) << 1) == 0; }
};

template <typename F>
__device__ int sturm_count_fast(const F* dg, const F* me2, int n, F x, bool& hit_zero) {
  using L = SturmLimits<F>;
  constexpr int kShift = (L::kBits == 11) ? 20 : 23, kMask = (1 << L::kBits) - 1;
  F pm = F(1), pc = dg[0] - x;
  int cnt = L::hi(pc) < 0;
  bool z = L::zero(pc);
  int hi_old = L::hi(pc);
  int i = 1;
  for (; i + 4 <= n; i += 4) {
    F dx[4], m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      dx[u] = dg[i + u] - x;
      m[u] = me2[i + u - 1];
    }
    const int ex = ((hi_old >> kShift) & kMask) - L::kBias;
    hi_old = L::hi(pc);
    if (ex > L::kThr || ex < -L::kThr) {
      const F sc = L::scale(ex < 0);
      dx[0] *= sc;
      m[0] *= sc;
      m[1] *= sc;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const F pn = fma(dx[u], pc, m[u] * pm);
      z |= L::zero(pn);
      cnt += (L::hi(pn) ^ L::hi(pc)) < 0;
      pm = pc;
      pc = pn;
    }
  }
  for (; i < n; ++i) {
    const F pn = fma(dg[i] - x, pc, me2[i - 1] * pm);
    z |= L::zero(pn);
    cnt += (L::hi(pn) ^ L::hi(pc)) < 0;
    pm = pc;
    pc = pn;
  }
  hit_zero = z;
  return cnt;
}

// One CTA per eigenvalue i (ascending order).  Multisection: the points
// a + h (t + 1), t < np, split [a, b] into np + 1 parts per round; the first
// point whose count exceeds i bounds eigenvalue i from above.  The counts run
// on T scaled by 2^-k >= 1/||T||_Gershgorin (exact).  The bracket is first
// narrowed in FP32 (128 points, ~7 bits per round) to a few FP32 ulps of
// ||T||, widened by a margin covering the FP32 counts' error, checked by two
// FP64 counts (the Gershgorin interval is used instead if the check fails),
// and refined in FP64 (128 points, 7 bits per round) down to 4e-16 ||T||.
// blockIdx.y = 1: the second job (work1, ev1), same n.
__global__ void __launch_bounds__(kBisectThreads) bisect_kernel(const double* work0, int n,
                                                                double* ev0,
                                                                const double* work1,
                                                                double* ev1) {
  const double* work = blockIdx.y ? work1 : work0;
  double* ev_out = blockIdx.y ? ev1 : ev0;
  __shared__ double sdg[kBisectMaxN], se2[kBisectMaxN], ndg[kBisectMaxN], nme2[kBisectMaxN];
  __shared__ float fdg[kBisectMaxN], fme2[kBisectMaxN];
  __shared__ unsigned masks[kBisectThreads / 32];
  __shared__ int s_cnt[2];
  const double* dg = work + (size_t)n * n;
  const double* v = dg + 3 * (size_t)n;       // e^2
  const double* p = v + n;                    // lo, hi, pivmin
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  const int i = blockIdx.x;
  const double lo = p[0], hi = p[1];
  const double pivmin = p[2];
  const double tn = fmax(fabs(lo), fabs(hi));
  // exact power-of-two scale with ||T|| <= sc (Gershgorin)
  const double sc = (tn > 0.0) ? exp2(ceil(log2(tn))) : 1.0;
  const double isc = 1.0 / sc;
  for (int t = tid; t < n; t += kBisectThreads) {
    sdg[t] = dg[t];
    se2[t] = (t + 1 < n) ? v[t] : 0.0;
    ndg[t] = sdg[t] * isc;
    nme2[t] = -se2[t] * (isc * isc);
    fdg[t] = static_cast<float>(ndg[t]);
    fme2[t] = static_cast<float>(nme2[t]);
  }
  __syncthreads();
  const double res = 4e-16 * tn;
  // exact count of eigenvalues below x (FP64, scaled; the safe recurrence
  // after an exact zero)
  auto count64 = [&](double x) {
    bool zero;
    int c = sturm_count_fast<double>(ndg, nme2, n, x * isc, zero);
    if (zero) c = sturm_count(sdg, se2, n, x, pivmin);
    return c;
  };
  // ---- FP32 phase ----
  constexpr int NPT = kBisectThreads;
  double a = lo, b = hi;
  {
    const double res32 = 64.0 * 1.1920928955078125e-07 * tn;
    for (int round = 0; round < 8 && b - a > res32; ++round) {
      const double h = (b - a) * (1.0 / (NPT + 1));
      const double xd = a + h * (tid + 1);
      bool zero;
      int c = sturm_count_fast<float>(fdg, fme2, n, static_cast<float>(xd * isc), zero);
      if (zero) c = count64(xd);
      const unsigned mask = __ballot_sync(0xffffffffu, c > i);
      if (lane == 0) masks[wrp] = mask;
      __syncthreads();
      int first = NPT;
#pragma unroll
      for (int w = NPT / 32 - 1; w >= 0; --w)
        if (masks[w]) first = w * 32 + __ffs(masks[w]) - 1;
      __syncthreads();
      const double na = (first == 0) ? a : a + h * first;
      const double nb = (first == NPT) ? b : a + h * (first + 1);
      if (!(nb < b || na > a)) break;
      a = na;
      b = nb;
    }
    // margin for the FP32 counts (and the rounding of x to FP32)
    const double mg = 16.0 * 1.1920928955078125e-07 * tn;
    a = fmax(lo, a - mg);
    b = fmin(hi, b + mg);
  }
  // ---- FP64 phase: 128 points per round (one warp per SMSP: B300 runs one
  // FP64 instruction per sub-partition at a time, so a round costs one
  // warp's recurrence whatever the number of warps).  The first round also
  // counts at a and b (threads 0 and NPT - 1 take the endpoints): if the
  // FP32 bracket does not hold eigenvalue i, it restarts from [lo, hi]. ----
  bool checked = false;
  for (int round = 0; round < 80; ++round) {
    const bool chk = !checked;
    if (!chk && b - a <= res) break;
    const double h = (b - a) * (1.0 / (NPT + 1));
    // evaluation points, increasing in t
    auto point = [&](int t) {
      return chk ? (t == 0 ? a : (t == NPT - 1 ? b : a + h * (t + 1))) : a + h * (t + 1);
    };
    const double x = point(tid);
    bool above;
    if (chk) {
      const int c = count64(x);
      above = c > i;
      if (tid == 0) s_cnt[0] = c;
      if (tid == NPT - 1) s_cnt[1] = c;
    } else {
      above = (x > a && x < b) ? (count64(x) > i) : (x >= b);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    if (lane == 0) masks[wrp] = mask;
    __syncthreads();
    if (chk) {
      checked = true;
      const bool ok = s_cnt[0] <= i && s_cnt[1] > i;
      __syncthreads();
      if (!ok) {                             // the bracket is wrong: restart
        a = lo;
        b = hi;
        continue;
      }
    }
    int first = NPT;
#pragma unroll
    for (int w = NPT / 32 - 1; w >= 0; --w)
      if (masks[w]) first = w * 32 + __ffs(masks[w]) - 1;
    __syncthreads();                          // masks are rewritten next round
    double na, nb;
    if (chk) {                                // 1 <= first <= NPT - 1 here
      na = point(first - 1);
      nb = point(first);
    } else {
      na = (first == 0) ? a : a + h * first;
      nb = (first == NPT) ? b : a + h * (first + 1);
    }
    if (!(nb < b || na > a)) break;          // no progress: bracket at resolution
    a = na;
    b = nb;
  }
  if (tid == 0) ev_out[i] = 0.5 * (a + b);
}

// sorted |lambda| (descending, ties by index) and the change to the previous.
// Non-negative doubles order like their bit patterns, so the ranking compares
// integers.
__global__ void spectrum_finish_kernel(const double* ev, int n, double* s_new, const double* s_old,
                                       int n_old, double* delta) {
  __shared__ double red[32], out;
  __shared__ long long key[kBisectMaxN];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) key[i] = __double_as_longlong(fabs(ev[i]));
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const long long ki = key[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const long long kj = key[j];
      rank += (kj > ki) || (kj == ki && j < i);
    }
    s_new[rank] = __longlong_as_double(ki);
  }
  __syncthreads();
  const int nm = n > n_old ? n : n_old;
  double acc = 0.0;
  for (int i = tid; i < nm; i += nt) {
    double x = (i < n) ? s_new[i] : 0.0;
    double y = (s_old != nullptr && i < n_old) ? s_old[i] : 0.0;
    acc += (x - y) * (x - y);
  }
  double tot = block_sum(acc, red, &out);
  if (tid == 0) if (delta) *delta = sqrt(tot);
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// I: the flat index type (32-bit whenever nrows * ncols fits, so that the
// row/column split and the index maps use 32-bit divisions).
template <typename I>
__device__ __forceinline__ long long map_off_i(const IdxMap& m, I i) {
  if (sizeof(I) == 4) return map_off32(m, static_cast<unsigned>(i));
  return map_off(m, static_cast<long long>(i));
}

template <bool SPLIT, typename I>
__global__ void gather_f32_k(const double* __restrict__ in, float* __restrict__ out,
                             float* __restrict__ lo, long long nrows, int ncols,
                             long long stride, const __grid_constant__ IdxMap rmap,
                             const __grid_constant__ IdxMap cmap) {
  const I tot = static_cast<I>(nrows * ncols), nc = static_cast<I>(ncols);
  for (I e = static_cast<I>(blockIdx.x) * blockDim.x + threadIdx.x; e < tot;
       e += static_cast<I>(gridDim.x) * blockDim.x) {
    const I r = e / nc, c = e - r * nc;
    const float x = static_cast<float>(in[map_off_i(rmap, r) + map_off_i(cmap, c)]);
    const long long o = static_cast<long long>(r) * stride + static_cast<long long>(c);
    if (SPLIT) tf32_split(x, out[o], lo[o]);
    else out[o] = x;
  }
}

template <bool SPLIT, typename I>
__global__ void gather_f32f_k(const float* __restrict__ in, float* __restrict__ out,
                              float* __restrict__ lo, long long nrows, int ncols,
                              long long stride, const __grid_constant__ IdxMap rmap,
                              const __grid_constant__ IdxMap cmap) {
  const I tot = static_cast<I>(nrows * ncols), nc = static_cast<I>(ncols);
  for (I e = static_cast<I>(blockIdx.x) * blockDim.x + threadIdx.x; e < tot;
       e += static_cast<I>(gridDim.x) * blockDim.x) {
    const I r = e / nc, c = e - r * nc;
    const float x = in[map_off_i(rmap, r) + map_off_i(cmap, c)];
    const long long o = static_cast<long long>(r) * stride + static_cast<long long>(c);
    if (SPLIT) tf32_split(x, out[o], lo[o]);
    else out[o] = x;
  }
}

__global__ void split_f32_k(float* __restrict__ x, float* __restrict__ lo, unsigned nrows,
                            unsigned ncols, unsigned long long stride) {
  const unsigned tot = nrows * ncols;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const unsigned r = e / ncols, c = e - r * ncols;
    const unsigned long long o = r * stride + c;
    float h, t;
    tf32_split(x[o], h, t);
    x[o] = h;
    lo[o] = t;
  }
}

}  // namespace

cudaError_t gather_f32f(const float* in, float* out, long long nrows, int ncols, long long stride,
                        IdxMap rmap, IdxMap cmap, cudaStream_t s, float* lo) {
  const long long tot = nrows * ncols;
  if (tot <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<long long>((tot + 255) / 256, 8192);
  const bool i32 = tot < (1ll << 32) - 2ll * 8192 * 256;
  if (lo && i32)
    gather_f32f_k<true, unsigned><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else if (lo)
    gather_f32f_k<true, long long><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else if (i32)
    gather_f32f_k<false, unsigned><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else
    gather_f32f_k<false, long long><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap,
                                                      cmap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gather_f32(const double* in, float* out, long long nrows, int ncols, long long stride,
                       IdxMap rmap, IdxMap cmap, cudaStream_t s, float* lo) {
  const long long tot = nrows * ncols;
  if (tot <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<long long>((tot + 255) / 256, 8192);
  const bool i32 = tot < (1ll << 32) - 2ll * 8192 * 256;
  if (lo && i32)
    gather_f32_k<true, unsigned><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else if (lo)
    gather_f32_k<true, long long><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else if (i32)
    gather_f32_k<false, unsigned><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap, cmap);
  else
    gather_f32_k<false, long long><<<g, 256, 0, s>>>(in, out, lo, nrows, ncols, stride, rmap,
                                                     cmap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t split_f32(float* x, float* lo, long long nrows, int ncols, long long stride,
                      cudaStream_t s) {
  const long long tot = nrows * ncols;
  if (tot <= 0) return cudaSuccess;
  if (tot >= (1ll << 32)) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)std::min<long long>((tot + 255) / 256, 8192);
  split_f32_k<<<g, 256, 0, s>>>(x, lo, (unsigned)nrows, (unsigned)ncols,
                                (unsigned long long)stride);
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
  if (nb > 296) nb = 296;   // 2 x 148 SMs, grid-stride: each block reduces the partials once
  if (nb < 1) nb = 1;
  scale_kernel<<<(unsigned)nb, 256, 0, s>>>(x, y, n, partials, nparts, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sym_edge(const double* Tin, double* Tout, int chi, int D2, cudaStream_t s) {
  long long n = (long long)chi * D2 * chi;
  if (n < (1ll << 32) - 256)
    sym_edge_kernel<unsigned><<<nblk(n), 256, 0, s>>>(Tin, Tout, chi, D2);
  else
    sym_edge_kernel<long long><<<nblk(n), 256, 0, s>>>(Tin, Tout, chi, D2);
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
  if (nT < (1ll << 32) - 256)
    sym_edge_kernel<unsigned><<<nblk(nT), 256, 0, s>>>(Tin, Tout, chi, D2);
  else
    sym_edge_kernel<long long><<<nblk(nT), 256, 0, s>>>(Tin, Tout, chi, D2);
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
// Tridiagonalisation, multisection and ranking of one corner (C1 == nullptr)
// or of two of the same size: with C1 the two clusters and the two sets of
// bisection CTAs share launches; s_new0 gets |eig(C0)| (no change measured),
// s_new gets |eig(C1)| and delta its change to s_new0.
static cudaError_t spectra(const double* C, int chi, double* work, double* s_new0,
                           const double* C1, double* work1, double* s_new,
                           const double* s_old, int chi_old, double* delta, int* err,
                           cudaStream_t s) {
  if (chi < 1 || chi > 1024) return cudaErrorInvalidValue;
  const int njobs = C1 ? 2 : 1;
  const size_t smem = (chi <= kSmemSpecMax) ? sizeof(double) * chi * (chi + 1) : 0;
  // one-time setup per device: shared-memory limits of the one-CTA and
  // cluster variants for their largest n, and whether the device can place a
  // 16-CTA cluster (its result is kept as the second key's status)
  device_once((const void*)spectrum_kernel, [] {
    cudaError_t r = cudaFuncSetAttribute(
        spectrum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(sizeof(double) * kSmemSpecMax * (kSmemSpecMax + 1)));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(spectrum_cluster_kernel<8, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(double) * (((size_t)kSpecClusterMaxN8 + 7) / 8 *
                                                           (kSpecClusterMaxN8 + 3) +
                                                       5 * (size_t)kSpecClusterMaxN8)));
    return r;
  });
  const bool ok16 =
      device_once((const void*)spectrum_cluster_kernel<16, false>, [] {
        auto k16 = spectrum_cluster_kernel<16, false>;
        const size_t smem16 = sizeof(double) * (((size_t)kSpecClusterMaxN16 + 15) / 16 *
                                                    (kSpecClusterMaxN16 + 3) +
                                                5 * (size_t)kSpecClusterMaxN16);
        cudaFuncSetAttribute(k16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16);
        // 16 CTAs per cluster is above the portable limit: allowed only where
        // the device can place such a cluster
        bool ok = cudaFuncSetAttribute(k16, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                      cudaSuccess &&
                  cudaFuncSetAttribute(spectrum_cluster_kernel<16, true>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                      cudaSuccess;
        if (ok) {
          cudaLaunchConfig_t q = {};
          q.gridDim = dim3(16);
          q.blockDim = dim3(256);
          q.dynamicSmemBytes = smem16;
          cudaLaunchAttribute qa[1];
          qa[0].id = cudaLaunchAttributeClusterDimension;
          qa[0].val.clusterDim.x = 16;
          qa[0].val.clusterDim.y = 1;
          qa[0].val.clusterDim.z = 1;
          q.attrs = qa;
          q.numAttrs = 1;
          int nclusters = 0;
          ok = cudaOccupancyMaxActiveClusters(&nclusters, k16, &q) == cudaSuccess &&
               nclusters >= 1;
        }
        cudaGetLastError();
        return ok ? cudaSuccess : cudaErrorNotSupported;
      }) == cudaSuccess;
  bool launched = false;
  int cs = 0;
  bool gmem = false;
  if (chi >= 3) {
    if (ok16 && chi >= kSpecCluster16From && chi <= kSpecClusterMaxN16) cs = 16;
    else if (chi <= kSpecClusterMaxN8) cs = 8;
    else if (ok16) { cs = 16; gmem = true; }   // rows in the work buffer
  }
  if (cs != 0) {
    auto kern = gmem ? spectrum_cluster_kernel<16, true>
                     : (cs == 8) ? spectrum_cluster_kernel<8, false>
                                 : spectrum_cluster_kernel<16, false>;
    const int nloc_max = (chi + cs - 1) / cs;
    const size_t csmem = sizeof(double) * ((gmem ? 0 : (size_t)nloc_max * chi) +
                                           3 * (size_t)nloc_max + 5 * (size_t)chi);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * njobs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = csmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, C, chi, work, C1 ? C1 : C, C1 ? work1 : work,
                                       njobs, err);
    if (e != cudaSuccess) return e;
    launched = true;
  }
  if (!launched) {
    spectrum_kernel<<<1, 1024, smem, s>>>(C, chi, work, err);
    if (C1) {
      note_launch();
      spectrum_kernel<<<1, 1024, smem, s>>>(C1, chi, work1, err);
    }
  }
  note_launch();
  double* ev = work + (size_t)chi * chi + 5 * (size_t)chi + 8;
  double* ev1 = C1 ? work1 + (size_t)chi * chi + 5 * (size_t)chi + 8 : ev;
  bisect_kernel<<<dim3(chi, njobs), kBisectThreads, 0, s>>>(work, chi, ev, C1 ? work1 : work, ev1);
  note_launch();
  if (C1) {
    spectrum_finish_kernel<<<1, 256, 0, s>>>(ev, chi, s_new0, nullptr, 0, nullptr);
    note_launch();
    spectrum_finish_kernel<<<1, 256, 0, s>>>(ev1, chi, s_new, s_new0, chi, delta);
  } else {
    spectrum_finish_kernel<<<1, 256, 0, s>>>(ev, chi, s_new, s_old, chi_old, delta);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t corner_spectrum(const double* C, int chi, double* work, double* s_new,
                            const double* s_old, int chi_old, double* delta, int* err,
                            cudaStream_t s) {
  return spectra(C, chi, work, nullptr, nullptr, nullptr, s_new, s_old, chi_old, delta, err, s);
}

cudaError_t corner_spectrum_pair(const double* C0, int chi0, double* work0, double* s0,
                                 const double* C1, int chi1, double* work1, double* s1,
                                 double* delta, int* err, cudaStream_t s) {
  if (chi0 == chi1)
    return spectra(C0, chi0, work0, s0, C1, work1, s1, nullptr, 0, delta, err, s);
  cudaError_t e = spectra(C0, chi0, work0, nullptr, nullptr, nullptr, s0, nullptr, 0, nullptr,
                          err, s);
  if (e != cudaSuccess) return e;
  return spectra(C1, chi1, work1, nullptr, nullptr, nullptr, s1, s0, chi0, delta, err, s);
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
