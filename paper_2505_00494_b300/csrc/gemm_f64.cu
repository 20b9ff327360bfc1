// FP64 CUDA-core contraction engine (any layout, through mixed-radix maps).
//
// Used by the plain FP64 path of every contraction in the QR-CTMRG step
// (QR-CTMRG paragraph, Fig. 1(e,f)), by the compact-WY updates of the
// Householder QR and by the reduced density matrices.  On B300 the FP64 pipe
// is narrow, so the kernel is arithmetic bound: a 64x64x16 shared-memory
// tile with a 4x4 register block per thread is enough to keep it busy.
#include "qrctm_internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>

namespace qrctm {

namespace {

constexpr int BM = 64, BK = 16, NT = 256;

// Element off of an operand stored as FP64, or as FP32 when f32 (the
// descriptor's storage flags; uniform over a launch).
__device__ __forceinline__ double ld_op(const double* p, bool f32, long long off) {
  return f32 ? static_cast<double>(reinterpret_cast<const float*>(p)[off]) : p[off];
}

// C[off] = v + beta C[off] in the result's storage type.
__device__ __forceinline__ void st_c(const Gemm& g, long long off, double v) {
  if (g.c_f32) {
    float* q = reinterpret_cast<float*>(g.C) + off;
    if (g.beta != 0.0) v += g.beta * static_cast<double>(*q);
    *q = static_cast<float>(v);
  } else {
    double* q = g.C + off;
    if (g.beta != 0.0) v += g.beta * *q;
    *q = v;
  }
}

// splits > 1 (batch == 1 only): CTA z handles K range [z*kc, (z+1)*kc) and
// writes its raw sums to g.part[z][M][N].  BN = 64 (4 x 4 per thread) or 48
// (4 x 3: for N a multiple of 48, such as chi = 144, no column of a tile idles).
template <int BN>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(Gemm g, int splits, long long kc) {
  constexpr int TN = BN / 16;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ long long aRow[BM], bCol[BN], aK[BK], bK[BK];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * BM;
  const long long ntiles_n = (g.N + BN - 1) / BN;
  for (long long ny = blockIdx.y; ny < ntiles_n; ny += gridDim.y) {
  const long long n0 = ny * BN;
  const long long kbeg = (splits > 1) ? (long long)blockIdx.z * kc : 0;
  const long long kend = (splits > 1) ? min(g.K, kbeg + kc) : g.K;
  for (long long b = (splits > 1) ? 0 : blockIdx.z; b < g.batch;
       b += (splits > 1) ? g.batch : gridDim.z) {
    const long long aB = map_off(g.a_b, b), bB = map_off(g.b_b, b), cB = map_off(g.c_b, b);
    __syncthreads();
    if (tid < BM) {
      long long m = m0 + tid;
      aRow[tid] = (m < g.M) ? map_off(g.a_m, m) : -1;
    } else if (tid < BM + BN) {
      long long n = n0 + tid - BM;
      bCol[tid - BM] = (n < g.N) ? map_off(g.b_n, n) : -1;
    }
    double acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

    for (long long k0 = kbeg; k0 < kend; k0 += BK) {
      if (tid < BK) {
        long long k = k0 + tid;
        aK[tid] = (k < kend) ? map_off(g.a_k, k) : -1;
      } else if (tid < 2 * BK) {
        long long k = k0 + tid - BK;
        bK[tid - BK] = (k < kend) ? map_off(g.b_k, k) : -1;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < (BM * BK) / NT; ++q) {
        int e = tid + NT * q;
        int r = e % BM, kk = e / BM;
        long long ro = aRow[r], ko = aK[kk];
        As[kk][r] = (ro >= 0 && ko >= 0) ? ld_op(g.A, g.a_f32, aB + ro + ko) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < (BN * BK) / NT; ++q) {
        int e = tid + NT * q;
        int c = e % BN, kk = e / BN;
        long long co = bCol[c], ko = bK[kk];
        Bs[kk][c] = (co >= 0 && ko >= 0) ? ld_op(g.B, g.b_f32, bB + co + ko) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double av[4], bv[TN];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (splits > 1) {
      double* P = g.part + (long long)blockIdx.z * g.M * g.N;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        long long m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          long long n = n0 + tx + 16 * j;
          if (n < g.N) P[m * g.N + n] = acc[i][j];
        }
      }
      continue;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
      long long ro = map_off(g.c_m, m);
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        long long n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        st_c(g, cB + ro + map_off(g.c_n, n), g.alpha * acc[i][j]);
      }
    }
  }
  }
}

// C(m,n) = alpha * sum_z part[z][m][n] + beta * C(m,n); a fixed summation
// order (four interleaved partial sums) keeps the result deterministic.
__global__ void splitk_reduce_kernel(Gemm g, int splits) {
  const long long MN = g.M * g.N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
       e += (long long)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int z = 0;
    for (; z + 4 <= splits; z += 4) {
      s0 += g.part[(long long)z * MN + e];
      s1 += g.part[(long long)(z + 1) * MN + e];
      s2 += g.part[(long long)(z + 2) * MN + e];
      s3 += g.part[(long long)(z + 3) * MN + e];
    }
    for (; z < splits; ++z) s0 += g.part[(long long)z * MN + e];
    const double s = (s0 + s1) + (s2 + s3);
    const long long m = e / g.N, n = e % g.N;
    st_c(g, map_off(g.c_m, m) + map_off(g.c_n, n), g.alpha * s);
  }
}

}  // namespace

cudaError_t device_once(const void* key, const std::function<cudaError_t()>& f) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({dev, key});
  if (it != done.end()) return it->second;
  e = f();
  done.emplace(std::make_pair(dev, key), e);
  return e;
}

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> count;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  std::lock_guard<std::mutex> lock(mu);
  auto it = count.find(dev);
  if (it != count.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 148;
  count[dev] = n;
  return n;
}

// Tiny outputs (M, N <= kThinMax, one batch entry, long K: a reduced density
// matrix or its trace partner over the whole environment): the tile kernel
// would compute a 64 x 48 tile for at most 16 useful entries.  Here each
// thread accumulates all M x N entries over a grid-stride range of k (the m
// and n offsets formed once), the block sums its threads in a fixed order
// into part[block][M N], and one more block adds the blocks' sums in block
// order and applies alpha, beta and the output maps.
constexpr int kThinMax = 4, kThinThreads = 256;

__global__ void __launch_bounds__(kThinThreads)
    gemm_f64_thin_k(const __grid_constant__ Gemm g, double* __restrict__ part) {
  __shared__ double red[kThinThreads / 32][kThinMax * kThinMax];
  const int M = (int)g.M, N = (int)g.N;
  long long am[kThinMax], bn[kThinMax];
#pragma unroll
  for (int i = 0; i < kThinMax; ++i) {
    am[i] = i < M ? map_off(g.a_m, i) : 0;
    bn[i] = i < N ? map_off(g.b_n, i) : 0;
  }
  double acc[kThinMax][kThinMax];
#pragma unroll
  for (int i = 0; i < kThinMax; ++i)
#pragma unroll
    for (int j = 0; j < kThinMax; ++j) acc[i][j] = 0.0;
  const bool k32 = g.K <= (long long)UINT32_MAX;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < g.K;
       k += (long long)gridDim.x * blockDim.x) {
    const long long ak = k32 ? map_off32(g.a_k, (unsigned)k) : map_off(g.a_k, k);
    const long long bk = k32 ? map_off32(g.b_k, (unsigned)k) : map_off(g.b_k, k);
    double a[kThinMax], b[kThinMax];
#pragma unroll
    for (int i = 0; i < kThinMax; ++i) {
      a[i] = i < M ? ld_op(g.A, g.a_f32, am[i] + ak) : 0.0;
      b[i] = i < N ? ld_op(g.B, g.b_f32, bk + bn[i]) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kThinMax; ++i)
#pragma unroll
      for (int j = 0; j < kThinMax; ++j)
        if (i < M && j < N) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kThinMax; ++i)
#pragma unroll
    for (int j = 0; j < kThinMax; ++j) {
      double v = acc[i][j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i * kThinMax + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < kThinMax * kThinMax) {
    double v = 0.0;
    for (int w = 0; w < kThinThreads / 32; ++w) v += red[w][threadIdx.x];
    part[(long long)blockIdx.x * kThinMax * kThinMax + threadIdx.x] = v;
  }
}

__global__ void gemm_f64_thin_finish_k(const __grid_constant__ Gemm g, const double* part,
                                       int blocks) {
  const int t = threadIdx.x, i = t / kThinMax, j = t % kThinMax;
  if (i >= g.M || j >= g.N) return;
  double v = 0.0;
  for (int b = 0; b < blocks; ++b) v += part[(long long)b * kThinMax * kThinMax + t];
  st_c(g, map_off(g.c_m, i) + map_off(g.c_n, j), g.alpha * v);
}

static unsigned long long g_launches = 0;
void note_launch(unsigned long long n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
unsigned long long launches_so_far() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

template <int BN>
cudaError_t gemm_f64_launch(const Gemm& g, cudaStream_t s) {
  long long gx = (g.M + BM - 1) / BM, gy = (g.N + BN - 1) / BN;
  if (gx > 0x7fffffffll) return cudaErrorInvalidValue;
  if (gy > 65535) gy = 65535;   // the kernel loops over the remaining N tiles
  const int nsm = device_sm_count();
  const long long tiles = gx * gy;
  int splits = 1;
  if (g.part != nullptr && g.batch == 1 && tiles < 2 * nsm && g.K >= 4 * BK) {
    long long want = (4ll * nsm + tiles - 1) / tiles;          // ~4 CTAs per SM
    long long by_k = g.K / (4 * BK);                           // >= 4 k-tiles per split
    long long by_mem = g.part_elems / (g.M * g.N);
    long long sp = std::min(std::min(want, by_k), std::min(by_mem, 65535ll));
    if (sp > 1) splits = (int)sp;
  }
  if (splits > 1) {
    long long kc = (g.K + splits - 1) / splits;
    kc = (kc + BK - 1) / BK * BK;
    splits = (int)((g.K + kc - 1) / kc);
    gemm_f64_kernel<BN><<<dim3((unsigned)gx, (unsigned)gy, splits), NT, 0, s>>>(g, splits, kc);
    note_launch();
    long long MN = g.M * g.N;
    long long nb = std::min<long long>((MN + 255) / 256, 4096);
    splitk_reduce_kernel<<<(unsigned)nb, 256, 0, s>>>(g, splits);
    note_launch();
    return cudaGetLastError();
  }
  int gz = g.batch < 65535 ? g.batch : 65535;
  gemm_f64_kernel<BN><<<dim3((unsigned)gx, (unsigned)gy, gz), NT, 0, s>>>(g, 1, 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemm_f64(const Gemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.batch == 1 && g.M <= kThinMax && g.N <= kThinMax && g.K >= 16384 && g.part != nullptr) {
    const int blocks = (int)std::min<long long>(
        std::min<long long>(2ll * device_sm_count(), (g.K + kThinThreads - 1) / kThinThreads),
        g.part_elems / (kThinMax * kThinMax));
    if (blocks >= 1) {
      gemm_f64_thin_k<<<blocks, kThinThreads, 0, s>>>(g, g.part);
      gemm_f64_thin_finish_k<<<1, kThinMax * kThinMax, 0, s>>>(g, g.part, blocks);
      note_launch(2);
      return cudaGetLastError();
    }
  }
  // the narrower tile where it leaves fewer idle columns in the last N tile
  const long long idle64 = (g.N + 63) / 64 * 64 - g.N, idle48 = (g.N + 47) / 48 * 48 - g.N;
  if (idle48 < idle64) return gemm_f64_launch<48>(g, s);
  return gemm_f64_launch<64>(g, s);
}

}  // namespace qrctm
