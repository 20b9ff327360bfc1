// Ket and bra layers of the on-site tensor absorbed into the edge, fused
// (QR-CTMRG paragraph: T' is built with the ket and bra layers of a absorbed
// one after the other, never forming the D^4 x D^4 double layer).
//
// For every (mu, b) pair -- mu the column of Q, b the third leg of T -- the
// slice X1[mu, b] is a D^2 x D^2 matrix with rows (u_b, k_b) and columns
// (u_k, k_k), and
//   Z [(u_b,k_b),(s,d_k,j_k)] = sum_{u_k,k_k} X1[(u_b,k_b),(u_k,k_k)] A[s,u_k,k_k,d_k,j_k]
//   X2[(d_k,j_k),(d_b,j_b)]   = sum_{s,u_b,k_b} Z[(u_b,k_b),(s,d_k,j_k)] A[s,u_b,k_b,d_b,j_b].
// Both contractions of a group of slices run in one CTA with Z held in shared
// memory, so the only HBM traffic is X1 in and X2 out.  Contractions this
// small (K = D^2 and d D^2) and this memory-heavy stay on the FP32 cores;
// accumulation is FP32, the precision class of the split path.
//
// Layouts (FP32):
//   X1  [(mu,b)][(u_b,k_b)] x (u_k,k_k), row stride D2p
//   Ak  [(s,d,r)] x (u,l), row stride D2p          (A[s,u,l,d,r])
//   Ab  [(d,r)] x (s,u,l), row stride dD2p          (A[s,u,l,d,r])
//   X2  [(mu,j_k,j_b)] x (b,d_k,d_b), row stride mp
// Instantiated for d = 2 and D = 2, 4 (D = 6 runs on the tensor cores,
// absorb_tc.cu).
#include "ctx.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace qrctm {

namespace {

using namespace ptx;

// Slices X1[g0 .. g0+ng) (contiguous, ng*D2*D2p floats) into shared memory
// by one bulk asynchronous copy completing on `bar`.
__device__ __forceinline__ void issue_slices(const float* X1, float* dst, uint32_t bar,
                                             long long g0, int ng, int D2, long long D2p) {
  const uint32_t bytes = (uint32_t)((size_t)ng * D2 * D2p * sizeof(float));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, bytes);
  bulk_load(smem_u32(dst), X1 + g0 * D2 * D2p, bytes, bar);
}

// One persistent CTA loops over batches of NG slices; the next batch is
// copied in (bulk async copy, double buffer) while the current one is
// contracted.  The buffer of a batch also stages its X2 block for the
// coalesced write-out.  Shapes are template parameters, so every index
// division is by a constant and the contraction loops unroll.
template <int D, int d, int NG>
struct AbsorbShape {
  static constexpr int D2 = D * D, dD2 = d * D2;
  static constexpr int R4 = D2 / 4, C8 = dD2 / 8;
  static constexpr int tpg1 = R4 * C8, tpg2 = R4 * R4;
  static constexpr int threads = NG * tpg2;
  static constexpr size_t xbuf = (size_t)NG * D2 * D2;   // floats per slice buffer
  static constexpr size_t smem_floats = 2 * xbuf + (size_t)NG * D2 * dD2 + 2 * (size_t)D2 * dD2;
};

template <int D, int d, int NG>
__global__ void __launch_bounds__(AbsorbShape<D, d, NG>::threads)
    absorb_fused_k(const float* __restrict__ X1, const float* __restrict__ Ak,
                   const float* __restrict__ Ab, float* __restrict__ X2, int ch, long long Akp,
                   long long Abp, long long mp, long long ngroups, int* err) {
  using S = AbsorbShape<D, d, NG>;
  constexpr int D2 = S::D2, dD2 = S::dD2, R4 = S::R4, C8 = S::C8, tpg1 = S::tpg1,
                tpg2 = S::tpg2, nt = S::threads;
  extern __shared__ __align__(128) float sm[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ int s_ok;
  __shared__ long long xbase[NG];   // X2 offset of slice g of the batch: (mu D2) mp + b D2
  const int tid = threadIdx.x;
  float* Xb0 = sm;                                  // [NG][D2][D2]  slices (then X2 staging)
  float* Xb1 = Xb0 + S::xbuf;
  float* Zs = Xb1 + S::xbuf;                        // [NG][D2][dD2]
  float* AkT = Zs + (size_t)NG * D2 * dD2;          // [D2][dD2]      AkT[k][c] = Ak[c][k]
  float* AbT = AkT + (size_t)D2 * dD2;              // [dD2][D2]      AbT[k][c] = Ab[c][k]
  const uint32_t bar0 = smem_u32(&mbar[0]), bar1 = smem_u32(&mbar[1]);
  const long long stride = (long long)gridDim.x * NG;
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long g0 = (long long)blockIdx.x * NG;
    if (g0 < ngroups)
      issue_slices(X1, Xb0, bar0, g0, (int)std::min<long long>(NG, ngroups - g0), D2, D2);
  }
  for (int e = tid; e < D2 * dD2; e += nt) {
    const int c = e / D2, k = e % D2;
    AkT[k * dD2 + c] = Ak[c * Akp + k];
  }
  for (int e = tid; e < D2 * dD2; e += nt) {
    const int c = e / dD2, k = e % dD2;
    AbT[k * D2 + c] = Ab[c * Abp + k];
  }
  // this thread's tiles (one of each contraction per slice group)
  const int g1 = tid / tpg1, rem1 = tid % tpg1, rb1 = (rem1 / C8) * 4, cb1 = (rem1 % C8) * 8;
  const int g2 = tid / tpg2, rem2 = tid % tpg2, rb2 = (rem2 / R4) * 4, cb2 = (rem2 % R4) * 4;
  // use n of buffer it & 1 (n = it >> 1) completes phase n of its mbarrier
  int it = 0;
  bool next_issued = false;
  if (tid == 0) s_ok = 1;
  for (long long g0 = (long long)blockIdx.x * NG; g0 < ngroups; g0 += stride, ++it) {
    const int ng = (int)std::min<long long>(NG, ngroups - g0);
    float* Xb = (it & 1) ? Xb1 : Xb0;
    const uint32_t bar = (it & 1) ? bar1 : bar0;
    __syncthreads();   // the other buffer's previous batch is fully written out
    if (tid < NG) {   // one 64-bit division per slice, not per element
      const long long gg = g0 + tid, mu = gg / ch;
      xbase[tid] = mu * D2 * mp + (gg - mu * ch) * D2;
    }
    const long long gn = g0 + stride;
    next_issued = gn < ngroups;
    if (tid == 0 && next_issued)
      issue_slices(X1, (it & 1) ? Xb0 : Xb1, (it & 1) ? bar0 : bar1, gn,
                   (int)std::min<long long>(NG, ngroups - gn), D2, D2);
    if (!mbar_wait_bounded(bar, (uint32_t)((it >> 1) & 1))) {
      atomicOr(err, ERRF_TIMEOUT);
      s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    // ket: Zs[g][r][c] = sum_k X[g][r][k] AkT[k][c]   (4 x 8 tile, k in steps of 4)
    for (int t = tid, g = g1; t < NG * tpg1; t += nt, g += nt / tpg1) {
      if (g >= ng) break;
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      const float* xa = Xb + ((size_t)g * D2 + rb1) * D2;
      const float* kb = AkT + cb1;
#pragma unroll 3
      for (int k = 0; k < D2; k += 4) {
        float av[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 a = *reinterpret_cast<const float4*>(xa + i * D2 + k);
          av[i][0] = a.x; av[i][1] = a.y; av[i][2] = a.z; av[i][3] = a.w;
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const float4 b0 = *reinterpret_cast<const float4*>(kb + (k + kk) * dD2);
          const float4 b1 = *reinterpret_cast<const float4*>(kb + (k + kk) * dD2 + 4);
          const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i][kk], bv[j], acc[i][j]);
        }
      }
      float* zo = Zs + ((size_t)g * D2 + rb1) * dD2 + cb1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        *reinterpret_cast<float4*>(zo + i * dD2) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(zo + i * dD2 + 4) =
            make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
      }
    }
    __syncthreads();
    // bra: out[g][r2][c2] = sum_{s,q} Zs[g][q][s*D2 + r2] AbT[s*D2 + q][c2]   (4 x 4 tile),
    // staged as Xb[g][(j_k,j_b)][(d_k,d_b)]  (r2 = d_k*D + j_k, c2 = d_b*D + j_b)
    if (g2 < ng) {
      const int g = g2;
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
      for (int s = 0; s < d; ++s) {
        const float* za = Zs + (size_t)g * D2 * dD2 + s * D2 + rb2;
        const float* ba = AbT + (size_t)s * D2 * D2 + cb2;
#pragma unroll 6
        for (int q = 0; q < D2; ++q) {
          const float4 a = *reinterpret_cast<const float4*>(za + q * dD2);
          const float4 b = *reinterpret_cast<const float4*>(ba + q * D2);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r2 = rb2 + i, dk = r2 / D, jk = r2 % D;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c2 = cb2 + j, db = c2 / D, jb = c2 % D;
          Xb[((size_t)g * D2 + jk * D + jb) * D2 + dk * D + db] = acc[i][j];
        }
      }
    }
    __syncthreads();
    // write out: consecutive slices of one mu are consecutive b, contiguous in X2
    for (int e = tid; e < NG * D2 * D2; e += nt) {
      const int dd = e % D2, g = (e / D2) % NG, jj = e / (D2 * NG);
      if (g >= ng) continue;
      X2[xbase[g] + (long long)jj * mp + dd] = Xb[((size_t)g * D2 + jj) * D2 + dd];
    }
  }
  // after an abandoned wait, let the copies still in flight land (bounded)
  // before the CTA's shared memory is released
  if (!s_ok && tid == 0) {
    mbar_wait_bounded((it & 1) ? bar1 : bar0, (uint32_t)((it >> 1) & 1));
    if (next_issued)
      mbar_wait_bounded(((it + 1) & 1) ? bar1 : bar0, (uint32_t)(((it + 1) >> 1) & 1));
  }
}

// FP64 ket + bra layers of one (mu, b) slice after another (the FP64 path,
// split layers, d = 2): the same contraction as above in FP64, for X1 in
// the slice-contiguous layout X1[(mu,b)][(u_b,k_b)][(u_k,k_k)] and X2 in the
// layout the FP64 projection reads, X2[(mu,b)][(d_k,j_k)][(d_b,j_b)].
//   Z [(u_b,k_b)][(s,d_k,j_k)] = sum_{u_k,k_k} X1 A[s,u_k,k_k,d_k,j_k]
//   X2[(d_k,j_k)][(d_b,j_b)]   = sum_{s,u_b,k_b} Z[(u_b,k_b)][(s,d_k,j_k)] A[s,u_b,k_b,d_b,j_b]
// Bound by the FP64 pipe (~2 FMA per clock per SM on B300): 2 d D^6 FMA per
// slice; per CTA of 8 warps, NG slices per batch copied in by one bulk
// asynchronous copy (double buffer), Z in shared memory, 4 x 4 register
// tiles for the ket and 2 x 4 for the bra so that both phases have D^4/4.5
// tiles per slice for 256 threads at D = 6.
template <int D, int NG, int NBUF>
struct Absorb64Shape {
  static constexpr int D2 = D * D, dD2 = 2 * D2, D4 = D2 * D2;
  static constexpr int threads = 256;
  static constexpr int ket_tiles = (D2 / 4) * (dD2 / 4);   // 4 x 4
  static constexpr int bra_tiles = (D2 / 2) * (D2 / 4);    // 2 x 4
  static constexpr size_t xbuf = (size_t)NG * D4;           // doubles per slice buffer
  static constexpr size_t smem_doubles =
      NBUF * xbuf + (size_t)NG * D2 * dD2 + 2 * (size_t)D2 * dD2;
};

// NBUF = 2: the next batch's copy overlaps this batch's contraction; NBUF = 1
// (D = 8: one slice of 32 KB, 224 KB in all) the copy is issued once the
// slice has been consumed -- its latency is small against the ~0.26 ms of
// FP64 work per slice.
template <int D, int NG, int NBUF>
__global__ void __launch_bounds__(256) absorb64_k(const double* __restrict__ X1,
                                                  const double* __restrict__ A,
                                                  double* __restrict__ X2, long long ngroups,
                                                  int* err) {
  using S = Absorb64Shape<D, NG, NBUF>;
  constexpr int D2 = S::D2, dD2 = S::dD2, D4 = S::D4, nt = S::threads;
  extern __shared__ __align__(128) double smd[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  double* Xb0 = smd;                                 // [NG][D2][D2]
  double* Xb1 = (NBUF == 2) ? Xb0 + S::xbuf : Xb0;
  double* Zs = Xb0 + NBUF * S::xbuf;                 // [NG][D2][dD2]
  double* AkT = Zs + (size_t)NG * D2 * dD2;          // [D2][dD2]: AkT[(u,l)][(s,d,r)] = A[s,u,l,d,r]
  double* Ab = AkT + (size_t)D2 * dD2;               // [dD2][D2]: Ab[(s,u,l)][(d,r)] = A[s,u,l,d,r]
  const uint32_t bar0 = smem_u32(&mbar[0]), bar1 = smem_u32(&mbar[1]);
  const long long stride = (long long)gridDim.x * NG;
  auto issue = [&](double* dst, uint32_t bar, long long g0, int ng) {
    const uint32_t bytes = (uint32_t)((size_t)ng * D4 * sizeof(double));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, bytes);
    bulk_load(smem_u32(dst), X1 + g0 * D4, bytes, bar);
  };
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long g0 = (long long)blockIdx.x * NG;
    if (g0 < ngroups) issue(Xb0, bar0, g0, (int)std::min<long long>(NG, ngroups - g0));
  }
  for (int e = tid; e < D2 * dD2; e += nt) {
    const int kq = e / dD2, cq = e % dD2;            // kq = (u,l), cq = (s,d,r)
    const int sq = cq / D2, dr = cq % D2;
    AkT[e] = A[(size_t)sq * D4 + (size_t)kq * D2 + dr];
    Ab[e] = A[e];
  }
  int it = 0;
  bool next_issued = false;
  if (tid == 0) s_ok = 1;
  for (long long g0 = (long long)blockIdx.x * NG; g0 < ngroups; g0 += stride, ++it) {
    const int ng = (int)std::min<long long>(NG, ngroups - g0);
    double* Xb = (it & 1) ? Xb1 : Xb0;
    const uint32_t bar = (it & 1) ? bar1 : bar0;
    __syncthreads();   // the other buffer's previous batch is consumed
    const long long gn = g0 + stride;
    next_issued = NBUF == 2 && gn < ngroups;   // with one buffer: set when issued below
    if (NBUF == 2 && tid == 0 && next_issued)
      issue((it & 1) ? Xb0 : Xb1, (it & 1) ? bar0 : bar1, gn, (int)std::min<long long>(NG, ngroups - gn));
    if (!mbar_wait_bounded(bar, (uint32_t)((it >> 1) & 1))) {
      atomicOr(err, ERRF_TIMEOUT);
      s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    // ket: Zs[g][r][c] = sum_k Xb[g][r][k] AkT[k][c]   (4 x 4 tiles)
    for (int t = tid; t < ng * S::ket_tiles; t += nt) {
      const int g = t / S::ket_tiles, q = t % S::ket_tiles;
      const int rb = (q / (dD2 / 4)) * 4, cb = (q % (dD2 / 4)) * 4;
      double acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
      const double* xa = Xb + ((size_t)g * D2 + rb) * D2;
      const double* kb = AkT + cb;
#pragma unroll 4
      for (int k = 0; k < D2; ++k) {
        const double2 b01 = *reinterpret_cast<const double2*>(kb + k * dD2);
        const double2 b23 = *reinterpret_cast<const double2*>(kb + k * dD2 + 2);
        const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double av = xa[i * D2 + k];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av, bv[j], acc[i][j]);
        }
      }
      double* zo = Zs + ((size_t)g * D2 + rb) * dD2 + cb;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        *reinterpret_cast<double2*>(zo + i * dD2) = make_double2(acc[i][0], acc[i][1]);
        *reinterpret_cast<double2*>(zo + i * dD2 + 2) = make_double2(acc[i][2], acc[i][3]);
      }
    }
    __syncthreads();
    // one buffer: the slices are consumed, the next batch's copy can start
    // (it lands while the bra runs)
    if (NBUF == 1 && gn < ngroups) {
      next_issued = true;
      if (tid == 0) issue(Xb0, (it & 1) ? bar0 : bar1, gn, (int)std::min<long long>(NG, ngroups - gn));
    }
    // bra: X2[g][r2][c2] = sum_{s,q} Zs[g][q][s D2 + r2] Ab[s D2 + q][c2]   (2 x 4 tiles)
    for (int t = tid; t < ng * S::bra_tiles; t += nt) {
      const int g = t / S::bra_tiles, q = t % S::bra_tiles;
      const int rb = (q / (D2 / 4)) * 2, cb = (q % (D2 / 4)) * 4;
      double acc[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const double* za = Zs + (size_t)g * D2 * dD2 + s2 * D2 + rb;
        const double* ba = Ab + (size_t)s2 * D2 * D2 + cb;
#pragma unroll 4
        for (int qq = 0; qq < D2; ++qq) {
          const double2 a = *reinterpret_cast<const double2*>(za + qq * dD2);
          const double2 b01 = *reinterpret_cast<const double2*>(ba + qq * D2);
          const double2 b23 = *reinterpret_cast<const double2*>(ba + qq * D2 + 2);
          const double av[2] = {a.x, a.y};
          const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
      }
      double* xo = X2 + (size_t)(g0 + g) * D4 + (size_t)rb * D2 + cb;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        *reinterpret_cast<double2*>(xo + i * D2) = make_double2(acc[i][0], acc[i][1]);
        *reinterpret_cast<double2*>(xo + i * D2 + 2) = make_double2(acc[i][2], acc[i][3]);
      }
    }
  }
  // after an abandoned wait, let the copies still in flight land (bounded)
  // before the CTA's shared memory is released
  if (!s_ok && tid == 0) {
    mbar_wait_bounded((it & 1) ? bar1 : bar0, (uint32_t)((it >> 1) & 1));
    if (next_issued)
      mbar_wait_bounded(((it + 1) & 1) ? bar1 : bar0, (uint32_t)(((it + 1) >> 1) & 1));
  }
}

using AbsorbKernel = void (*)(const float*, const float*, const float*, float*, int, long long,
                              long long, long long, long long, int*);

struct AbsorbVariant {
  AbsorbKernel k;
  int NG, threads;
  size_t smem;
};

// Instantiated shapes (d = 2, D = 2, 4); D = 6 runs in absorb_tc.cu, other
// shapes take the two-contraction tensor-core path.
template <int D, int NG>
AbsorbVariant absorb_variant() {
  using S = AbsorbShape<D, 2, NG>;
  return AbsorbVariant{absorb_fused_k<D, 2, NG>, NG, S::threads, sizeof(float) * S::smem_floats};
}

bool absorb_lookup(int d, int D, AbsorbVariant* v) {
  if (d != 2) return false;
  switch (D) {
    case 2: *v = absorb_variant<2, 256>(); return true;    // 256 threads
    case 4: *v = absorb_variant<4, 16>(); return true;     // 256 threads
    case 8: *v = absorb_variant<8, 2>(); return true;      // 512 threads
    default: return false;
  }
}

}  // namespace

// The fused FP32 kernel is used up to D = 6; at D = 8 (K = 64 and 128) the
// two tensor-core contractions through Z are faster on B300 (11.9 against
// 16.5 ms per step at chi = 512), at D = 6 the two are even (0.40 ms).
bool absorb_fused_ok(int d, int D) {
  AbsorbVariant v;
  return D <= 6 && absorb_lookup(d, D, &v);
}

cudaError_t absorb_fused(const float* X1, const float* Ak, const float* Ab, float* X2, int ch,
                         int D, int d, long long D2p, long long dD2p, long long mp, int* err,
                         cudaStream_t s) {
  AbsorbVariant v;
  if (!absorb_lookup(d, D, &v)) return cudaErrorInvalidValue;
  // slices are copied whole: rows must be unpadded (D^2 % 4 == 0 makes D2p == D^2)
  // and X1 16-byte aligned for the bulk copies
  if (D2p != (long long)D * D || (reinterpret_cast<uintptr_t>(X1) & 15) != 0)
    return cudaErrorInvalidValue;
  // X2 rows are written in 16-byte pieces
  if ((mp & 3) != 0 || (reinterpret_cast<uintptr_t>(X2) & 15) != 0) return cudaErrorInvalidValue;
  const long long ngroups = (long long)ch * ch;
  const int nsm = device_sm_count();
  cudaError_t e = cudaFuncSetAttribute(v.k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)v.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.k, v.threads, v.smem);
  per_sm = std::max(1, per_sm);
  const long long iters = (ngroups + v.NG - 1) / v.NG;
  const unsigned grid = (unsigned)std::min<long long>(iters, (long long)nsm * per_sm);
  v.k<<<grid, v.threads, v.smem, s>>>(X1, Ak, Ab, X2, ch, D2p, dD2p, mp, ngroups, err);
  note_launch();
  return cudaGetLastError();
}

// FP64 ket + bra for the FP64 path at d = 2, D = 4 and 6 (X1 slice-contiguous,
// X2 in the projection's layout); other shapes keep the two FP64 GEMMs.
bool absorb64_ok(int d, int D) { return d == 2 && (D == 4 || D == 6 || D == 8); }

template <int D, int NG, int NBUF>
cudaError_t absorb64_launch(const double* X1, const double* A, double* X2, long long ngroups,
                            int* err, cudaStream_t s) {
  using S = Absorb64Shape<D, NG, NBUF>;
  const void* kf = (const void*)absorb64_k<D, NG, NBUF>;
  const size_t smem = sizeof(double) * S::smem_doubles;
  cudaError_t e = device_once(kf, [kf, smem] {
    return cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const long long iters = (ngroups + NG - 1) / NG;
  const unsigned grid = (unsigned)std::min<long long>(iters, device_sm_count());
  absorb64_k<D, NG, NBUF><<<grid, S::threads, smem, s>>>(X1, A, X2, ngroups, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t absorb64(const double* X1, const double* A, double* X2, long long ngroups, int d, int D,
                     int* err, cudaStream_t s) {
  if (!absorb64_ok(d, D) || (reinterpret_cast<uintptr_t>(X1) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(X2) & 15) != 0)
    return cudaErrorInvalidValue;
  if (D == 8) return absorb64_launch<8, 1, 1>(X1, A, X2, ngroups, err, s);   // 224 KB
  if (D == 6) return absorb64_launch<6, 4, 2>(X1, A, X2, ngroups, err, s);   // 207 KB
  return absorb64_launch<4, 8, 2>(X1, A, X2, ngroups, err, s);              // 74 KB
}

}  // namespace qrctm
