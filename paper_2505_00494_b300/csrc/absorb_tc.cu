// Ket and bra layers of the on-site tensor absorbed into the edge on the
// tensor cores (QR-CTMRG paragraph: T' is built with the ket and bra layers
// of the double layer absorbed one after the other), d = 2, D = 6.
//
// For every (mu, b) pair the slice X1[mu, b] is a D^2 x D^2 matrix with rows
// (u_b, k_b) and columns (u_k, k_k), and
//   Z [(u_b,k_b),(s,d_k,j_k)] = sum_{u_k,k_k} X1[(u_b,k_b),(u_k,k_k)] A[s,u_k,k_k,d_k,j_k]
//   X2[(d_k,j_k),(d_b,j_b)]   = sum_{s,u_b,k_b} Z[(u_b,k_b),(s,d_k,j_k)] A[s,u_b,k_b,d_b,j_b].
// A tile is three slices: 108 of the 128 rows of one tcgen05 MMA.
//   ket: D1[(g,u_b,k_b)][(s,d_k,j_k)] = X1 rows (A operand in tensor memory,
//        K = 36 padded to 40) x A_ket (B operand, shared memory, N = 80);
//   Z' : D1 is drained from tensor memory and written transposed into a
//        shared-memory operand with rows (g,d_k,j_k) and K index (s,u_b,k_b);
//   bra: D2[(g,d_k,j_k)][(d_b,j_b)] = Z' (A operand, shared memory, K = 72)
//        x A_bra (B operand, shared memory, N = 48);
//   X2 : D2 is drained, staged in shared memory and written out as
//        contiguous 144-byte row segments.
// Every operand is split into TF32 head and tail planes (the split of the
// contraction engine): per 8-wide K slice head*head accumulates in a main
// accumulator and head*tail + tail*head in a correction accumulator (both
// FP32 in tensor memory), summed when drained.  Z goes through FP32 once,
// as in the two-launch route.  Shared-memory operands are K-major with the
// 128-byte swizzle (rows of 32 FP32, 8-row atoms of 1024 bytes).
//
// Layouts (FP32, as in absorb.cu):
//   X1  [(mu,b)][(u_b,k_b)] x (u_k,k_k), row stride D2p (= 36)
//   Ak  [(s,d,r)] x (u,l), row stride D2p          (A[s,u,l,d,r])
//   Ab  [(d,r)] x (s,u,l), row stride dD2p (= 72)  (A[s,u,l,d,r])
//   X2  [(mu,j_k,j_b)] x (b,d_k,d_b), row stride mp
// Sixteen warps: warps w, w + 4, w + 8 and w + 12 serve TMEM lane quarter w
// (tile rows 32 w .. 32 w + 31) and split the columns of each row between
// them in 16-column pieces, so that every SM sub-partition has four warps to
// hide latencies; thread 0 issues the MMAs.  Every mbarrier wait is bounded; a wait that runs out
// raises ERRF_TIMEOUT and the CTA unwinds, freeing tensor memory.
#include "ctx.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace qrctm {

namespace {

constexpr int kD2 = 36;               // D^2 at D = 6
constexpr int kDD2 = 72;              // d D^2 at d = 2
constexpr int kGT = 3;                // slices per tile (108 of 128 rows)
constexpr int kThreads = 512;        // warps w, w+4, w+8, w+12 share TMEM lane quarter w
constexpr int kKetN = 80;             // ket N (72 used), multiple of 16 for M = 128
constexpr int kBraN = 48;             // bra N (36 used)
// shared-memory regions (bytes from a 1024-aligned base); K-major SW128
// blocks of rows x 128 bytes
constexpr int kAkBlock = kKetN * 128;          // 10240: one 32-wide K block of A_ket
constexpr int kAbBlock = kBraN * 128;          // 6144
constexpr int kZBlock = 128 * 128;             // 16384
constexpr int kOffAkH = 0;
constexpr int kOffAkL = kOffAkH + 2 * kAkBlock;
constexpr int kOffAbH = kOffAkL + 2 * kAkBlock;
constexpr int kOffAbL = kOffAbH + 3 * kAbBlock;
constexpr int kOffZH = kOffAbL + 3 * kAbBlock;
constexpr int kOffZL = kOffZH + 3 * kZBlock;
constexpr int kOffStg = kOffZL + 3 * kZBlock;
constexpr int kStgRow = kGT * kD2;             // 108 floats per staged row
constexpr int kOffBar = kOffStg + kD2 * kStgRow * 4;
constexpr int kSmem = kOffBar + 64 + 1024;     // + alignment slack
static_assert(kOffZH % 1024 == 0 && kOffAbH % 1024 == 0 && kOffAkL % 1024 == 0 &&
                  kOffAbL % 1024 == 0 && kOffZL % 1024 == 0,
              "SW128 operand blocks must be 1024-byte aligned");
static_assert(kSmem <= 232448, "shared memory");
// tensor-memory columns
constexpr uint32_t kD1Main = 0, kD1Corr = 96, kD2Main = 192, kD2Corr = 256;
constexpr uint32_t kAHi = 320, kALo = 384;     // X1 rows, K padded to 64
constexpr uint32_t kTmemCols = 512;

using namespace ptx;

__global__ void __launch_bounds__(kThreads, 1)
    absorb_tc_kernel(const float* __restrict__ X1, const float* __restrict__ Ak,
                     const float* __restrict__ Ab, float* __restrict__ X2, int ch, long long mp,
                     long long ngroups, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float* stg = reinterpret_cast<float*>(base + kOffStg);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kOffBar);     // [0] ket, [1] bra
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffBar + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(base + kOffBar + 24);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sb = smem_u32(base);
  const uint32_t bar_ket = smem_u32(&bars[0]), bar_bra = smem_u32(&bars[1]);

  // resident B operands: A_ket (80 x 64, used 72 x 36) and A_bra (48 x 96,
  // used 36 x 72), head and tail planes
  for (int e = tid; e < kKetN * 64; e += kThreads) {
    const int r = e >> 6, k = e & 63;
    const float v = (r < kDD2 && k < kD2) ? Ak[r * kD2 + k] : 0.f;
    float h, t;
    tf32_split(v, h, t);
    const uint32_t o = sw128_off(r, k, kAkBlock);
    *reinterpret_cast<float*>(base + kOffAkH + o) = h;
    *reinterpret_cast<float*>(base + kOffAkL + o) = t;
  }
  for (int e = tid; e < kBraN * 96; e += kThreads) {
    const int r = e / 96, k = e % 96;
    const float v = (r < kD2 && k < kDD2) ? Ab[r * kDD2 + k] : 0.f;
    float h, t;
    tf32_split(v, h, t);
    const uint32_t o = sw128_off(r, k, kAbBlock);
    *reinterpret_cast<float*>(base + kOffAbH + o) = h;
    *reinterpret_cast<float*>(base + kOffAbL + o) = t;
  }
  if (tid == 0) {
    mbar_init(bar_ket, 1);
    mbar_init(bar_bra, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int quarter = warp & 3, part = warp >> 2;   // part: 16-column piece owner
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
  constexpr uint32_t idesc_ket = idesc_tf32(128, kKetN), idesc_bra = idesc_tf32(128, kBraN);
  // this thread's tile row: slice g_loc = row / 36, row (u_b,k_b) = row % 36
  // of the ket; row (d_k,j_k) = row % 36 of the bra
  const int row = quarter * 32 + (tid & 31);
  const int g_loc = row / kD2, rin = row % kD2;
  const long long ntiles = (ngroups + kGT - 1) / kGT;
  // X1 rows of a tile -> head and tail into tensor memory (K 36 used of 64)
  auto load_a = [&](long long tile) {
    const long long g0 = tile * kGT;
    const int gcount = (int)std::min<long long>(kGT, ngroups - g0);
    const bool valid = g_loc < gcount;
    const float* src = X1 + ((g0 + g_loc) * kD2 + rin) * (long long)kD2;
    // part p: columns 16 p .. 16 p + 15 of the K range 0..63 (36 used)
    float hv[16], tv[16];
    float4 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int col = 16 * part + 4 * c;
      if (valid && col < kD2) v[c] = *reinterpret_cast<const float4*>(src + col);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      tf32_split(v[c].x, hv[4 * c], tv[4 * c]);
      tf32_split(v[c].y, hv[4 * c + 1], tv[4 * c + 1]);
      tf32_split(v[c].z, hv[4 * c + 2], tv[4 * c + 2]);
      tf32_split(v[c].w, hv[4 * c + 3], tv[4 * c + 3]);
    }
    tmem_st16(lane_base + kAHi + 16 * part, hv);
    tmem_st16(lane_base + kALo + 16 * part, tv);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  };
  // staged rows out: row (j_k, j_b) of slice g goes to X2 row (mu*36 + j_k*6 +
  // j_b), columns b*36 .. b*36 + 35 (16-byte pieces)
  auto write_out = [&](long long tile) {
    const long long g0 = tile * kGT;
    const int gcount = (int)std::min<long long>(kGT, ngroups - g0);
    for (int e = tid; e < kD2 * gcount * 9; e += kThreads) {
      const int piece = e % 9, rg = e / 9, g = rg % gcount, rho = rg / gcount;
      const long long G = g0 + g;
      const long long mu = G / ch, bb = G % ch;
      const float4 v = *reinterpret_cast<const float4*>(stg + rho * kStgRow + g * kD2 + piece * 4);
      *reinterpret_cast<float4*>(X2 + (mu * kD2 + rho) * mp + bb * kD2 + piece * 4) = v;
    }
  };
  // Per tile: ket MMAs (tile i) while the previous tile's X2 rows are written
  // out; the D1 drain into Z'; bra MMAs while the next tile's X1 rows are
  // loaded into tensor memory; the D2 drain into the staging rows.
  int it = 0;
  long long tile = blockIdx.x;
  if (tile < ntiles) load_a(tile);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  long long prev = -1;
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    const long long g0 = tile * kGT;
    const int gcount = (int)std::min<long long>(kGT, ngroups - g0);
    const bool valid = g_loc < gcount;
    // ket: 5 K slices of 8 (K = 40), three MMAs each
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < 5; ++ks) {
        const uint32_t kb = (uint32_t)(ks >> 2) * kAkBlock + (uint32_t)(ks & 3) * 32;
        const uint64_t bh = desc_sw128(sb + kOffAkH + kb), bl = desc_sw128(sb + kOffAkL + kb);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        umma_tf32_tmem_a(tmem + kD1Main, tmem + kAHi + ks * 8, bh, idesc_ket, acc);
        umma_tf32_tmem_a(tmem + kD1Corr, tmem + kAHi + ks * 8, bl, idesc_ket, acc);
        umma_tf32_tmem_a(tmem + kD1Corr, tmem + kALo + ks * 8, bh, idesc_ket, 1u);
      }
      umma_commit(bar_ket);
    }
    if (prev >= 0) write_out(prev);
    if (!mbar_wait_bounded(bar_ket, it & 1)) {
      atomicOr(err, ERRF_TIMEOUT);
      *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // Z row (g, u_b, k_b) -> Z'[(g, d_k, j_k)][(s, u_b, k_b)], head and tail
    // 16-column pieces: part p takes piece p, part 0 also piece 4 (columns 64..71)
#pragma unroll
    for (int cc = 0; cc < 5; ++cc) {
      if (!(cc == part || (cc == 4 && part == 0))) continue;
      float zm[16], zc[16];
      tmem_ld16(lane_base + kD1Main + cc * 16, zm);
      tmem_ld16(lane_base + kD1Corr + cc * 16, zc);
      if (valid) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = cc * 16 + i;                 // (s, d_k, j_k)
          if (n < kDD2) {
            const int s = n / kD2, dj = n % kD2;
            float h, t;
            tf32_split(zm[i] + zc[i], h, t);
            const uint32_t o = sw128_off(g_loc * kD2 + dj, s * kD2 + rin, kZBlock);
            *reinterpret_cast<float*>(base + kOffZH + o) = h;
            *reinterpret_cast<float*>(base + kOffZL + o) = t;
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // bra: 9 K slices of 8 (K = 72)
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < 9; ++ks) {
        const uint32_t za = (uint32_t)(ks >> 2) * kZBlock + (uint32_t)(ks & 3) * 32;
        const uint32_t ab = (uint32_t)(ks >> 2) * kAbBlock + (uint32_t)(ks & 3) * 32;
        const uint64_t ah = desc_sw128(sb + kOffZH + za), al = desc_sw128(sb + kOffZL + za);
        const uint64_t bh = desc_sw128(sb + kOffAbH + ab), bl = desc_sw128(sb + kOffAbL + ab);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        umma_tf32_ss(tmem + kD2Main, ah, bh, idesc_bra, acc);
        umma_tf32_ss(tmem + kD2Corr, ah, bl, idesc_bra, acc);
        umma_tf32_ss(tmem + kD2Corr, al, bh, idesc_bra, 1u);
      }
      umma_commit(bar_bra);
    }
    // the next tile's X1 rows into tensor memory (the ket MMAs that read the
    // A region are complete)
    if (tile + gridDim.x < ntiles) load_a(tile + gridDim.x);
    if (!mbar_wait_bounded(bar_bra, it & 1)) {
      atomicOr(err, ERRF_TIMEOUT);
      *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // X2 row (g, d_k, j_k), columns (d_b, j_b) -> staging [(j_k, j_b)][(g, d_k, d_b)]
    // 16-column pieces: part p < 3 takes columns 16 p .. 16 p + 15 (36 used)
    if (part < 3) {
      float xm[16], xc[16];
      const int dk = rin / 6, jk = rin % 6;
      tmem_ld16(lane_base + kD2Main + 16 * part, xm);
      tmem_ld16(lane_base + kD2Corr + 16 * part, xc);
      if (valid) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = 16 * part + i;
          if (n < kD2) {
            const int db = n / 6, jb = n % 6;
            stg[(jk * 6 + jb) * kStgRow + g_loc * kD2 + dk * 6 + db] = xm[i] + xc[i];
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    prev = tile;
  }
  if (!*abort_flag && prev >= 0) write_out(prev);
  // teardown: tensor memory is freed after every MMA has completed (a wait
  // that ran out is retried, bounded, before the CTA exits)
  __syncthreads();
  if (*abort_flag && tid == 0) {
    mbar_wait_bounded(bar_ket, it & 1);
    mbar_wait_bounded(bar_bra, it & 1);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

bool absorb_tc_ok(int d, int D) { return d == 2 && D == 6; }

cudaError_t absorb_tc(const float* X1, const float* Ak, const float* Ab, float* X2, int ch,
                      long long D2p, long long dD2p, long long mp, int* err, cudaStream_t s) {
  if (D2p != kD2 || dD2p != kDD2) return cudaErrorInvalidValue;
  // 16-byte row pieces of X2 and X1
  if ((mp & 3) != 0 || (reinterpret_cast<uintptr_t>(X2) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(X1) & 15) != 0)
    return cudaErrorInvalidValue;
  const long long ngroups = (long long)ch * ch;
  cudaError_t e = device_once((const void*)absorb_tc_kernel, [] {
    return cudaFuncSetAttribute(absorb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmem);
  });
  if (e != cudaSuccess) return e;
  const long long ntiles = (ngroups + kGT - 1) / kGT;
  const unsigned grid = (unsigned)std::min<long long>(ntiles, device_sm_count());
  absorb_tc_kernel<<<grid, kThreads, kSmem, s>>>(X1, Ak, Ab, X2, ch, mp, ngroups, err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
