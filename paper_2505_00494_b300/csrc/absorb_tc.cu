// Ket and bra layers of the on-site tensor absorbed into the edge on the
// tensor cores (QR-CTMRG paragraph: T' is built with the ket and bra layers
// of the double layer absorbed one after the other), d = 2, D = 6.
//
// For every (mu, b) pair the slice X1[mu, b] is a D^2 x D^2 matrix with rows
// (u_b, k_b) and columns (u_k, k_k), and
//   Z [(u_b,k_b),(s,d_k,j_k)] = sum_{u_k,k_k} X1[(u_b,k_b),(u_k,k_k)] A[s,u_k,k_k,d_k,j_k]
//   X2[(d_k,j_k),(d_b,j_b)]   = sum_{s,u_b,k_b} Z[(u_b,k_b),(s,d_k,j_k)] A[s,u_b,k_b,d_b,j_b].
// A tile is three consecutive slices g = (mu, b) (108 X1 rows).
//   ket: Z transposed,
//        D1[(s,d_k,j_k)][(g,u_b,k_b)] = A_ket (A operand, tensor memory,
//        72 of 128 lanes, K = 36 padded to 40) x X1 rows (B operand, shared
//        memory, N = 112 of which 108 used);
//   Z' : D1 is drained from tensor memory; the lane of row (s,d_k,j_k)
//        holds the 36 values (u_b,k_b) of each slice, a contiguous K range of
//        the bra's A operand Z'[(g,d_k,j_k)][(s,u_b,k_b)], written as 16-byte
//        vectors into the 128-byte-swizzled K-major layout;
//   bra: D2[(g,d_k,j_k)][(d_b,j_b)] = Z' (A operand, shared memory, K = 72)
//        x A_bra (B operand, shared memory, N = 48 of which 36 used);
//   X2 : D2 is drained into one dense 36 x 36 staging box per slice and each
//        box goes to X2 by one TMA tensor store.
// Every operand is split into TF32 head and tail planes (the split of the
// contraction engine): per 8-wide K slice head*head accumulates in a main
// accumulator and head*tail + tail*head in a correction accumulator (both
// FP32 in tensor memory), summed when drained.  Z goes through FP32 once,
// as in the two-launch route.
//
// Layouts (FP32, as in absorb.cu):
//   X1  [(mu,b)][(u_b,k_b)] x (u_k,k_k), row stride 36
//   Ak  [(s,d,r)] x (u,l), row stride 36           (A[s,u,l,d,r])
//   Ab  [(d,r)] x (s,u,l), row stride 72           (A[s,u,l,d,r])
//   X2  [(mu,j_k,j_b)] x (b,d_k,d_b), row stride mp
//
// Schedule per tile t (one CTA of sixteen warps per SM, persistent): the
// ket MMAs of t run while the X2 boxes of t - 1 are drained and stored;
// then the warps of tensor-memory lane quarters 0-2 drain D1 into Z' while
// the quarter-3 warps write the next tile's X1 rows (prefetched into
// registers one tile ahead) into the B-operand planes; one thread then
// queues the bra MMAs of t followed by the ket MMAs of t + 1, so that the
// D2 drain of t overlaps the ket of t + 1.  Every mbarrier wait is bounded;
// a wait that runs out raises ERRF_TIMEOUT and the CTA unwinds, freeing
// tensor memory.
#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace qrctm {

namespace {

constexpr int kD2 = 36;               // D^2 at D = 6
constexpr int kDD2 = 72;              // d D^2 at d = 2
constexpr int kGT = 3;                // slices per tile
constexpr int kRows = kGT * kD2;      // 108 X1 rows per tile
constexpr int kThreads = 512;         // warps w, w+4, w+8, w+12 share TMEM lane quarter w
constexpr int kKetN = 112;            // ket N (108 used), multiple of 16 for M = 128
constexpr int kBraN = 48;             // bra N (36 used)
constexpr int kPrefetch = 8;          // X1 float4 pieces per quarter-3 thread (972 / 128)
// shared-memory regions (bytes from a 1024-aligned base); K-major SW128
// blocks of rows x 128 bytes
constexpr int kXBlock = kKetN * 128;           // 14336: one 32-wide K block of the X1 rows
constexpr int kAbBlock = kBraN * 128;          // 6144
constexpr int kZBlock = 128 * 128;             // 16384
constexpr int kOffXH = 0;
constexpr int kOffXL = kOffXH + 2 * kXBlock;
constexpr int kOffAbH = kOffXL + 2 * kXBlock;
constexpr int kOffAbL = kOffAbH + 3 * kAbBlock;
constexpr int kOffZH = kOffAbL + 3 * kAbBlock;
constexpr int kOffZL = kOffZH + 3 * kZBlock;
constexpr int kStgSlot = 5248;                 // 36 x 36 floats rounded up to 128 bytes
constexpr int kOffStg = kOffZL + 3 * kZBlock;
constexpr int kOffBar = kOffStg + kGT * kStgSlot;
constexpr int kSmem = kOffBar + 64 + 1024;     // + alignment slack
static_assert(kOffXL % 1024 == 0 && kOffAbH % 1024 == 0 && kOffAbL % 1024 == 0 &&
                  kOffZH % 1024 == 0 && kOffZL % 1024 == 0 && kOffStg % 128 == 0 &&
                  kStgSlot % 128 == 0,
              "SW128 operand blocks must be 1024-byte aligned, TMA boxes 128-byte aligned");
static_assert(kSmem <= 232448, "shared memory");
static_assert(kPrefetch * 128 >= kRows * 9, "X1 prefetch covers the tile");
// tensor-memory columns
constexpr uint32_t kD1Main = 0, kD1Corr = 128, kD2Main = 256, kD2Corr = 320;
constexpr uint32_t kAHi = 384, kALo = 448;     // A_ket rows, K padded to 48
constexpr uint32_t kTmemCols = 512;

using namespace ptx;

// byte offset of the 16-byte chunk (row r, K chunk kc = K / 4) of a K-major
// SW128 operand whose 32-wide K blocks are `block` bytes apart
__device__ __forceinline__ uint32_t sw128_chunk(int r, int kc, int block) {
  return (uint32_t)((kc >> 3) * block + r * 128 + (((kc & 7) ^ (r & 7)) << 4));
}

// TF32 head and tail of x on the integer and FP32 pipes (round to nearest,
// ties away from zero, as tf32_split): x = head + tail exactly for finite x.
// The hardware conversion instruction has a lower issue rate.
__device__ __forceinline__ void split_rna(float x, float& head, float& tail) {
  head = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  tail = __uint_as_float((__float_as_uint(x - head) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void store_split4(unsigned char* base, uint32_t off_h, uint32_t off_l,
                                             float4 v) {
  float4 h, t;
  split_rna(v.x, h.x, t.x);
  split_rna(v.y, h.y, t.y);
  split_rna(v.z, h.z, t.z);
  split_rna(v.w, h.w, t.w);
  *reinterpret_cast<float4*>(base + off_h) = h;
  *reinterpret_cast<float4*>(base + off_l) = t;
}

__global__ void __launch_bounds__(kThreads, 1)
    absorb_tc_kernel(const __grid_constant__ CUtensorMap tmX2, const float* __restrict__ X1,
                     const float* __restrict__ Ak, const float* __restrict__ Ab, int ch,
                     long long ngroups, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // mbarriers: ket MMAs complete, bra MMAs complete (two issuing threads),
  // every MMA complete (teardown)
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffBar + 24);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(base + kOffBar + 28);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, part = warp >> 2;   // TMEM lane quarter, column share
  const uint32_t sb = smem_u32(base);
  const uint32_t bar_ket = smem_u32(&bars[0]), bar_bra = smem_u32(&bars[1]);
  const uint32_t bar_fin = smem_u32(&bars[2]);
  const long long ntiles = (ngroups + kGT - 1) / kGT;

  // X1 and Z' operand planes start at zero: K pads, rows 108..127 and the
  // unused K range of Z' stay zero (finite) for the whole launch
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < (kOffAbH - kOffXH) / 16; e += kThreads)
    reinterpret_cast<float4*>(base + kOffXH)[e] = zero4;
  for (int e = tid; e < (kOffStg - kOffZH) / 16; e += kThreads)
    reinterpret_cast<float4*>(base + kOffZH)[e] = zero4;
  // resident A_bra (bra B operand): 48 x 96, used 36 x 72, head and tail
  for (int e = tid; e < kBraN * 96; e += kThreads) {
    const int r = e / 96, k = e % 96;
    const float v = (r < kD2 && k < kDD2) ? Ab[r * kDD2 + k] : 0.f;
    float h, t;
    split_rna(v, h, t);
    const uint32_t o = sw128_off(r, k, kAbBlock);
    *reinterpret_cast<float*>(base + kOffAbH + o) = h;
    *reinterpret_cast<float*>(base + kOffAbL + o) = t;
  }
  if (tid == 0) {
    mbar_init(bar_ket, 1);
    mbar_init(bar_bra, 2);
    mbar_init(bar_fin, 3);
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
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
  // A_ket into tensor memory (ket A operand): lane L = row (s, d_k, j_k),
  // zero beyond row 72; K columns 0..47 of the head and tail planes, zero
  // beyond K = 36; part p < 3 writes columns 16 p .. 16 p + 15
  if (part < 3) {
    const int L = quarter * 32 + lane;
    float hv[16], tv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = 16 * part + i;
      const float v = (L < kDD2 && k < kD2) ? Ak[L * kD2 + k] : 0.f;
      split_rna(v, hv[i], tv[i]);
    }
    tmem_st16(lane_base + kAHi + 16 * part, hv);
    tmem_st16(lane_base + kALo + 16 * part, tv);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  constexpr uint32_t idesc_ket = idesc_tf32(128, kKetN), idesc_bra = idesc_tf32(128, kBraN);

  // X1 rows of a tile (quarter-3 warps): 108 rows x 9 float4 pieces,
  // prefetched into registers one tile ahead, then split into the B-operand
  // head and tail planes
  const int q3 = part * 32 + lane;
  float4 pre[kPrefetch];
  auto prefetch = [&](long long tl) {
    const long long g0 = tl * kGT;
    const int n4 = (int)std::min<long long>(kGT, ngroups - g0) * kD2 * 9;
    const float* src = X1 + g0 * (kD2 * kD2);
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int e = q3 + 128 * u;
      pre[u] = (e < n4) ? __ldg(reinterpret_cast<const float4*>(src + (e / 9) * kD2 + (e % 9) * 4))
                        : zero4;
    }
  };
  auto store_x1 = [&](long long tl) {
    const long long g0 = tl * kGT;
    const int n4 = (int)std::min<long long>(kGT, ngroups - g0) * kD2 * 9;
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int e = q3 + 128 * u;
      if (e < n4) {
        const uint32_t o = sw128_chunk(e / 9, e % 9, kXBlock);
        store_split4(base, kOffXH + o, kOffXL + o, pre[u]);
      }
    }
  };
  // MMA issue (one thread): descriptors are formed once; a K slice of 8
  // advances the start address by 32 bytes inside a 128-byte row, the next
  // 32-wide K block by one block (start-address field in 16-byte units)
  auto issue_ket = [&]() {
    const uint64_t dXH = desc_sw128(sb + kOffXH), dXL = desc_sw128(sb + kOffXL);
#pragma unroll
    for (int ks = 0; ks < 5; ++ks) {
      const uint64_t kb = (uint64_t)(((ks >> 2) * kXBlock + (ks & 3) * 32) >> 4);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      umma_tf32_tmem_a(tmem + kD1Main, tmem + kAHi + ks * 8, dXH + kb, idesc_ket, acc);
      umma_tf32_tmem_a(tmem + kD1Corr, tmem + kAHi + ks * 8, dXL + kb, idesc_ket, acc);
      umma_tf32_tmem_a(tmem + kD1Corr, tmem + kALo + ks * 8, dXH + kb, idesc_ket, 1u);
    }
    umma_commit(bar_ket);
  };
  // bra: the main products (head x head) and the correction products
  // (head x tail, tail x head) go to different accumulators and are issued
  // by two threads, each committing to the bra barrier
  auto issue_bra = [&](bool corr) {
    const uint64_t dZH = desc_sw128(sb + kOffZH), dZL = desc_sw128(sb + kOffZL);
    const uint64_t dAH = desc_sw128(sb + kOffAbH), dAL = desc_sw128(sb + kOffAbL);
#pragma unroll
    for (int ks = 0; ks < 9; ++ks) {
      const uint64_t za = (uint64_t)(((ks >> 2) * kZBlock + (ks & 3) * 32) >> 4);
      const uint64_t ab = (uint64_t)(((ks >> 2) * kAbBlock + (ks & 3) * 32) >> 4);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      if (!corr) {
        umma_tf32_ss(tmem + kD2Main, dZH + za, dAH + ab, idesc_bra, acc);
      } else {
        umma_tf32_ss(tmem + kD2Corr, dZH + za, dAL + ab, idesc_bra, acc);
        umma_tf32_ss(tmem + kD2Corr, dZL + za, dAH + ab, idesc_bra, 1u);
      }
    }
    umma_commit(bar_bra);
  };
  // D1 -> Z' (quarters 0-2): the lane of row (s, d_k, j_k) writes, for each
  // slice g, the K range s*36 .. s*36 + 35 of Z' row (g, d_k, j_k); 16-column
  // pieces of D1, part p takes pieces 2p and 2p + 1 (part 3: piece 6).  The
  // loops are not unrolled over pieces: warps of one SM sub-partition run
  // different pieces, and unrolled per-piece code overflows the instruction
  // cache.
  auto drain_d1 = [&](int gcount) {
    const int L = quarter * 32 + lane;
    const bool lv = L < kDD2;
    const int s = L >= kD2 ? 1 : 0, dj = L - s * kD2;
    const int pend = min(2 * part + 2, min(7, (gcount * kD2 + 15) / 16));
#pragma unroll 1
    for (int piece = 2 * part; piece < pend; ++piece) {
      float zm[16], zc[16];
      tmem_ld16x2(lane_base + kD1Main + piece * 16, lane_base + kD1Corr + piece * 16, zm, zc);
      if (lv) {
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const int n0 = piece * 16 + c4 * 4;        // column (g, u_b, k_b) of the chunk
          const int g = n0 / kD2, kk = n0 - g * kD2;
          if (g < gcount) {
            const float4 v = make_float4(zm[4 * c4] + zc[4 * c4], zm[4 * c4 + 1] + zc[4 * c4 + 1],
                                         zm[4 * c4 + 2] + zc[4 * c4 + 2],
                                         zm[4 * c4 + 3] + zc[4 * c4 + 3]);
            const uint32_t o = sw128_chunk(g * kD2 + dj, s * 9 + (kk >> 2), kZBlock);
            store_split4(base, kOffZH + o, kOffZL + o, v);
          }
        }
      }
    }
  };
  // D2 -> staging (parts 0-2, 16-column pieces, 36 of 48 used): the lane of
  // row (g, d_k, j_k) writes box g at row (j_k, j_b), column (d_k, d_b)
  auto drain_d2 = [&](int gcount) {
    if (part >= 3) return;
    const int L = quarter * 32 + lane;
    const int g = L / kD2, dj = L % kD2, dk = dj / 6, jk = dj % 6;
    float xm[16], xc[16];
    tmem_ld16x2(lane_base + kD2Main + 16 * part, lane_base + kD2Corr + 16 * part, xm, xc);
    if (g < gcount) {
      float* stg = reinterpret_cast<float*>(base + kOffStg + g * kStgSlot) + jk * 6 * kD2 + dk * 6;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = 16 * part + i;                 // (d_b, j_b)
        const int db = n / 6, jb = n - db * 6;
        if (n < kD2) stg[jb * kD2 + db] = xm[i] + xc[i];
      }
    }
  };

  // Per tile: wait for the ket; D1 -> Z' (quarters 0-2) while the quarter-3
  // warps write the next X1 rows; one block barrier; thread 0 issues the
  // bra's main products, thread 32 its correction products and thread 64
  // the next tile's ket; wait for the bra; D2 -> staging; one block barrier;
  // thread 0 stores the boxes (TMA) while the next ket runs.
  long long tile = blockIdx.x;
  int it = 0;
  if (tile < ntiles && quarter == 3) {
    prefetch(tile);
    store_x1(tile);
    if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tile < ntiles && tid == 64) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    issue_ket();
  }
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    const long long g0 = tile * kGT;
    const int gcount = (int)std::min<long long>(kGT, ngroups - g0);
    const long long next = tile + gridDim.x;
    const bool has_next = next < ntiles;
    // ket of this tile complete: D1 readable, the X1 planes free
    if (!mbar_wait_bounded(bar_ket, it & 1)) {
      atomicOr(err, ERRF_TIMEOUT);
      *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (quarter < 3) {
      drain_d1(gcount);
    } else if (has_next) {
      store_x1(next);
      if (next + gridDim.x < ntiles) prefetch(next + gridDim.x);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (tid == 0) bulk_wait_read_all();   // the previous tile's boxes have left the staging
    __syncthreads();
    if (tid == 0 || tid == 32 || (tid == 64 && has_next)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 64) issue_ket();
      else issue_bra(tid == 32);
    }
    // bra complete: D2 readable (the next tile's ket runs meanwhile)
    if (!mbar_wait_bounded(bar_bra, it & 1)) {
      atomicOr(err, ERRF_TIMEOUT);
      *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    drain_d2(gcount);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      for (int g = 0; g < gcount; ++g) {
        const long long G = g0 + g;
        const int mu = (int)(G / ch), bb = (int)(G % ch);
        tma_store_2d(&tmX2, bb * kD2, mu * kD2, sb + kOffStg + g * kStgSlot);
      }
      bulk_commit();
    }
  }
  // teardown: every issued MMA completes before tensor memory is freed (one
  // more commit tracks all of them), every box store before the CTA exits
  __syncthreads();
  if (tid == 0 || tid == 32 || tid == 64) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    umma_commit(bar_fin);
  }
  if (tid == 0) {
    if (!mbar_wait_bounded(bar_fin, 0)) atomicOr(err, ERRF_TIMEOUT);
    bulk_wait_all();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
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
  // 16-byte X1 row pieces; X2 rows 16-byte aligned for the TMA boxes
  if ((mp & 3) != 0 || (reinterpret_cast<uintptr_t>(X2) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(X1) & 15) != 0)
    return cudaErrorInvalidValue;
  const long long m = (long long)ch * kD2;
  if (m > (1ll << 31) - 1) return cudaErrorInvalidValue;
  CUtensorMap tm;
  if (!make_map_2d_f32(&tm, X2, m, m, mp, kD2, kD2)) return cudaErrorInvalidValue;
  const long long ngroups = (long long)ch * ch;
  cudaError_t e = device_once((const void*)absorb_tc_kernel, [] {
    return cudaFuncSetAttribute(absorb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmem);
  });
  if (e != cudaSuccess) return e;
  const long long ntiles = (ngroups + kGT - 1) / kGT;
  const unsigned grid = (unsigned)std::min<long long>(ntiles, device_sm_count());
  absorb_tc_kernel<<<grid, kThreads, kSmem, s>>>(tm, X1, Ak, Ab, ch, ngroups, err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
