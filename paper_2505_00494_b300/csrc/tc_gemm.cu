// Split-precision contraction on the 5th-generation tensor cores (tcgen05).
//
// D[b](m,n) = alpha * sum_k A[b](m,k) B[b](n,k) + beta * D[b](m,n)
//
// A and B are FP32, K-contiguous ("K-major"), read by TMA into 128-byte
// swizzled shared-memory tiles (32 FP32 of K per row).  Four converter warps
// split every element in place into a TF32 head hi = rna_tf32(x) and an FP32
// tail lo = x - hi (exact), written to a second tile of the same layout.  One
// elected thread issues, per 8-wide K slice, three kind::tf32 MMAs
//     hi(A) hi(B) + hi(A) lo(B) + lo(A) hi(B)
// into one FP32 accumulator in tensor memory (the lo*lo term, ~2^-22
// relative, is dropped; the tensor core keeps 10 mantissa bits of lo, so each
// product carries ~2^-21 relative error before FP32 accumulation).
// The same four warps then read the accumulator (tcgen05.ld) and store it
// through mixed-radix index maps in FP32 or FP64.
//
// Warp roles (192 threads): 0 = TMA producer, 1 = TMEM owner + MMA issuer,
// 2..5 = converters, then epilogue (together they cover the four TMEM lane
// quarters).  Every mbarrier wait is bounded; on timeout the kernel raises
// ERRF_TIMEOUT in the error word and unwinds (TMEM is always freed).
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "qrctm_internal.cuh"
#include "tc_gemm.cuh"

namespace qrctm {

namespace {

constexpr int BM = 128;           // rows per tile = TMEM lanes
constexpr int BK = 32;            // FP32 elements of K per swizzled row (128 B)
constexpr int NTHREADS = 192;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false on timeout or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && *abort_flag) return false;
  }
  atomicOr(err, ERRF_TIMEOUT);
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* tm, int x, int y, int z,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), version bits for the tcgen05 family.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11,"
      " %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29,"
      " %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_head(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 4;          // 16 KB
  static constexpr int B_BYTES = BN * BK * 4;
  static constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);   // x and lo tiles
  static constexpr int STAGES = std::min(4, (210 * 1024) / STAGE_BYTES);
  // main accumulator at column 0, correction accumulator at column HALF
  static constexpr int HALF = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr int TMEM_COLS = 2 * HALF;
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + 1024 + 2 * BN * 8;
};

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, const TcArgs args) {
  using C = Cfg<BN>;
  constexpr int S = C::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* tiles = base;
  unsigned char* ctrl = base + S * C::STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ctrl);        // full[S], conv[S], empty[S], accf
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + 8 * (3 * S + 1));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctrl + 8 * (3 * S + 1) + 8);
  long long* col_off = reinterpret_cast<long long*>(ctrl + 1024);
  long long* col_off32 = col_off + BN;

  auto xA = [&](int s) { return tiles + s * C::STAGE_BYTES; };
  auto loA = [&](int s) { return tiles + s * C::STAGE_BYTES + C::A_BYTES; };
  auto xB = [&](int s) { return tiles + s * C::STAGE_BYTES + 2 * C::A_BYTES; };
  auto loB = [&](int s) { return tiles + s * C::STAGE_BYTES + 2 * C::A_BYTES + C::B_BYTES; };
  const uint32_t full0 = smem_u32(&bars[0]), conv0 = smem_u32(&bars[S]),
                 empty0 = smem_u32(&bars[2 * S]), accf = smem_u32(&bars[3 * S]);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int z = blockIdx.z / args.ksplit, kz = blockIdx.z % args.ksplit;
  int issued = 0;   // TMA k-blocks issued (producer lane only)
  const int nkb_all = (int)((args.K + BK - 1) / BK);
  const int kb0 = kz * args.kb_per_split;
  const int nkb = max(0, min(nkb_all - kb0, args.kb_per_split));

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(conv0 + 8 * s, 4);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const int za = args.a_batched ? z : 0, zb = args.b_batched ? z : 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        if (kb >= S && !mbar_wait(empty0 + 8 * s, ((kb / S) - 1) & 1, abort_flag, args.err)) break;
        mbar_arrive_expect_tx(full0 + 8 * s, C::A_BYTES + C::B_BYTES);
        tma_load(smem_u32(xA(s)), &tmA, (kb0 + kb) * BK, (int)m0, za, full0 + 8 * s);
        tma_load(smem_u32(xB(s)), &tmB, (kb0 + kb) * BK, n0, zb, full0 + 8 * s);
        issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, BN);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % S;
        ok = mbar_wait(conv0 + 8 * s, (kb / S) & 1, abort_flag, args.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(xA(s)), al = smem_u32(loA(s));
        const uint32_t bh = smem_u32(xB(s)), bl = smem_u32(loB(s));
        // head*head into the main accumulator; the two head*tail terms into
        // a separate one, so that the tensor core's truncating accumulation
        // never adds ~2^-11-sized terms to the large running sum
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint32_t off = ks * 32;   // 8 TF32 = 32 bytes along K
          const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
          umma_tf32(tmem, desc_sw128(ah + off), desc_sw128(bh + off), idesc, acc);
          umma_tf32(tmem + C::HALF, desc_sw128(ah + off), desc_sw128(bl + off), idesc, acc);
          umma_tf32(tmem + C::HALF, desc_sw128(al + off), desc_sw128(bh + off), idesc, 1u);
        }
        umma_commit(empty0 + 8 * s);
      }
      umma_commit(accf);
    }
  } else {
    // ---------------- converters (warps 2..5) ----------------
    const int t = threadIdx.x - 64;   // 0..127
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(full0 + 8 * s, (kb / S) & 1, abort_flag, args.err)) break;
      float4* xa = reinterpret_cast<float4*>(xA(s));
      float4* la = reinterpret_cast<float4*>(loA(s));
#pragma unroll
      for (int i = 0; i < (BM * BK / 4) / 128; ++i) {
        const int idx = t + 128 * i;
        float4 v = xa[idx], h, l;
        h.x = tf32_head(v.x); h.y = tf32_head(v.y); h.z = tf32_head(v.z); h.w = tf32_head(v.w);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        xa[idx] = h;
        la[idx] = l;
      }
      float4* xb = reinterpret_cast<float4*>(xB(s));
      float4* lb = reinterpret_cast<float4*>(loB(s));
      for (int idx = t; idx < BN * BK / 4; idx += 128) {
        float4 v = xb[idx], h, l;
        h.x = tf32_head(v.x); h.y = tf32_head(v.y); h.z = tf32_head(v.z); h.w = tf32_head(v.w);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        xb[idx] = h;
        lb[idx] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv0 + 8 * s);
    }
    // ---------------- epilogue ----------------
    for (int j = t; j < BN; j += 128) {
      const long long n = (long long)n0 + j;
      col_off[j] = (n < args.N) ? map_off(args.c_n, n) : 0;
      if (args.C32) col_off32[j] = (n < args.N) ? map_off(args.c32_n, n) : 0;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const bool ok = mbar_wait(accf, 0, abort_flag, args.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int q = warp & 3;                 // TMEM lane quarter of this warp
      const int row = q * 32 + lane;
      const long long m = (long long)m0 + row;
      const bool mvalid = m < args.M;
      const bool split = args.ksplit > 1 || args.partials_only;
      const long long base_off =
          split ? (((long long)z * args.ksplit + kz) * args.M + (mvalid ? m : 0)) * args.N
                : map_off(args.c_b, z) + (mvalid ? map_off(args.c_m, m) : 0);
      const long long row32 = (args.C32 && mvalid) ? map_off(args.c32_m, m) : 0;
      const bool col_unit = args.c_n.nd > 0 && args.c_n.str[0] == 1;
#pragma unroll 1
      for (int c = 0; c < (BN + 31) / 32; ++c) {
        float v[32], w[32];
        const uint32_t ta = tmem + (static_cast<uint32_t>(q * 32) << 16) + c * 32;
        tmem_ld32(ta, v);
        tmem_ld32(ta + C::HALF, w);
        if (!split && !args.c_fp64 && args.beta == 0.0 && col_unit) {
          // FP32 output whose lowest column digit has unit stride: the 32 x 32
          // chunk goes through shared memory (the idle pipeline buffers: every
          // MMA has completed) and is written with the lanes along the columns
          float* stg = reinterpret_cast<float*>(tiles) + (warp & 3) * (32 * 33);
          const float al = static_cast<float>(args.alpha);
#pragma unroll
          for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = al * (v[j] + w[j]);
          __syncwarp();
          const int jj = c * 32 + lane;
          const bool cvalid = jj < BN && (long long)n0 + jj < args.N;
          const long long co = cvalid ? col_off[jj] : 0;
          float* outp = static_cast<float*>(args.C);
          for (int rr = 0; rr < 32; ++rr) {
            const long long bo = __shfl_sync(0xffffffffu, base_off, rr);
            const int valid_r = __shfl_sync(0xffffffffu, mvalid ? 1 : 0, rr);
            if (valid_r && cvalid) outp[bo + co] = stg[rr * 33 + lane];
          }
          __syncwarp();
          continue;
        }
        if (!mvalid) continue;
        if (split) {
          float* p = args.part + base_off + n0 + c * 32;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int jj = c * 32 + j;
            if (jj < BN && (long long)n0 + jj < args.N) p[j] = v[j] + w[j];
          }
          continue;
        }
        // all loads of the old values first (they would otherwise wait on
        // the stores before them), then the results
        const int nv = min(32, min(BN - c * 32, (int)(args.N - n0 - c * 32)));
        if (!args.c_fp64) {
          // FP32 output: FP32 arithmetic (B300's FP64 pipe would otherwise
          // bound the epilogue)
          const float al = static_cast<float>(args.alpha), be = static_cast<float>(args.beta);
          float* p = static_cast<float*>(args.C) + base_off;
          float o[32];
          if (be != 0.f) {
#pragma unroll
            for (int j = 0; j < 32; ++j) o[j] = (j < nv) ? p[col_off[c * 32 + j]] : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float r = al * (v[j] + w[j]);
            if (be != 0.f) r = fmaf(be, o[j], r);
            if (j < nv) p[col_off[c * 32 + j]] = r;
          }
          continue;
        }
        double r[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = args.alpha * static_cast<double>(v[j] + w[j]);
        if (args.beta != 0.0) {
          double old[32];
          const double* p = static_cast<const double*>(args.C) + base_off;
#pragma unroll
          for (int j = 0; j < 32; ++j) old[j] = (j < nv) ? p[col_off[c * 32 + j]] : 0.0;
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = fma(args.beta, old[j], r[j]);
        }
        {
          double* p = static_cast<double*>(args.C) + base_off;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nv) p[col_off[c * 32 + j]] = r[j];
          if (args.C32) {
            float* p32 = args.C32 + row32;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv) p32[col_off32[c * 32 + j]] = static_cast<float>(r[j]);
          }
        }
      }
    }
  }
  // teardown: the TMEM owner frees the accumulator after everyone is done
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && warp == 0 && lane == 0) {
    // drain TMA copies that may still be in flight before the CTA exits:
    // wait (bounded) for the last issued use of every stage
    for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb)
      for (uint32_t i = 0; i < (1u << 20); ++i)
        if (mbar_try_wait(full0 + 8 * (kb % S), (kb / S) & 1)) break;
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Persistent variant (BN <= 128): one CTA per SM walks the output tiles; the
// TMEM accumulator pair is double buffered so that four dedicated epilogue
// warps drain tile i while the MMA warp already accumulates tile i + 1, and
// the TMA / converter ring runs on across tile boundaries.
//
// Warps (320 threads): 0 = TMA producer, 1 = TMEM owner + MMA issuer,
// 2..5 = converters, 6..9 = epilogue (warp w reads TMEM lane quarter w % 4).
// ---------------------------------------------------------------------------
constexpr int NTHREADS_P = 320;

template <int BN>
struct CfgP {
  static constexpr int A_BYTES = BM * BK * 4;
  static constexpr int B_BYTES = BN * BK * 4;
  static constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);
  static constexpr int STG_BYTES = 4 * 32 * 33 * 4;                 // epilogue staging
  // as many ring stages as fit the 227 KB opt-in limit next to the rest
  static constexpr int STAGES =
      std::min(4, (232448 - 2048 - STG_BYTES - 2 * BN * 8) / STAGE_BYTES);
  static constexpr int HALF = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;
  static constexpr int TMEM_COLS = 4 * HALF;                        // 2 buffers x (main, corr)
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + STG_BYTES + 1024 + 2 * BN * 8;
};

template <int BN>
__global__ void __launch_bounds__(NTHREADS_P, 1)
    tc_tf32x3_persist(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const TcArgs args) {
  using C = CfgP<BN>;
  static_assert(BN <= 128, "double-buffered accumulators need BN <= 128");
  constexpr int S = C::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* tiles = base;
  float* stg_all = reinterpret_cast<float*>(base + S * C::STAGE_BYTES);
  unsigned char* ctrl = base + S * C::STAGE_BYTES + C::STG_BYTES;
  // full[S], conv[S], empty[S], accf[2], acce[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ctrl);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + 8 * (3 * S + 4));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctrl + 8 * (3 * S + 4) + 8);
  volatile int* epi_stop = reinterpret_cast<volatile int*>(ctrl + 8 * (3 * S + 4) + 16);
  long long* col_off = reinterpret_cast<long long*>(ctrl + 1024);
  long long* col_off32 = col_off + BN;

  auto xA = [&](int s) { return tiles + s * C::STAGE_BYTES; };
  auto loA = [&](int s) { return tiles + s * C::STAGE_BYTES + C::A_BYTES; };
  auto xB = [&](int s) { return tiles + s * C::STAGE_BYTES + 2 * C::A_BYTES; };
  auto loB = [&](int s) { return tiles + s * C::STAGE_BYTES + 2 * C::A_BYTES + C::B_BYTES; };
  const uint32_t full0 = smem_u32(&bars[0]), conv0 = smem_u32(&bars[S]),
                 empty0 = smem_u32(&bars[2 * S]), accf0 = smem_u32(&bars[3 * S]),
                 acce0 = smem_u32(&bars[3 * S + 2]);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long mt = (args.M + BM - 1) / BM, nt = (args.N + BN - 1) / BN;
  const long long zt = (long long)args.batch * args.ksplit;
  const long long ntiles = mt * nt * zt;
  const int nkb_all = (int)((args.K + BK - 1) / BK);
  // tile t -> (z, kz, m0, n0), n fastest
  auto tile_of = [&](long long t, int& z, int& kz, long long& m0, int& n0, int& nkb, int& kb0) {
    const long long tn = t % nt, tm = (t / nt) % mt, tz = t / (nt * mt);
    z = (int)(tz / args.ksplit);
    kz = (int)(tz % args.ksplit);
    m0 = tm * BM;
    n0 = (int)(tn * BN);
    kb0 = kz * args.kb_per_split;
    nkb = max(0, min(nkb_all - kb0, args.kb_per_split));
  };
  int issued = 0;   // TMA k-blocks issued (producer lane only)

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(conv0 + 8 * s, 4);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);
    }
    *abort_flag = 0;
    *epi_stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int kbg = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int z, kz, n0, nkb, kb0;
        long long m0;
        tile_of(t, z, kz, m0, n0, nkb, kb0);
        const int za = args.a_batched ? z : 0, zb = args.b_batched ? z : 0;
        for (int kb = 0; kb < nkb; ++kb, ++kbg) {
          const int s = kbg % S;
          if (kbg >= S && !mbar_wait(empty0 + 8 * s, ((kbg / S) - 1) & 1, abort_flag, args.err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full0 + 8 * s, C::A_BYTES + C::B_BYTES);
          tma_load(smem_u32(xA(s)), &tmA, (kb0 + kb) * BK, (int)m0, za, full0 + 8 * s);
          tma_load(smem_u32(xB(s)), &tmB, (kb0 + kb) * BK, n0, zb, full0 + 8 * s);
          issued = kbg + 1;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, BN);
      int kbg = 0, it = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        int z, kz, n0, nkb, kb0;
        long long m0;
        tile_of(t, z, kz, m0, n0, nkb, kb0);
        const int ab = it & 1;
        // the epilogue must have drained this accumulator buffer (use it - 2)
        if (it >= 2 && !mbar_wait(acce0 + 8 * ab, ((it >> 1) - 1) & 1, abort_flag, args.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dmain = tmem + ab * 2 * C::HALF, dcorr = dmain + C::HALF;
        for (int kb = 0; kb < nkb; ++kb, ++kbg) {
          const int s = kbg % S;
          ok = mbar_wait(conv0 + 8 * s, (kbg / S) & 1, abort_flag, args.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = smem_u32(xA(s)), al = smem_u32(loA(s));
          const uint32_t bh = smem_u32(xB(s)), bl = smem_u32(loB(s));
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint32_t off = ks * 32;
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            umma_tf32(dmain, desc_sw128(ah + off), desc_sw128(bh + off), idesc, acc);
            umma_tf32(dcorr, desc_sw128(ah + off), desc_sw128(bl + off), idesc, acc);
            umma_tf32(dcorr, desc_sw128(al + off), desc_sw128(bh + off), idesc, 1u);
          }
          umma_commit(empty0 + 8 * s);
        }
        if (ok) umma_commit(accf0 + 8 * ab);
      }
    }
  } else if (warp < 6) {
    // ---------------- converters (warps 2..5) ----------------
    const int t4 = threadIdx.x - 64;   // 0..127
    int kbg = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int z, kz, n0, nkb, kb0;
      long long m0;
      tile_of(t, z, kz, m0, n0, nkb, kb0);
      for (int kb = 0; kb < nkb; ++kb, ++kbg) {
        const int s = kbg % S;
        if (!mbar_wait(full0 + 8 * s, (kbg / S) & 1, abort_flag, args.err)) {
          ok = false;
          break;
        }
        float4* xa = reinterpret_cast<float4*>(xA(s));
        float4* la = reinterpret_cast<float4*>(loA(s));
#pragma unroll
        for (int i = 0; i < (BM * BK / 4) / 128; ++i) {
          const int idx = t4 + 128 * i;
          float4 v = xa[idx], h, l;
          h.x = tf32_head(v.x); h.y = tf32_head(v.y); h.z = tf32_head(v.z); h.w = tf32_head(v.w);
          l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
          xa[idx] = h;
          la[idx] = l;
        }
        float4* xb = reinterpret_cast<float4*>(xB(s));
        float4* lb = reinterpret_cast<float4*>(loB(s));
        for (int idx = t4; idx < BN * BK / 4; idx += 128) {
          float4 v = xb[idx], h, l;
          h.x = tf32_head(v.x); h.y = tf32_head(v.y); h.z = tf32_head(v.z); h.w = tf32_head(v.w);
          l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
          xb[idx] = h;
          lb[idx] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(conv0 + 8 * s);
      }
    }
  } else {
    // ---------------- epilogue (warps 6..9) ----------------
    const int te = threadIdx.x - 192;   // 0..127
    const int q = warp & 3;             // TMEM lane quarter of this warp
    float* stg = stg_all + q * (32 * 33);
    const bool col_unit = args.c_n.nd > 0 && args.c_n.str[0] == 1;
    const bool split = args.ksplit > 1 || args.partials_only;
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      int z, kz, n0, nkb, kb0;
      long long m0;
      tile_of(t, z, kz, m0, n0, nkb, kb0);
      const int ab = it & 1;
      asm volatile("bar.sync 2, 128;" ::: "memory");   // previous tile's offsets are dead
      for (int j = te; j < BN; j += 128) {
        const long long n = (long long)n0 + j;
        col_off[j] = (n < args.N) ? map_off(args.c_n, n) : 0;
        if (args.C32) col_off32[j] = (n < args.N) ? map_off(args.c32_n, n) : 0;
      }
      asm volatile("bar.sync 2, 128;" ::: "memory");
      // a failed wait stops all four epilogue warps together: the flag is
      // written only before the barrier below and read only after it
      if (!mbar_wait(accf0 + 8 * ab, (it >> 1) & 1, abort_flag, args.err) && lane == 0)
        *epi_stop = 1;
      asm volatile("bar.sync 2, 128;" ::: "memory");
      if (*epi_stop) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = q * 32 + lane;
      const long long m = m0 + row;
      const bool mvalid = m < args.M;
      const long long base_off =
          split ? (((long long)z * args.ksplit + kz) * args.M + (mvalid ? m : 0)) * args.N
                : map_off(args.c_b, z) + (mvalid ? map_off(args.c_m, m) : 0);
      const long long row32 = (args.C32 && mvalid) ? map_off(args.c32_m, m) : 0;
      const uint32_t dmain = tmem + ab * 2 * C::HALF;
#pragma unroll 1
      for (int c = 0; c < (BN + 31) / 32; ++c) {
        float v[32], w[32];
        const uint32_t ta = dmain + (static_cast<uint32_t>(q * 32) << 16) + c * 32;
        tmem_ld32(ta, v);
        tmem_ld32(ta + C::HALF, w);
        const int nv = min(32, min(BN - c * 32, (int)(args.N - n0 - c * 32)));
        if (!split && !args.c_fp64 && args.beta == 0.0 && col_unit) {
          const float al = static_cast<float>(args.alpha);
#pragma unroll
          for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = al * (v[j] + w[j]);
          __syncwarp();
          const bool cvalid = lane < nv;
          const long long co = cvalid ? col_off[c * 32 + lane] : 0;
          float* outp = static_cast<float*>(args.C);
          for (int rr = 0; rr < 32; ++rr) {
            const long long bo = __shfl_sync(0xffffffffu, base_off, rr);
            const int valid_r = __shfl_sync(0xffffffffu, mvalid ? 1 : 0, rr);
            if (valid_r && cvalid) outp[bo + co] = stg[rr * 33 + lane];
          }
          __syncwarp();
          continue;
        }
        if (!mvalid) continue;
        if (split) {
          float* p = args.part + base_off + n0 + c * 32;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nv) p[j] = v[j] + w[j];
          continue;
        }
        if (!args.c_fp64) {
          const float al = static_cast<float>(args.alpha), be = static_cast<float>(args.beta);
          float* p = static_cast<float*>(args.C) + base_off;
          float o[32];
          if (be != 0.f) {
#pragma unroll
            for (int j = 0; j < 32; ++j) o[j] = (j < nv) ? p[col_off[c * 32 + j]] : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float r = al * (v[j] + w[j]);
            if (be != 0.f) r = fmaf(be, o[j], r);
            if (j < nv) p[col_off[c * 32 + j]] = r;
          }
          continue;
        }
        double r[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = args.alpha * static_cast<double>(v[j] + w[j]);
        double* p = static_cast<double*>(args.C) + base_off;
        if (args.beta != 0.0) {
          double old[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) old[j] = (j < nv) ? p[col_off[c * 32 + j]] : 0.0;
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = fma(args.beta, old[j], r[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nv) p[col_off[c * 32 + j]] = r[j];
        if (args.C32) {
          float* p32 = args.C32 + row32;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nv) p32[col_off32[c * 32 + j]] = static_cast<float>(r[j]);
        }
      }
      // this accumulator buffer may be overwritten by tile it + 2
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * ab);
    }
  }
  // teardown: the TMEM owner frees the accumulators after everyone is done
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && warp == 0 && lane == 0) {
    for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb)
      for (uint32_t i = 0; i < (1u << 20); ++i)
        if (mbar_try_wait(full0 + 8 * (kb % S), (kb / S) & 1)) break;
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// out(b,m,n) = alpha * sum_z part[b][z][m][n] + beta * out: FP64 sums in a
// fixed order (four interleaved partial sums, then their pairwise sum)
__global__ void tc_splitk_reduce(const TcArgs a, int batch) {
  const long long MN = a.M * a.N;
  const long long tot = MN * batch;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / MN, r = e % MN, m = r / a.N, n = r % a.N;
    const float* p = a.part + b * a.ksplit * MN + r;
    // compensated FP32 sum (TwoSum per term, Knuth): s + c carries the sum of
    // the partials to ~2^-48 of their magnitude, like an FP64 sum, at FP32
    // speed (B300's FP64 pipe would bound this pass)
    float sh = 0.f, se = 0.f;
    for (int z = 0; z < a.ksplit; ++z) {
      const float x = p[(long long)z * MN];
      const float t = sh + x;
      const float bp = t - sh;
      se += (sh - (t - bp)) + (x - bp);
      sh = t;
    }
    const double acc = static_cast<double>(sh) + static_cast<double>(se);
    const long long off = map_off(a.c_b, b) + map_off(a.c_m, m) + map_off(a.c_n, n);
    double v = a.alpha * acc;
    if (a.c_fp64) {
      double* o = static_cast<double*>(a.C) + off;
      if (a.beta != 0.0) v += a.beta * *o;
      *o = v;
      if (a.C32) a.C32[map_off(a.c32_m, m) + map_off(a.c32_n, n)] = static_cast<float>(v);
    } else {
      float* o = static_cast<float*>(a.C) + off;
      if (a.beta != 0.0) v += a.beta * static_cast<double>(*o);
      *o = static_cast<float>(v);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// 3-D map over (K, rows, batch) of FP32, box (32, box_rows, 1), 128-byte swizzle.
bool make_map(CUtensorMap* tm, const TcOperand& op, int box_rows) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(op.ptr) & 15) != 0) return false;
  if ((op.row_stride * 4) % 16 != 0 || (op.batch_stride * 4) % 16 != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows,
                        (cuuint64_t)(op.batch > 0 ? op.batch : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)op.row_stride * 4,
                           (cuuint64_t)(op.batch_stride > 0 ? op.batch_stride : op.row_stride *
                                                                                   op.rows) * 4};
  cuuint32_t box[3] = {BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(op.ptr), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, bool PERSIST>
cudaError_t launch_bn(const TcGemm& g, cudaStream_t s) {
  const int smem_bytes = PERSIST ? CfgP<BN>::SMEM : Cfg<BN>::SMEM;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = PERSIST ? cudaFuncSetAttribute(tc_tf32x3_persist<BN <= 128 ? BN : 128>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem_bytes)
                            : cudaFuncSetAttribute(tc_tf32x3_kernel<BN>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem_bytes);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  CUtensorMap ta, tb;
  if (!make_map(&ta, g.A, BM) || !make_map(&tb, g.B, BN)) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = g.M; a.N = g.N; a.K = g.K;
  a.C = g.C; a.c_fp64 = g.c_fp64 ? 1 : 0;
  a.c_m = g.c_m; a.c_n = g.c_n; a.c_b = g.c_b;
  a.alpha = g.alpha; a.beta = g.beta;
  a.a_batched = g.A.batch > 1 ? 1 : 0;
  a.b_batched = g.B.batch > 1 ? 1 : 0;
  a.err = g.err;
  // K chunks: at most 512 of K (16 blocks) per chunk, more chunks when the
  // output grid alone cannot fill the GPU; partials are summed by compensated
  // FP32 arithmetic
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const long long tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * std::max(1, g.batch);
  const int nkb = (int)((g.K + BK - 1) / BK);
  int ksplit = 1, kbps = nkb;
  if (g.part != nullptr && nkb > 2) {
    // K within one 512-wide chunk: split for occupancy only when the output
    // grid is far too small for the GPU (otherwise the reduction pass costs
    // more than the shorter K loop saves)
    const bool fill = nkb > 16 || tiles * 4 < nsm;
    long long want = std::max<long long>((nkb + 15) / 16,
                                         fill ? (2ll * nsm + tiles - 1) / tiles : 1);
    want = std::min<long long>(want, nkb / 2);
    const long long cap = g.part_elems / (g.M * g.N * std::max(1, g.batch));
    want = std::min<long long>(want, cap);
    if (g.max_ksplit > 0) want = std::min<long long>(want, g.max_ksplit);
    if (want > 1) {
      kbps = (int)((nkb + want - 1) / want);
      ksplit = (nkb + kbps - 1) / kbps;
    }
  }
  if (g.partials_only) {
    if (g.part == nullptr ||
        (long long)ksplit * g.M * g.N * std::max(1, g.batch) > g.part_elems)
      return cudaErrorInvalidValue;
    if (g.ksplit_out) *g.ksplit_out = ksplit;
  }
  if (g.C32 != nullptr && (!g.c_fp64 || g.batch > 1)) return cudaErrorInvalidValue;
  a.ksplit = ksplit;
  a.kb_per_split = kbps;
  a.part = g.part;
  a.partials_only = g.partials_only ? 1 : 0;
  a.C32 = g.C32;
  a.c32_m = g.c32_m;
  a.c32_n = g.c32_n;
  if ((long long)std::max(1, g.batch) * ksplit > 65535) return cudaErrorInvalidValue;
  a.batch = std::max(1, g.batch);
  if (PERSIST) {
    const long long ntiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * a.batch * ksplit;
    const unsigned grid = (unsigned)std::min<long long>(ntiles, nsm);
    tc_tf32x3_persist<BN <= 128 ? BN : 128><<<grid, NTHREADS_P, smem_bytes, s>>>(ta, tb, a);
  } else {
    dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN),
              (unsigned)(std::max(1, g.batch) * ksplit));
    tc_tf32x3_kernel<BN><<<grid, NTHREADS, smem_bytes, s>>>(ta, tb, a);
  }
  note_launch();
  if (ksplit > 1 && !g.partials_only) {
    const long long tot = g.M * g.N * std::max(1, g.batch);
    tc_splitk_reduce<<<(unsigned)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(
        a, std::max(1, g.batch));
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_tc(const TcGemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (g.A.rows < 1 || g.B.rows < 1 || g.A.K != g.K || g.B.K != g.K) return cudaErrorInvalidValue;
  if (g.batch > 65535 || g.M > (1ll << 31) - BM) return cudaErrorInvalidValue;
  // the persistent kernel (double-buffered accumulators, BN <= 128) except
  // for 128 < N <= 256, where one wider tile avoids re-reading A per N tile
  const long long N = g.N;
  if (N <= 32) return launch_bn<32, true>(g, s);
  if (N <= 48) return launch_bn<48, true>(g, s);
  if (N <= 64) return launch_bn<64, true>(g, s);
  if (N <= 80) return launch_bn<80, true>(g, s);
  if (N <= 128) return launch_bn<128, true>(g, s);
  if (N <= 144) return launch_bn<144, false>(g, s);
  if (N <= 256) return launch_bn<256, false>(g, s);
  return launch_bn<128, true>(g, s);
}

}  // namespace qrctm
