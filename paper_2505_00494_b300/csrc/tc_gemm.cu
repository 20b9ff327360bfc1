// Split-precision contraction on the 5th-generation tensor cores (tcgen05).
//
// D[b](m,n) = alpha * sum_k A[b](m,k) B[b](n,k) + beta * D[b](m,n)
//
// A and B are FP32, K-contiguous ("K-major"), read by TMA into 128-byte
// swizzled shared-memory tiles (32 FP32 of K per row).  Every element is split
// into a TF32 head and a TF32 tail, and one elected thread issues, per 8-wide
// K slice, three kind::tf32 MMAs
//     head(A) head(B) -> main,   head(A) tail(B) + tail(A) head(B) -> corr
// into two FP32 accumulators in tensor memory, summed by the epilogue, which
// stores the result through mixed-radix index maps in FP32 or FP64.  A is
// staged into tensor memory (the MMAs read it there), B stays in shared
// memory; the kernel below describes the split and the warp roles.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "qrctm_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace qrctm {

namespace {

constexpr int BM = 128;           // rows per tile = TMEM lanes
constexpr int BK = 32;            // FP32 elements of K per swizzled row (128 B)
constexpr int NTHREADS = 320;     // 2 + 4 converter + 4 epilogue warps
constexpr int NCONV = 4;          // converter warps

using namespace ptx;

// Bounded wait of the pipeline roles: gives up when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  return mbar_wait_abortable(bar, parity, abort_flag, err, ERRF_TIMEOUT);
}


// alpha * (double) x with no FP64 multiply for alpha = +-1 (alpha is the same
// for the whole launch): on B300 the widening itself already issues at the
// FP64 rate
__device__ __forceinline__ double widen_scaled(double alpha, float x) {
  if (alpha == 1.0) return static_cast<double>(x);
  if (alpha == -1.0) return static_cast<double>(-x);
  return alpha * static_cast<double>(x);
}

// ---------------------------------------------------------------------------
// Epilogue (both kernels).  The 128 epilogue threads first fill the tile's
// output offsets in shared memory (one row each, columns strided); each warp
// then drains the 32 accumulator rows of its TMEM lane quarter in 32 x 32
// chunks: main + correction summed, staged transposed in shared memory and
// written one row per instruction with the lanes along the columns (coalesced
// where the lowest column digit has unit stride; the row loop is unrolled so
// that many stores are in flight).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void epi_offsets(const TcArgs& a, int bn, int t, long long m0, int n0,
                                            int z, int kz, long long* col_off,
                                            long long* col_off32, long long* row_off,
                                            long long* row_off32) {
  const bool split = a.ksplit > 1 || a.partials_only;
  // (M, N < 2^31: the index maps take their digits with 32-bit divisions)
  for (int j = t; j < bn; j += 128) {
    const long long n = (long long)n0 + j;
    const bool ok = n < a.N;
    // split partials: part[b][z][m][n], the column index itself
    col_off[j] = split ? n : (ok ? map_off32(a.c_n, (unsigned)n) : 0);
    if (a.C32) col_off32[j] = ok ? map_off32(a.c32_n, (unsigned)n) : 0;
  }
  const long long m = m0 + t;
  const bool ok = m < a.M;
  row_off[t] = split ? (((long long)z * a.ksplit + kz) * a.M + (ok ? m : 0)) * a.N
                     : map_off32(a.c_b, (unsigned)z) + (ok ? map_off32(a.c_m, (unsigned)m) : 0);
  if (a.C32) row_off32[t] = ok ? map_off32(a.c32_m, (unsigned)m) : 0;
}

template <int BN>
__device__ __forceinline__ void epi_rows(const TcArgs& a, uint32_t acc, uint32_t half, int q,
                                         int lane, long long m0, int n0, float* stg,
                                         const long long* col_off, const long long* col_off32,
                                         const long long* row_off, const long long* row_off32) {
  const bool split = a.ksplit > 1 || a.partials_only;
  const long long rv = a.M - m0 - q * 32;
  if (rv <= 0) return;                      // warp-uniform: no valid row in this quarter
  const int rows = rv < 32 ? (int)rv : 32;
  const long long* ro = row_off + q * 32;
  const long long* ro32 = row_off32 + q * 32;
  // an output whose rows, not columns, are contiguous is written with the
  // lanes along the rows (one lane = one accumulator row: no staging)
  const bool row_major_out = split || (a.c_n.nd > 0 && a.c_n.str[0] == 1);
  if (!row_major_out && a.c_m.nd > 0 && a.c_m.str[0] == 1) {
    const bool rvalid = lane < rows;
    const long long myro = rvalid ? ro[lane] : 0;
    const long long myro32 = (rvalid && a.C32) ? ro32[lane] : 0;
#pragma unroll 1
    for (int c = 0; c < (BN + 31) / 32; ++c) {
      float v[32], w[32];
      const uint32_t ta = acc + (static_cast<uint32_t>(q * 32) << 16) + c * 32;
      tmem_ld32(ta, v);
      tmem_ld32(ta + half, w);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += w[j];
      if (!rvalid) continue;
      const long long nrem = a.N - n0 - c * 32;
      const int nv = (int)(nrem < BN - c * 32 ? nrem : BN - c * 32);   // valid if j < nv
      // a one-digit column map is computed, not read from shared memory;
      // either way each half's offsets and old values are loaded before its
      // stores (the compiler cannot move shared-memory loads across global
      // stores it cannot prove disjoint)
      const bool cn1 = a.c_n.nd == 1;
      const long long cs = a.c_n.str[0], nc0 = (long long)n0 + c * 32;
      auto coff = [&](int j) -> long long {
        return cn1 ? (nc0 + j) * cs : col_off[c * 32 + (j < nv ? j : 0)];
      };
      if (!a.c_fp64) {
        float* p = static_cast<float*>(a.C) + myro;
        const float al = static_cast<float>(a.alpha), be = static_cast<float>(a.beta);
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 16) {   // halves: 16 loads in flight
          long long o[16];
          float r[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) o[u] = coff(j0 + u);
#pragma unroll
          for (int u = 0; u < 16; ++u) r[u] = al * v[j0 + u];
          if (be != 0.f) {
            float old[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) old[u] = (j0 + u < nv) ? p[o[u]] : 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) r[u] = fmaf(be, old[u], r[u]);
          }
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (j0 + u < nv) p[o[u]] = r[u];
        }
      } else {
        double* p = static_cast<double*>(a.C) + myro;
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 16) {   // halves: 16 doubles in flight
          long long o[16];
          double r[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) o[u] = coff(j0 + u);
          if (a.beta != 0.0) {
#pragma unroll
            for (int u = 0; u < 16; ++u) r[u] = (j0 + u < nv) ? p[o[u]] : 0.0;
#pragma unroll
            for (int u = 0; u < 16; ++u)
              r[u] = fma(a.beta, r[u], widen_scaled(a.alpha, v[j0 + u]));
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) r[u] = widen_scaled(a.alpha, v[j0 + u]);
          }
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (j0 + u < nv) p[o[u]] = r[u];
          if (a.C32) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (j0 + u < nv)
                a.C32[myro32 + col_off32[c * 32 + j0 + u]] = static_cast<float>(r[u]);
          }
        }
      }
    }
    return;
  }
  // FP32 rows contiguous in n (split-K partials, or an FP32 output whose
  // column map is the identity): each thread stores its own row's 32 columns
  // from its registers, in 16-byte pieces where the row start allows, with
  // no staging and no per-element offsets
  if (split || (!a.c_fp64 && a.c_n.nd == 1 && a.c_n.str[0] == 1)) {
    const bool rvalid = lane < rows;
    float* base = split ? a.part : static_cast<float*>(a.C);
    const long long myro = rvalid ? ro[lane] : 0;
    const float al = split ? 1.f : static_cast<float>(a.alpha);
    const float be = split ? 0.f : static_cast<float>(a.beta);
#pragma unroll 1
    for (int c = 0; c < (BN + 31) / 32; ++c) {
      float v[32], w[32];
      const uint32_t ta = acc + (static_cast<uint32_t>(q * 32) << 16) + c * 32;
      tmem_ld32(ta, v);
      tmem_ld32(ta + half, w);
      const long long nrem = a.N - n0 - c * 32;
      if (!rvalid || nrem <= 0) continue;
      const int nv = nrem < 32 ? (int)nrem : 32;
      float* p = base + myro + n0 + c * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = al * (v[j] + w[j]);
      if (nv == 32 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        float4* p4 = reinterpret_cast<float4*>(p);
        if (be != 0.f) {
          float4 old[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) old[u] = p4[u];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            v[4 * u] = fmaf(be, old[u].x, v[4 * u]);
            v[4 * u + 1] = fmaf(be, old[u].y, v[4 * u + 1]);
            v[4 * u + 2] = fmaf(be, old[u].z, v[4 * u + 2]);
            v[4 * u + 3] = fmaf(be, old[u].w, v[4 * u + 3]);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          p4[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nv) p[j] = (be != 0.f) ? fmaf(be, p[j], v[j]) : v[j];
      }
    }
    return;
  }
#pragma unroll 1
  for (int c = 0; c < (BN + 31) / 32; ++c) {
    float v[32], w[32];
    const uint32_t ta = acc + (static_cast<uint32_t>(q * 32) << 16) + c * 32;
    tmem_ld32(ta, v);
    tmem_ld32(ta + half, w);
#pragma unroll
    for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j] + w[j];
    __syncwarp();
    const int jj = c * 32 + lane;
    const bool cvalid = jj < BN && (long long)n0 + jj < a.N;
    // rows in groups of 8: offsets and staged values are loaded before the
    // group's stores (the compiler cannot move shared-memory loads across
    // global stores it cannot prove disjoint)
    if (cvalid) {
      const long long co = col_off[jj];
      const long long co32 = (a.c_fp64 && a.C32) ? col_off32[jj] : 0;
#pragma unroll 1
      for (int r0 = 0; r0 < rows; r0 += 8) {
        long long o[8], o32[8];
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          o[u] = ro[r0 + u] + co;
          x[u] = stg[(r0 + u) * 33 + lane];
          if (a.C32) o32[u] = ro32[r0 + u] + co32;
        }
        if (split) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (r0 + u < rows) a.part[o[u]] = x[u];
        } else if (!a.c_fp64) {
          // FP32 output in FP32 arithmetic (B300's FP64 pipe would bound it)
          float* p = static_cast<float*>(a.C);
          const float al = static_cast<float>(a.alpha), be = static_cast<float>(a.beta);
          if (be != 0.f) {
            float old[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) old[u] = (r0 + u < rows) ? p[o[u]] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = fmaf(be, old[u], al * x[u]);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] *= al;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (r0 + u < rows) p[o[u]] = x[u];
        } else {
          double* p = static_cast<double*>(a.C);
          double r[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) r[u] = widen_scaled(a.alpha, x[u]);
          if (a.beta != 0.0) {
            double old[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) old[u] = (r0 + u < rows) ? p[o[u]] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) r[u] = fma(a.beta, old[u], r[u]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (r0 + u < rows) p[o[u]] = r[u];
          if (a.C32) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (r0 + u < rows) a.C32[o32[u]] = static_cast<float>(r[u]);
          }
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// The kernel.  Tile = 128 rows (TMEM lanes) x BN columns; NBUF accumulator
// buffers, each a (main, correction) pair of BN-wide FP32 regions in tensor
// memory.  NBUF = 2: persistent (one CTA per SM walks the tiles; the epilogue
// drains tile i while the MMAs accumulate tile i + 1).  NBUF = 1: one tile
// per CTA (the wide-N shapes, whose accumulators leave no room for a second
// buffer).
//
// Split of an FP32 value x (TF32x3): head = rna_tf32(x), tail = rna_tf32(x -
// head), with x - head exact in FP32 and |tail| <= 2^-11 |x|; the two
// roundings leave x represented to 2^-22 |x| and the dropped tail(A) tail(B)
// term is below 2^-22 |ab|.  Rounding is an integer add and mask on the bit
// pattern (round half away from zero at bit 13): the conversion
// instruction's throughput would bound the kernel.  A NaN x keeps itself as
// head, so it reaches the result.
//
// Operand staging: TMA brings the raw A (128 x 32) and B (BN x 32) tiles of
// each 32-wide K block into shared memory.  Four converter warps then
//   * split B in shared memory: head in place of the raw tile, tail plane
//     beside it, and
//   * move the A tile into tensor memory, head and tail side by side (each
//     thread one row = one TMEM lane),
// so that the three MMAs per 8-wide K slice,
//     head(A) head(B) -> main,  head(A) tail(B) + tail(A) head(B) -> corr,
// read A from tensor memory and only B from shared memory: the contraction
// is bound by shared-memory bandwidth, and this removes the three reads of A
// per K slice and the A planes from it.
//
// Warps (320 threads): 0 = TMA producer, 1 = TMEM owner + MMA issuer,
// 2..5 = converters (warp w: the rows of TMEM lane quarter w % 4),
// 6..9 = epilogue.  Every mbarrier wait is
// bounded; on timeout the kernel raises ERRF_TIMEOUT in the error word and
// unwinds (TMEM is always freed).
// ---------------------------------------------------------------------------
template <int BN, int NBUF, int PRE>
struct Cfg {
  static constexpr bool PRE_A = PRE == 2, PRE_B = PRE >= 1;
  static constexpr int A_BYTES = BM * BK * 4;                       // 16 KB
  static constexpr int B_BYTES = BN * BK * 4;
  static constexpr int A_PLANES = PRE_A ? 2 : 1;
  // A (and tail(A) when A comes pre-split), B, tail(B)
  static constexpr int STAGE_BYTES = A_PLANES * A_BYTES + 2 * B_BYTES;
  static constexpr int TX_BYTES = A_PLANES * A_BYTES + (PRE_B ? 2 : 1) * B_BYTES;
  static constexpr int STG_BYTES = 4 * 32 * 33 * 4;                 // epilogue staging
  static constexpr int OFF_BYTES = 2 * BN * 8 + 2 * BM * 8;         // column and row offsets
  static constexpr int STAGES =
      std::min(4, (232448 - 2048 - STG_BYTES - OFF_BYTES) / STAGE_BYTES);
  static constexpr int HALF = (BN + 31) / 32 * 32;                  // TMEM columns per region
  static constexpr int ACC_COLS = NBUF * 2 * HALF;
  // (head, tail) x 32 columns per A stage; none when A comes pre-split (read from shared memory)
  static constexpr int A_STAGES = PRE_A ? 0 : std::min(4, (512 - ACC_COLS) / 64);
  static constexpr int A_COL0 = ACC_COLS;
  static constexpr int TMEM_COLS = 512;
  static constexpr int NBAR = 3 * STAGES + A_STAGES + 2 * NBUF;
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + STG_BYTES + 1024 + OFF_BYTES;
  static_assert(STAGES >= 2 && (PRE_A || A_STAGES >= 2), "tile does not fit the SM");
  static_assert(ACC_COLS + 64 * A_STAGES <= TMEM_COLS, "tensor memory overflow");
  static_assert(8 * NBAR + 24 <= 1024, "control block overflow");
};

template <int BN, int NBUF, int PRE>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmAlo,
                     const __grid_constant__ CUtensorMap tmBlo, const TcArgs args) {
  using C = Cfg<BN, NBUF, PRE>;
  constexpr int S = C::STAGES, AS = C::A_STAGES, ASM = AS > 0 ? AS : 1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* tiles = base;
  float* stg_all = reinterpret_cast<float*>(base + S * C::STAGE_BYTES);
  unsigned char* ctrl = base + S * C::STAGE_BYTES + C::STG_BYTES;
  // full[S], conv[S], empty[S], tfree[AS], accf[NBUF], acce[NBUF]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ctrl);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + 8 * C::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctrl + 8 * C::NBAR + 8);
  volatile int* epi_stop = reinterpret_cast<volatile int*>(ctrl + 8 * C::NBAR + 16);
  long long* col_off = reinterpret_cast<long long*>(ctrl + 1024);
  long long* col_off32 = col_off + BN;
  long long* row_off = col_off32 + BN;
  long long* row_off32 = row_off + BM;

  auto xA = [&](int s) { return tiles + s * C::STAGE_BYTES; };
  auto loA = [&](int s) { return tiles + s * C::STAGE_BYTES + C::A_BYTES; };   // PRE_A only
  auto xB = [&](int s) { return tiles + s * C::STAGE_BYTES + C::A_PLANES * C::A_BYTES; };
  auto loB = [&](int s) {
    return tiles + s * C::STAGE_BYTES + C::A_PLANES * C::A_BYTES + C::B_BYTES;
  };
  const uint32_t full0 = smem_u32(&bars[0]), conv0 = smem_u32(&bars[S]),
                 empty0 = smem_u32(&bars[2 * S]), tfree0 = smem_u32(&bars[3 * S]),
                 accf0 = smem_u32(&bars[3 * S + AS]), acce0 = smem_u32(&bars[3 * S + AS + NBUF]);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long mt = (args.M + BM - 1) / BM, nt = (args.N + BN - 1) / BN;
  const long long zt = (long long)args.batch * args.ksplit;
  const long long ntiles = mt * nt * zt;
  const int nkb_all = (int)((args.K + BK - 1) / BK);
  // tile t -> (z, kz, m0, n0), n fastest (neighbouring CTAs share A rows in L2);
  // the host keeps the tile count below 2^31, so 32-bit divisions suffice
  const unsigned ntu = (unsigned)nt, mtu = (unsigned)mt, ksu = (unsigned)args.ksplit;
  auto tile_of = [&](long long t, int& z, int& kz, long long& m0, int& n0, int& nkb, int& kb0) {
    const unsigned tu = (unsigned)t, q = tu / ntu, tn = tu - q * ntu, tz = q / mtu,
                   tm = q - tz * mtu;
    z = (int)(tz / ksu);
    kz = (int)(tz - (unsigned)z * ksu);
    m0 = (long long)tm * BM;
    n0 = (int)(tn * BN);
    kb0 = kz * args.kb_per_split;
    nkb = max(0, min(nkb_all - kb0, args.kb_per_split));
  };
  int issued = 0;   // TMA k-blocks issued (producer lane only)

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(conv0 + 8 * s, NCONV);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int s = 0; s < AS; ++s) mbar_init(tfree0 + 8 * s, 1);
    for (int b = 0; b < NBUF; ++b) {
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
          mbar_arrive_expect_tx(full0 + 8 * s, C::TX_BYTES);
          tma_load_3d(smem_u32(xA(s)), &tmA, (kb0 + kb) * BK, (int)m0, za, full0 + 8 * s);
          if (C::PRE_A)
            tma_load_3d(smem_u32(loA(s)), &tmAlo, (kb0 + kb) * BK, (int)m0, za, full0 + 8 * s);
          tma_load_3d(smem_u32(xB(s)), &tmB, (kb0 + kb) * BK, n0, zb, full0 + 8 * s);
          if (C::PRE_B)
            tma_load_3d(smem_u32(loB(s)), &tmBlo, (kb0 + kb) * BK, n0, zb, full0 + 8 * s);
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
        const int ab = it % NBUF;
        // the epilogue must have drained this accumulator buffer (use it - NBUF)
        if (it >= NBUF &&
            !mbar_wait(acce0 + 8 * ab, ((it / NBUF) - 1) & 1, abort_flag, args.err))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dmain = tmem + ab * 2 * C::HALF, dcorr = dmain + C::HALF;
        for (int kb = 0; kb < nkb; ++kb, ++kbg) {
          const int s = kbg % S, sa = kbg % ASM;
          // both operands pre-split: the TMA landing is all the MMAs wait for
          ok = mbar_wait((C::PRE_A ? full0 : conv0) + 8 * s, (kbg / S) & 1, abort_flag, args.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t bh = smem_u32(xB(s)), bl = smem_u32(loB(s));
          // head*head into the main accumulator; the two head*tail terms into
          // a separate one, so that the tensor core's truncating accumulation
          // never adds ~2^-11-sized terms to the large running sum
          if (C::PRE_A) {
            const uint32_t ah = smem_u32(xA(s)), al = smem_u32(loA(s));
#pragma unroll
            for (int ks = 0; ks < BK / 8; ++ks) {
              const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
              const uint64_t dah = desc_sw128(ah + ks * 32), dbh = desc_sw128(bh + ks * 32);
              umma_tf32_ss(dmain, dah, dbh, idesc, acc);
              umma_tf32_ss(dcorr, dah, desc_sw128(bl + ks * 32), idesc, acc);
              umma_tf32_ss(dcorr, desc_sw128(al + ks * 32), dbh, idesc, 1u);
            }
            umma_commit(empty0 + 8 * s);    // shared-memory stage free
          } else {
            const uint32_t ah = tmem + C::A_COL0 + sa * 64, al = ah + 32;
#pragma unroll
            for (int ks = 0; ks < BK / 8; ++ks) {
              const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
              umma_tf32_tmem_a(dmain, ah + ks * 8, desc_sw128(bh + ks * 32), idesc, acc);
              umma_tf32_tmem_a(dcorr, ah + ks * 8, desc_sw128(bl + ks * 32), idesc, acc);
              umma_tf32_tmem_a(dcorr, al + ks * 8, desc_sw128(bh + ks * 32), idesc, 1u);
            }
            umma_commit(empty0 + 8 * s);    // shared-memory stage free
            umma_commit(tfree0 + 8 * sa);   // tensor-memory A stage free
          }
        }
        if (ok) umma_commit(accf0 + 8 * ab);
      }
    }
  } else if (warp < 2 + NCONV && !C::PRE_A) {
    // ---------------- converters (warps 2..5) ----------------
    // (idle when both operands come pre-split)
    const int tc = threadIdx.x - 64;            // 0..127
    const int q = warp & 3;                     // TMEM lane quarter
    const int row = q * 32 + lane;              // A row = TMEM lane
    int kbg = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int z, kz, n0, nkb, kb0;
      long long m0;
      tile_of(t, z, kz, m0, n0, nkb, kb0);
      for (int kb = 0; kb < nkb; ++kb, ++kbg) {
        const int s = kbg % S, sa = kbg % ASM;
        ok = mbar_wait(full0 + 8 * s, (kbg / S) & 1, abort_flag, args.err);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        // B (unless it came pre-split): head in place, tail plane in the same
        // swizzled layout
        float4* xb = reinterpret_cast<float4*>(xB(s));
        float4* lb = reinterpret_cast<float4*>(loB(s));
#pragma unroll 2
        for (int idx = tc; idx < (C::PRE_B ? 0 : BN * BK / 4); idx += 32 * NCONV) {
          const float4 v = xb[idx];
          float4 hd, tl;
          tf32_split(v.x, hd.x, tl.x);
          tf32_split(v.y, hd.y, tl.y);
          tf32_split(v.z, hd.z, tl.z);
          tf32_split(v.w, hd.w, tl.w);
          xb[idx] = hd;
          lb[idx] = tl;
        }
        // this thread's A row: 16-byte chunk c of row r sits at chunk c ^ (r % 8)
        float hv[32], tv[32];
        const unsigned char* ar = xA(s) + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(ar + ((c ^ (row & 7)) << 4));
          hv[4 * c] = v.x; hv[4 * c + 1] = v.y; hv[4 * c + 2] = v.z; hv[4 * c + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) tf32_split(hv[i], hv[i], tv[i]);
        // the MMAs of the K block that used this TMEM stage last must be done;
        // the warp proceeds (tcgen05.st is warp-collective) only if every lane saw it
        if (kbg >= AS) ok = mbar_wait(tfree0 + 8 * sa, ((kbg / ASM) - 1) & 1, abort_flag, args.err);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ta = tmem + (static_cast<uint32_t>(q * 32) << 16) + C::A_COL0 + sa * 64;
        tmem_st32(ta, hv);
        tmem_st32(ta + 32, tv);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(conv0 + 8 * s);
      }
    }
  } else if (warp >= 2 + NCONV) {
    // ---------------- epilogue (warps 6..9) ----------------
    const int te = threadIdx.x - 64 - 32 * NCONV;   // 0..127
    const int q = warp & 3;             // TMEM lane quarter of this warp
    float* stg = stg_all + q * (32 * 33);
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      int z, kz, n0, nkb, kb0;
      long long m0;
      tile_of(t, z, kz, m0, n0, nkb, kb0);
      const int ab = it % NBUF;
      asm volatile("bar.sync 2, 128;" ::: "memory");   // previous tile's offsets are dead
      epi_offsets(args, BN, te, m0, n0, z, kz, col_off, col_off32, row_off, row_off32);
      asm volatile("bar.sync 2, 128;" ::: "memory");
      // a failed wait stops all four epilogue warps together: the flag is
      // written only before the barrier below and read only after it
      if (!mbar_wait(accf0 + 8 * ab, (it / NBUF) & 1, abort_flag, args.err) && lane == 0)
        *epi_stop = 1;
      asm volatile("bar.sync 2, 128;" ::: "memory");
      if (*epi_stop) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      epi_rows<BN>(args, tmem + ab * 2 * C::HALF, C::HALF, q, lane, m0, n0, stg, col_off,
                   col_off32, row_off, row_off32);
      // this accumulator buffer may be overwritten by tile it + NBUF
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * ab);
    }
  }
  // teardown: the TMEM owner frees tensor memory after everyone is done
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

// out(b,m,n) = alpha * sum_z part[b][z][m][n] + beta * out.  Lanes run along
// 32 consecutive outputs (coalesced); the 8 warps of a block form 8 / wz
// output groups of wz warps each, the wz warps of a group striding over z.
// Each lane adds its terms in a fixed order by compensated FP32 arithmetic
// (TwoSum per term, Knuth: sh + se carries the sum to ~2^-48 of its
// magnitude without the FP64 pipe) and the group's warps meet in FP64 in
// warp order.  wz = 1 for a large output (each warp owns its outputs, no
// barrier); wz up to 8 for a thin output with a long K, whose few outputs
// would otherwise leave a handful of threads walking hundreds of partials
// each.  I: the flat index type (32-bit whenever batch*M*N fits).
constexpr int kReduceWarps = 8;

__device__ __forceinline__ void two_sum_add(float& sh, float& se, float x) {
  const float t = sh + x;
  const float bp = t - sh;
  se += (sh - (t - bp)) + (x - bp);
  sh = t;
}

template <typename I>
__device__ __forceinline__ long long out_off(const IdxMap& m, I i) {
  return sizeof(I) == 4 ? map_off32(m, static_cast<unsigned>(i))
                        : map_off(m, static_cast<long long>(i));
}

template <typename I>
__device__ __forceinline__ void reduce_store(const TcArgs& a, I e, I MN, I N, double acc) {
  const I b = e / MN, r = e - b * MN, m = r / N, n = r - m * N;
  const long long off = out_off(a.c_b, b) + out_off(a.c_m, m) + out_off(a.c_n, n);
  const double v = a.alpha == 1.0 ? acc : a.alpha * acc;
  if (a.c_fp64) {
    double* o = static_cast<double*>(a.C) + off;
    const double w = a.beta != 0.0 ? fma(a.beta, *o, v) : v;
    *o = w;
    if (a.C32) a.C32[out_off(a.c32_m, m) + out_off(a.c32_n, n)] = static_cast<float>(w);
  } else {
    float* o = static_cast<float*>(a.C) + off;
    *o = static_cast<float>(a.beta != 0.0 ? fma(a.beta, static_cast<double>(*o), v) : v);
  }
}

template <typename I>
__global__ void __launch_bounds__(32 * kReduceWarps)
    tc_splitk_reduce(const __grid_constant__ TcArgs a, int batch, int wz) {
  __shared__ double red[kReduceWarps][2][32];
  const I N = static_cast<I>(a.N), MN = static_cast<I>(a.M) * N, tot = MN * static_cast<I>(batch);
  const int kz = a.ksplit, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int groups = kReduceWarps / wz, g = warp / wz, zw = warp - g * wz;
  const I step = static_cast<I>(gridDim.x) * groups * 32;
  for (I base = static_cast<I>(blockIdx.x) * groups * 32; base < tot; base += step) {
    const I e = base + g * 32 + lane;
    float sh = 0.f, se = 0.f;
    if (e < tot) {
      const I b = e / MN, r = e - b * MN;
      const float* p = a.part + (long long)b * kz * (long long)MN + r;
      int z = zw;
      for (; z + 3 * wz < kz; z += 4 * wz) {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldcg(p + (long long)(z + u * wz) * MN);
#pragma unroll
        for (int u = 0; u < 4; ++u) two_sum_add(sh, se, x[u]);
      }
      for (; z < kz; z += wz) two_sum_add(sh, se, __ldcg(p + (long long)z * MN));
    }
    if (wz == 1) {
      if (e < tot) reduce_store(a, e, MN, N, static_cast<double>(sh) + static_cast<double>(se));
      continue;
    }
    red[warp][0][lane] = static_cast<double>(sh);
    red[warp][1][lane] = static_cast<double>(se);
    __syncthreads();
    if (zw == 0 && e < tot) {
      double acc = red[warp][0][lane] + red[warp][1][lane];
      for (int w = 1; w < wz; ++w) acc += red[warp + w][0][lane] + red[warp + w][1][lane];
      reduce_store(a, e, MN, N, acc);
    }
    __syncthreads();
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

}  // namespace

// 2-D map over an FP32 matrix (cols x rows, row stride in elements), box
// (box_cols, box_rows), no swizzle: the shared-memory side of a copy is a
// dense box.
bool make_map_2d_f32(CUtensorMap* tm, const float* base, long long cols, long long rows,
                     long long row_stride, int box_cols, int box_rows) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (row_stride * 4) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

template <int BN, int NBUF, int PRE>
cudaError_t launch_bn(const TcGemm& g, cudaStream_t s) {
  using C = Cfg<BN, NBUF, PRE>;
  // the shared-memory limit is a per-device attribute of the kernel
  cudaError_t ea = device_once((const void*)tc_tf32x3_kernel<BN, NBUF, PRE>, [] {
    return cudaFuncSetAttribute(tc_tf32x3_kernel<BN, NBUF, PRE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (ea != cudaSuccess) return ea;
  // tail planes (pre-split operands) share the layout of their head planes
  TcOperand alo = g.A, blo = g.B;
  if (C::PRE_A) alo.ptr = g.A.lo;
  if (C::PRE_B) blo.ptr = g.B.lo;
  CUtensorMap ta, tb, tal, tbl;
  if (!make_map(&ta, g.A, BM) || !make_map(&tb, g.B, BN) || !make_map(&tal, alo, BM) ||
      !make_map(&tbl, blo, BN))
    return cudaErrorInvalidValue;
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
  const int nsm = device_sm_count();
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
  // NBUF = 2: one CTA per SM walks the tiles; NBUF = 1: one tile per CTA
  const long long ntiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * a.batch * ksplit;
  if (ntiles > (1ll << 31) - 1) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(NBUF == 2 ? std::min<long long>(ntiles, nsm) : ntiles);
  tc_tf32x3_kernel<BN, NBUF, PRE><<<grid, NTHREADS, C::SMEM, s>>>(ta, tb, tal, tbl, a);
  note_launch();
  if (ksplit > 1 && !g.partials_only) {
    const long long tot = g.M * g.N * std::max(1, g.batch);
    // warps over z only while the outputs alone would not fill the GPU
    int wz = 1;
    if (tot < 32ll * kReduceWarps * 4 * device_sm_count())
      while (wz < kReduceWarps && wz < ksplit) wz *= 2;
    const long long per_block = 32ll * (kReduceWarps / wz);
    const unsigned blocks = (unsigned)std::min<long long>((tot + per_block - 1) / per_block, 8192);
    if (tot < (1ll << 31))
      tc_splitk_reduce<unsigned><<<blocks, 32 * kReduceWarps, 0, s>>>(a, std::max(1, g.batch), wz);
    else
      tc_splitk_reduce<unsigned long long>
          <<<blocks, 32 * kReduceWarps, 0, s>>>(a, std::max(1, g.batch), wz);
    note_launch();
  }
  return cudaGetLastError();
}

template <int BN, int NBUF>
cudaError_t launch_pre(const TcGemm& g, cudaStream_t s) {
  if (g.A.lo != nullptr) return launch_bn<BN, NBUF, 2>(g, s);
  if (g.B.lo != nullptr) return launch_bn<BN, NBUF, 1>(g, s);
  return launch_bn<BN, NBUF, 0>(g, s);
}

}  // namespace

cudaError_t gemm_tc(const TcGemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (g.A.rows < 1 || g.B.rows < 1 || g.A.K != g.K || g.B.K != g.K) return cudaErrorInvalidValue;
  // a pre-split A is taken with a pre-split B only (A's head plane must not
  // be split again)
  if (g.A.lo != nullptr && g.B.lo == nullptr) return cudaErrorInvalidValue;
  if (g.batch > 65535 || g.M > (1ll << 31) - BM || g.N > (1ll << 31) - 256)
    return cudaErrorInvalidValue;
  // double-buffered accumulators up to 96 columns per tile (tensor memory
  // holds 2 x (main, correction) x 96 columns next to two A stages); N in
  // (96, 128] as two 64-column tiles (short-K streams, whose epilogue must
  // overlap); N in (128, 192] as one single-buffered tile (A is staged once
  // per row block).
  // Wider N: 192-column single-buffered tiles when K is long enough for the
  // main loop to dwarf the exposed epilogue (half the operand traffic and
  // conversions per output of 96-column tiles), else 96-column tiles whose
  // epilogue overlaps the next tile.
  const long long N = g.N;
  if (N <= 32) return launch_pre<32, 2>(g, s);
  if (N <= 64) return launch_pre<64, 2>(g, s);
  if (N <= 96) return launch_pre<96, 2>(g, s);
  if (N <= 128) return launch_pre<64, 2>(g, s);    // two double-buffered tiles
  if (N <= 144) return launch_pre<144, 1>(g, s);
  if (N <= 192 || g.K >= 512) return launch_pre<192, 1>(g, s);
  // both operands pre-split (no tensor-memory A stages): 128-column
  // double-buffered tiles fill tensor memory with accumulators and cut the
  // shared-memory operand traffic per output, when there are tiles enough
  if (g.A.lo != nullptr && ((g.M + BM - 1) / BM) * ((N + 127) / 128) * std::max(1, g.batch) >= 296)
    return launch_bn<128, 2, 2>(g, s);
  return launch_pre<96, 2>(g, s);
}

}  // namespace qrctm
