// Contraction dispatch for the energy and the adjoint passes.
//
// Every contraction of the reduced density matrices and of the reverse
// passes is described once, as a descriptor with index maps (Gemm): operands
// and result in FP64, or in FP32 where the descriptor's storage flags say so
// (the gradient tape of a split context).  A context in split precision runs
// them on the TF32x3 tensor-core engine: each operand is gathered through its
// maps into a K-contiguous FP32 copy (row stride padded to 16 bytes,
// batch-major), the product accumulates on the tensor cores, and the
// epilogue writes the result through the descriptor's output maps with alpha
// and beta.  Traces and the energy reduction that follow stay in FP64, and so
// do contractions with a thin output (fewer than 16 rows or columns: long
// reductions into a few numbers, memory bound).  An FP64 context runs every
// descriptor on the FP64 CUDA-core engine.
#include "ctx.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace qrctm {

namespace {

inline long long pad4(long long x) { return (x + 3) & ~3ll; }

bool zero_map(const IdxMap& m) {
  for (int t = 0; t < m.nd; ++t)
    if (m.str[t] != 0) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Operand gathers: out[b][r][k] (row stride ldk, batch stride nr * ldk) =
// in[bm(b) + rm(r) + km(k)], FP64 -> FP32.  Rows are numbered rb = b nr + r,
// so that out row rb starts at out + rb * ldk.  Two tilings, chosen by which
// index runs through the input with unit stride:
//  * along k (the K index's lowest digit has stride 1): a block takes about
//    8192 elements (up to 128 rows x 1024 k); the row offsets and the k
//    offsets are formed once per block into shared memory and every element
//    costs one load and one store, lanes along k for both;
//  * along rows (a digit of the row index has stride 1): the rows are
//    enumerated in an order v that makes that digit the fastest (two maps of
//    v: the input offset and the output row); a block reads a 128 (v) x 32
//    (k) tile with lanes along v, transposes it through shared memory and
//    writes it with lanes along k.
// Both are bound by the latency of their loads, not by their arithmetic: a
// lane keeps 8 to 16 independent loads in flight, and the per-block offsets
// use 32-bit digit divisions where the row index fits.
// ---------------------------------------------------------------------------
constexpr int kGatherThreads = 256;
constexpr int kKRowsMax = 128, kKCols = 1024, kKElems = 8192, kKUnroll = 4;
constexpr int kRTileElems = 4096;   // elements per row-mode tile

// Offset of row rb = b nr + r (kNarrow: 32-bit digit divisions, rb < 2^32).
template <bool kNarrow>
__device__ __forceinline__ long long row_offset(const IdxMap& bm, const IdxMap& rm, long long nr,
                                                long long rb) {
  if (kNarrow) {
    const unsigned r32 = (unsigned)rb, n32 = (unsigned)nr, b = r32 / n32;
    return map_off32(bm, b) + map_off32(rm, r32 - b * n32);
  }
  const long long b = rb / nr;
  return map_off(bm, b) + map_off(rm, rb - b * nr);
}

template <bool kNarrow>
__device__ __forceinline__ long long vmap(const IdxMap& m, long long v) {
  return kNarrow ? map_off32(m, (unsigned)v) : map_off(m, v);
}

// Lanes along k; each warp takes kKUnroll rows at a time, so that a lane has
// that many independent loads in flight per k.
template <bool kNarrow, typename T>
__global__ void __launch_bounds__(kGatherThreads)
    gather_along_k(const T* __restrict__ in, float* __restrict__ out, long long rows,
                   long long nr, long long nk, long long ldk, int rb_tile, int k_tile,
                   long long nkt, const __grid_constant__ IdxMap bm,
                   const __grid_constant__ IdxMap rm, const __grid_constant__ IdxMap km) {
  __shared__ long long roff[kKRowsMax];
  __shared__ long long koff[kKCols];
  const long long kt = blockIdx.x % nkt, rt = blockIdx.x / nkt;
  const long long rb0 = rt * rb_tile, k0 = kt * k_tile;
  const int nrow = (int)std::min<long long>(rb_tile, rows - rb0);
  const int ncol = (int)std::min<long long>(k_tile, nk - k0);
  for (int i = threadIdx.x; i < nrow; i += blockDim.x)
    roff[i] = row_offset<kNarrow>(bm, rm, nr, rb0 + i);
  for (int j = threadIdx.x; j < ncol; j += blockDim.x)
    koff[j] = map_off32(km, (unsigned)(k0 + j));
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i0 = warp * kKUnroll; i0 < nrow; i0 += (kGatherThreads / 32) * kKUnroll) {
    const int nu = nrow - i0 < kKUnroll ? nrow - i0 : kKUnroll;
    const T* src[kKUnroll];
    float* dst[kKUnroll];
#pragma unroll
    for (int u = 0; u < kKUnroll; ++u) {
      const int i = std::min(i0 + u, nrow - 1);
      src[u] = in + roff[i];
      dst[u] = out + (rb0 + i) * ldk + k0;
    }
#pragma unroll 2
    for (int j = lane; j < ncol; j += 32) {
      const long long ko = koff[j];
      T v[kKUnroll];
#pragma unroll
      for (int u = 0; u < kKUnroll; ++u)
        if (u < nu) v[u] = src[u][ko];
#pragma unroll
      for (int u = 0; u < kKUnroll; ++u)
        if (u < nu) dst[u][j] = static_cast<float>(v[u]);
    }
  }
}

// Lanes along the row order v, a TR x (4096 / TR) tile transposed through
// shared memory, written with lanes along k.  TR (16 ... 128) follows the
// number of rows: an operand of 36 or 72 rows and a K of 746496 would leave
// most of a 128-row tile empty.
template <bool kNarrow, typename T, int TR>
__global__ void __launch_bounds__(kGatherThreads)
    gather_along_rows(const T* __restrict__ in, float* __restrict__ out, long long rows,
                      long long nk, long long ldk, long long nkt,
                      const __grid_constant__ IdxMap vin, const __grid_constant__ IdxMap vout,
                      const __grid_constant__ IdxMap km) {
  constexpr int TK = kRTileElems / TR;
  __shared__ float tile[TK][TR + 1];
  __shared__ long long roff[TR], orow[TR], koff[TK];
  const long long kt = blockIdx.x % nkt, rt = blockIdx.x / nkt;
  const long long v0 = rt * TR, k0 = kt * TK;
  const int nrow = (int)std::min<long long>(TR, rows - v0);
  const int ncol = (int)std::min<long long>(TK, nk - k0);
  const int t = threadIdx.x;
  for (int i = t; i < nrow; i += kGatherThreads) {
    roff[i] = vmap<kNarrow>(vin, v0 + i);
    orow[i] = vmap<kNarrow>(vout, v0 + i);
  }
  for (int j = t; j < ncol; j += kGatherThreads) koff[j] = map_off32(km, (unsigned)(k0 + j));
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRTileElems / kGatherThreads; ++q) {   // rows fastest: reads along v
    const int e = t + kGatherThreads * q, i = e % TR, j = e / TR;
    if (i < nrow && j < ncol) tile[j][i] = static_cast<float>(in[roff[i] + koff[j]]);
  }
  __syncthreads();
#pragma unroll 4
  for (int q = 0; q < kRTileElems / kGatherThreads; ++q) {   // k fastest: writes along k
    const int e = t + kGatherThreads * q, j = e % TK, i = e / TK;
    if (i < nrow && j < ncol) out[orow[i] * ldk + k0 + j] = tile[j][i];
  }
}

// Merge neighbouring digits that continue one another (stride of the upper =
// radix x stride of the lower) and drop inner digits of radix 1: the same
// offsets with fewer divisions.
IdxMap merge_digits(const IdxMap& m) {
  IdxMap r{};
  r.nd = 0;
  for (int t = 0; t < m.nd; ++t) {
    const bool last = t == m.nd - 1;
    if (!last && m.rad[t] == 1) continue;
    if (r.nd > 0) {
      const int p = r.nd - 1;
      const long long run = (long long)r.rad[p] * r.str[p];
      if (m.str[t] == run && (last || (long long)r.rad[p] * m.rad[t] <= INT32_MAX)) {
        if (!last) r.rad[p] *= m.rad[t];
        continue;  // the merged digit is the last one when t is
      }
    }
    r.rad[r.nd] = last ? 1 : m.rad[t];
    r.str[r.nd] = m.str[t];
    ++r.nd;
  }
  if (r.nd == 0) { r.nd = 1; r.rad[0] = 1; r.str[0] = 0; }
  return r;
}

// Explicit digits of the combined row index rb = b nr + r: radix, input
// stride and output place value of each.  False when a map's lower radices
// do not divide its index range or the digits are too many for one map.
struct RowDigits {
  int nd;
  long long rad[kMaxDigits], str[kMaxDigits], place[kMaxDigits];
};
bool row_digits(const IdxMap& bm, long long nb, const IdxMap& rm, long long nr, RowDigits& d) {
  d.nd = 0;
  auto add = [&](const IdxMap& m, long long n, long long place0) {
    long long prod = 1;
    for (int t = 0; t < m.nd; ++t) {
      long long rad = m.rad[t];
      if (t == m.nd - 1) {
        if (n % prod != 0) return false;
        rad = n / prod;
      }
      if (rad == 1) continue;
      if (d.nd == kMaxDigits) return false;
      d.rad[d.nd] = rad;
      d.str[d.nd] = m.str[t];
      d.place[d.nd] = place0 * prod;
      ++d.nd;
      prod *= rad;
    }
    return prod == n;
  };
  return add(rm, nr, 1) && (nb == 1 || add(bm, nb, nr));
}

// Length of the unit-stride run of a map's lowest digit (1 if none).
long long unit_run(const IdxMap& m, long long n) {
  if (m.str[0] != 1 && m.str[0] != -1) return 1;
  return m.nd == 1 ? n : m.rad[0];
}

// How one gather runs: the tiling, its grid and the maps it takes.
struct GatherPlan {
  bool along_rows;
  IdxMap bm, rm, km;  // digits merged
  IdxMap vin, vout;   // along rows: input offset and output row of v
  long long blocks, nkt;
  int rb_tile, k_tile;
  int tr;       // row-mode tile height
  bool narrow;  // row indices below 2^32: 32-bit digit divisions
};

bool plan_gather(long long nb, long long nr, long long nk, const IdxMap& bm0, const IdxMap& rm0,
                 const IdxMap& km0, GatherPlan& p) {
  const long long rows = nb * nr;
  if (nk > (long long)UINT32_MAX) return false;
  p.narrow = rows <= (long long)UINT32_MAX;
  p.bm = merge_digits(bm0);
  p.rm = merge_digits(rm0);
  p.km = merge_digits(km0);
  // the longest unit-stride run among the row digits
  RowDigits rd;
  int u = -1;
  if (row_digits(p.bm, nb, p.rm, nr, rd))
    for (int t = 0; t < rd.nd; ++t)
      if ((rd.str[t] == 1 || rd.str[t] == -1) && (u < 0 || rd.rad[t] > rd.rad[u])) u = t;
  for (int t = 0; u >= 0 && t < rd.nd; ++t)
    if (rd.rad[t] > INT32_MAX) u = -1;
  // row-mode tile height: the least padding over the rows (the taller on a tie)
  p.tr = 128;
  for (int tr = 64; tr >= 16; tr /= 2)
    if ((rows + tr - 1) / tr * tr - rows < (rows + p.tr - 1) / p.tr * p.tr - rows) p.tr = tr;
  p.nkt = (nk + kRTileElems / p.tr - 1) / (kRTileElems / p.tr);
  p.blocks = ((rows + p.tr - 1) / p.tr) * p.nkt;
  p.along_rows = u >= 0 && rd.rad[u] > unit_run(p.km, nk) && p.blocks <= INT32_MAX;
  if (p.along_rows) {
    // rows in the order: digit u first, then the others from the lowest up
    p.vin = IdxMap{};
    p.vout = IdxMap{};
    p.vin.nd = p.vout.nd = rd.nd;
    int o = 0;
    auto put = [&](int t) {
      p.vin.rad[o] = p.vout.rad[o] = (int)rd.rad[t];
      p.vin.str[o] = rd.str[t];
      p.vout.str[o] = rd.place[t];
      ++o;
    };
    put(u);
    for (int t = 0; t < rd.nd; ++t)
      if (t != u) put(t);
    p.rb_tile = p.tr;
    p.k_tile = kRTileElems / p.tr;
    return true;
  }
  p.k_tile = (int)std::min<long long>(nk, kKCols);
  p.rb_tile = std::max(1, std::min(kKRowsMax, kKElems / p.k_tile));
  p.nkt = (nk + p.k_tile - 1) / p.k_tile;
  p.blocks = ((rows + p.rb_tile - 1) / p.rb_tile) * p.nkt;
  return p.blocks <= INT32_MAX;
}

template <typename T>
cudaError_t gather3_t(const T* in, float* out, long long nb, long long nr, long long nk,
                      long long ldk, const IdxMap& bm, const IdxMap& rm, const IdxMap& km,
                      cudaStream_t s) {
  const long long rows = nb * nr;
  if (rows <= 0 || nk <= 0) return cudaSuccess;
  GatherPlan p;
  if (!plan_gather(nb, nr, nk, bm, rm, km, p)) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)p.blocks;
  if (p.along_rows) {
    auto launch = [&](auto tr_tag) {
      constexpr int TR = decltype(tr_tag)::value;
      if (p.narrow)
        gather_along_rows<true, T, TR><<<grid, kGatherThreads, 0, s>>>(in, out, rows, nk, ldk,
                                                                       p.nkt, p.vin, p.vout, p.km);
      else
        gather_along_rows<false, T, TR><<<grid, kGatherThreads, 0, s>>>(
            in, out, rows, nk, ldk, p.nkt, p.vin, p.vout, p.km);
    };
    switch (p.tr) {
      case 16: launch(std::integral_constant<int, 16>{}); break;
      case 32: launch(std::integral_constant<int, 32>{}); break;
      case 64: launch(std::integral_constant<int, 64>{}); break;
      default: launch(std::integral_constant<int, 128>{}); break;
    }
  } else if (p.narrow) {
    gather_along_k<true, T><<<grid, kGatherThreads, 0, s>>>(in, out, rows, nr, nk, ldk, p.rb_tile,
                                                            p.k_tile, p.nkt, p.bm, p.rm, p.km);
  } else {
    gather_along_k<false, T><<<grid, kGatherThreads, 0, s>>>(
        in, out, rows, nr, nk, ldk, p.rb_tile, p.k_tile, p.nkt, p.bm, p.rm, p.km);
  }
  note_launch();
  return cudaGetLastError();
}

// in holds doubles, or floats when f32 (an operand the tape keeps in FP32)
cudaError_t gather3(const void* in, bool f32, float* out, long long nb, long long nr,
                    long long nk, long long ldk, const IdxMap& bm, const IdxMap& rm,
                    const IdxMap& km, cudaStream_t s) {
  return f32 ? gather3_t(static_cast<const float*>(in), out, nb, nr, nk, ldk, bm, rm, km, s)
             : gather3_t(static_cast<const double*>(in), out, nb, nr, nk, ldk, bm, rm, km, s);
}

}  // namespace

size_t mm_split_floats(const Gemm& g) {
  const long long Ka = pad4(g.K), B = std::max(1, g.batch);
  const long long nbA = zero_map(g.a_b) ? 1 : B, nbB = zero_map(g.b_b) ? 1 : B;
  return (size_t)(Ka * (nbA * g.M + nbB * g.N));
}

cudaError_t gemm_run(qrctm_ctx* c, const Gemm& g) { return gemm_run_kchunked(c, g, 0); }

cudaError_t gemm_run_kchunked(qrctm_ctx* c, const Gemm& g, long long kchunk) {
  // contractions with a thin output (a reduction over a long index into a
  // few numbers, memory bound) or whose operand copies would not fit the
  // scratch stay on the FP64 engine
  if (!c->mm_split || std::min(g.M, g.N) < 16 || mm_split_floats(g) > c->mm32_floats)
    return gemm_f64(g, c->st);
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (kchunk < 0 || (kchunk & 3) != 0) return cudaErrorInvalidValue;
  const long long Ka = pad4(g.K), B = std::max(1, g.batch);
  const bool shA = zero_map(g.a_b), shB = zero_map(g.b_b);
  const long long nbA = shA ? 1 : B, nbB = shB ? 1 : B;
  float* A32 = c->mm32;
  float* B32 = A32 + pad4(nbA * g.M * Ka);
  cudaError_t e;
  if ((e = gather3(g.A, g.a_f32, A32, nbA, g.M, g.K, Ka, g.a_b, g.a_m, g.a_k, c->st)) !=
      cudaSuccess)
    return e;
  if ((e = gather3(g.B, g.b_f32, B32, nbB, g.N, g.K, Ka, g.b_b, g.b_n, g.b_k, c->st)) !=
      cudaSuccess)
    return e;
  // K in chunks (kchunk > 0): every chunk accumulates in FP32 on the tensor
  // cores and is added to the FP64 result by the epilogue (beta = 1 after the
  // first), so no FP32 sum runs over more than kchunk terms
  const long long kc = kchunk > 0 ? kchunk : g.K;
  for (long long k0 = 0; k0 < g.K; k0 += kc) {
    const long long kn = std::min(kc, g.K - k0);
    TcGemm t{};
    t.A = TcOperand{A32 + k0, g.M, kn, Ka, (int)nbA, g.M * Ka};
    t.B = TcOperand{B32 + k0, g.N, kn, Ka, (int)nbB, g.N * Ka};
    t.M = g.M; t.N = g.N; t.K = kn; t.batch = (int)B;
    t.C = g.C; t.c_fp64 = !g.c_f32;
    t.c_m = g.c_m; t.c_n = g.c_n; t.c_b = g.c_b;
    t.alpha = g.alpha; t.beta = k0 == 0 ? g.beta : 1.0;
    t.err = c->err;
    t.part = c->tc_part; t.part_elems = c->tc_part_elems;
    if ((e = gemm_tc(t, c->st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qrctm
