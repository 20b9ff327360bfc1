// Contraction dispatch for the energy and the adjoint passes.
//
// Every contraction of the reduced density matrices and of the reverse
// passes is described once, as an FP64 descriptor with index maps (Gemm).
// A context in split precision runs them on the TF32x3 tensor-core engine:
// each operand is gathered through its maps into a K-contiguous FP32 copy
// (row stride padded to 16 bytes, batch-major), the product accumulates on
// the tensor cores, and the epilogue writes the FP64 result through the
// descriptor's output maps with alpha and beta.  Traces and the energy
// reduction that follow stay in FP64, and so do contractions with a thin
// output (fewer than 16 rows or columns: long reductions into a few numbers,
// memory bound).  An FP64 context runs every descriptor on the FP64
// CUDA-core engine.
#include "ctx.cuh"
#include "tc_gemm.cuh"

#include <algorithm>

namespace qrctm {

namespace {

inline long long pad4(long long x) { return (x + 3) & ~3ll; }

bool zero_map(const IdxMap& m) {
  for (int t = 0; t < m.nd; ++t)
    if (m.str[t] != 0) return false;
  return true;
}

// out[b][r][k] (row stride ldk, batch stride ldb) = in[bm(b) + rm(r) + km(k)].
// One warp per piece of an output row (up to 1024 elements, so that a few
// long rows still spread over the GPU): the row's offset bm(b) + rm(r) is
// formed once per piece and the K offsets with 32-bit digit divisions (a
// per-element decomposition of the flat index in 64 bits made the gather
// instruction bound); rows shorter than 32 are packed R = 32 / nk to a warp.
__global__ void gather3_f32_k(const double* __restrict__ in, float* __restrict__ out, long long nb,
                              long long nr, long long nk, long long ldk, long long ldb,
                              IdxMap bm, IdxMap rm, IdxMap km) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long rows = nb * nr;
  if (nk >= 32) {
    constexpr long long kChunk = 1024;
    const long long nch = (nk + kChunk - 1) / kChunk;
    for (long long t = warp0; t < rows * nch; t += nwarps) {
      const long long rb = t / nch, k0 = (t - rb * nch) * kChunk;
      const long long r = rb % nr, b = rb / nr;
      const long long base = map_off(bm, b) + map_off(rm, r);
      float* o = out + b * ldb + r * ldk;
      const unsigned kend = (unsigned)std::min(nk, k0 + kChunk);
      for (unsigned k = (unsigned)k0 + lane; k < kend; k += 32)
        o[k] = static_cast<float>(in[base + map_off32(km, k)]);
    }
  } else {
    const int R = 32 / (int)nk, sub = lane / (int)nk, kk = lane % (int)nk;
    const long long koff = map_off32(km, (unsigned)kk);
    for (long long rb0 = warp0 * R; rb0 < rows; rb0 += nwarps * R) {
      const long long rb = rb0 + sub;
      if (sub >= R || rb >= rows) continue;
      const long long r = rb % nr, b = rb / nr;
      out[b * ldb + r * ldk + kk] =
          static_cast<float>(in[map_off(bm, b) + map_off(rm, r) + koff]);
    }
  }
}

cudaError_t gather3(const double* in, float* out, long long nb, long long nr, long long nk,
                    long long ldk, const IdxMap& bm, const IdxMap& rm, const IdxMap& km,
                    cudaStream_t s) {
  const long long tot = nb * nr * nk;
  if (tot <= 0) return cudaSuccess;
  gather3_f32_k<<<(unsigned)std::min<long long>((tot + 255) / 256, 16384), 256, 0, s>>>(
      in, out, nb, nr, nk, ldk, nr * ldk, bm, rm, km);
  note_launch();
  return cudaGetLastError();
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
  if ((e = gather3(g.A, A32, nbA, g.M, g.K, Ka, g.a_b, g.a_m, g.a_k, c->st)) != cudaSuccess)
    return e;
  if ((e = gather3(g.B, B32, nbB, g.N, g.K, Ka, g.b_b, g.b_n, g.b_k, c->st)) != cudaSuccess)
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
    t.C = g.C; t.c_fp64 = true;
    t.c_m = g.c_m; t.c_n = g.c_n; t.c_b = g.c_b;
    t.alpha = g.alpha; t.beta = k0 == 0 ? g.beta : 1.0;
    t.err = c->err;
    t.part = c->tc_part; t.part_elems = c->tc_part_elems;
    if ((e = gemm_tc(t, c->st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qrctm
