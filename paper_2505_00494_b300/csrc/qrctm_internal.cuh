// Internal declarations shared by the QR-CTMRG CUDA sources.
//
// Every contraction of the method is expressed as a (batched) matrix product
// whose operands and result are addressed through mixed-radix index maps:
// an index i is split into digits (innermost first) and each digit carries
// its own element stride.  This lets one GEMM kernel read and write every
// tensor layout of the step (reshape + permute folded into the addressing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

namespace qrctm {

// ---------------------------------------------------------------------------
// Per-device host state.  Kernel attributes (the dynamic shared-memory
// limit, the non-portable cluster size) are set per device, and devices may
// differ in SM count, so one-time setup is keyed by (current device, key).
// device_once runs f the first time a (device, key) pair is met, under a
// lock (a concurrent first call waits for it), and returns f's result then
// and on every later call for that pair.
// ---------------------------------------------------------------------------
cudaError_t device_once(const void* key, const std::function<cudaError_t()>& f);
// SM count of the current device (looked up once per device).
int device_sm_count();

// ---------------------------------------------------------------------------
// Mixed-radix index map: offset(i) = sum_t digit_t(i) * str[t].
// digit_0 = i % rad[0], digit_1 = (i / rad[0]) % rad[1], ...; the last used
// digit takes the remaining quotient (its radix is ignored).
// ---------------------------------------------------------------------------
constexpr int kMaxDigits = 6;
struct IdxMap {
  int nd;
  int rad[kMaxDigits];
  long long str[kMaxDigits];
};

static inline IdxMap im0() { IdxMap m{}; m.nd = 1; m.rad[0] = 1; m.str[0] = 0; return m; }
static inline IdxMap im1(long long s0) { IdxMap m{}; m.nd = 1; m.rad[0] = 1; m.str[0] = s0; return m; }
static inline IdxMap im2(int r0, long long s0, long long s1) {
  IdxMap m{}; m.nd = 2; m.rad[0] = r0; m.str[0] = s0; m.str[1] = s1; return m;
}
static inline IdxMap im3(int r0, int r1, long long s0, long long s1, long long s2) {
  IdxMap m{}; m.nd = 3; m.rad[0] = r0; m.rad[1] = r1; m.str[0] = s0; m.str[1] = s1; m.str[2] = s2;
  return m;
}
static inline IdxMap im4(int r0, int r1, int r2, long long s0, long long s1, long long s2,
                         long long s3) {
  IdxMap m{}; m.nd = 4; m.rad[0] = r0; m.rad[1] = r1; m.rad[2] = r2;
  m.str[0] = s0; m.str[1] = s1; m.str[2] = s2; m.str[3] = s3; return m;
}
static inline IdxMap im5(int r0, int r1, int r2, int r3, long long s0, long long s1,
                         long long s2, long long s3, long long s4) {
  IdxMap m{}; m.nd = 5; m.rad[0] = r0; m.rad[1] = r1; m.rad[2] = r2; m.rad[3] = r3;
  m.str[0] = s0; m.str[1] = s1; m.str[2] = s2; m.str[3] = s3; m.str[4] = s4; return m;
}

__host__ __device__ __forceinline__ long long map_off(const IdxMap& m, long long i) {
  long long off = 0;
#pragma unroll
  for (int t = 0; t < kMaxDigits; ++t) {
    if (t >= m.nd) break;
    if (t == m.nd - 1) {
      off += i * m.str[t];
    } else {
      long long q = i / m.rad[t];
      off += (i - q * m.rad[t]) * m.str[t];
      i = q;
    }
  }
  return off;
}

// The same for an index below 2^32: the digits come from 32-bit divisions
// (a 64-bit division is a long instruction sequence).
__host__ __device__ __forceinline__ long long map_off32(const IdxMap& m, unsigned i) {
  long long off = 0;
#pragma unroll
  for (int t = 0; t < kMaxDigits; ++t) {
    if (t >= m.nd) break;
    if (t == m.nd - 1) {
      off += (long long)i * m.str[t];
    } else {
      const unsigned r = static_cast<unsigned>(m.rad[t]), q = i / r;
      off += (long long)(i - q * r) * m.str[t];
      i = q;
    }
  }
  return off;
}

// C[b](m,n) = alpha * sum_k A[b](m,k) B[b](k,n) + beta * C[b](m,n)
// If `part` is set and the output grid is too small to fill the GPU, the K
// range is split over CTAs; partial sums go to `part` (part_elems doubles)
// and a second kernel adds them in a fixed order (deterministic).
struct Gemm {
  long long M, N, K;
  int batch;
  const double* A; IdxMap a_m, a_k, a_b;
  const double* B; IdxMap b_k, b_n, b_b;
  double* C;       IdxMap c_m, c_n, c_b;
  double alpha, beta;
  double* part;
  long long part_elems;
  // the operand (or result) is stored as FP32: its pointer holds floats
  // (both engines read and write such operands; arithmetic as before)
  bool a_f32, b_f32, c_f32;
};

static inline Gemm gemm_init() {
  Gemm g{};
  g.part = nullptr;
  g.part_elems = 0;
  g.a_f32 = g.b_f32 = g.c_f32 = false;
  g.batch = 1;
  g.a_b = im0(); g.b_b = im0(); g.c_b = im0();
  g.alpha = 1.0; g.beta = 0.0;
  return g;
}

// Process-wide count of kernels launched by this library (for reporting).
void note_launch(unsigned long long n = 1);
unsigned long long launches_so_far();

// FP64 CUDA-core contraction (any layout).  Returns cudaGetLastError().
cudaError_t gemm_f64(const Gemm& g, cudaStream_t s);

// FP32 value of a double by moving its bits (sign, exponent rebiased, the
// mantissa truncated to 23 bits) and back: B300 runs the FP64<->FP32
// conversions on its FP64 pipe (64 clocks each, one at a time per
// sub-partition), integer moves cost a few clocks.  Valid for |x| with a
// normal FP32 exponent; callers check the range first.
static __device__ __forceinline__ float f32_of_bits(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  return __uint_as_float((hi & 0x80000000u) | ((((hi >> 20) & 0x7ffu) - 896u) << 23) |
                         ((hi & 0xfffffu) << 3) | (lo >> 29));
}
static __device__ __forceinline__ double f64_of_bits(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned hi = (fb & 0x80000000u) | ((((fb >> 23) & 0xffu) + 896u) << 20) |
                      ((fb >> 3) & 0xfffffu);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(fb << 29));
}

// FP64 reciprocal from an FP32 seed r0 by one third-order step: with
// e = 1 - x r0 (|e| <= 2^-22), 1/x = r0 (1 + e + e^2 + ...), and
// r0 (1 + e + e^2) leaves e^3 < 2^-66 (three dependent FP64 operations, no
// long-latency IEEE divide sequence on the scalar path; results within an
// ulp).  The range test and the seed's conversions are integer operations.
static __device__ __forceinline__ double rcp_nr(double x) {
  const unsigned e = (static_cast<unsigned>(__double2hiint(x)) >> 20) & 0x7ffu;
  if (e < 1023u - 100u || e > 1023u + 100u) return 1.0 / x;   // outside the seed's range
  const double r = f64_of_bits(1.0f / f32_of_bits(x));
  const double d = fma(-x, r, 1.0);
  return fma(r, fma(d, d, d), r);
}

// 1/sqrt(a) in FP64 from the FP32 estimate y0 by one third-order step: with
// e = 1 - a y0^2 (y0^2 exact in FP64, |e| <= 2^-20),
// 1/sqrt(a) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + ...), truncated after
// e^2 (error 5e^3/16 < 2^-61; five dependent FP64 operations), for a inside
// [2^-100, 2^100].
static __device__ __forceinline__ double rsqrt_nr(double a) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(a));
  const unsigned e = (hi >> 20) & 0x7ffu;
  if ((hi >> 31) || e < 1023u - 100u || e > 1023u + 100u) return 1.0 / sqrt(a);
  const double y = f64_of_bits(rsqrtf(f32_of_bits(a)));
  const double d = fma(-a, y * y, 1.0);
  return fma(y * d, fma(d, 0.375, 0.5), y);
}

// Nearest TF32 (ties away from zero) of a finite x: add half a TF32 unit to
// the magnitude bits and clear the 13 dropped ones (a carry moves into the
// exponent, as rounding up to the next binade should).
static __device__ __forceinline__ float tf32_rna_bits(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Split of an FP32 x for the TF32x3 contraction: x = head + tail, both TF32
// (x - head is exact in FP32 and |tail| <= 2^-11 |x|); a NaN stays the head
// (Inf gives a NaN tail).
static __device__ __forceinline__ void tf32_split(float x, float& head, float& tail) {
  head = (x == x) ? tf32_rna_bits(x) : x;
  tail = tf32_rna_bits(x - head);
}

// ---------------------------------------------------------------------------
// Device-side error flag bits (written by kernels, read by the host).
// ---------------------------------------------------------------------------
enum : int {
  ERRF_NUMERIC = 1,      // NaN/Inf or zero norm met
  ERRF_TIMEOUT = 2,      // a bounded wait ran out
  ERRF_BOUNDS = 4,       // a size check inside a kernel failed
};

// Arrival counter for cooperative launches.  `count` only grows during a
// launch: CTA b publishes its data, then adds 1; a CTA that needs round r
// (r = 1, 2, ...) of all P CTAs waits until count >= r P.  At exit every CTA
// adds 1 to `exit`, and the last one puts both words back to zero, so the
// next launch starts from zero without a host-side reset.  Waits are bounded;
// on timeout ERRF_TIMEOUT is raised and the wait returns false.
struct GridBar {
  unsigned int count;
  unsigned int exit;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Called by one thread after the CTA's published writes (ordered before it by
// a block or warp barrier).
__device__ __forceinline__ void grid_arrive(GridBar* bar) {
  // release: the CTA's published writes (ordered before this by a block or
  // warp barrier) become visible before the count does
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
}

// Default bound of a grid wait, in polls (each poll after the first 64 sleeps
// ~32 ns on top of its L2 round trip: about a second in all).
constexpr long long kGridWaitSpins = 1ll << 25;

// Called by one thread; true once count >= target.  After `limit` polls the
// wait gives up: ERRF_TIMEOUT is raised and false returned.
__device__ __forceinline__ bool grid_wait(GridBar* bar, unsigned int target, int* err,
                                          long long limit) {
  long long spins = 0;
  while (ld_acquire_gpu(&bar->count) < target) {
    if (++spins > limit) {
      atomicOr(err, ERRF_TIMEOUT);
      return false;
    }
    if (spins > 64) __nanosleep(32);
  }
  return true;
}

// Called by one thread of every CTA as its last action.
__device__ __forceinline__ void grid_exit(GridBar* bar, unsigned int nblocks) {
  __threadfence();
  if (atomicAdd(&bar->exit, 1u) == nblocks - 1) {
    atomicExch(&bar->count, 0u);
    atomicExch(&bar->exit, 0u);
  }
}

// ---------------------------------------------------------------------------
// Householder QR (unpivoted, diag(R) >= 0) of a column-major m x n matrix.
// ---------------------------------------------------------------------------
struct QrWork {
  double* splitk;   // split-K partial sums (kSplitKElems doubles)
  double* W;        // m x n working copy (column-major)
  double* V;        // m x n explicit reflectors (column-major, unit diagonal)
  double* Tf;       // nb x nb x npanel compact-WY factors
  double* Y;        // nb x n scratch
  double* Y2;       // nb x n scratch
  double* part;     // partial sums of the panel kernel
  GridBar* bar;
  int* err;
  // optional host callback around every panel launch (begin = 1, end = 0),
  // used for per-phase timing
  void (*hook)(void* user, int begin);
  void* hook_user;
  // bound of the panel's grid waits (polls) and arrivals expected beyond the
  // CTAs launched (0; a positive value makes every wait run out, which only
  // the timeout test asks for); qr_carve sets the defaults
  long long wait_spins;
  unsigned int wait_extra;
  // panel rounds: two columns per grid-wide exchange (guarded) when true,
  // one column per exchange when false.  The paired round forms the second
  // reflector's norm from Gram sums, whose rounding leaves its Householder
  // transform orthogonal only to ~1e-13 on ill-conditioned panels (one
  // column per exchange: ~1e-15); qr_carve chooses one column (the FP64
  // path), the split-precision QR, whose trailing update and Q are FP32-class,
  // two.
  bool pair_rounds;
  int ncols;              // columns of the factorisation (n)
};
constexpr long long kSplitKElems = 1ll << 21;   // 16 MB of split-K partials
size_t qr_work_bytes(int m, int n);
QrWork qr_carve(void* base, int m, int n);
int qr_panel_grid(int m);
cudaError_t householder_qr_f64(int m, int n, const double* M, double* Q, double* R_rowmajor,
                               const QrWork& w, cudaStream_t s);
constexpr int kQrPanel = 32;   // panel width of the blocked QR
// Factor panel columns j0..j0+nbj of w.W in place (FP64 Householder):
// reflectors into w.V, tau and a G-sized scratch returned.  With X32 set,
// FP32 copies of the reflectors also go to X32[c][i] and V32[c][i] (row
// stride ldx) and Vt32[i][c] (row stride ldv).  With src32 set the panel's
// columns are read from the FP32 rows src32[c][i] (stride ldx) instead of w.W.
cudaError_t qr_panel_step(int m, int j0, int nbj, const QrWork& w, cudaStream_t s, double** G_out,
                          double** tau_out, float* X32 = nullptr, long long ldx = 0,
                          float* Vt32 = nullptr, const float* src32 = nullptr,
                          float* V32 = nullptr, long long ldv = 0);
cudaError_t qr_tfactor(const double* G, const double* tau, double* Tp, int nbj, cudaStream_t s);
cudaError_t qr_extract_r(const double* W, double* R, int m, int n, cudaStream_t s);
// Split-precision variant (tensor-core compact-WY products); f32 holds
// qr_split_floats(m, n) floats, part the tensor-core split-K partial sums.
size_t qr_split_floats(int m, int n);
cudaError_t householder_qr_split(int m, int n, const double* M, double* R, const QrWork& w,
                                 float* f32, float* Q32, bool x32_ready, float* part,
                                 long long part_elems, cudaStream_t s);
// FP32 copy of the input inside f32 (row c = column c of M, row stride
// pad4(m)); a caller that writes it itself passes x32_ready = true.
float* qr_split_x32(float* f32);

// out[r * stride + c] = (float) in[map(rmap, r) + map(cmap, c)], 0 <= c < ncols.
// With lo set, the FP32 value is split (tf32_split): out gets the TF32 head,
// lo[r * stride + c] the TF32 tail.
cudaError_t gather_f32f(const float* in, float* out, long long nrows, int ncols, long long stride,
                        IdxMap rmap, IdxMap cmap, cudaStream_t s, float* lo = nullptr);
cudaError_t gather_f32(const double* in, float* out, long long nrows, int ncols, long long stride,
                       IdxMap rmap, IdxMap cmap, cudaStream_t s, float* lo = nullptr);
// In place: x[r * stride + c] -> its TF32 head, lo[r * stride + c] = its TF32 tail.
cudaError_t split_f32(float* x, float* lo, long long nrows, int ncols, long long stride,
                      cudaStream_t s);

// ---------------------------------------------------------------------------
// Elementwise / reduction kernels.
// ---------------------------------------------------------------------------
cudaError_t c4v_symmetrize(int d, int D, const double* X, double* Y, cudaStream_t s);
cudaError_t sum_squares_partials(const double* x, long long n, double* partials, int nparts,
                                 cudaStream_t s);
cudaError_t scale_by_inv_norm(const double* x, double* y, long long n, const double* partials,
                              int nparts, int* err, cudaStream_t s);
// C <- (C + C^T)/2 and T[a,k,b] <- (T[a,k,b] + T[b,k,a])/2, then each / ||.||_F
cudaError_t sym_norm_env(const double* Cin, const double* Tin, double* Cout, double* Tout,
                         int chi, int D2, double* partials, int* err, cudaStream_t s);
cudaError_t sym_edge(const double* Tin, double* Tout, int chi, int D2, cudaStream_t s);
cudaError_t init_env_kernel(int d, int D, const double* A, double* C0, double* T0,
                            cudaStream_t s);
cudaError_t double_layer_kernel(int d, int D, const double* A, double* a, cudaStream_t s);
cudaError_t set_identity_cols(double* Q, int m, int n, cudaStream_t s);
cudaError_t corner_spectrum(const double* C, int chi, double* work, double* s_new,
                            const double* s_old, int chi_old, double* delta, int* err,
                            cudaStream_t s);
// |eig(C0)| -> s0 and |eig(C1)| -> s1 with delta = ||s1 - s0||; for equal
// sizes the two corners share one set of launches (two clusters, two rows
// of bisection CTAs).
cudaError_t corner_spectrum_pair(const double* C0, int chi0, double* work0, double* s0,
                                 const double* C1, int chi1, double* work1, double* s1,
                                 double* delta, int* err, cudaStream_t s);
cudaError_t fill_zero(double* p, long long n, cudaStream_t s);
cudaError_t axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t s);

}  // namespace qrctm
