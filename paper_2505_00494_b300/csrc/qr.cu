// Blocked Householder QR of the reduced corner (QR-CTMRG paragraph: the
// isometry Q of an unpivoted QR of ct replaces the eigenvectors U).
//
// Layout: the m x n input is column-major (each column of ct contiguous).
// Panels of nb <= 32 columns are factored by one cooperative kernel spread
// over the whole GPU (one bounded arrival round per column, FP64 sums);
// the trailing matrix and the explicit Q are updated with the compact WY
// form H_1...H_nb = I - V T V^T through the contraction engine.
//
// Reflector choice: H x = ||x|| e_1 with v = x - ||x|| e_1, whose first entry
// is evaluated as -sigma / (x_0 + ||x||) when x_0 > 0 (Parlett's rearrangement,
// no cancellation).  This yields diag(R) >= 0 directly, the sign convention
// under which the thin QR of a full-rank matrix is unique.
#include "qrctm_internal.cuh"

#include <algorithm>

namespace qrctm {

namespace {

constexpr int NB = 32;       // panel width (one warp lane per panel column)
constexpr int PT = 256;      // threads per panel CTA (8 row lanes x 32 columns)
constexpr int PMAX = 1024;   // upper bound on panel CTAs (scratch sizing)
constexpr size_t kPanelTileMax = 160 * 1024;   // shared-memory panel tile limit

__host__ __device__ inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Reflector scalars of a column with pivot value x0 and sigma = sum_{i>c}
// x_i^2 > 0: mu = sqrt(x0^2 + sigma) (returned as rmu = 1/mu and mu),
// w = x0 - mu (= -sigma / (x0 + mu) for x0 > 0, no cancellation) and
// inv_w = 1/w.  tau = -w/mu follows when asked for.  The column loop forms
// the same values by the same operations (1/sigma on a second warp), so both
// agree bit for bit; the _rn intrinsics keep the compiler from contracting
// the products into different fused operations at the two sites.
__device__ __forceinline__ void reflector(double x0, double sigma, double* rmu, double* mu,
                                          double* inv_w, double* tau) {
  const double a = fma(x0, x0, sigma);
  const double y = rsqrt_nr(a);
  const double m = __dmul_rn(a, y);
  *rmu = y;
  *mu = m;
  // x0 > 0 from the bits (an FP64 compare would take a 64-clock FP64 slot)
  const int x0h = __double2hiint(x0);
  if (x0h >= 0 && (x0h | __double2loint(x0)) != 0) {
    const double xm = __dadd_rn(x0, m);
    *inv_w = __dmul_rn(-xm, rcp_nr(sigma));
    if (tau) *tau = sigma * y * rcp_nr(xm);       // -w/mu with w = -sigma/(x0 + mu)
  } else {
    const double w = __dsub_rn(x0, m);
    *inv_w = rcp_nr(w);
    if (tau) *tau = -w * y;
  }
}

// Panel factorisation, one cooperative launch over the GPU.  With TILE, each
// CTA keeps its block of panel rows (rows_per_cta x nb doubles) in shared
// memory for the whole factorisation, so that a column step touches global
// memory only for the cross-CTA sums and the published pivot row; the tile
// is written back (R entries, reflectors) at the end.  Without TILE (very
// tall panels) the same steps run on W in global memory.
//
// Column step j (c = j0 + j the pivot row), once every CTA has added its
// partial sums of column j into the column's accumulator row (slot 0:
// sigma = sum_{i>c} x_i^2, slot t: s_t = sum_{i>c} x_i y_{t,i} for column
// j + t) and arrived, and the owner of row c has published that row (x_0
// and the y_{t,0}):
//   mu = sqrt(x_0^2 + sigma), w = x_0 - mu, tau = -w / mu,
//   v = x / w (v_0 = 1),   y_t -= tau (y_{t,0} + s_t / w) v,   R_cc = mu,
//   R_{c,j+t} = y_{t,0} - tau (y_{t,0} + s_t / w).
// Since tau / w = -1/mu, the rows below c need only 1/mu and 1/w:
//   v_i = x_i / w,   y_{t,i} += (y_{t,0} + s_t / w) / mu * x_i,
// so the scalar chain between the arrival and the row pass is one
// reciprocal square root and one reciprocal; tau and the R entries of the
// pivot rows are formed once after the column loop, from the saved sums
// (sigma_j, s_{t,j}) and the pivot rows, which no later column touches.
// Warp 0 waits, reads the accumulator and forms the multipliers; one block
// barrier hands them to the row pass.  The pass over a CTA's rows that
// applies reflector j also accumulates the partial sums of column j + 1 (the
// updated value of column j + 1 on a row reaches the other lanes by a warp
// shuffle), two rows at a time; a second block barrier gathers them and
// warp 0 adds them into column j + 1's accumulator row (FP64 atomics; the
// order of the additions across CTAs is not fixed) and arrives.
//
// part: accumulator rows [column][NB] (zeroed before the first panel of a
// factorisation), then the pivot rows rowb[2][NB].
template <bool TILE>
__global__ void __launch_bounds__(PT) qr_panel_kernel(double* __restrict__ W,
                                                      double* __restrict__ V,
                                                      double* __restrict__ tau_out,
                                                      double* __restrict__ part, GridBar* bar,
                                                      int* err, int m, int j0, int nb,
                                                      int rows_per_cta, float* __restrict__ X32,
                                                      long long ldx, float* __restrict__ Vt32,
                                                      const float* __restrict__ src32,
                                                      float* __restrict__ V32, long long ldv,
                                                      long long wait_spins, unsigned wait_extra) {
  const int P = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;   // wrp = row lane (0..7)
  const long long r_begin = (long long)j0 + (long long)b * rows_per_cta;
  const long long r_end = std::min<long long>(m, r_begin + rows_per_cta);
  const int rows = (int)std::max<long long>(0, r_end - r_begin);
  double* accum = part + (size_t)j0 * NB;          // row jc: column j0 + jc
  double* rowb = part + 2 * (size_t)PMAX * NB;
  __shared__ double red[8][NB];
  __shared__ double coef_s[NB];   // per lane: new y_t = y_t + coef_s[t] x on rows below c
  __shared__ double ssum[NB][NB]; // column j: sigma (slot 0) and s_t (slot t)
  __shared__ double tau_s[NB];
  __shared__ double iw_s[NB];     // 1/w of column j (R entries after the loop)
  __shared__ double x0_s[NB];     // pivot value x_0 of column j as published
  __shared__ double rsig_s;       // 1/sigma of the current column (warp 1)
  __shared__ int s_ok;
  extern __shared__ double tile[];                 // [rows][NB + 1]
  // element (global row i, panel column jc)
  auto at = [&](long long i, int jc) -> double& {
    if (TILE) return tile[(i - r_begin) * (NB + 1) + jc];
    return W[((long long)j0 + jc) * m + i];
  };
  // the eight row lanes' partial sums of a slot: warps 0-3 (one per SM
  // sub-partition, whose FP64 pipes work in parallel) fold warps 4-7 in,
  // then warp 0 adds the four (3 FP64 adds on its pipe instead of 7)
  auto fold8 = [&]() {
    if (wrp < 4) {
      red[wrp][lane] += red[wrp + 4][lane];
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  };
  auto sum4 = [&](int t) { return (red[0][t] + red[1][t]) + (red[2][t] + red[3][t]); };
  // warp 0: add the partial sums (lane t = slot t, nslots of them) into the
  // accumulator row of panel column col, then arrive
  auto publish = [&](int col, double v, int nslots) {
    if (wrp == 0) {
      if (lane < nslots) atomicAdd(accum + (size_t)col * NB + lane, v);
      __syncwarp();
      if (lane == 0) grid_arrive(bar);
    }
  };
  if (TILE) {
    // panel columns from W (FP64) or, when src32 is set, from the FP32 rows
    // src32[c][i] (row stride ldx) of a trailing matrix kept in FP32
    for (int e = threadIdx.x; e < rows * nb; e += PT) {
      const int r = e % rows, jc = e / rows;
      tile[r * (NB + 1) + jc] =
          src32 ? static_cast<double>(src32[((long long)j0 + jc) * ldx + r_begin + r])
                : W[((long long)j0 + jc) * m + r_begin + r];
    }
    __syncthreads();
  }
  // partial sums of column 0 (slot t = lane) and the pivot row j0
  {
    const long long c = j0;
    double acc = 0.0;
    if (lane < nb)
      for (long long i = std::max<long long>(r_begin, c + 1) + wrp; i < r_end; i += 8)
        acc = fma(at(i, 0), at(i, lane), acc);
    red[wrp][lane] = acc;
    if (c >= r_begin && c < r_end && (int)threadIdx.x < nb) rowb[threadIdx.x] = at(c, threadIdx.x);
    __syncthreads();
    fold8();
    publish(0, (wrp == 0) ? sum4(lane) : 0.0, nb);
  }

  int done = 0;
  for (int j = 0; j < nb; ++j) {
    const int buf = j & 1;
    const long long c = (long long)j0 + j;
    const int nrem = nb - j - 1;
    const bool last = (j + 1 >= nb);
    if (wrp == 1) {
      // 1/sigma for a pivot x_0 > 0 (1/w = -(x_0 + mu)/sigma), formed on a
      // second SM sub-partition while warp 0 forms 1/mu: FP64 instructions
      // of one sub-partition do not overlap
      int okw = 1;
      if (lane == 0)
        okw = grid_wait(bar, (unsigned)P * (unsigned)(j + 1) + wait_extra, err, wait_spins) ? 1 : 0;
      __syncwarp();
      if (lane == 0) {
        double rs = 0.0;
        if (okw) {
          const double sg = __ldcg(accum + (size_t)j * NB);
          if (((__double2hiint(sg) & 0x7fffffff) | __double2loint(sg)) != 0) rs = rcp_nr(sg);
        }
        rsig_s = rs;
      }
      asm volatile("bar.arrive 3, 64;" ::: "memory");
    } else if (wrp == 0) {
      int okw = 1;
      if (lane == 0)
        okw = grid_wait(bar, (unsigned)P * (unsigned)(j + 1) + wait_extra, err, wait_spins) ? 1 : 0;
      __syncwarp();                                        // orders lane 0's acquire first
      okw = __shfl_sync(0xffffffffu, okw, 0);
      double y0 = 0.0, st = 0.0;
      if (okw && lane <= nrem) {
        y0 = __ldcg(rowb + buf * NB + lane);               // x_0 (lane 0), y_{t,0} (lane t)
        st = __ldcg(accum + (size_t)j * NB + lane);        // sigma (lane 0), s_t (lane t)
      }
      ssum[j][lane] = st;
      if (lane == 0) x0_s[j] = y0;
      double rmu = 0.0, inv_w = 0.0, xm = 0.0;
      // st != 0 and x_0 > 0 from the bits (an FP64 compare takes a 64-clock
      // FP64 slot); the scalars are those of reflector(), operation for
      // operation, so the values after the loop agree bit for bit
      const bool nz = ((__double2hiint(st) & 0x7fffffff) | __double2loint(st)) != 0;
      const int x0h = __double2hiint(y0);
      const bool pos = x0h >= 0 && (x0h | __double2loint(y0)) != 0;
      if (lane == 0 && nz) {
        const double a = fma(y0, y0, st);
        rmu = rsqrt_nr(a);
        const double m = __dmul_rn(a, rmu);
        if (pos) xm = __dadd_rn(y0, m);
        else inv_w = rcp_nr(__dsub_rn(y0, m));
      }
      asm volatile("bar.sync 3, 64;" ::: "memory");       // warp 1's 1/sigma
      if (lane == 0 && nz && pos) inv_w = __dmul_rn(-xm, rsig_s);
      // sigma = 0: x is zero below c, v = e_1 (tau = 0 or 2); the rows
      // below c are left as they are (multipliers 0)
      rmu = __shfl_sync(0xffffffffu, rmu, 0);
      inv_w = __shfl_sync(0xffffffffu, inv_w, 0);
      double mult = 0.0;
      if (lane == 0) mult = inv_w;
      else if (lane <= nrem) mult = rmu * fma(st, inv_w, y0);
      coef_s[lane] = mult;
      if (lane == 0) s_ok = okw;
    }
    __syncthreads();
    if (!s_ok) break;
    double acc = 0.0, acc2 = 0.0;
    {
      const double mult = coef_s[lane];
      const bool active = (lane <= nrem);
      const bool upd = (lane >= 1 && active);
      long long i = std::max<long long>(r_begin, c + 1) + wrp;
      // two rows per pass (independent FMA chains), then the odd one
      for (; i + 8 < r_end; i += 16) {
        const double x1 = at(i, j), x2 = at(i + 8, j);
        const double o1 = upd ? at(i, j + lane) : 0.0;
        const double o2 = upd ? at(i + 8, j + lane) : 0.0;
        const double n1 = fma(mult, x1, o1), n2 = fma(mult, x2, o2);
        __syncwarp();
        if (active) {
          at(i, j + lane) = n1;
          at(i + 8, j + lane) = n2;
        }
        if (!last) {
          const double xn1 = __shfl_sync(0xffffffffu, n1, 1);   // updated column j + 1
          const double xn2 = __shfl_sync(0xffffffffu, n2, 1);
          if (upd) {
            if (i > c + 1) acc = fma(xn1, n1, acc);
            else rowb[(buf ^ 1) * NB + lane - 1] = n1;       // pivot row of column j + 1
            acc2 = fma(xn2, n2, acc2);
          }
        }
      }
      for (; i < r_end; i += 8) {
        const double x = at(i, j);
        const double old = upd ? at(i, j + lane) : 0.0;
        const double nv = fma(mult, x, old);
        __syncwarp();
        if (active) at(i, j + lane) = nv;
        if (!last) {
          const double xn = __shfl_sync(0xffffffffu, nv, 1);
          if (upd) {
            if (i > c + 1) acc = fma(xn, nv, acc);
            else rowb[(buf ^ 1) * NB + lane - 1] = nv;
          }
        }
      }
    }
    done = j + 1;
    if (last) break;
    red[wrp][lane] = acc + acc2;                           // slot lane - 1 of column j + 1
    __syncthreads();
    fold8();
    publish(j + 1, (wrp == 0 && lane < nrem) ? sum4(lane + 1) : 0.0, nrem);
  }
  __syncthreads();
  // tau and the pivot rows (R_cc = mu, R_{c,j+t} = y_{t,0} - tau (y_{t,0} +
  // s_t / w)) of the factored columns: one lane per column, from the saved
  // sums and the published pivot values.  CTA 0 needs tau of every column;
  // a CTA holding pivot rows needs its own columns.  A NaN or Inf anywhere
  // in the panel reaches tau or mu.
  const bool has_pivots = r_begin < (long long)j0 + done;
  if ((b == 0 || has_pivots) && wrp == 0 && lane < done) {
    const long long c = (long long)j0 + lane;
    const double sigma = ssum[lane][0];
    const double x0 = x0_s[lane];        // = at(c, lane) on the owner of row c
    double tau = 0.0, iw = 0.0, mu = fabs(x0);
    if (sigma != 0.0) {
      double rmu;
      reflector(x0, sigma, &rmu, &mu, &iw, &tau);
    } else {
      tau = (x0 < 0.0) ? 2.0 : 0.0;
    }
    if (!(tau == tau) || isinf(tau) || !(mu == mu) || isinf(mu)) atomicOr(err, ERRF_NUMERIC);
    tau_s[lane] = tau;
    iw_s[lane] = iw;
    if (c >= r_begin && c < r_end) at(c, lane) = mu;
  }
  __syncthreads();
  if (has_pivots) {
    for (int e = threadIdx.x; e < done * NB; e += PT) {
      const int jj = e / NB, t = e % NB;
      const long long c = (long long)j0 + jj;
      if (t >= 1 && jj + t < nb && c >= r_begin && c < r_end) {
        const double y0 = at(c, jj + t);
        at(c, jj + t) = y0 - tau_s[jj] * fma(ssum[jj][t], iw_s[jj], y0);
      }
    }
    __syncthreads();
  }
  // write back: panel rows of W (R above/on the diagonal, reflectors below)
  // and the explicit reflectors V (zero above the unit diagonal); optionally
  // FP32 copies of V for the tensor-core WY products: X32[c][i] and V32[c][i]
  // (rows c, row stride ldx) and Vt32[i][c] (row stride ldv)
  for (int e = threadIdx.x; e < rows * nb; e += PT) {
    const int r = e % rows, jc = e / rows;
    const long long i = r_begin + r, c = (long long)j0 + jc;
    const double x = at(i, jc);
    if (TILE) W[c * m + i] = x;
    const double v = (i < c) ? 0.0 : (i == c ? 1.0 : x);
    V[c * m + i] = v;
    if (X32) {
      const float vf = static_cast<float>(v);
      X32[c * ldx + i] = vf;
      V32[c * ldx + i] = vf;
      Vt32[i * ldv + c] = vf;
    }
  }
  // tau of the panel columns for the compact-WY factor (built after the kernel)
  if (b == 0 && threadIdx.x < (unsigned)nb) tau_out[threadIdx.x] = tau_s[threadIdx.x];
  if (threadIdx.x == 0) grid_exit(bar, (unsigned)P);
}

// Cancellation guard of a paired round: column b's reflector norm
// sigma_b = |x_b + m_b x_a|^2 (rows below its pivot) is formed from the
// pair's Gram sums; it is used only when it keeps at least this fraction of
// M_b = G_bb + 2 |m_b G_ab| + m_b^2 G_aa (so its relative rounding error
// stays below ~2^10 ulp); otherwise the round factors column a alone.
constexpr double kPairGuard = 1.0 / 1024.0;

// Placement of the pair kernel's padded Gram-sum accumulators inside the
// panel scratch: past the accumulator rows of the one-column kernel, the
// pivot rows, G and tau; kPairAccCap doubles are free there.
constexpr int kPairAccStride = 16;
constexpr size_t kPairAccOff = ((size_t)2 * PMAX * NB + 4 * NB + NB * NB + NB + 15) & ~size_t(15);
constexpr size_t kPairAccCap = (size_t)2 * PMAX * NB + 2 * NB + (size_t)PMAX * NB * NB - kPairAccOff;

// Panel factorisation with up to two columns per grid-wide exchange.  The
// single-column kernel above needs one exchange of partial sums per column;
// here a round factors columns a = j and b = j + 1 (pivot rows c, c + 1) from
// one exchange of the pair's Gram sums over the rows below both pivots,
//   G_at = sum x_a y_t,  G_bt = sum x_b y_t   (t >= a, resp. t >= b),
// and the two pivot rows (published by their owners).  Column a's reflector
// follows from sigma_a = G_aa + x_a[c+1]^2 and s_t = G_at + x_a[c+1] y_t[c+1]
// exactly as in the single-column kernel (multipliers m_t: y_t += m_t x_a on
// the rows below c).  After it, on the rows below c + 1,
//   x_b' = x_b + m_b x_a,  y_t' = y_t + m_t x_a,  so
//   sigma_b = G_bb + 2 m_b G_ab + m_b^2 G_aa,
//   s_t'    = G_bt + m_t G_ab + m_b G_at + m_b m_t G_aa,
// and column b's reflector (pivot value x_b[c+1] + m_b x_a[c+1], multipliers
// n_t) is applied in the same row pass: y_t'' = y_t' + n_t x_b'.  The row
// pass then accumulates the Gram sums of the next pair over the rows below
// its pivots and the owners publish those two pivot rows.  When sigma_b
// fails the cancellation guard (or only one column is left) the round
// factors column a alone and the next pair starts at b.  Every CTA takes the
// same decision from the same sums.  Accumulators: per round starting at
// panel column p, two rows of NB doubles (Gram sums of columns p and p + 1);
// pivot rows rowb[buffer][2][NB].
template <bool TILE>
__global__ void __launch_bounds__(PT) qr_panel2_kernel(double* __restrict__ W,
                                                       double* __restrict__ V,
                                                       double* __restrict__ tau_out,
                                                       double* __restrict__ part, GridBar* bar,
                                                       int* err, int m, int j0, int nb,
                                                       int rows_per_cta, float* __restrict__ X32,
                                                       long long ldx, float* __restrict__ Vt32,
                                                       const float* __restrict__ src32,
                                                       float* __restrict__ V32, long long ldv,
                                                       long long wait_spins, unsigned wait_extra,
                                                       double* __restrict__ acc_base, int as) {
  const int P = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;   // wrp = row lane (0..7)
  const long long r_begin = (long long)j0 + (long long)b * rows_per_cta;
  const long long r_end = std::min<long long>(m, r_begin + rows_per_cta);
  const int rows = (int)std::max<long long>(0, r_end - r_begin);
  // Gram-sum accumulators: round at panel column p, slot (r, t) at
  // accum[((p * 2 + r) * NB + t) * as] (as = 16: one 128-byte line per sum, so
  // the grid's atomic additions spread over the L2 slices)
  double* accum = acc_base + (size_t)j0 * 2 * NB * as;
  double* rowb = part + 2 * (size_t)PMAX * NB;      // [buffer][pivot row 0/1][NB]
  __shared__ double red[8][2][NB];
  __shared__ double cfa[NB];      // lane 0: 1/w_a; lane t >= 1: m_t
  __shared__ double cfb[NB];      // lane 1: 1/w_b; lane t >= 2: n_t
  __shared__ double ssum[NB][NB]; // column j: sigma (slot 0) and s_t (slot t)
  __shared__ double tau_s[NB];
  __shared__ double iw_s[NB];
  __shared__ double x0_s[NB];     // pivot value of column j when its reflector was formed
  __shared__ double rsig_s;       // 1/sigma_a (warp 1)
  __shared__ double rsigb_s;      // 1/sigma_b (warp 2)
  __shared__ double sc_rmu, sc_inw;    // reflector a: 1/mu_a, 1/w_a (warp 0)
  __shared__ double sc_rmub, sc_iwb;   // reflector b: 1/mu_b, 1/w_b (warp 1)
  __shared__ int s_ok, s_k, s_kr;
  extern __shared__ double tile[];
  auto at = [&](long long i, int jc) -> double& {
    if (TILE) return tile[(i - r_begin) * (NB + 1) + jc];
    return W[((long long)j0 + jc) * m + i];
  };
  auto fold8 = [&]() {
    if (wrp < 4) {
      red[wrp][0][lane] += red[wrp + 4][0][lane];
      red[wrp][1][lane] += red[wrp + 4][1][lane];
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  };
  auto sum4 = [&](int s, int t) {
    return (red[0][s][t] + red[1][s][t]) + (red[2][s][t] + red[3][s][t]);
  };
  if (TILE) {
    for (int e = threadIdx.x; e < rows * nb; e += PT) {
      const int r = e % rows, jc = e / rows;
      tile[r * (NB + 1) + jc] =
          src32 ? static_cast<double>(src32[((long long)j0 + jc) * ldx + r_begin + r])
                : W[((long long)j0 + jc) * m + r_begin + r];
    }
    __syncthreads();
  }
  // Gram sums of the first pair over rows > j0 + 1, and pivot rows j0, j0 + 1
  {
    const long long c = j0;
    double acc1 = 0.0, acc2 = 0.0;
    if (lane < nb) {
      for (long long i = std::max<long long>(r_begin, c + 2) + wrp; i < r_end; i += 8) {
        const double y = at(i, lane);
        acc1 = fma(at(i, 0), y, acc1);
        if (nb > 1) acc2 = fma(at(i, 1), y, acc2);
      }
    }
    red[wrp][0][lane] = acc1;
    red[wrp][1][lane] = acc2;
    for (int q = 0; q < 2; ++q)
      if (c + q >= r_begin && c + q < r_end && (int)threadIdx.x < nb)
        rowb[q * NB + threadIdx.x] = at(c + q, threadIdx.x);
    __syncthreads();
    fold8();
    if (wrp == 0) {
      double* acc = accum;
      if (lane < nb) atomicAdd(acc + (size_t)lane * as, sum4(0, lane));
      if (lane >= 1 && lane < nb) atomicAdd(acc + (size_t)(NB + lane) * as, sum4(1, lane));
      __syncwarp();
      if (lane == 0) grid_arrive(bar);
    }
  }

  int done = 0, round = 0;
  while (done < nb) {
    const int p = done;                     // first column of this round
    const int buf = round & 1;
    const long long c = (long long)j0 + p;  // pivot row of column p
    const int nrem = nb - p - 1;            // columns right of p
    const double* acc = accum + (size_t)p * 2 * NB * as;
    const double* rb = rowb + (size_t)buf * 2 * NB;
    const unsigned target = (unsigned)P * (unsigned)(round + 1) + wait_extra;
    // Scalars of the round, spread over three warps on three SM
    // sub-partitions (FP64 instructions of one sub-partition do not overlap):
    //   warp 0: reflector a (lane 0), then the per-column quantities m_t,
    //           y_t'[c+1], s_t' (all lanes), then n_t;
    //   warp 1: 1/sigma_a, then reflector b (from m_b, sigma_b, x_b'[c+1]);
    //   warp 2: 1/sigma_b and the cancellation guard.
    // Each waits on the grid barrier and loads its inputs itself, so no L2
    // round trip follows a block barrier.  Barriers: 3 (warp 1 -> 0: 1/sigma_a),
    // 4 (warp 0 -> 1, 2: rmu_a, 1/w_a), 6 (warp 2 -> 1: 1/sigma_b),
    // 5 (warps 1, 2 -> 0: reflector b and the decision).
    if (wrp == 1 || wrp == 2) {
      int okw = 1;
      if (lane == 0) okw = grid_wait(bar, target, err, wait_spins) ? 1 : 0;
      // column a at row c+1, column b at rows c, c+1, and the Gram sums G_aa,
      // G_ab, G_bb (over rows > c+1)
      double ra1 = 0.0, g00 = 0.0, rb0 = 0.0, rb1 = 0.0, g01 = 0.0, g11 = 0.0;
      if (lane == 0 && okw) {
        ra1 = (c + 1 < m) ? __ldcg(rb + NB) : 0.0;
        g00 = __ldcg(acc);
        if (nrem >= 1) {
          rb0 = __ldcg(rb + 1);
          rb1 = __ldcg(rb + NB + 1);
          g01 = __ldcg(acc + as);
          g11 = __ldcg(acc + (size_t)(NB + 1) * as);
        }
      }
      if (wrp == 1) {
        if (lane == 0) {
          // 1/sigma_a for a pivot x_0 > 0 (sigma_a as warp 0 forms it)
          const double sg = fma(ra1, ra1, g00);
          double rs = 0.0;
          if (okw && (((__double2hiint(sg) & 0x7fffffff) | __double2loint(sg)) != 0))
            rs = rcp_nr(sg);
          rsig_s = rs;
        }
        __syncwarp();
        asm volatile("bar.arrive 3, 64;" ::: "memory");
      }
      __syncwarp();
      asm volatile("bar.sync 4, 96;" ::: "memory");        // rmu_a, 1/w_a from warp 0
      // m_b, sigma_b and x_b'[c+1] exactly as warp 0 forms m_t, y_t'[c+1]
      double mb = 0.0, sb = 0.0, xb0 = 0.0, rmub = 0.0, iwb = 0.0, xm = 0.0;
      bool nzb = false, pos = false;
      if (lane == 0 && nrem >= 1) {
        const double st1 = fma(ra1, rb1, g01);
        mb = sc_rmu * fma(st1, sc_inw, rb0);
        sb = fma(mb, fma(mb, g00, 2.0 * g01), g11);
        nzb = ((__double2hiint(sb) & 0x7fffffff) | __double2loint(sb)) != 0;
        if (wrp == 2) {
          rsigb_s = nzb ? rcp_nr(sb) : 0.0;
        } else {
          // reflector b, operation for operation as reflector() forms it
          xb0 = fma(mb, ra1, rb1);
          const int xh = __double2hiint(xb0);
          pos = xh >= 0 && (xh | __double2loint(xb0)) != 0;
          if (nzb) {
            const double a = fma(xb0, xb0, sb);
            rmub = rsqrt_nr(a);
            const double mm = __dmul_rn(a, rmub);
            if (pos) xm = __dadd_rn(xb0, mm);
            else iwb = rcp_nr(__dsub_rn(xb0, mm));
          }
        }
      }
      if (wrp == 2) {
        __syncwarp();
        asm volatile("bar.arrive 6, 64;" ::: "memory");
        if (lane == 0) {
          bool safe = false;
          if (nrem >= 1) {
            const double Mb = fma(mb * mb, g00, fma(2.0 * fabs(mb), fabs(g01), g11));
            safe = (sb >= kPairGuard * Mb) && (sb == sb) && (c + 1 < m);
          }
          s_k = safe ? 2 : 1;
        }
      } else {
        __syncwarp();
        asm volatile("bar.sync 6, 64;" ::: "memory");      // 1/sigma_b from warp 2
        if (lane == 0 && nrem >= 1) {
          if (nzb && pos) iwb = __dmul_rn(-xm, rsigb_s);
          sc_rmub = rmub;
          sc_iwb = iwb;
          ssum[p + 1][0] = sb;
          x0_s[p + 1] = xb0;
        }
      }
      __syncwarp();
      asm volatile("bar.arrive 5, 96;" ::: "memory");
    } else if (wrp == 0) {
      int okw = 1;
      if (lane == 0) okw = grid_wait(bar, target, err, wait_spins) ? 1 : 0;
      __syncwarp();                                        // orders lane 0's acquire first
      okw = __shfl_sync(0xffffffffu, okw, 0);
      // lane t: column p + t at rows c, c+1; Gram sums G_{p,p+t}, G_{p+1,p+t}
      double r0 = 0.0, r1 = 0.0, g0 = 0.0, g1 = 0.0;
      if (okw && lane <= nrem) {
        r0 = __ldcg(rb + lane);
        r1 = (c + 1 < m) ? __ldcg(rb + NB + lane) : 0.0;
        g0 = __ldcg(acc + (size_t)lane * as);
        g1 = __ldcg(acc + (size_t)(NB + lane) * as);
      }
      // column a's sums over rows > c: sigma (lane 0), s_t (lane t)
      const double ra1 = __shfl_sync(0xffffffffu, r1, 0);
      const double st = fma(ra1, r1, g0);
      ssum[p][lane] = st;
      if (lane == 0) x0_s[p] = r0;
      double rmu = 0.0, inv_w = 0.0, xm = 0.0;
      const bool nz = ((__double2hiint(st) & 0x7fffffff) | __double2loint(st)) != 0;
      const int x0h = __double2hiint(r0);
      const bool pos = x0h >= 0 && (x0h | __double2loint(r0)) != 0;
      if (lane == 0 && nz) {
        const double a = fma(r0, r0, st);
        rmu = rsqrt_nr(a);
        const double mm = __dmul_rn(a, rmu);
        if (pos) xm = __dadd_rn(r0, mm);
        else inv_w = rcp_nr(__dsub_rn(r0, mm));
      }
      __syncwarp();
      asm volatile("bar.sync 3, 64;" ::: "memory");       // warp 1's 1/sigma_a
      if (lane == 0 && nz && pos) inv_w = __dmul_rn(-xm, rsig_s);
      if (lane == 0) {
        sc_rmu = rmu;
        sc_inw = inv_w;
      }
      __syncwarp();
      asm volatile("bar.arrive 4, 96;" ::: "memory");
      rmu = __shfl_sync(0xffffffffu, rmu, 0);
      inv_w = __shfl_sync(0xffffffffu, inv_w, 0);
      double ma = 0.0;                                    // m_t (lane t >= 1), 1/w_a (lane 0)
      if (lane == 0) ma = inv_w;
      else if (lane <= nrem) ma = rmu * fma(st, inv_w, r0);
      cfa[lane] = ma;
      // pivot row c+1 after reflector a and s_t' for lanes t >= 2
      const double y1 = fma(ma, ra1, r1);
      const double mb = __shfl_sync(0xffffffffu, ma, 1);
      const double gaa = __shfl_sync(0xffffffffu, g0, 0);
      const double gab = __shfl_sync(0xffffffffu, g0, 1);
      const double sp = fma(ma, fma(mb, gaa, gab), fma(mb, g0, g1));
      if (lane >= 2) ssum[p + 1][lane - 1] = sp;
      __syncwarp();
      asm volatile("bar.sync 5, 96;" ::: "memory");       // reflector b and the decision
      const int k = (nrem >= 1) ? s_k : 1;
      double nbc = 0.0;
      if (k == 2) {
        const double rmub = sc_rmub, iwb = sc_iwb;
        if (lane == 1) nbc = iwb;
        else if (lane >= 2 && lane <= nrem) nbc = rmub * fma(sp, iwb, y1);
      }
      cfb[lane] = nbc;
      if (lane == 0) {
        s_ok = okw;
        s_kr = k;
      }
    }
    __syncthreads();
    if (!s_ok) break;
    const int k = s_kr;
    const int nnext = nb - p - k;           // columns left after this round
    double acc1 = 0.0, acc2 = 0.0;
    {
      const double ca = cfa[lane], cb = cfb[lane];
      const bool active = (lane <= nrem);
      const bool upda = (lane >= 1 && active);
      // pivot rows of the next round: c + k, c + k + 1; Gram sums below them
      const long long q0 = c + k, q1 = c + k + 1;
      const int la = k, lb = k + 1;          // lanes of the next pair's columns
      // one row: any row (the pivot rows of this and the next round included)
      auto row1 = [&](long long i) {
        const double xa = at(i, p);
        const double old = upda ? at(i, p + lane) : 0.0;
        double y = fma(ca, xa, old);        // lane 0: v_a = x_a / w_a
        if (k == 2 && i > c + 1) {
          // lane 1: v_b = x_b' / w_b; lanes t >= 2: y_t'' = y_t' + n_t x_b'
          // in one instruction (cb = 0 beyond nrem: y unchanged)
          const double xb = __shfl_sync(0xffffffffu, y, 1);
          if (lane >= 1) y = fma(cb, xb, lane == 1 ? 0.0 : y);
        }
        __syncwarp();
        if (active) at(i, p + lane) = y;
        if (nnext > 0) {
          const double ya = __shfl_sync(0xffffffffu, y, la & 31);
          const double yb = __shfl_sync(0xffffffffu, y, lb & 31);
          if (i == q0 || i == q1) {
            if (lane >= k && active)
              rowb[(size_t)(buf ^ 1) * 2 * NB + (i == q1 ? NB : 0) + (lane - k)] = y;
          } else if (i > q1) {
            if (lane >= k && active) acc1 = fma(ya, y, acc1);
            if (lane >= k + 1 && active) acc2 = fma(yb, y, acc2);
          }
        }
      };
      long long i = std::max<long long>(r_begin, c + 1) + wrp;
      for (; i < r_end && i <= q1; i += 8) row1(i);
      if (nrem < 16) {
        // at most 16 live columns: rows i (lanes 0-15) and i + 8 (lanes
        // 16-31) share each FP64 instruction, which costs the same for any
        // number of active lanes; rows here are below both pivots
        const int t = lane & 15, half = lane & 16;
        const long long off = half ? 8 : 0;
        const double pca = cfa[t], pcb = cfb[t];
        const bool pact = t <= nrem, pupd = t >= 1 && pact;
        double pacc1 = 0.0, pacc2 = 0.0;
        for (; i < r_end; i += 16) {
          const long long ir = i + off;
          const bool rv = ir < r_end;
          const double xa = rv ? at(ir, p) : 0.0;
          const double old = (rv && pupd) ? at(ir, p + t) : 0.0;
          double y = fma(pca, xa, old);
          if (k == 2) {
            const double xb = __shfl_sync(0xffffffffu, y, half | 1);
            if (t >= 1) y = fma(pcb, xb, t == 1 ? 0.0 : y);
          }
          __syncwarp();
          if (rv && pact) at(ir, p + t) = y;
          if (nnext > 0) {
            const double ya = __shfl_sync(0xffffffffu, y, half | la);
            const double yb = __shfl_sync(0xffffffffu, y, half | lb);
            if (rv && pact && t >= k) pacc1 = fma(ya, y, pacc1);
            if (rv && pact && t >= k + 1) pacc2 = fma(yb, y, pacc2);
          }
        }
        // lane t (< 16) collects both halves' sums of column p + t
        pacc1 += __shfl_down_sync(0xffffffffu, pacc1, 16);
        pacc2 += __shfl_down_sync(0xffffffffu, pacc2, 16);
        if (lane < 16) {
          acc1 += pacc1;
          acc2 += pacc2;
        }
      } else {
      // rows below the next pivots, two at a time (independent chains: a
      // dependent FP64 operation costs 64 clocks on B300)
      double acc1b = 0.0, acc2b = 0.0;
      for (; i + 8 < r_end; i += 16) {
        const double xa1 = at(i, p), xa2 = at(i + 8, p);
        const double o1 = upda ? at(i, p + lane) : 0.0;
        const double o2 = upda ? at(i + 8, p + lane) : 0.0;
        double y1 = fma(ca, xa1, o1), y2 = fma(ca, xa2, o2);
        if (k == 2) {
          const double xb1 = __shfl_sync(0xffffffffu, y1, 1);
          const double xb2 = __shfl_sync(0xffffffffu, y2, 1);
          if (lane >= 1) {
            y1 = fma(cb, xb1, lane == 1 ? 0.0 : y1);
            y2 = fma(cb, xb2, lane == 1 ? 0.0 : y2);
          }
        }
        __syncwarp();
        if (active) {
          at(i, p + lane) = y1;
          at(i + 8, p + lane) = y2;
        }
        if (nnext > 0) {
          const double ya1 = __shfl_sync(0xffffffffu, y1, la & 31);
          const double ya2 = __shfl_sync(0xffffffffu, y2, la & 31);
          const double yb1 = __shfl_sync(0xffffffffu, y1, lb & 31);
          const double yb2 = __shfl_sync(0xffffffffu, y2, lb & 31);
          if (lane >= k && active) {
            acc1 = fma(ya1, y1, acc1);
            acc1b = fma(ya2, y2, acc1b);
          }
          if (lane >= k + 1 && active) {
            acc2 = fma(yb1, y1, acc2);
            acc2b = fma(yb2, y2, acc2b);
          }
        }
      }
      for (; i < r_end; i += 8) row1(i);
      acc1 += acc1b;
      acc2 += acc2b;
      }
    }
    done = p + k;
    ++round;
    if (done >= nb) break;
    red[wrp][0][lane] = acc1;
    red[wrp][1][lane] = acc2;
    __syncthreads();
    fold8();
    // warp 0 adds slot row 0, warp 1 slot row 1 (two sub-partitions); warp 0
    // arrives once warp 1's additions are issued (the barrier orders them
    // before the release)
    if (wrp == 0 || wrp == 1) {
      double* an = accum + (size_t)done * 2 * NB * as;
      const int t = lane + k;                // red lane of the next round's column done + lane
      if (wrp == 0) {
        if (lane < nnext) atomicAdd(an + (size_t)lane * as, sum4(0, t));
        __syncwarp();
        asm volatile("bar.sync 7, 64;" ::: "memory");
        if (lane == 0) grid_arrive(bar);
      } else {
        if (lane >= 1 && lane < nnext) atomicAdd(an + (size_t)(NB + lane) * as, sum4(1, t));
        __syncwarp();
        asm volatile("bar.arrive 7, 64;" ::: "memory");
      }
    }
  }
  __syncthreads();
  // tau and the pivot rows, as in the single-column kernel
  const bool has_pivots = r_begin < (long long)j0 + done;
  if ((b == 0 || has_pivots) && wrp == 0 && lane < done) {
    const long long c = (long long)j0 + lane;
    const double sigma = ssum[lane][0];
    const double x0 = x0_s[lane];
    double tau = 0.0, iw = 0.0, mu = fabs(x0);
    if (sigma != 0.0) {
      double rmu;
      reflector(x0, sigma, &rmu, &mu, &iw, &tau);
    } else {
      tau = (x0 < 0.0) ? 2.0 : 0.0;
    }
    if (!(tau == tau) || isinf(tau) || !(mu == mu) || isinf(mu)) atomicOr(err, ERRF_NUMERIC);
    tau_s[lane] = tau;
    iw_s[lane] = iw;
    if (c >= r_begin && c < r_end) at(c, lane) = mu;
  }
  __syncthreads();
  if (has_pivots) {
    for (int e = threadIdx.x; e < done * NB; e += PT) {
      const int jj = e / NB, t = e % NB;
      const long long c = (long long)j0 + jj;
      if (t >= 1 && jj + t < nb && c >= r_begin && c < r_end) {
        const double y0 = at(c, jj + t);
        at(c, jj + t) = y0 - tau_s[jj] * fma(ssum[jj][t], iw_s[jj], y0);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rows * nb; e += PT) {
    const int r = e % rows, jc = e / rows;
    const long long i = r_begin + r, c = (long long)j0 + jc;
    const double x = at(i, jc);
    if (TILE) W[c * m + i] = x;
    const double v = (i < c) ? 0.0 : (i == c ? 1.0 : x);
    V[c * m + i] = v;
    if (X32) {
      const float vf = static_cast<float>(v);
      X32[c * ldx + i] = vf;
      V32[c * ldx + i] = vf;
      Vt32[i * ldv + c] = vf;
    }
  }
  if (b == 0 && threadIdx.x < (unsigned)nb) tau_out[threadIdx.x] = tau_s[threadIdx.x];
  if (threadIdx.x == 0) grid_exit(bar, (unsigned)P);
}

// T (upper triangular, nb x nb, row stride NB): T_jj = tau_j,
// T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j], with G = V^T V of the panel.
__global__ void qr_tfactor_kernel(const double* __restrict__ G, const double* __restrict__ tau,
                                  double* __restrict__ Tf, int nb) {
  __shared__ double Gs[NB][NB + 1];
  __shared__ double Ts[NB][NB + 1];
  __shared__ double taus[NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    Gs[e / nb][e % nb] = G[(e / nb) * NB + (e % nb)];
    Ts[e / nb][e % nb] = 0.0;
  }
  for (int e = threadIdx.x; e < nb; e += blockDim.x) taus[e] = tau[e];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    double val = 0.0;
    const int i = threadIdx.x;
    if (i < j) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int l = i;
      for (; l + 4 <= j; l += 4) {
        v0 = fma(Ts[i][l], Gs[l][j], v0);
        v1 = fma(Ts[i][l + 1], Gs[l + 1][j], v1);
        v2 = fma(Ts[i][l + 2], Gs[l + 2][j], v2);
        v3 = fma(Ts[i][l + 3], Gs[l + 3][j], v3);
      }
      for (; l < j; ++l) v0 = fma(Ts[i][l], Gs[l][j], v0);
      val = -taus[j] * ((v0 + v1) + (v2 + v3));
    }
    __syncthreads();
    if (i < j) Ts[i][j] = val;
    if (i == j) Ts[j][j] = taus[j];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x)
    Tf[(e / nb) * NB + (e % nb)] = Ts[e / nb][e % nb];
}

__global__ void extract_r_kernel(const double* __restrict__ W, double* __restrict__ R, int m,
                                 int n) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  R[e] = (j >= i) ? W[(long long)j * m + i] : 0.0;
}

__global__ void set_identity_cols_kernel(double* Q, int m, int n) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  long long col = e / m, row = e % m;
  Q[e] = (row == col) ? 1.0 : 0.0;
}

}  // namespace

// Factor panel p (columns j0..j0+nbj) of w.W in place: FP64 Householder
// reflectors into w.V, tau and the Gram-based T factor into w.Tf (stride NB).
// gram_tc: compute G = V^T V with the caller's contraction (nullptr = FP64).
cudaError_t qr_panel_step(int m, int j0, int nbj, const QrWork& w, cudaStream_t s, double** G_out,
                          double** tau_out, float* X32, long long ldx, float* Vt32,
                          const float* src32, float* V32, long long ldv) {
  const int mr = m - j0;
  int P = qr_panel_grid(mr);
  double* W = w.W; double* V = w.V; double* part = w.part;
  double* Gp = w.part + 2 * (size_t)PMAX * NB + 4 * NB;   // after the pivot rows [2][2][NB]
  double* taup = Gp + NB * NB;
  GridBar* bar = w.bar; int* err = w.err;
  int m_ = m, j0_ = j0, nb_ = nbj;
  float* x32 = X32;
  float* vt32 = Vt32;
  float* v32 = V32;
  const float* s32 = src32;
  long long ldx_ = ldx, ldv_ = ldv;
  long long spins_ = w.wait_spins > 0 ? w.wait_spins : kGridWaitSpins;
  unsigned extra_ = w.wait_extra;
  // one accumulator row of NB doubles per column of the whole factorisation
  if (j0 + nbj > 2 * PMAX) return cudaErrorInvalidValue;
  cudaError_t e = cudaErrorUnknown;
  if (w.hook) w.hook(w.hook_user, 1);
  // the first panel of a factorisation clears every column's accumulator
  if (j0 == 0 &&
      (e = cudaMemsetAsync(part, 0, sizeof(double) * 2 * (size_t)PMAX * NB, s)) != cudaSuccess) {
    if (w.hook) w.hook(w.hook_user, 0);
    return e;
  }
  // cooperative launch, one CTA per SM at most: every CTA adds its partial
  // sums into the column's accumulator and arrives on the counter
  int rpc = (mr + P - 1) / P;

  const size_t tile = sizeof(double) * (size_t)rpc * (NB + 1);
  if (src32 != nullptr && tile > kPanelTileMax) {
    if (w.hook) w.hook(w.hook_user, 0);
    return cudaErrorInvalidValue;   // an FP32 source needs the tiled path
  }
  // two columns per grid-wide exchange where the accumulator rows fit (two
  // rows of NB per round start: j0 + nb <= PMAX); one column otherwise.  The
  // pair kernel's sums sit one per 128-byte line past the pivot rows, G and
  // tau (zeroed with the first panel), or packed when the factorisation is
  // too wide for that region.
  const bool pair = w.pair_rounds && j0 + nbj <= PMAX;
  double* acc_base = part;
  int as = 1;
  if (pair && (size_t)w.ncols * 2 * NB * kPairAccStride <= kPairAccCap) {
    acc_base = part + kPairAccOff;
    as = kPairAccStride;
    if (j0 == 0 && (e = cudaMemsetAsync(acc_base, 0, sizeof(double) * (size_t)w.ncols * 2 * NB *
                                                         kPairAccStride, s)) != cudaSuccess) {
      if (w.hook) w.hook(w.hook_user, 0);
      return e;
    }
  }
  void* args[] = {&W, &V, &taup, &part, &bar, &err, &m_, &j0_, &nb_, &rpc, &x32, &ldx_, &vt32,
                  &s32, &v32, &ldv_, &spins_, &extra_, &acc_base, &as};
  const void* kt = pair ? (const void*)qr_panel2_kernel<true> : (const void*)qr_panel_kernel<true>;
  const void* kg = pair ? (const void*)qr_panel2_kernel<false> : (const void*)qr_panel_kernel<false>;
  if (tile <= kPanelTileMax) {
    // the shared-memory limit is a per-device attribute of the kernel
    e = device_once(kt, [kt] {
      return cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPanelTileMax);
    });
    if (e != cudaSuccess) {
      if (w.hook) w.hook(w.hook_user, 0);
      return e;
    }
    e = cudaLaunchCooperativeKernel(kt, dim3(P), dim3(PT), args, tile, s);
  } else {
    e = cudaLaunchCooperativeKernel(kg, dim3(P), dim3(PT), args, 0, s);
  }
  if (w.hook) w.hook(w.hook_user, 0);
  if (e != cudaSuccess) return e;
  note_launch();
  *G_out = Gp;
  *tau_out = taup;
  return cudaSuccess;
}

cudaError_t qr_tfactor(const double* G, const double* tau, double* Tp, int nbj, cudaStream_t s) {
  qr_tfactor_kernel<<<1, NB, 0, s>>>(G, tau, Tp, nbj);
  note_launch();
  return cudaGetLastError();
}

cudaError_t qr_extract_r(const double* W, double* R, int m, int n, cudaStream_t s) {
  long long tot = (long long)n * n;
  extract_r_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W, R, m, n);
  note_launch();
  return cudaGetLastError();
}

int qr_panel_grid(int mrows) {
  const int nsm = device_sm_count();
  int p = (mrows + 31) / 32;
  return std::max(1, std::min(std::min(p, nsm), PMAX));
}

size_t qr_work_bytes(int m, int n) {
  const int npan = (n + NB - 1) / NB;
  size_t b = 0;
  b += align_up(sizeof(double) * (size_t)kSplitKElems);     // split-K partials
  b += align_up(sizeof(double) * (size_t)m * n);            // W
  b += align_up(sizeof(double) * (size_t)m * n);            // V
  b += align_up(sizeof(double) * (size_t)NB * NB * npan);   // Tf
  b += align_up(sizeof(double) * (size_t)NB * n);           // Y
  b += align_up(sizeof(double) * (size_t)NB * n);           // Y2
  b += align_up(sizeof(double) * ((size_t)2 * PMAX * NB + 2 * NB + (size_t)PMAX * NB * NB));
  b += align_up(sizeof(GridBar));
  b += align_up(sizeof(int));
  return b;
}

QrWork qr_carve(void* base, int m, int n) {
  const int npan = (n + NB - 1) / NB;
  char* p = static_cast<char*>(base);
  QrWork w;
  w.hook = nullptr;
  w.hook_user = nullptr;
  w.splitk = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)kSplitKElems);
  w.W = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)m * n);
  w.V = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)m * n);
  w.Tf = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)NB * NB * npan);
  w.Y = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)NB * n);
  w.Y2 = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * (size_t)NB * n);
  w.part = reinterpret_cast<double*>(p);
  p += align_up(sizeof(double) * ((size_t)2 * PMAX * NB + 2 * NB + (size_t)PMAX * NB * NB));
  w.bar = reinterpret_cast<GridBar*>(p); p += align_up(sizeof(GridBar));
  w.err = reinterpret_cast<int*>(p);
  w.wait_spins = kGridWaitSpins;
  w.wait_extra = 0;
  w.pair_rounds = false;
  w.ncols = n;
  return w;
}

cudaError_t set_identity_cols(double* Q, int m, int n, cudaStream_t s) {
  long long tot = (long long)m * n;
  set_identity_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Q, m, n);
  note_launch();
  return cudaGetLastError();
}

// M (m x n, column-major, m >= n) -> Q (m x n, column-major), R (n x n, row-major).
// The grid barrier in `w` must be zero on entry; it is left zero on exit.
cudaError_t householder_qr_f64(int m, int n, const double* M, double* Q, double* R,
                               const QrWork& w, cudaStream_t s) {
  if (m < n || n <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(w.W, M, sizeof(double) * (size_t)m * n,
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  const int npan = (n + NB - 1) / NB;
  for (int p = 0; p < npan; ++p) {
    const int j0 = p * NB;
    const int nbj = std::min(NB, n - j0);
    const int mr = m - j0;
    double* Tp = w.Tf + (size_t)p * NB * NB;
    double *Gp, *taup;
    if ((e = qr_panel_step(m, j0, nbj, w, s, &Gp, &taup)) != cudaSuccess) return e;
    {
      // G = V_p^T V_p over the panel rows (reflectors are zero above their
      // unit diagonal), then T from G and tau
      Gemm g = gemm_init();
      g.part = w.splitk; g.part_elems = kSplitKElems;
      g.M = nbj; g.N = nbj; g.K = mr;
      g.A = w.V + (size_t)j0 * m + j0; g.a_m = im1(m); g.a_k = im1(1);
      g.B = w.V + (size_t)j0 * m + j0; g.b_k = im1(1); g.b_n = im1(m);
      g.C = Gp; g.c_m = im1(NB); g.c_n = im1(1);
      if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
      qr_tfactor_kernel<<<1, NB, 0, s>>>(Gp, taup, Tp, nbj);
      note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int n2 = n - j0 - nbj;
    if (n2 > 0) {
      Gemm g = gemm_init();
      g.part = w.splitk; g.part_elems = kSplitKElems;
      // Y = V^T W2   (nbj x n2, K = mr)
      g.M = nbj; g.N = n2; g.K = mr;
      g.A = w.V + (size_t)j0 * m + j0; g.a_m = im1(m); g.a_k = im1(1);
      g.B = w.W + (size_t)(j0 + nbj) * m + j0; g.b_k = im1(1); g.b_n = im1(m);
      g.C = w.Y; g.c_m = im1(n2); g.c_n = im1(1);
      if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
      // Y2 = T^T Y   (nbj x n2, K = nbj)
      g.M = nbj; g.N = n2; g.K = nbj;
      g.A = Tp; g.a_m = im1(1); g.a_k = im1(NB);
      g.B = w.Y; g.b_k = im1(n2); g.b_n = im1(1);
      g.C = w.Y2; g.c_m = im1(n2); g.c_n = im1(1);
      if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
      // W2 -= V Y2   (mr x n2, K = nbj)
      g.M = mr; g.N = n2; g.K = nbj;
      g.A = w.V + (size_t)j0 * m + j0; g.a_m = im1(1); g.a_k = im1(m);
      g.B = w.Y2; g.b_k = im1(n2); g.b_n = im1(1);
      g.C = w.W + (size_t)(j0 + nbj) * m + j0; g.c_m = im1(1); g.c_n = im1(m);
      g.alpha = -1.0; g.beta = 1.0;
      if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    }
  }
  {
    long long tot = (long long)n * n;
    extract_r_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w.W, R, m, n);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // Q = H_1 ... H_n [I; 0], applying the panels in reverse order
  if ((e = set_identity_cols(Q, m, n, s)) != cudaSuccess) return e;
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * NB;
    const int nbj = std::min(NB, n - j0);
    const int mr = m - j0, nq = n - j0;
    const double* Tp = w.Tf + (size_t)p * NB * NB;
    Gemm g = gemm_init();
    g.part = w.splitk; g.part_elems = kSplitKElems;
    // Y = V^T Qs   (nbj x nq, K = mr)
    g.M = nbj; g.N = nq; g.K = mr;
    g.A = w.V + (size_t)j0 * m + j0; g.a_m = im1(m); g.a_k = im1(1);
    g.B = Q + (size_t)j0 * m + j0; g.b_k = im1(1); g.b_n = im1(m);
    g.C = w.Y; g.c_m = im1(nq); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    // Y2 = T Y
    g.M = nbj; g.N = nq; g.K = nbj;
    g.A = Tp; g.a_m = im1(NB); g.a_k = im1(1);
    g.B = w.Y; g.b_k = im1(nq); g.b_n = im1(1);
    g.C = w.Y2; g.c_m = im1(nq); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    // Qs -= V Y2
    g.M = mr; g.N = nq; g.K = nbj;
    g.A = w.V + (size_t)j0 * m + j0; g.a_m = im1(1); g.a_k = im1(m);
    g.B = w.Y2; g.b_k = im1(nq); g.b_n = im1(1);
    g.C = Q + (size_t)j0 * m + j0; g.c_m = im1(1); g.c_n = im1(m);
    g.alpha = -1.0; g.beta = 1.0;
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qrctm
