// Device side of the L-BFGS variational optimisation (Automatic
// differentiation paragraph): the two-loop recursion, trial points and
// curvature pairs.  The parameter vector has d D^4 <= 2^16 entries, so every
// kernel is one block of 1024 threads; reductions run in a fixed order.
#include "ctx.cuh"

namespace qrctm {

namespace {

constexpr int kOptThreads = 1024;

// Sum over the block; every thread gets the result.  red: 33 doubles.
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = ln < (int)(blockDim.x >> 5) ? red[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (ln == 0) red[32] = v;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__device__ double block_dot(const double* x, const double* y, int n, double* red) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += x[i] * y[i];
  return block_sum(t, red);
}

// p = -H g over the cnt newest pairs of the ring (slot of the newest:
// head - 1), H0 = (s.y / y.y) I of the newest pair; out[0] = g.p,
// out[1] = p.p.  q: n doubles of scratch.
__global__ void __launch_bounds__(kOptThreads)
lbfgs_direction_k(int n, int cnt, int head, int hist, const double* __restrict__ S,
                  const double* __restrict__ Y, const double* __restrict__ g,
                  double* __restrict__ q, double* __restrict__ p, double* __restrict__ out) {
  __shared__ double red[33];
  __shared__ double alpha[32], rho[32];
  for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] = g[i];
  __syncthreads();
  for (int j = 0; j < cnt; ++j) {          // newest first
    const int sl = (head - 1 - j + 2 * hist) % hist;
    const double* s = S + (size_t)sl * n;
    const double* y = Y + (size_t)sl * n;
    const double sy = block_dot(s, y, n, red);
    const double a = block_dot(s, q, n, red) / sy;
    if (threadIdx.x == 0) { alpha[j] = a; rho[j] = 1.0 / sy; }
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] -= a * y[i];
    __syncthreads();
  }
  if (cnt > 0) {
    const int sl = (head - 1 + hist) % hist;
    const double* s = S + (size_t)sl * n;
    const double* y = Y + (size_t)sl * n;
    const double gam = block_dot(s, y, n, red) / block_dot(y, y, n, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] *= gam;
    __syncthreads();
  }
  for (int j = cnt - 1; j >= 0; --j) {     // oldest first
    const int sl = (head - 1 - j + 2 * hist) % hist;
    const double* s = S + (size_t)sl * n;
    const double* y = Y + (size_t)sl * n;
    const double b = rho[j] * block_dot(y, q, n, red);
    const double c = alpha[j] - b;
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] += c * s[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = -q[i];
  __syncthreads();
  const double gp = block_dot(g, p, n, red);
  const double pp = block_dot(p, p, n, red);
  if (threadIdx.x == 0) { out[0] = gp; out[1] = pp; }
}

// xt = x + a p
__global__ void __launch_bounds__(kOptThreads)
lbfgs_trial_k(int n, const double* __restrict__ x, double a, const double* __restrict__ p,
              double* __restrict__ xt) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) xt[i] = x[i] + a * p[i];
}

// s = xt - x, y = gt - g; out[0] = s.y, out[1] = s.s, out[2] = y.y
__global__ void __launch_bounds__(kOptThreads)
lbfgs_pair_k(int n, const double* __restrict__ xt, const double* __restrict__ x,
             const double* __restrict__ gt, const double* __restrict__ g, double* __restrict__ s,
             double* __restrict__ y, double* __restrict__ out) {
  __shared__ double red[33];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s[i] = xt[i] - x[i];
    y[i] = gt[i] - g[i];
  }
  __syncthreads();
  const double sy = block_dot(s, y, n, red);
  const double ss = block_dot(s, s, n, red);
  const double yy = block_dot(y, y, n, red);
  if (threadIdx.x == 0) { out[0] = sy; out[1] = ss; out[2] = yy; }
}

}  // namespace

cudaError_t lbfgs_direction(int n, int cnt, int head, int hist, const double* S, const double* Y,
                            const double* g, double* q, double* p, double* out, cudaStream_t s) {
  if (cnt < 0 || cnt > hist || hist > 32) return cudaErrorInvalidValue;
  lbfgs_direction_k<<<1, kOptThreads, 0, s>>>(n, cnt, head, hist, S, Y, g, q, p, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t lbfgs_trial(int n, const double* x, double a, const double* p, double* xt,
                        cudaStream_t s) {
  lbfgs_trial_k<<<1, kOptThreads, 0, s>>>(n, x, a, p, xt);
  note_launch();
  return cudaGetLastError();
}

cudaError_t lbfgs_pair(int n, const double* xt, const double* x, const double* gt,
                       const double* g, double* s_out, double* y_out, double* out,
                       cudaStream_t s) {
  lbfgs_pair_k<<<1, kOptThreads, 0, s>>>(n, xt, x, gt, g, s_out, y_out, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
