// Classical networks fed directly (Discussion: QR-CTMRG applies to classical
// partition functions): the boundary built from the network tensor, and the
// partition function per site / one-site expectation values at the fixed
// point.  FP64 throughout.
//
// Network tensor a[u][l][d][r] (bond b), environment C[a][b], T[a][k][b] with
// k < b the inner leg.  Observables (normalisations of C and T cancel):
//   E[x][p][y]     = sum C[x,s] T[s,p,t] C[t,y]                (C T C)
//   Z00            = Tr C^4 = sum_ij C2[i,j] C2[j,i],  C2 = C C
//   Z10            = sum E[x,p,y] E[y,p,x]                       (2x1 ring)
//   F[x][p][q][z]  = sum_y E[x,p,y] T[y,q,z]
//   H[z][x][p][q]  = sum_{r,s} F[z,r,s,x] a[p,s,r,q]
//   Z11            = sum F[x,p,q,z] H[z,x,p,q]                   (3x3 patch)
//   kappa = Z11 Z00 / Z10^2,  <O> = Z11(a_obs) / Z11(a).
#include <algorithm>

#include "ctx.cuh"

namespace qrctm {

namespace {

constexpr int kDotBlocks = 256;

// C0[d][r] = sum_{u,l} v[u] v[l] a[u,l,d,r];  T0[u][r][d] = sum_l v[l] a[u,l,d,r]
__global__ void network_boundary_k(int b, const double* __restrict__ a,
                                   const double* __restrict__ v, double* __restrict__ C0,
                                   double* __restrict__ T0) {
  const long long b2 = (long long)b * b, b3 = b2 * b;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b3;
       e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e / b2), r = (int)((e / b) % b), dd = (int)(e % b);
    double t = 0.0;
    for (int l = 0; l < b; ++l) {
      const double vl = v ? v[l] : 1.0;
      t += vl * a[((u * b2 + (long long)l * b + dd) * b) + r];
    }
    T0[e] = t;   // e = (u*b + r)*b + d
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b2;
       e += (long long)gridDim.x * blockDim.x) {
    const int dd = (int)(e / b), r = (int)(e % b);
    double t = 0.0;
    for (int u = 0; u < b; ++u) {
      const double vu = v ? v[u] : 1.0;
      for (int l = 0; l < b; ++l) {
        const double vl = v ? v[l] : 1.0;
        t += vu * vl * a[((u * b2 + (long long)l * b + dd) * b) + r];
      }
    }
    C0[e] = t;
  }
}

// part[blockIdx.x] = sum over this block's share of x[xm(i)] * y[ym(i)], i < n
__global__ void map_dot_k(const double* __restrict__ x, const __grid_constant__ IdxMap xm,
                          const double* __restrict__ y, const __grid_constant__ IdxMap ym,
                          long long n, double* __restrict__ part) {
  __shared__ double red[256 / 32];
  double t = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    t += x[map_off(xm, i)] * y[map_off(ym, i)];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) red[w] = t;
  __syncthreads();
  if (w == 0) {
    t = ln < (int)(blockDim.x >> 5) ? red[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (ln == 0) part[blockIdx.x] = t;
  }
}

// out[k] = sum of part[k*kDotBlocks .. + nblk) in a fixed order (one warp per k)
__global__ void dot_finish_k(const double* __restrict__ part, int nblk, int nk,
                             double* __restrict__ out) {
  const int k = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (k >= nk) return;
  double t = 0.0;
  for (int i = ln; i < nblk; i += 32) t += part[k * kDotBlocks + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (ln == 0) out[k] = t;
}

cudaError_t map_dot(const double* x, IdxMap xm, const double* y, IdxMap ym, long long n,
                    double* part, cudaStream_t s) {
  map_dot_k<<<kDotBlocks, 256, 0, s>>>(x, xm, y, ym, n, part);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t network_boundary(int b, const double* a, const double* v, double* C0, double* T0,
                             cudaStream_t s) {
  const long long b3 = (long long)b * b * b;
  const unsigned nb = (unsigned)std::min<long long>((b3 + 255) / 256, 1024);
  network_boundary_k<<<nb, 256, 0, s>>>(b, a, v, C0, T0);
  note_launch();
  return cudaGetLastError();
}

// Z[0..3] = (Z00, Z10, Z11(a), Z11(a_obs)) into c->e_d (Z[3] only with a_obs).
cudaError_t network_traces(qrctm_ctx* c, const double* a_obs) {
  const int ch = c->chi_cur, b = c->D2;
  const long long bc = (long long)b * ch, b2 = (long long)b * b;
  cudaStream_t s = c->st;
  double* E = c->Mcm;     // [x][p][y]   chi*b*chi
  double* G1 = c->Q;      // [x][p][t]   chi*b*chi
  double* C2 = c->Craw;   // chi*chi
  double* F = c->X1;      // [x][p][q][z]  (chi b)^2
  double* H = c->X2;      // [z][x][p][q]  (chi b)^2
  double* part = c->partials;
  cudaError_t e;
  // C2 = C C
  {
    Gemm g = gemm_ctx(c);
    g.M = ch; g.N = ch; g.K = ch;
    g.A = c->C; g.a_m = im1(ch); g.a_k = im1(1);
    g.B = c->C; g.b_k = im1(ch); g.b_n = im1(1);
    g.C = C2; g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
  }
  // G1[x,(p,t)] = sum_s C[x,s] T[s,(p,t)];  E[(x,p),y] = sum_t G1[(x,p),t] C[t,y]
  {
    Gemm g = gemm_ctx(c);
    g.M = ch; g.N = bc; g.K = ch;
    g.A = c->C; g.a_m = im1(ch); g.a_k = im1(1);
    g.B = c->T; g.b_k = im1(bc); g.b_n = im1(1);
    g.C = G1; g.c_m = im1(bc); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    g = gemm_ctx(c);
    g.M = bc; g.N = ch; g.K = ch;
    g.A = G1; g.a_m = im1(ch); g.a_k = im1(1);
    g.B = c->C; g.b_k = im1(ch); g.b_n = im1(1);
    g.C = E; g.c_m = im1(ch); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
  }
  // F[(x,p),(q,z)] = sum_y E[(x,p),y] T[y,(q,z)]
  {
    Gemm g = gemm_ctx(c);
    g.M = bc; g.N = bc; g.K = ch;
    g.A = E; g.a_m = im1(ch); g.a_k = im1(1);
    g.B = c->T; g.b_k = im1(bc); g.b_n = im1(1);
    g.C = F; g.c_m = im1(bc); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
  }
  // Z00: C2[i,j] C2[j,i];  Z10: E[x,p,y] E[y,p,x]
  if ((e = map_dot(C2, im1(1), C2, im2(ch, ch, 1), (long long)ch * ch, part, s)) != cudaSuccess)
    return e;
  if ((e = map_dot(E, im1(1), E, im3(ch, b, bc, ch, 1), bc * ch, part + kDotBlocks, s)) !=
      cudaSuccess)
    return e;
  // H[(z,x),(p,q)] = sum_{(r,s)} F[z,r,s,x] a[p,s,r,q], then Z11 = sum F[x,p,q,z] H[z,x,p,q]
  const double* nets[2] = {c->a, a_obs};
  const int nk = a_obs ? 4 : 3;
  for (int t = 0; t < (a_obs ? 2 : 1); ++t) {
    Gemm g = gemm_ctx(c);
    g.M = (long long)ch * ch; g.N = b2; g.K = b2;
    g.A = F; g.a_m = im2(ch, 1, b2 * ch); g.a_k = im2(b, ch, bc);
    g.B = nets[t]; g.b_k = im2(b, b2, b); g.b_n = im2(b, 1, b2 * b);
    g.C = H; g.c_m = im1(b2); g.c_n = im1(1);
    if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
    if ((e = map_dot(F, im1(1), H, im4(ch, b, b, b2 * ch, 1, b, b2), bc * bc,
                     part + (2 + t) * kDotBlocks, s)) != cudaSuccess)
      return e;
  }
  dot_finish_k<<<1, 32 * nk, 0, s>>>(part, kDotBlocks, nk, c->e_d);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qrctm
