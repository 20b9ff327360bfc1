// Standard C4v CTMRG step (Standard CTMRG paragraph, Fig. 1(d)): the method
// QR-CTMRG is compared against.  The enlarged corner Ct (chi D^2 square) is
// built by the same contraction chain as the QR step's T' (reduced corner,
// then the edge and both layers of A), symmetrised into a dense FP64 matrix,
// fully diagonalised (cuSOLVER dsyevd, the library eigensolver of the
// comparison method), and the chi eigenvectors of largest |eigenvalue| (ties
// by index) form the isometry U:  C' = U^T Ct U = diag(eigenvalues),
// T' = U^T (T a) U,  then the usual symmetrisation and normalisation.
#include <cusolverDn.h>

#include "ctx.cuh"

namespace qrctm {

namespace {

// E[i + j m] = (Ct(i,j) + Ct(j,i)) / 2 with Ct(i,j) = X2[rmap(i) + cmap(j)]
__global__ void sym_corner_dense_k(const double* __restrict__ X2, double* __restrict__ E,
                                   long long m, const __grid_constant__ IdxMap rmap,
                                   const __grid_constant__ IdxMap cmap) {
  const long long tot = m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % m, j = e / m;
    E[e] = 0.5 * (X2[map_off(rmap, i) + map_off(cmap, j)] + X2[map_off(rmap, j) + map_off(cmap, i)]);
  }
}

// idx[rank] = i for the eigenvalues ranked by |w| descending, ties by index
__global__ void rank_eigs_k(const double* __restrict__ w, int m, int keep, int* __restrict__ idx,
                            const int* info, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && *info != 0) atomicOr(err, ERRF_NUMERIC);
  if (i >= m) return;
  const double ai = fabs(w[i]);
  int rank = 0;
  for (int j = 0; j < m; ++j) {
    const double aj = fabs(w[j]);
    rank += (aj > ai) || (aj == ai && j < i);
  }
  if (rank < keep) idx[rank] = i;
}

// U[:, r] = E[:, idx[r]] (column-major m x keep); Cd = diag(w[idx[r]])
__global__ void gather_eigs_k(const double* __restrict__ E, const double* __restrict__ w,
                              const int* __restrict__ idx, long long m, int keep,
                              double* __restrict__ U, double* __restrict__ Cd) {
  const long long tot = m * keep;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % m, r = e / m;
    U[e] = E[(long long)idx[r] * m + i];
  }
  const long long tc = (long long)keep * keep;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tc;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / keep), b = (int)(e % keep);
    Cd[e] = (a == b) ? w[idx[a]] : 0.0;
  }
}

}  // namespace

// dsyevd's workspace is only known once a solver handle exists (host-only
// planning cannot query it).  Measured requests on B300 (CUDA 13): 4.15 n^2
// doubles at n = 1024, 4.03 n^2 at n = 5184; 5 n^2 + 64 n + 2^20 is reserved.
// A larger request fails the step with cudaErrorMemoryAllocation.
size_t eigen_work_doubles(long long m) { return (size_t)(5 * m * m + 64 * m + (1ll << 20)); }

cudaError_t eigen_step(qrctm_ctx* c, int ci, int co) {
  const int D = c->D, D2 = c->D2;
  const long long D3 = (long long)D2 * D, D4 = (long long)D2 * D2;
  const long long m = (long long)ci * D2;
  if (c->eig_E == nullptr || co > m) return cudaErrorInvalidValue;
  cudaError_t e;
  {
    PhaseScope ps(c, QRCTM_PH_CT);
    if ((e = reduced_corner(c, c->C, c->T, ci, c->Mcm)) != cudaSuccess) return e;
  }
  // X2 <- enlarged corner (the first half of renorm_edge with P = ct)
  if ((e = renorm_edge(c, c->Mcm, ci, c->T, ci, nullptr)) != cudaSuccess) return e;
  {
    PhaseScope ps(c, QRCTM_PH_QR);   // the decomposition phase of this method
    // Ct((b,l),(r,j)) = X2[r,b,l_k,j_k,l_b,j_b]
    const X2Maps xm = x2_maps(c, ci);
    const IdxMap ct_row = xm.ct_row, ct_col = xm.ct_col;
    sym_corner_dense_k<<<(unsigned)std::min<long long>((m * m + 255) / 256, 65535), 256, 0, c->st>>>(
        c->X2, c->eig_E, m, ct_row, ct_col);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cusolverDnHandle_t h = static_cast<cusolverDnHandle_t>(c->solver);
    if (h == nullptr) {
      if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return cudaErrorUnknown;
      c->solver = h;
    }
    if (cusolverDnSetStream(h, c->st) != CUSOLVER_STATUS_SUCCESS) return cudaErrorUnknown;
    int lwork = 0;
    if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)m,
                                    c->eig_E, (int)m, c->eig_w, &lwork) != CUSOLVER_STATUS_SUCCESS)
      return cudaErrorUnknown;
    if ((size_t)lwork > c->eig_work_doubles) return cudaErrorMemoryAllocation;
    if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)m, c->eig_E,
                         (int)m, c->eig_w, c->eig_work, lwork, c->eig_info) !=
        CUSOLVER_STATUS_SUCCESS)
      return cudaErrorUnknown;
    note_launch();
    rank_eigs_k<<<(unsigned)((m + 255) / 256), 256, 0, c->st>>>(c->eig_w, (int)m, co, c->eig_idx,
                                                                c->eig_info, c->err);
    note_launch();
    gather_eigs_k<<<(unsigned)std::min<long long>((m * co + 255) / 256, 65535), 256, 0, c->st>>>(
        c->eig_E, c->eig_w, c->eig_idx, m, co, c->Q, c->Craw);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = renorm_edge(c, c->Q, co, c->T, ci, c->Traw)) != cudaSuccess) return e;
  {
    PhaseScope ps(c, QRCTM_PH_SYMNORM);
    if ((e = sym_norm_env(c->Craw, c->Traw, c->C, c->T, co, D2, c->partials, c->err, c->st)) !=
        cudaSuccess)
      return e;
  }
  c->chi_cur = co;
  c->iters += 1;
  return cudaSuccess;
}

void eigen_release(qrctm_ctx* c) {
  if (c->solver) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(c->solver));
  c->solver = nullptr;
}

}  // namespace qrctm
