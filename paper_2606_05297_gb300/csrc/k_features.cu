// k_features.cu -- state features for the learned proposal: <n_r>, <n_r^2> per
// mode in one streaming pass, and <a_i^dag a_j> for a list of mode pairs, one
// pass per pair.  Plain FP64 on the caller's complex128 state (a few flops per
// amplitude); fixed grid, one partial sum per CTA per output, so the results
// are deterministic.
#include "cvq_internal.cuh"

namespace cvq {

template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_features_diag(const __grid_constant__ SectorDev S,
                                                            const double2* __restrict__ psi,
                                                            double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  __syncthreads();
  double acc[2 * LMAX];
#pragma unroll
  for (int k = 0; k < 2 * LMAX; ++k) acc[k] = 0.0;
  const int L = S.L;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, L, S.N, Gs);
    const double2 v = psi[x];
    const double p2 = fma(v.x, v.x, v.y * v.y);
#pragma unroll
    for (int r = 0; r < LMAX; ++r) {
      if (r < L) {
        const double n = (double)occ_get(w, r);
        acc[r] = fma(p2, n, acc[r]);
        acc[LMAX + r] = fma(p2, n * n, acc[LMAX + r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < LMAX; ++r) {
    if (r < L) {
      const double a = block_sum(acc[r]);
      if (threadIdx.x == 0) partial[(size_t)r * NBLK + blockIdx.x] = a;
      const double b = block_sum(acc[LMAX + r]);
      if (threadIdx.x == 0) partial[(size_t)(L + r) * NBLK + blockIdx.x] = b;
    }
  }
}

constexpr int MAX_FEATURE_PAIRS = 240;
struct PairArg {
  int n;
  int pi[MAX_FEATURE_PAIRS], pj[MAX_FEATURE_PAIRS];
};

// <a_i^dag a_j> = sum_x conj(psi[x]) sqrt(n_i (n_j + 1)) psi[x - e_i + e_j]
template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_features_pairs(const __grid_constant__ SectorDev S,
                                                             const __grid_constant__ PairArg a,
                                                             const double2* __restrict__ psi,
                                                             double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ double sqn[DMAX * DMAX];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int k = threadIdx.x; k < DMAX * DMAX; k += blockDim.x) sqn[k] = sqrt((double)k);
  __syncthreads();
  const int L = S.L, Dm1 = S.D - 1;
  for (int p = 0; p < a.n; ++p) {
    const int i = a.pi[p], j = a.pj[p];
    double re = 0.0, im = 0.0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
      uint64_t wR = 0;
      const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, L, S.N, Gs, &wR);
      const int ni = occ_get(w, i), nj = occ_get(w, j);
      if (ni < 1 || nj >= Dm1) continue;
      int64_t y;
      if (KIND == CVQ_BKC) {
        const int64_t f = 2 * x + (occ_get(w, L - 1) & 1);
        y = (f - S.stride[i] + S.stride[j]) >> 1;
      } else {
        y = x + bh_move_delta(w, wR, i, j, -1, L, Gs);
      }
      const double c = sqn[ni * (nj + 1)];
      const double2 u = psi[x], v = psi[y];
      // conj(u) * c v
      re = fma(c, fma(u.x, v.x, u.y * v.y), re);
      im = fma(c, fma(u.x, v.y, -u.y * v.x), im);
    }
    const double sr = block_sum(re);
    if (threadIdx.x == 0) partial[(size_t)(2 * L + 2 * p) * NBLK + blockIdx.x] = sr;
    const double si = block_sum(im);
    if (threadIdx.x == 0) partial[(size_t)(2 * L + 2 * p + 1) * NBLK + blockIdx.x] = si;
  }
}

cudaError_t launch_features(const SectorDev& S, const double2* psi, const int* pi, const int* pj, int npairs,
                            double* partial, cudaStream_t st) {
  if (npairs < 0 || npairs > MAX_FEATURE_PAIRS) return cudaErrorInvalidValue;
  if (S.kind == CVQ_BH) k_features_diag<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, psi, partial);
  else k_features_diag<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, psi, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || npairs == 0) return e;
  PairArg a;
  a.n = npairs;
  for (int p = 0; p < npairs; ++p) {
    a.pi[p] = pi[p];
    a.pj[p] = pj[p];
  }
  if (S.kind == CVQ_BH) k_features_pairs<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, a, psi, partial);
  else k_features_pairs<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, a, psi, partial);
  return cudaGetLastError();
}

}  // namespace cvq
