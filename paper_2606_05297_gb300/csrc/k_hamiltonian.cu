// k_hamiltonian.cu -- matrix-free sector matvec sigma = H psi with the fused
// energy reduction Re <psi|sigma> (Sec. IV.A/B), the Eq. (grad) pool screen
// g_k = 2 Re <H psi|A_k psi>, the fixed-order final reduction, and the
// Lanczos vector update used for E0.
//
// Every kernel runs a fixed grid (NBLK CTAs x NTHREADS threads) in grid-stride
// loops and leaves one partial sum per CTA, so the reductions are
// deterministic for a given sector.  The matvec and the screen work on df
// states (df.cuh); the Lanczos update works on the caller's complex128 vectors.
#include "cvq_internal.cuh"
#include "k_ham_impl.cuh"

namespace cvq {

template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_apply_H(const __grid_constant__ SectorDev S, const cdf* __restrict__ psi,
                                                      cdf* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ HSmem H;
  if (KIND == CVQ_BH) load_G(Gs, S);
  load_htabs(H, S);
  __syncthreads();
  dfacc eacc;
  acc_zero(eacc);
  apply_H_range<KIND>(S, Gs, H, psi, sigma, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, S.dim,
                      (int64_t)gridDim.x * blockDim.x, eacc);
  if (partial) {
    const double s = block_sum(acc_to_double(eacc));
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

cudaError_t launch_apply_H(const SectorDev& S, const cdf* psi, cdf* sigma, double* partial, cudaStream_t st) {
  if (S.kind == CVQ_BH) k_apply_H<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, psi, sigma, partial);
  else k_apply_H<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, psi, sigma, partial);
  return cudaGetLastError();
}

// ------------------------------------------------------------ screen

// c times a df, exact when c is 0, +-1 or a power of two (all c_plus here)
__device__ __forceinline__ df df_scale(df a, float c) { return df_make(a.h * c, a.l * c); }

// Row rule of a pool generator: (A psi)[x] = cp F(x, x+m) psi[x+m]
// - conj(cp) F(x, x-m) psi[x-m] for the move m = (di on mode i, dj on mode j),
// or i f(n(x)) psi[x] for a diagonal generator.  Per element the kernel
// accumulates Re sum_x conj(sigma[x]) (A psi)[x].
template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_screen(const __grid_constant__ SectorDev S, const GateArg* __restrict__ pool,
                                                     const __grid_constant__ SubsetArg sub, const cdf* __restrict__ psi,
                                                     const cdf* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ float2 sq[DMAX][5];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) (&sq[0][0])[e] = (&S.tab->sq[0][0])[e];
  __syncthreads();
  const int L = S.L, Dm1 = S.D - 1;
  for (int k = 0; k < sub.n; ++k) {
    const GateArg& op = pool[sub.idx[k]];
    const int i = op.i, j = op.t.single ? -1 : op.j;
    const int di = op.t.di, dj = op.t.dj, dg = op.t.diag;
    const float cpr = (float)op.t.cp_re, cpi = (float)op.t.cp_im;
    dfacc acc;
    acc_zero(acc);
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
      uint64_t wR = 0;
      const uint64_t w = unrank<KIND>(x, S, Gs, &wR);
      const cdf s = sigma[x];
      const int ni = occ_get(w, i);
      if (dg) {
        const int f = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, j);
        if (f) {
          const cdf p = psi[x];
          dfacc c;  // Re(conj(s) * i f p) = f (s.im p.re - s.re p.im)
          acc_zero(c);
          acc_mac(c, im_of(s), re_of(p));
          acc_mac(c, df_neg(re_of(s)), im_of(p));
          acc_macf(acc, acc_get(c), (float)f);
        }
        continue;
      }
      const int nj = (j >= 0) ? occ_get(w, j) : 0;
      const int64_t f = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
      if (ni + di >= 0 && ni + di <= Dm1 && (j < 0 || (nj + dj >= 0 && nj + dj <= Dm1))) {
        df F = df_make(sq[ni][di + 2].x, sq[ni][di + 2].y);
        if (j >= 0) F = df_mul(F, df_make(sq[nj][dj + 2].x, sq[nj][dj + 2].y));
        const cdf q = psi[moved_index<KIND>(x, w, wR, f, i, di, j, dj, S, Gs)];
        dfacc z;  // Re(cp conj(s) q)
        acc_zero(z);
        if (cpr != 0.f) {
          acc_mac(z, df_scale(re_of(s), cpr), re_of(q));
          acc_mac(z, df_scale(im_of(s), cpr), im_of(q));
        }
        if (cpi != 0.f) {
          acc_mac(z, df_scale(re_of(s), -cpi), im_of(q));
          acc_mac(z, df_scale(im_of(s), cpi), re_of(q));
        }
        acc_mac(acc, F, acc_get(z));
      }
      if (ni - di >= 0 && ni - di <= Dm1 && (j < 0 || (nj - dj >= 0 && nj - dj <= Dm1))) {
        df F = df_make(sq[ni][2 - di].x, sq[ni][2 - di].y);
        if (j >= 0) F = df_mul(F, df_make(sq[nj][2 - dj].x, sq[nj][2 - dj].y));
        const cdf q = psi[moved_index<KIND>(x, w, wR, f, i, -di, j, -dj, S, Gs)];
        dfacc z;  // Re(-conj(cp) conj(s) q)
        acc_zero(z);
        if (cpr != 0.f) {
          acc_mac(z, df_scale(re_of(s), -cpr), re_of(q));
          acc_mac(z, df_scale(im_of(s), -cpr), im_of(q));
        }
        if (cpi != 0.f) {
          acc_mac(z, df_scale(re_of(s), -cpi), im_of(q));
          acc_mac(z, df_scale(im_of(s), cpi), re_of(q));
        }
        acc_mac(acc, F, acc_get(z));
      }
    }
    const double r = block_sum(acc_to_double(acc));
    if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = r;
  }
}

cudaError_t launch_screen(const SectorDev& S, const GateArg* pool_ops, const SubsetArg& sub, const cdf* psi,
                          const cdf* sigma, double* partial, cudaStream_t st) {
  if (sub.n <= 0) return cudaSuccess;
  if (S.kind == CVQ_BH) k_screen<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, pool_ops, sub, psi, sigma, partial);
  else k_screen<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, pool_ops, sub, psi, sigma, partial);
  return cudaGetLastError();
}

// ------------------------------------------------------------ reduce

__global__ void k_reduce(const double* __restrict__ partial, int nblk, double scale, double* __restrict__ out) {
  const int r = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partial[(size_t)r * nblk + b];
  v = block_sum(v);
  if (threadIdx.x == 0) out[r] = scale * v;
}

cudaError_t launch_reduce(const double* partial, int nred, int nblk, double scale, double* out, cudaStream_t st) {
  if (nred <= 0) return cudaSuccess;
  k_reduce<<<nred, NTHREADS, 0, st>>>(partial, nblk, scale, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ Lanczos

__global__ void __launch_bounds__(NTHREADS) k_lanczos_update(int64_t dim, const double2* __restrict__ vp,
                                                             const double2* __restrict__ v, double2* __restrict__ w,
                                                             const double* __restrict__ alpha,
                                                             const double* __restrict__ beta_prev,
                                                             double* __restrict__ partial) {
  const double a = alpha[0], b = beta_prev[0];
  double acc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    double2 t = w[x];
    const double2 c = v[x];
    t.x = fma(-a, c.x, t.x);
    t.y = fma(-a, c.y, t.y);
    if (b != 0.0) {
      const double2 q = vp[x];
      t.x = fma(-b, q.x, t.x);
      t.y = fma(-b, q.y, t.y);
    }
    w[x] = t;
    acc = fma(t.x, t.x, acc);
    acc = fma(t.y, t.y, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// beta = sqrt(sum of partials) (fixed order), v_next = w / beta.
__global__ void __launch_bounds__(NTHREADS) k_lanczos_scale(int64_t dim, const double2* __restrict__ w,
                                                            double2* __restrict__ vn, const double* __restrict__ partial,
                                                            double* __restrict__ beta) {
  __shared__ double nb;
  double v = 0.0;
  for (int b = threadIdx.x; b < NBLK; b += blockDim.x) v += partial[b];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    nb = sqrt(v);
    if (blockIdx.x == 0) beta[0] = nb;
  }
  __syncthreads();
  const double inv = (nb > 0.0) ? 1.0 / nb : 1.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    const double2 t = w[x];
    vn[x] = make_double2(t.x * inv, t.y * inv);
  }
}

cudaError_t launch_lanczos_update(const SectorDev& S, const double2* v_prev, const double2* v, double2* w,
                                  const double* alpha, const double* beta_prev, double* partial, cudaStream_t st) {
  k_lanczos_update<<<NBLK, NTHREADS, 0, st>>>(S.dim, v_prev, v, w, alpha, beta_prev, partial);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_scale(const SectorDev& S, const double2* w, double2* v_next, const double* partial,
                                 double* beta, cudaStream_t st) {
  k_lanczos_scale<<<NBLK, NTHREADS, 0, st>>>(S.dim, w, v_next, partial, beta);
  return cudaGetLastError();
}

}  // namespace cvq
