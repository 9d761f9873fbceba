// k_hamiltonian.cu -- matrix-free sector matvec sigma = H psi with the fused
// energy reduction Re <psi|sigma> (Sec. IV.A/B), the Eq. (grad) pool screen
// g_k = 2 Re <H psi|A_k psi>, and the fixed-order final reduction.
//
// Every kernel runs a fixed grid (NBLK CTAs x NTHREADS threads) in grid-stride
// loops and leaves one partial sum per CTA, so the reductions are
// deterministic for a given sector.
#include "cvq_internal.cuh"

namespace cvq {

__device__ __forceinline__ double block_sum_h(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

struct SectorTables {
  int64_t G[LMAX][DMAX + 1];
  double sqf[DMAX][5];
};

__device__ __forceinline__ void load_tables(SectorTables& T, const SectorDev& S) {
  for (int e = threadIdx.x; e < LMAX * (DMAX + 1); e += blockDim.x) T.G[e / (DMAX + 1)][e % (DMAX + 1)] = S.G[e / (DMAX + 1)][e % (DMAX + 1)];
  for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) T.sqf[e / 5][e % 5] = S.sqf[e / 5][e % 5];
  __syncthreads();
}

template <int KIND>
__device__ __forceinline__ uint64_t unrank(int64_t x, const SectorDev& S, const SectorTables& T) {
  return (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, S.L, S.N, T.G);
}

// Index of the tuple w moved by (dr on mode r, ds on mode s); f is the BKC
// full index of w.
template <int KIND>
__device__ __forceinline__ int64_t moved_index(uint64_t w, int64_t f, int r, int dr, int s, int ds, const SectorDev& S,
                                               const SectorTables& T) {
  if (KIND == CVQ_BKC) {
    int64_t g = f + (int64_t)dr * S.stride[r];
    if (s >= 0) g += (int64_t)ds * S.stride[s];
    return g >> 1;
  } else {
    uint64_t v = occ_shift(w, r, dr);
    if (s >= 0) v = occ_shift(v, s, ds);
    return bh_rank(v, S.L, S.N, T.G);
  }
}

template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_apply_H(const __grid_constant__ SectorDev S, const double2* __restrict__ psi,
                                                      double2* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ SectorTables T;
  load_tables(T, S);
  const int L = S.L, Dm1 = S.D - 1;
  double eacc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = unrank<KIND>(x, S, T);
    const int64_t f = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
    const double2 p = psi[x];
    double dg = 0.0;
    for (int r = 0; r < L; ++r) {
      const double n = (double)occ_get(w, r);
      dg += S.nn1[r] * n * (n - 1.0) + S.n2[r] * n * n + S.n1[r] * n;
    }
    double ar = dg * p.x, ai = dg * p.y;
    for (int b = 0; b < S.nb; ++b) {
      const int r = b, s = (b + 1 == L) ? 0 : b + 1;
      const int nr = occ_get(w, r), ns = occ_get(w, s);
      const double h = S.hop[b];
      if (h != 0.0) {
        if (ns >= 1 && nr < Dm1) {   // <x| a_r^dag a_s |x - e_r + e_s>... neighbour x + e_r - e_s
          const double c = h * T.sqf[nr][3] * T.sqf[ns][1];
          const double2 q = psi[moved_index<KIND>(w, f, r, +1, s, -1, S, T)];
          ar = fma(c, q.x, ar);
          ai = fma(c, q.y, ai);
        }
        if (nr >= 1 && ns < Dm1) {   // neighbour x - e_r + e_s
          const double c = h * T.sqf[nr][1] * T.sqf[ns][3];
          const double2 q = psi[moved_index<KIND>(w, f, r, -1, s, +1, S, T)];
          ar = fma(c, q.x, ar);
          ai = fma(c, q.y, ai);
        }
      }
      const double pc = S.pair[b];
      if (KIND == CVQ_BKC && pc != 0.0) {
        if (nr < Dm1 && ns < Dm1) {  // neighbour x + e_r + e_s (a_r a_s lowers it to x)
          const double c = pc * T.sqf[nr][3] * T.sqf[ns][3];
          const double2 q = psi[moved_index<KIND>(w, f, r, +1, s, +1, S, T)];
          ar = fma(c, q.x, ar);
          ai = fma(c, q.y, ai);
        }
        if (nr >= 1 && ns >= 1) {    // neighbour x - e_r - e_s
          const double c = pc * T.sqf[nr][1] * T.sqf[ns][1];
          const double2 q = psi[moved_index<KIND>(w, f, r, -1, s, -1, S, T)];
          ar = fma(c, q.x, ar);
          ai = fma(c, q.y, ai);
        }
      }
    }
    sigma[x] = make_double2(ar, ai);
    eacc = fma(p.x, ar, eacc);
    eacc = fma(p.y, ai, eacc);
  }
  if (partial) {
    const double s = block_sum_h(eacc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

cudaError_t launch_apply_H(const SectorDev& S, const double2* psi, double2* sigma, double* partial, cudaStream_t st) {
  if (S.kind == CVQ_BH) k_apply_H<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, psi, sigma, partial);
  else k_apply_H<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, psi, sigma, partial);
  return cudaGetLastError();
}

// ------------------------------------------------------------ screen

// Row rule of a pool generator: (A psi)[x] = cp F(x, x+m) psi[x+m]
// - conj(cp) F(x, x-m) psi[x-m] for the move m = (di on mode i, dj on mode j),
// or i f(n(x)) psi[x] for a diagonal generator.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_screen(const __grid_constant__ SectorDev S, const GateArg* __restrict__ pool,
                                                     const __grid_constant__ SubsetArg sub, const double2* __restrict__ psi,
                                                     const double2* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ SectorTables T;
  load_tables(T, S);
  const int L = S.L, Dm1 = S.D - 1;
  for (int k = 0; k < sub.n; ++k) {
    const GateArg& op = pool[sub.idx[k]];
    const int i = op.i, j = op.t.single ? -1 : op.j;
    const int di = op.t.di, dj = op.t.dj, dg = op.t.diag;
    const double2 cp = make_double2(op.t.cp_re, op.t.cp_im);
    double acc = 0.0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
      const uint64_t w = unrank<KIND>(x, S, T);
      const double2 s = sigma[x];
      const int ni = occ_get(w, i);
      if (dg) {
        int f;
        if (dg == 1) f = ni * ni;
        else if (dg == 2) f = ni * (ni - 1);
        else if (dg == 3) f = ni;
        else f = ni * occ_get(w, j);
        const double2 p = psi[x];
        // Re(conj(s) * i f p)
        acc = fma((double)f, fma(s.y, p.x, -s.x * p.y), acc);
        continue;
      }
      const int nj = (j >= 0) ? occ_get(w, j) : 0;
      const int64_t f = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
      double tr = 0.0, ti = 0.0;
      if (ni + di >= 0 && ni + di <= Dm1 && (j < 0 || (nj + dj >= 0 && nj + dj <= Dm1))) {
        const double F = T.sqf[ni][di + 2] * (j >= 0 ? T.sqf[nj][dj + 2] : 1.0);
        const double2 q = psi[moved_index<KIND>(w, f, i, di, j, dj, S, T)];
        tr += F * (cp.x * q.x - cp.y * q.y);
        ti += F * (cp.x * q.y + cp.y * q.x);
      }
      if (ni - di >= 0 && ni - di <= Dm1 && (j < 0 || (nj - dj >= 0 && nj - dj <= Dm1))) {
        const double F = T.sqf[ni][2 - di] * (j >= 0 ? T.sqf[nj][2 - dj] : 1.0);
        const double2 q = psi[moved_index<KIND>(w, f, i, -di, j, -dj, S, T)];
        // -conj(cp) * q
        tr -= F * (cp.x * q.x + cp.y * q.y);
        ti -= F * (cp.x * q.y - cp.y * q.x);
      }
      acc = fma(s.x, tr, acc);
      acc = fma(s.y, ti, acc);
    }
    const double r = block_sum_h(acc);
    if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = r;
  }
}

cudaError_t launch_screen(const SectorDev& S, const GateArg* pool_ops, const SubsetArg& sub, const double2* psi,
                          const double2* sigma, double* partial, cudaStream_t st) {
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
  v = block_sum_h(v);
  if (threadIdx.x == 0) out[r] = scale * v;
}

cudaError_t launch_reduce(const double* partial, int nred, int nblk, double scale, double* out, cudaStream_t st) {
  if (nred <= 0) return cudaSuccess;
  k_reduce<<<nred, NTHREADS, 0, st>>>(partial, nblk, scale, out);
  return cudaGetLastError();
}

}  // namespace cvq

namespace cvq {

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
  const double s = block_sum_h(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// beta = sqrt(sum of partials) (fixed order), v_next = w / beta.
__global__ void __launch_bounds__(NTHREADS) k_lanczos_scale(int64_t dim, const double2* __restrict__ w,
                                                            double2* __restrict__ vn, const double* __restrict__ partial,
                                                            double* __restrict__ beta) {
  __shared__ double nb;
  double v = 0.0;
  for (int b = threadIdx.x; b < NBLK; b += blockDim.x) v += partial[b];
  v = block_sum_h(v);
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
