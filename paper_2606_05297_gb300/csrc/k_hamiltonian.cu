// k_hamiltonian.cu -- matrix-free sector matvec sigma = H psi with the fused
// energy reduction Re <psi|sigma> (Sec. IV.A/B), the Eq. (grad) pool screen
// g_k = 2 Re <H psi|A_k psi>, the fixed-order final reduction, and the
// Lanczos vector update used for E0.
//
// Every kernel runs a fixed grid (NBLK CTAs x NTHREADS threads, the screen
// screen_grid CTAs) in grid-stride loops and leaves one partial sum per CTA, so
// the reductions are deterministic for a given sector.  The matvec and the screen work on df
// states (df.cuh); the Lanczos update works on the caller's complex128 vectors.
#include "cvq_internal.cuh"
#include "k_ham_impl.cuh"

namespace cvq {

template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_apply_H(const __grid_constant__ SectorDev S, const cdf* __restrict__ psi,
                                                      cdf* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ HSmem H;
  __shared__ int32_t Dp[(KIND == CVQ_BH) ? LMAX : 1][DMAX + 1];
  __shared__ uint64_t wbuf[(KIND == CVQ_BH) ? NTHREADS / 32 * 32 * WALK_RMAX : 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  load_htabs(H, S);
  __syncthreads();
  if (KIND == CVQ_BH) load_dhop(Dp, Gs, S);
  __syncthreads();
  dfacc eacc;
  acc_zero(eacc);
  if (KIND == CVQ_BH)
    bh_walk(S, Gs, wbuf, 0, S.dim,
            [&](int64_t x, uint64_t w) { apply_H_one<KIND>(S, Gs, Dp, H, psi, sigma, x, w, eacc); });
  else
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

// Pool screen, Eq. (grad): for a generator A = cp G - conj(cp) G^dag whose
// ladder string G moves x by delta (and G^dag by -delta),
//   Re <sigma|A psi> = Re(cp Z_delta) - Re(conj(cp) Z_{-delta}),
//   Z_delta = sum_x F_delta(x) conj(sigma[x]) psi[x + delta],
// with F_delta(x) the ladder factor of the move; for a diagonal generator
// A = i f(n), Re <sigma|A psi> = sum_x f(x) Re(conj(sigma[x]) i psi[x]).
// Every pool element that moves by the same delta (both phases of a beam
// splitter or squeezer, for instance) shares one Z, so the kernel streams
// one neighbour read per distinct shift instead of two per element.  Shifts
// are taken SCREEN_CHUNK at a time: a chunk's accumulators stay in registers
// while each CTA walks its share of the sector, then leave one partial per CTA
// (rows 2s and 2s + 1 for Re and Im of shift s, row 2 nsh + d for diagonal
// function d).
// Resident CTAs per SM: four for the Kitaev chain (64 registers), three for
// Bose-Hubbard (its rank walk needs about 80).  The grid is that many per SM,
// screen_grid, so that no second partial wave runs; row e of the partials has
// one slot per CTA.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS, KIND == CVQ_BKC ? 4 : 3) k_screen(const __grid_constant__ SectorDev S,
                                                     const __grid_constant__ ScreenArg a, const cdf* __restrict__ psi,
                                                     const cdf* __restrict__ sigma, double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ float2 sq[DMAX][5];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) (&sq[0][0])[e] = (&S.tab->sq[0][0])[e];
  __syncthreads();
  const int nc_sh = (a.nsh + SCREEN_CHUNK - 1) / SCREEN_CHUNK, nc_dg = (a.ndg + SCREEN_CHUNK - 1) / SCREEN_CHUNK;
  for (int c = 0; c < nc_sh + nc_dg; ++c) {
    const bool isdg = c >= nc_sh;
    const int base = (isdg ? c - nc_sh : c) * SCREEN_CHUNK;
    const int cnt = min(SCREEN_CHUNK, (isdg ? a.ndg : a.nsh) - base);
    dfacc zr[SCREEN_CHUNK], zi[SCREEN_CHUNK];
    screen_chunk<KIND>(S, Gs, sq, isdg, (isdg ? a.dg : a.sh) + base, cnt, psi, sigma,
                       (int64_t)blockIdx.x * blockDim.x + threadIdx.x, S.dim, (int64_t)gridDim.x * blockDim.x, zr, zi);
    // one reduction for the chunk: value 2k and 2k + 1 are Re Z and Im Z of
    // shift k (rows 2 (base + k) and 2 (base + k) + 1), or value k is D of
    // diagonal function k (row 2 nsh + base + k)
    const int m = isdg ? cnt : 2 * cnt, q = threadIdx.x;
    const double s = block_sums<2 * SCREEN_CHUNK>(
        [&](int k) {
          return acc_to_double(isdg ? zr[k & (SCREEN_CHUNK - 1)] : ((k & 1) ? zi[k >> 1] : zr[k >> 1]));
        },
        m);
    if (q < m) partial[(size_t)(isdg ? 2 * a.nsh + base + q : 2 * base + q) * gridDim.x + blockIdx.x] = s;
  }
}

// g_k = 2 [Re(cp Z_+) - Re(conj(cp) Z_-)], or 2 D_d for a diagonal generator.
__global__ void k_screen_epilogue(const __grid_constant__ ScreenMap m, int nsh, const double* __restrict__ z,
                                  double* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.n) return;
  const int4 e = m.e[k];
  const double2 cp = m.cp[k];
  if (e.x) {
    grad[k] = 2.0 * z[2 * nsh + e.y];
  } else {
    const double pr = z[2 * e.y], pi = z[2 * e.y + 1], mr = z[2 * e.z], mi = z[2 * e.z + 1];
    grad[k] = 2.0 * ((cp.x * pr - cp.y * pi) - (cp.x * mr + cp.y * mi));
  }
}

int screen_grid(const SectorDev& S) { return (NBLK / 4) * (S.kind == CVQ_BH ? 3 : 4); }

cudaError_t launch_screen(const SectorDev& S, const ScreenArg& a, const cdf* psi, const cdf* sigma, double* partial,
                          cudaStream_t st) {
  if (a.nsh + a.ndg <= 0) return cudaSuccess;
  const int grid = screen_grid(S);
  if (S.kind == CVQ_BH) k_screen<CVQ_BH><<<grid, NTHREADS, 0, st>>>(S, a, psi, sigma, partial);
  else k_screen<CVQ_BKC><<<grid, NTHREADS, 0, st>>>(S, a, psi, sigma, partial);
  return cudaGetLastError();
}

cudaError_t launch_screen_epilogue(const ScreenMap& m, int nsh, const double* z, double* grad, cudaStream_t st) {
  if (m.n <= 0) return cudaSuccess;
  k_screen_epilogue<<<(m.n + 127) / 128, 128, 0, st>>>(m, nsh, z, grad);
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

// The n gradient rows (scale 2) and the energy row after them (scale 1) in one
// launch, each row summed as k_reduce sums it.
__global__ void k_reduce_eg(const double* __restrict__ partial, int n, int nblk, double* __restrict__ E,
                            double* __restrict__ grad) {
  const int r = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partial[(size_t)r * nblk + b];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    if (r < n) grad[r] = 2.0 * v;
    else E[0] = 1.0 * v;
  }
}

cudaError_t launch_reduce_eg(const double* partial, int n, int nblk, double* E, double* grad, cudaStream_t st) {
  k_reduce_eg<<<n + 1, NTHREADS, 0, st>>>(partial, n, nblk, E, grad);
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
