// k_noalloc.cu -- a pool screen that allocates nothing and needs no caller
// workspace.
//
// Some callers cannot allocate device memory at the moment they need a
// screen: code running while a stream is being captured into a CUDA graph
// (cudaMalloc is not allowed there), real-time loops that cannot afford the
// device-wide synchronisation cudaMalloc implies, and hosts that hand all of
// the device's memory to their own allocator.  cvq_screen_subset_noalloc
// serves them: it reads the caller's complex128 state directly, forms each
// row of H psi on the fly, and keeps its per-CTA partial sums in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>

#include "cvq_internal.cuh"

namespace cvq {

const SectorDev* internal_sector(const cvq_sector* s);
const GateArg* internal_pool_ops(const cvq_pool* p, const cvq_sector** sec, int* K);
int internal_fail(int code, const char* msg);

constexpr int NOALLOC_MAX_SUBSET = 64;

// Shared by every call on a device: NOALLOC_MAX_SUBSET x NBLK partial sums
// (311,296 bytes).  Every call overwrites the rows it uses before reading
// them, so nothing has to start at zero; calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_SUBSET * NBLK];

__device__ __forceinline__ cdf load_c128(const double2* p, int64_t x) {
  const double2 v = p[x];
  return make_cdf(df_from_double(v.x), df_from_double(v.y));
}

__device__ __forceinline__ df df_scale_c(df a, float c) { return df_make(a.h * c, a.l * c); }

// Index of tuple w (index x) moved by (dr on r, ds on s).
template <int KIND>
__device__ __forceinline__ int64_t na_moved(int64_t x, uint64_t w, uint64_t wR, int64_t f, int r, int dr, int s, int ds,
                                            const SectorDev& S, const int64_t (*G)[DMAX + 1]) {
  if (KIND == CVQ_BKC) {
    int64_t g = f + (int64_t)dr * S.stride[r];
    if (s >= 0) g += (int64_t)ds * S.stride[s];
    return g >> 1;
  }
  return x + bh_move_delta(w, wR, r, s, dr, S.L, G);
}

// For every screened element k: partial[k][cta] = sum over this CTA's
// amplitudes of Re conj((H psi)[x]) (A_k psi)[x], with (H psi)[x] formed from
// the Hamiltonian row of x.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_screen_noalloc(const __grid_constant__ SectorDev S,
                                                             const GateArg* __restrict__ pool,
                                                             const __grid_constant__ SubsetArg sub,
                                                             const double2* __restrict__ psi, double* __restrict__ partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ float2 dE[LMAX][DMAX];
  __shared__ float2 P[4][DMAX][DMAX];
  __shared__ float2 sq[DMAX][5];
  __shared__ float2 hop[LMAX], pair[LMAX];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) (&dE[0][0])[e] = (&S.tab->diagE[0][0])[e];
  for (int e = threadIdx.x; e < 4 * DMAX * DMAX; e += blockDim.x) (&P[0][0][0])[e] = (&S.tab->P[0][0][0])[e];
  for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) (&sq[0][0])[e] = (&S.tab->sq[0][0])[e];
  for (int e = threadIdx.x; e < LMAX; e += blockDim.x) {
    hop[e] = S.tab->hop[e];
    pair[e] = S.tab->pair[e];
  }
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
      const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, L, S.N, Gs, &wR);
      const int64_t f = (KIND == CVQ_BKC) ? 2 * x + (occ_get(w, L - 1) & 1) : 0;
      // sigma = (H psi)[x]
      const cdf p = load_c128(psi, x);
      dfacc dgs;
      acc_zero(dgs);
      for (int r = 0; r < L; ++r) {
        const float2 e = dE[r][occ_get(w, r)];
        acc_add(dgs, df_make(e.x, e.y));
      }
      const df d = acc_get(dgs);
      dfacc sr_, si_;
      acc_zero(sr_);
      acc_zero(si_);
      acc_mac(sr_, d, re_of(p));
      acc_mac(si_, d, im_of(p));
      for (int b = 0; b < S.nb; ++b) {
        const int r = b, s = (b + 1 == L) ? 0 : b + 1;
        const int nr = occ_get(w, r), ns = occ_get(w, s);
        const df h = df_make(hop[b].x, hop[b].y);
        if (h.h != 0.f) {
          if (ns >= 1 && nr < Dm1) {
            const df c = df_mul(h, df_make(P[0][nr][ns].x, P[0][nr][ns].y));
            const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, r, +1, s, -1, S, Gs));
            acc_mac(sr_, c, re_of(q));
            acc_mac(si_, c, im_of(q));
          }
          if (nr >= 1 && ns < Dm1) {
            const df c = df_mul(h, df_make(P[1][nr][ns].x, P[1][nr][ns].y));
            const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, r, -1, s, +1, S, Gs));
            acc_mac(sr_, c, re_of(q));
            acc_mac(si_, c, im_of(q));
          }
        }
        if (KIND == CVQ_BKC) {
          const df pc = df_make(pair[b].x, pair[b].y);
          if (pc.h != 0.f) {
            if (nr < Dm1 && ns < Dm1) {
              const df c = df_mul(pc, df_make(P[2][nr][ns].x, P[2][nr][ns].y));
              const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, r, +1, s, +1, S, Gs));
              acc_mac(sr_, c, re_of(q));
              acc_mac(si_, c, im_of(q));
            }
            if (nr >= 1 && ns >= 1) {
              const df c = df_mul(pc, df_make(P[3][nr][ns].x, P[3][nr][ns].y));
              const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, r, -1, s, -1, S, Gs));
              acc_mac(sr_, c, re_of(q));
              acc_mac(si_, c, im_of(q));
            }
          }
        }
      }
      const cdf sg = make_cdf(acc_get(sr_), acc_get(si_));
      // (A_k psi)[x] and its overlap with sigma
      const int ni = occ_get(w, i);
      if (dg) {
        const int fv = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, j);
        if (fv) {
          dfacc c;
          acc_zero(c);
          acc_mac(c, im_of(sg), re_of(p));
          acc_mac(c, df_neg(re_of(sg)), im_of(p));
          acc_macf(acc, acc_get(c), (float)fv);
        }
        continue;
      }
      const int nj = (j >= 0) ? occ_get(w, j) : 0;
      if (ni + di >= 0 && ni + di <= Dm1 && (j < 0 || (nj + dj >= 0 && nj + dj <= Dm1))) {
        df F = df_make(sq[ni][di + 2].x, sq[ni][di + 2].y);
        if (j >= 0) F = df_mul(F, df_make(sq[nj][dj + 2].x, sq[nj][dj + 2].y));
        const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, i, di, j, dj, S, Gs));
        dfacc z;
        acc_zero(z);
        if (cpr != 0.f) {
          acc_mac(z, df_scale_c(re_of(sg), cpr), re_of(q));
          acc_mac(z, df_scale_c(im_of(sg), cpr), im_of(q));
        }
        if (cpi != 0.f) {
          acc_mac(z, df_scale_c(re_of(sg), -cpi), im_of(q));
          acc_mac(z, df_scale_c(im_of(sg), cpi), re_of(q));
        }
        acc_mac(acc, F, acc_get(z));
      }
      if (ni - di >= 0 && ni - di <= Dm1 && (j < 0 || (nj - dj >= 0 && nj - dj <= Dm1))) {
        df F = df_make(sq[ni][2 - di].x, sq[ni][2 - di].y);
        if (j >= 0) F = df_mul(F, df_make(sq[nj][2 - dj].x, sq[nj][2 - dj].y));
        const cdf q = load_c128(psi, na_moved<KIND>(x, w, wR, f, i, -di, j, -dj, S, Gs));
        dfacc z;
        acc_zero(z);
        if (cpr != 0.f) {
          acc_mac(z, df_scale_c(re_of(sg), -cpr), re_of(q));
          acc_mac(z, df_scale_c(im_of(sg), -cpr), im_of(q));
        }
        if (cpi != 0.f) {
          acc_mac(z, df_scale_c(re_of(sg), -cpi), im_of(q));
          acc_mac(z, df_scale_c(im_of(sg), cpi), re_of(q));
        }
        acc_mac(acc, F, acc_get(z));
      }
    }
    const double r = block_sum(acc_to_double(acc));
    if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = r;
  }
}

// 2 x the fixed-order sum of each row of partials.
__global__ void k_noalloc_reduce(const double* __restrict__ partial, double* __restrict__ out) {
  const int r = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < NBLK; b += blockDim.x) v += partial[(size_t)r * NBLK + b];
  v = block_sum(v);
  if (threadIdx.x == 0) out[r] = 2.0 * v;
}

// Device address of the scratch array, looked up once per device.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[256];

static int noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return internal_fail(CVQ_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return internal_fail(CVQ_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_partial);
    if (e != cudaSuccess || !ptr) return internal_fail(CVQ_ECUDA, "cudaGetSymbolAddress of the screen scratch failed");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return CVQ_OK;
}

}  // namespace cvq

using namespace cvq;

extern "C" int cvq_screen_subset_noalloc(const cvq_sector* s, const cvq_pool* p, const cvq_c128* psi,
                                         const int* subset, int n_subset, double* grad_dev, void* stream) {
  if (!s || !p || !psi || !subset || !grad_dev) return internal_fail(CVQ_EINVAL, "null argument");
  const cvq_sector* owner = nullptr;
  int K = 0;
  const GateArg* ops = internal_pool_ops(p, &owner, &K);
  if (owner != s) return internal_fail(CVQ_EINVAL, "pool belongs to another sector");
  if (n_subset < 1 || n_subset > NOALLOC_MAX_SUBSET)
    return internal_fail(CVQ_EINVAL, "n_subset must be in [1, 64] for cvq_screen_subset_noalloc");
  SubsetArg sub;
  sub.n = n_subset;
  for (int k = 0; k < n_subset; ++k) {
    if (subset[k] < 0 || subset[k] >= K) return internal_fail(CVQ_EINVAL, "subset entry outside the pool");
    sub.idx[k] = subset[k];
  }
  double* scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  const SectorDev& S = *internal_sector(s);
  cudaStream_t st = (cudaStream_t)stream;
  if (S.kind == CVQ_BH)
    k_screen_noalloc<CVQ_BH><<<NBLK, NTHREADS, 0, st>>>(S, ops, sub, (const double2*)psi, scratch);
  else
    k_screen_noalloc<CVQ_BKC><<<NBLK, NTHREADS, 0, st>>>(S, ops, sub, (const double2*)psi, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(CVQ_ECUDA, cudaGetErrorString(e));
  k_noalloc_reduce<<<n_subset, NTHREADS, 0, st>>>(scratch, grad_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(CVQ_ECUDA, cudaGetErrorString(e));
  return CVQ_OK;
}
