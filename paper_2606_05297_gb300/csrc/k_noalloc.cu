// k_noalloc.cu -- a pool screen that allocates nothing and needs no caller
// workspace.
//
// Some callers cannot allocate device memory at the moment they need a
// screen: latency-critical loops that cannot pay for the device-wide
// synchronisation a cudaMalloc brings, host applications whose own caching
// allocator has already reserved all of the device's memory (a cudaMalloc by
// this library would then fail), and plug-ins that a host process hands fixed
// buffers and forbids allocating.  cvq_screen_subset_noalloc serves them: it
// reads the caller's complex128 state directly, forms each row of H psi on
// the fly (once per pass of eight screened elements), and keeps its per-CTA
// partial sums in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
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

// Screened elements handled per pass over the sector: each pass forms every
// row of H psi once and shares it among this many elements.
constexpr int NOALLOC_CHUNK = 8;

// For every screened element k: partial[k][cta] = sum over this CTA's
// amplitudes of Re conj((H psi)[x]) (A_k psi)[x], with (H psi)[x] formed from
// the Hamiltonian row of x once per pass of NOALLOC_CHUNK elements.
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
  __shared__ int4 emv[NOALLOC_CHUNK];   // (i, j or -1, di, dj) of the pass's elements
  __shared__ int edg[NOALLOC_CHUNK];    // diagonal function (0: a ladder move)
  __shared__ float2 ecp[NOALLOC_CHUNK]; // c_plus
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) (&dE[0][0])[e] = (&S.tab->diagE[0][0])[e];
  for (int e = threadIdx.x; e < 4 * DMAX * DMAX; e += blockDim.x) (&P[0][0][0])[e] = (&S.tab->P[0][0][0])[e];
  for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) (&sq[0][0])[e] = (&S.tab->sq[0][0])[e];
  for (int e = threadIdx.x; e < LMAX; e += blockDim.x) {
    hop[e] = S.tab->hop[e];
    pair[e] = S.tab->pair[e];
  }
  const int L = S.L, Dm1 = S.D - 1;
  for (int c0 = 0; c0 < sub.n; c0 += NOALLOC_CHUNK) {
    const int cnt = min(NOALLOC_CHUNK, sub.n - c0);
    __syncthreads();  // the previous pass has finished reading the element tables
    if (threadIdx.x < cnt) {
      const GateArg& op = pool[sub.idx[c0 + threadIdx.x]];
      emv[threadIdx.x] = make_int4(op.i, op.t.single ? -1 : op.j, op.t.di, op.t.dj);
      edg[threadIdx.x] = op.t.diag;
      ecp[threadIdx.x] = make_float2((float)op.t.cp_re, (float)op.t.cp_im);
    }
    __syncthreads();
    dfacc acc[NOALLOC_CHUNK];
#pragma unroll
    for (int q = 0; q < NOALLOC_CHUNK; ++q) acc_zero(acc[q]);
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
      // Re(conj(sigma) i psi) = sigma.im psi.re - sigma.re psi.im, shared by the diagonal elements
      dfacc cd;
      acc_zero(cd);
      acc_mac(cd, im_of(sg), re_of(p));
      acc_mac(cd, df_neg(re_of(sg)), im_of(p));
      const df cdv = acc_get(cd);
      // (A_k psi)[x] of each element of the pass and its overlap with sigma
#pragma unroll
      for (int q = 0; q < NOALLOC_CHUNK; ++q) {
        if (q >= cnt) continue;
        const int4 mv = emv[q];
        const int i = mv.x, j = mv.y, di = mv.z, dj = mv.w, dg = edg[q];
        const float cpr = ecp[q].x, cpi = ecp[q].y;
        const int ni = occ_get(w, i);
        if (dg) {
          const int fv = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, j);
          if (fv) acc_macf(acc[q], cdv, (float)fv);
          continue;
        }
        const int nj = (j >= 0) ? occ_get(w, j) : 0;
        if (ni + di >= 0 && ni + di <= Dm1 && (j < 0 || (nj + dj >= 0 && nj + dj <= Dm1))) {
          df F = df_make(sq[ni][di + 2].x, sq[ni][di + 2].y);
          if (j >= 0) F = df_mul(F, df_make(sq[nj][dj + 2].x, sq[nj][dj + 2].y));
          const cdf qa = load_c128(psi, na_moved<KIND>(x, w, wR, f, i, di, j, dj, S, Gs));
          dfacc z;
          acc_zero(z);
          if (cpr != 0.f) {
            acc_mac(z, df_scale_c(re_of(sg), cpr), re_of(qa));
            acc_mac(z, df_scale_c(im_of(sg), cpr), im_of(qa));
          }
          if (cpi != 0.f) {
            acc_mac(z, df_scale_c(re_of(sg), -cpi), im_of(qa));
            acc_mac(z, df_scale_c(im_of(sg), cpi), re_of(qa));
          }
          acc_mac(acc[q], F, acc_get(z));
        }
        if (ni - di >= 0 && ni - di <= Dm1 && (j < 0 || (nj - dj >= 0 && nj - dj <= Dm1))) {
          df F = df_make(sq[ni][2 - di].x, sq[ni][2 - di].y);
          if (j >= 0) F = df_mul(F, df_make(sq[nj][2 - dj].x, sq[nj][2 - dj].y));
          const cdf qa = load_c128(psi, na_moved<KIND>(x, w, wR, f, i, -di, j, -dj, S, Gs));
          dfacc z;
          acc_zero(z);
          if (cpr != 0.f) {
            acc_mac(z, df_scale_c(re_of(sg), -cpr), re_of(qa));
            acc_mac(z, df_scale_c(im_of(sg), -cpr), im_of(qa));
          }
          if (cpi != 0.f) {
            acc_mac(z, df_scale_c(re_of(sg), -cpi), im_of(qa));
            acc_mac(z, df_scale_c(im_of(sg), cpi), re_of(qa));
          }
          acc_mac(acc[q], F, acc_get(z));
        }
      }
    }
    const double r = block_sums<NOALLOC_CHUNK>([&](int q) { return acc_to_double(acc[q]); }, cnt);
    if ((int)threadIdx.x < cnt) partial[(size_t)(c0 + threadIdx.x) * NBLK + blockIdx.x] = r;
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

// Device address of the scratch array.  In host code the array's name is
// only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with the device current, once per device and CUDA
// context: the cache remembers the context it was filled in (cuCtxGetId, a
// number never reused within a process), so after a device reset, which makes
// a new context with its own copy of the array, the address is looked up again
// instead of pointing into the old one.
typedef int (*PfnCtxGetCurrent)(void**);
typedef int (*PfnCtxGetId)(void*, unsigned long long*);

struct ScratchSlot {
  unsigned long long ctx_id;
  double* ptr;
};

static std::mutex g_noalloc_mu;
static ScratchSlot g_noalloc_slot[256];
static PfnCtxGetCurrent g_ctx_get_current = nullptr;
static PfnCtxGetId g_ctx_get_id = nullptr;

// Id of the calling thread's current CUDA context (0 if it has none yet);
// the caller holds g_noalloc_mu.
static int current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1 ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2)
      return internal_fail(CVQ_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
    g_ctx_get_current = (PfnCtxGetCurrent)f1;
    g_ctx_get_id = (PfnCtxGetId)f2;
  }
  void* ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0) return internal_fail(CVQ_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && g_ctx_get_id(ctx, id) != 0) return internal_fail(CVQ_ECUDA, "cuCtxGetId failed");
  return CVQ_OK;
}

static int noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return internal_fail(cvq_status_from_cuda((int)e), cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return internal_fail(CVQ_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned long long id = 0;
  if (int rc = current_context_id(&id)) return rc;
  ScratchSlot& slot = g_noalloc_slot[dev];
  if (id == 0 || slot.ptr == nullptr || slot.ctx_id != id) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_partial);
    if (e != cudaSuccess || !ptr)
      return internal_fail(e != cudaSuccess ? cvq_status_from_cuda((int)e) : CVQ_ECUDA,
                           "cudaGetSymbolAddress of the screen scratch failed");
    slot.ptr = ptr;
    if (int rc = current_context_id(&slot.ctx_id)) {  // the lookup has made the primary context current
      slot.ptr = nullptr;
      return rc;
    }
  }
  *out = slot.ptr;
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
  if (e != cudaSuccess) return internal_fail(cvq_status_from_cuda((int)e), cudaGetErrorString(e));
  k_noalloc_reduce<<<n_subset, NTHREADS, 0, st>>>(scratch, grad_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(cvq_status_from_cuda((int)e), cudaGetErrorString(e));
  return CVQ_OK;
}
