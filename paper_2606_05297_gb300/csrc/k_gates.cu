// k_gates.cu -- gate engine: per-call block unitaries, forward gate
// application exp(theta A) psi (Sec. IV.B, O_r = exp(theta_r A_r)) and the
// fused reverse step of the adjoint gradient, in double-float arithmetic.
//
// A gate acts block-diagonally: with every mode other than the gate's fixed
// (an "orbit"), the generator couples only the occupation pairs (a, b) of the
// gate's modes that are joined by its move, so each orbit splits into small
// blocks.  One thread owns one orbit (Kitaev chain) or one orbit of a fixed
// pair occupation M (Bose-Hubbard), reads its block amplitudes once,
// multiplies them by the b x b block unitary staged in shared memory and
// writes them back in place.  Runs of consecutive diagonal gates (K, R, CK,
// n(n-1)) are one streaming phase multiply.
#include "cvq_internal.cuh"
#include "k_diag_impl.cuh"
#include "k_gate_impl.cuh"

namespace cvq {

// ------------------------------------------------------------ conversions

__global__ void __launch_bounds__(NTHREADS) k_to_df(int64_t dim, const double2* __restrict__ src, cdf* __restrict__ dst) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[x];
    dst[x] = make_cdf(df_from_double(v.x), df_from_double(v.y));
  }
}

__global__ void __launch_bounds__(NTHREADS) k_from_df(int64_t dim, const cdf* __restrict__ src, double2* __restrict__ dst) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    const cdf v = src[x];
    dst[x] = make_double2(df_to_double(re_of(v)), df_to_double(im_of(v)));
  }
}

cudaError_t launch_to_df(int64_t dim, const double2* src, cdf* dst, cudaStream_t st) {
  k_to_df<<<NBLK, NTHREADS, 0, st>>>(dim, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_from_df(int64_t dim, const cdf* src, double2* dst, cudaStream_t st) {
  k_from_df<<<NBLK, NTHREADS, 0, st>>>(dim, src, dst);
  return cudaGetLastError();
}

// ------------------------------------------------------------ build

// Block unitaries of every gate g of the call: one CTA per (gate, block), so
// the FP64 work spreads over the GPU.
__global__ void k_build(const __grid_constant__ BuildArgs a, const TypeDesc* __restrict__ types, PoolDev P,
                        cdf* __restrict__ U) {
  const int g = blockIdx.x;
  if (g >= a.n) return;
  const TypeDesc& t = types[a.type_of[g]];
  if (t.diag) return;  // diagonal gates are applied from per-run phase tables
  __shared__ double2 ph[MAX_BEXT];
  build_block_unitary(t, a.theta[g], P, U + (size_t)g * a.ustride, blockIdx.y, ph,
                      a.D ? a.D + (size_t)g * a.ustride : nullptr);
}

cudaError_t launch_build_gates(const BuildArgs& a, const TypeDesc* types_dev, PoolDev P, cdf* U, cudaStream_t st) {
  if (a.n <= 0 || a.maxblk <= 0) return cudaSuccess;
  k_build<<<dim3(a.n, a.maxblk), 128, 0, st>>>(a, types_dev, P, U);
  return cudaGetLastError();
}

// ------------------------------------------------------------ block gates

// Defined in k_gate_impl.cuh, instantiated in k_gate_{bh,bkc}_{fwd,adj}.cu.
template <int KIND, bool ADJ>
void launch_block(const SectorDev& S, const GateArg& g, PoolDev P, const cdf* src, cdf* dst, cdf* lam, double* partial,
                  size_t sm, cudaStream_t st);
template <int KIND, bool ADJ>
void set_block_smem_limit(int bytes);

template <bool ADJ>
static cudaError_t launch_gate_impl(const SectorDev& S, const GateArg& g, PoolDev P, const cdf* src, cdf* dst,
                                    cdf* lam, double* partial, cudaStream_t st) {
  if (g.tm.idx && src == dst && !g.t.diag) return launch_tile_gate(g, P, dst, lam, partial, ADJ, st);
  // The largest gate table: a two-mode gate at cutoff 16 has at most
  // 2 * (1^2 + ... + 15^2) + 16^2 = 2736 block entries and at most 64 blocks.
  constexpr int kMaxNu = 2816, kMaxBlocks = 64;
  if (g.t.diag || g.t.nu > kMaxNu || g.t.nblocks > kMaxBlocks) return cudaErrorInvalidValue;
  // the largest gate (cutoff 16) needs ~150 KB: tables plus 256 staging columns of 16 entries
  constexpr int kMaxSmem = 200 * 1024;
  const size_t sm = gate_smem_bytes(g.t, S.kind);
  if (sm > (size_t)kMaxSmem) return cudaErrorInvalidValue;
  // one opt-in to the largest dynamic shared memory a gate can need (a
  // function-local static: done once, also when several host threads launch)
  static const bool attr_set = [] {
    set_block_smem_limit<CVQ_BH, ADJ>(kMaxSmem);
    set_block_smem_limit<CVQ_BKC, ADJ>(kMaxSmem);
    return true;
  }();
  (void)attr_set;
  if (S.kind == CVQ_BH) launch_block<CVQ_BH, ADJ>(S, g, P, src, dst, lam, partial, sm, st);
  else launch_block<CVQ_BKC, ADJ>(S, g, P, src, dst, lam, partial, sm, st);
  return cudaGetLastError();
}

cudaError_t launch_gate(const SectorDev& S, const GateArg& g, PoolDev P, const cdf* src, cdf* dst, cudaStream_t st) {
  return launch_gate_impl<false>(S, g, P, src, dst, nullptr, nullptr, st);
}

cudaError_t launch_gate_adjoint(const SectorDev& S, const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial,
                                cudaStream_t st) {
  return launch_gate_impl<true>(S, g, P, psi, psi, lam, partial, st);
}

// ------------------------------------------------------------ diagonal runs

// One run per launch, phase tables built on the host in FP64.  NACC: the
// gradient accumulators of the reverse pass (diag_run_acc); with 24 the
// registers allow two CTAs per SM, so the grid is NBLK / 2 and CTA 0 zeroes
// the other half of each gradient row's partial slots.
template <int KIND, bool ADJ, bool KEEP, int NACC>
__global__ void __launch_bounds__(NTHREADS, NACC > DIAG_ACC ? 2 : 4)
    k_diag_run(const __grid_constant__ SectorDev S, const __grid_constant__ DiagRunArg a, const cdf* src, cdf* dst,
               cdf* lam, double* partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ cdf T[LMAX][DMAX];
  __shared__ cdf TP[MAX_RUN_PAIRS][DMAX * DMAX];
  __shared__ uint64_t wbuf[(KIND == CVQ_BH) ? NTHREADS / 32 * 32 * WALK_RMAX : 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) T[e / DMAX][e % DMAX] = a.T[e / DMAX][e % DMAX];
  for (int e = threadIdx.x; e < a.npair * DMAX * DMAX; e += blockDim.x)
    TP[e / (DMAX * DMAX)][e % (DMAX * DMAX)] = a.TP[e / (DMAX * DMAX)][e % (DMAX * DMAX)];
  __syncthreads();
  // Reverse: gradients of the run's first NACC gates; the host launches
  // k_diag_grad beforehand for the rest.
  dfacc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc_zero(acc[k]);
  if (KIND == CVQ_BH)
    bh_walk(S, Gs, wbuf, 0, S.dim,
            [&](int64_t x, uint64_t w) { diag_run_one<ADJ, NACC, DiagRunArg, KEEP>(S, T, TP, a, src, dst, lam, x, w, acc); });
  else
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x)
      diag_run_one<ADJ, NACC, DiagRunArg, KEEP>(S, T, TP, a, src, dst, lam, x, bkc_unrank(x, S), acc);
  if (ADJ) {
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      if (k < a.m) {
        const double s = block_sum(acc_to_double(acc[k]));
        if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = s;
        if (blockIdx.x == 0)
          for (int e = gridDim.x + threadIdx.x; e < NBLK; e += blockDim.x) partial[(size_t)k * NBLK + e] = 0.0;
      }
    }
  }
}

// Two CTAs per SM (its 16 accumulators take about 120 registers), so half the
// NBLK partial slots of each gradient row; CTA 0 zeroes the other half.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS, 2) k_diag_grad(const __grid_constant__ SectorDev S,
                                                        const __grid_constant__ DiagGradArg a, const cdf* psi,
                                                        const cdf* lam, double* partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ uint64_t wbuf[(KIND == CVQ_BH) ? NTHREADS / 32 * 32 * WALK_RMAX : 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  __syncthreads();
  dfacc acc[DIAG_GRAD_ACC];
#pragma unroll
  for (int k = 0; k < DIAG_GRAD_ACC; ++k) acc_zero(acc[k]);
  if (KIND == CVQ_BH)
    bh_walk(S, Gs, wbuf, 0, S.dim,
            [&](int64_t x, uint64_t w) { diag_grad_one<DIAG_GRAD_ACC>(a, psi, lam, x, w, acc); });
  else
    diag_grad_range<KIND, DIAG_GRAD_ACC>(S, Gs, a, psi, lam, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, S.dim,
                                         (int64_t)gridDim.x * blockDim.x, acc);
#pragma unroll
  for (int k = 0; k < DIAG_GRAD_ACC; ++k) {
    if (k < a.m) {
      const double s = block_sum(acc_to_double(acc[k]));
      if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = s;
      if (blockIdx.x == 0)
        for (int e = gridDim.x + threadIdx.x; e < NBLK; e += blockDim.x) partial[(size_t)k * NBLK + e] = 0.0;
    }
  }
}

cudaError_t launch_diag_grad(const SectorDev& S, const DiagGradArg& a, const cdf* psi, const cdf* lam, double* partial,
                             cudaStream_t st) {
  if (S.kind == CVQ_BH) k_diag_grad<CVQ_BH><<<NBLK / 2, NTHREADS, 0, st>>>(S, a, psi, lam, partial);
  else k_diag_grad<CVQ_BKC><<<NBLK / 2, NTHREADS, 0, st>>>(S, a, psi, lam, partial);
  return cudaGetLastError();
}

template <int KIND>
static void launch_diag_run_kind(const SectorDev& S, const DiagRunArg& a, const cdf* src, cdf* dst, cdf* lam,
                                 double* partial, bool adjoint, cudaStream_t st, bool keep_psi) {
  if (!adjoint) {
    k_diag_run<KIND, false, false, DIAG_ACC><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
  } else if (diag_run_acc(a.m) == DIAG_ACC) {
    if (keep_psi) k_diag_run<KIND, true, true, DIAG_ACC><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
    else k_diag_run<KIND, true, false, DIAG_ACC><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
  } else {
    if (keep_psi)
      k_diag_run<KIND, true, true, DIAG_ACC_LONG><<<NBLK / 2, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
    else
      k_diag_run<KIND, true, false, DIAG_ACC_LONG><<<NBLK / 2, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
  }
}

cudaError_t launch_diag_run(const SectorDev& S, const DiagRunArg& a, const cdf* src, cdf* dst, cdf* lam,
                            double* partial, bool adjoint, cudaStream_t st, bool keep_psi) {
  if (keep_psi && !adjoint) return cudaErrorInvalidValue;
  if (S.kind == CVQ_BH) launch_diag_run_kind<CVQ_BH>(S, a, src, dst, lam, partial, adjoint, st, keep_psi);
  else launch_diag_run_kind<CVQ_BKC>(S, a, src, dst, lam, partial, adjoint, st, keep_psi);
  return cudaGetLastError();
}

}  // namespace cvq
