// k_gate_impl.cuh -- block gate kernels (forward and reverse), instantiated
// once per (sector kind, direction) in k_gate_{bh,bkc}_{fwd,adj}.cu so that
// the translation units compile in parallel.
#pragma once

#include "cvq_internal.cuh"

namespace cvq {

// ------------------------------------------------------------ block math

struct BkcIdx {  // member (a, b) of an orbit with base f0: (f0 + a s_i + b s_j) >> 1
  int64_t f0, si, sj;
  __host__ __device__ __forceinline__ int64_t operator()(int2 m) const { return (f0 + m.x * si + m.y * sj) >> 1; }
};

struct BhIdx {   // member (a, M - a): rank of member (0, M) plus the rank change of moving a bosons j -> i
  uint64_t w0, wR0;
  int64_t r0;
  int i, j, L;
  const int64_t (*G)[DMAX + 1];
  __host__ __device__ __forceinline__ int64_t operator()(int2 m) const {
    return m.x ? r0 + bh_move_delta(w0, wR0, i, j, m.x, L, G) : r0;
  }
};

// out += u * v (complex df), accumulating the real and imaginary parts
template <bool REALU>
__device__ __forceinline__ void cmac(dfacc& ar, dfacc& ai, cdf u, cdf v) {
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  if (!REALU) {
    acc_mac(ar, df_neg(im_of(u)), im_of(v));
    acc_mac(ai, im_of(u), re_of(v));
  }
}

// out += conj(u) * v
template <bool REALU>
__device__ __forceinline__ void cmac_conj(dfacc& ar, dfacc& ai, cdf u, cdf v) {
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  if (!REALU) {
    acc_mac(ar, im_of(u), im_of(v));
    acc_mac(ai, df_neg(im_of(u)), re_of(v));
  }
}

template <int B, bool REALU, class IDX>
__device__ __forceinline__ void block_fwd(const cdf* __restrict__ Ub, const int2* __restrict__ mem, const IDX& idx,
                                          const cdf* src, cdf* dst) {
  int64_t x[B];
  cdf in[B];
#pragma unroll
  for (int l = 0; l < B; ++l) {
    x[l] = idx(mem[l]);
    in[l] = src[x[l]];
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    dfacc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
#pragma unroll
    for (int l = 0; l < B; ++l) cmac<REALU>(ar, ai, Ub[k * B + l], in[l]);
    dst[x[k]] = make_cdf(acc_get(ar), acc_get(ai));
  }
}

// Reverse step for one block.  With the tridiagonal generator
// A[k][k+1] = cp F_k, A[k+1][k] = -conj(cp) F_k the gradient term
// Re sum_k conj(lam_k) (A psi)_k equals sum_k F_k Re(cp z_k),
// z_k = conj(lam_k) psi_{k+1} - lam_{k+1} conj(psi_k).  Then psi <- U^dag psi,
// lam <- U^dag lam.
template <int B, bool REALU, class IDX>
__device__ __forceinline__ void block_adj(const cdf* __restrict__ Ub, const int2* __restrict__ mem,
                                          const float2* __restrict__ F, float cpr, float cpi, const IDX& idx, cdf* psi,
                                          cdf* lam, dfacc& gacc) {
  int64_t x[B];
  cdf ps[B], la[B];
#pragma unroll
  for (int l = 0; l < B; ++l) {
    x[l] = idx(mem[l]);
    ps[l] = psi[x[l]];
    la[l] = lam[x[l]];
  }
#pragma unroll
  for (int k = 0; k + 1 < B; ++k) {
    const df Fk = df_make(F[k].x, F[k].y);
    if (cpr != 0.f) {  // Re z_k
      dfacc z;
      acc_zero(z);
      acc_mac(z, re_of(la[k]), re_of(ps[k + 1]));
      acc_mac(z, im_of(la[k]), im_of(ps[k + 1]));
      acc_mac(z, df_neg(re_of(la[k + 1])), re_of(ps[k]));
      acc_mac(z, df_neg(im_of(la[k + 1])), im_of(ps[k]));
      const df zr = acc_get(z);
      acc_mac(gacc, Fk, df_make(zr.h * cpr, zr.l * cpr));
    }
    if (cpi != 0.f) {  // -Im z_k
      dfacc z;
      acc_zero(z);
      acc_mac(z, re_of(la[k]), im_of(ps[k + 1]));
      acc_mac(z, df_neg(im_of(la[k])), re_of(ps[k + 1]));
      acc_mac(z, df_neg(im_of(la[k + 1])), re_of(ps[k]));
      acc_mac(z, re_of(la[k + 1]), im_of(ps[k]));
      const df zi = acc_get(z);
      acc_mac(gacc, Fk, df_make(-zi.h * cpi, -zi.l * cpi));
    }
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    dfacc pr, pi, lr, li;
    acc_zero(pr);
    acc_zero(pi);
    acc_zero(lr);
    acc_zero(li);
#pragma unroll
    for (int l = 0; l < B; ++l) {
      const cdf u = Ub[l * B + k];  // conj(U_lk)
      cmac_conj<REALU>(pr, pi, u, ps[l]);
      cmac_conj<REALU>(lr, li, u, la[l]);
    }
    psi[x[k]] = make_cdf(acc_get(pr), acc_get(pi));
    lam[x[k]] = make_cdf(acc_get(lr), acc_get(li));
  }
}

#define CVQ_BLOCK_SWITCH(B, CALL)                    \
  switch (B) {                                       \
    case 1: { constexpr int BB = 1; CALL; } break;   \
    case 2: { constexpr int BB = 2; CALL; } break;   \
    case 3: { constexpr int BB = 3; CALL; } break;   \
    case 4: { constexpr int BB = 4; CALL; } break;   \
    case 5: { constexpr int BB = 5; CALL; } break;   \
    case 6: { constexpr int BB = 6; CALL; } break;   \
    case 7: { constexpr int BB = 7; CALL; } break;   \
    case 8: { constexpr int BB = 8; CALL; } break;   \
    case 9: { constexpr int BB = 9; CALL; } break;   \
    case 10: { constexpr int BB = 10; CALL; } break; \
    case 11: { constexpr int BB = 11; CALL; } break; \
    case 12: { constexpr int BB = 12; CALL; } break; \
    case 13: { constexpr int BB = 13; CALL; } break; \
    case 14: { constexpr int BB = 14; CALL; } break; \
    case 15: { constexpr int BB = 15; CALL; } break; \
    case 16: { constexpr int BB = 16; CALL; } break; \
    default: break;                                  \
  }

// ------------------------------------------------------------ orbit enumeration

// Kitaev chain: number of orbits of a gate on `nm` modes (1 or 2).  Orbits are
// split in two halves by the parity class q of the gate modes' occupation sum;
// within a half, the lowest-stride outer mode absorbs the parity constraint so
// consecutive threads touch consecutive amplitudes.
__host__ __device__ __forceinline__ int64_t bkc_items(const SectorDev& S, int nm) {
  int64_t n = 1;
  for (int r = 0; r < S.L - nm; ++r) n *= S.D;
  return n;  // = 1 when no outer mode exists
}

__host__ __device__ __forceinline__ void bkc_orbit(const SectorDev& S, int i, int j, int64_t t, int64_t items, int64_t& f0,
                                          int& q) {
  const int nm = (j >= 0) ? 2 : 1;
  if (S.L == nm) {  // no outer mode: one orbit, class fixed by the sector parity
    f0 = 0;
    q = S.parity;
    return;
  }
  const int64_t halfn = items / 2;
  q = (t >= halfn) ? 1 : 0;
  const int64_t u = t - q * halfn;
  const int pout = (S.parity - q) & 1;
  int lo = S.L - 1;
  while (lo == i || lo == j) --lo;
  const int64_t rlow = u % S.half;
  int64_t rest = u / S.half;
  int64_t f = 0;
  int par = 0;
  for (int r = S.L - 1; r >= 0; --r) {
    if (r == i || r == j || r == lo) continue;
    const int64_t qq = rest / S.D;
    const int n = (int)(rest - qq * S.D);
    rest = qq;
    f += (int64_t)n * S.stride[r];
    par += n;
  }
  const int nlo = (int)(2 * rlow) + ((pout - par) & 1);
  f += (int64_t)nlo * S.stride[lo];
  f0 = f;
}

// Bose-Hubbard two-mode orbit t: class M (= n_i + n_j) and the tuple of its
// first member (n_i, n_j) = (0, M).
__host__ __device__ __forceinline__ uint64_t bh_orbit(const SectorDev& S, const int64_t (*G)[DMAX + 1], int i, int j,
                                             int64_t t, int& M) {
  M = 0;
  while (M < S.N && t >= S.bh2_off[M + 1]) ++M;
  const int64_t u = t - S.bh2_off[M];
  const uint64_t wo = bh_unrank(u, S.L - 2, S.N - M, G);
  uint64_t w = (uint64_t)M << (4 * j);
  int k = 0;
  for (int r = 0; r < S.L; ++r) {
    if (r == i || r == j) continue;
    w |= (uint64_t)occ_get(wo, k) << (4 * r);
    ++k;
  }
  return w;
}

// ------------------------------------------------------------ block kernels

struct GateSmem {
  cdf* U;
  int2* mem;
  float2* F;
  BlockDesc* blk;
};

__device__ __forceinline__ GateSmem stage_gate(const GateArg& g, PoolDev P, bool needF, char* smem) {
  GateSmem s;
  const TypeDesc& t = g.t;
  s.U = reinterpret_cast<cdf*>(smem);
  s.blk = reinterpret_cast<BlockDesc*>(s.U + t.nu);
  int nmem = 0, nf = 0;
  for (int bi = 0; bi < t.nblocks; ++bi) {
    const BlockDesc bd = P.blk[t.blk_base + bi];
    nmem = max(nmem, bd.mem_off + bd.size);
    nf = max(nf, bd.f_off + bd.size - 1);
  }
  s.mem = reinterpret_cast<int2*>(s.blk + t.nblocks);
  s.F = reinterpret_cast<float2*>(s.mem + nmem);
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) s.U[e] = g.U[e];
  for (int e = threadIdx.x; e < t.nblocks; e += blockDim.x) s.blk[e] = P.blk[t.blk_base + e];
  for (int e = threadIdx.x; e < nmem; e += blockDim.x) s.mem[e] = P.mem[t.mem_base + e];
  if (needF)
    for (int e = threadIdx.x; e < nf; e += blockDim.x) s.F[e] = P.F[t.f_base + e];
  __syncthreads();
  return s;
}

template <int KIND, bool ADJ, bool REALU>
__global__ void __launch_bounds__(NTHREADS) k_gate_block(const __grid_constant__ SectorDev S, const __grid_constant__ GateArg g,
                                                         PoolDev P, const cdf* src, cdf* dst, cdf* lam,
                                                         double* partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  const GateSmem sm = stage_gate(g, P, ADJ, smem);
  const TypeDesc& t = g.t;
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  dfacc gacc;
  acc_zero(gacc);
  const int nm = t.single ? 1 : 2;
  const int j = t.single ? -1 : g.j;
  const int64_t items = (KIND == CVQ_BKC) ? bkc_items(S, nm) : S.bh2_off[S.N + 1];
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (int64_t)gridDim.x * blockDim.x) {
    int cls;
    BkcIdx bidx;
    BhIdx hidx;
    if (KIND == CVQ_BKC) {
      bkc_orbit(S, g.i, j, it, items, bidx.f0, cls);
      bidx.si = S.stride[g.i];
      bidx.sj = (j >= 0) ? S.stride[j] : 0;
    } else {
      hidx.w0 = bh_orbit(S, Gs, g.i, j, it, cls);
      hidx.wR0 = bh_suffix(hidx.w0, S.L);
      hidx.r0 = bh_rank(hidx.w0, S.L, S.N, Gs);
      hidx.i = g.i;
      hidx.j = j;
      hidx.L = S.L;
      hidx.G = Gs;
    }
    for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
      const BlockDesc bd = sm.blk[bi];
      const cdf* Ub = sm.U + bd.u_off;
      const int2* mem = sm.mem + bd.mem_off;
      if (KIND == CVQ_BKC) {
        if (ADJ) { CVQ_BLOCK_SWITCH(bd.size, (block_adj<BB, REALU>(Ub, mem, sm.F + bd.f_off, cpr, cpi, bidx, dst, lam, gacc))) }
        else { CVQ_BLOCK_SWITCH(bd.size, (block_fwd<BB, REALU>(Ub, mem, bidx, src, dst))) }
      } else {
        if (ADJ) { CVQ_BLOCK_SWITCH(bd.size, (block_adj<BB, REALU>(Ub, mem, sm.F + bd.f_off, cpr, cpi, hidx, dst, lam, gacc))) }
        else { CVQ_BLOCK_SWITCH(bd.size, (block_fwd<BB, REALU>(Ub, mem, hidx, src, dst))) }
      }
    }
  }
  if (ADJ) {
    const double s = block_sum(acc_to_double(gacc));
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}


// Launch of the block kernel of one gate (REALU chosen from the gate type).
template <int KIND, bool ADJ>
void launch_block(const SectorDev& S, const GateArg& g, PoolDev P, const cdf* src, cdf* dst, cdf* lam, double* partial,
                  size_t sm, cudaStream_t st) {
  if (g.t.realu) k_gate_block<KIND, ADJ, true><<<NBLK, NTHREADS, sm, st>>>(S, g, P, src, dst, lam, partial);
  else k_gate_block<KIND, ADJ, false><<<NBLK, NTHREADS, sm, st>>>(S, g, P, src, dst, lam, partial);
}

// One opt-in per kernel to the largest dynamic shared memory a gate can need.
template <int KIND, bool ADJ>
void set_block_smem_limit(int bytes) {
  cudaFuncSetAttribute(k_gate_block<KIND, ADJ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_gate_block<KIND, ADJ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace cvq
