// k_gate_impl.cuh -- block gate kernels (forward and reverse), instantiated
// once per (sector kind, direction) in k_gate_{bh,bkc}_{fwd,adj}.cu so that
// the translation units compile in parallel.
//
// A thread owns one orbit of the gate (the occupations of every other mode
// fixed) and walks its blocks.  Each block's amplitudes are staged in the
// thread's own column of shared memory (entry l of thread t at l*NTHREADS+t,
// so a warp's accesses never share a bank) together with their sector
// indices; the block unitary is read from shared memory as a broadcast.  The
// block size is a runtime loop bound, so the code does not grow with it.
#pragma once

#include "cvq_internal.cuh"

namespace cvq {

// ------------------------------------------------------------ member indices

struct BkcIdx {  // member (a, b) of an orbit with base f0: (f0 + a s_i + b s_j) >> 1
  int64_t f0, si, sj;
  __host__ __device__ __forceinline__ int64_t operator()(int2 m) const { return (f0 + m.x * si + m.y * sj) >> 1; }
};

template <class T>
struct BhIdxT {  // member (a, M - a): rank of member (0, M) plus the rank change of moving a bosons j -> i
  uint64_t w0, wR0;
  T r0;
  int i, j, L;
  const T (*G)[DMAX + 1];
  __host__ __device__ __forceinline__ int64_t operator()(int2 m) const {
    return (int64_t)(m.x ? r0 + bh_move_delta(w0, wR0, i, j, m.x, L, G) : r0);
  }
};
using BhIdx = BhIdxT<int64_t>;

// ------------------------------------------------------------ complex df helpers

template <bool REALU>
__device__ __forceinline__ void cmac(dfacc& ar, dfacc& ai, cdf u, cdf v) {  // += u v
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  if (!REALU) {
    acc_mac(ar, df_neg(im_of(u)), im_of(v));
    acc_mac(ai, im_of(u), re_of(v));
  }
}

template <bool REALU>
__device__ __forceinline__ void cmac_conj(dfacc& ar, dfacc& ai, cdf u, cdf v) {  // += conj(u) v
  acc_mac(ar, re_of(u), re_of(v));
  acc_mac(ai, re_of(u), im_of(v));
  if (!REALU) {
    acc_mac(ar, im_of(u), im_of(v));
    acc_mac(ai, df_neg(im_of(u)), re_of(v));
  }
}

// One product of a block-unitary entry with an amplitude when the entry is
// real (even k - l, or a real generator) or purely imaginary (odd k - l):
// 2 df products instead of 4.  CONJ uses conj(u).
template <bool REALU, bool CONJ>
__device__ __forceinline__ void cmac_cb(dfacc& ar, dfacc& ai, cdf u, cdf v, int odd) {
  if (REALU || !odd) {
    const df a = re_of(u);
    acc_mac(ar, a, re_of(v));
    acc_mac(ai, a, im_of(v));
  } else {  // u = i b: u v = -b v.im + i b v.re
    const df b = CONJ ? df_neg(im_of(u)) : im_of(u);
    acc_mac(ar, df_neg(b), im_of(v));
    acc_mac(ai, b, re_of(v));
  }
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

__host__ __device__ __forceinline__ void bkc_orbit(const SectorDev& S, int i, int j, int64_t t, int64_t items,
                                                   int64_t& f0, int& q) {
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

// Bose-Hubbard two-mode orbit u of class M (= n_i + n_j): the tuple of its
// first member (n_i, n_j) = (0, M), built from the u-th composition of N - M
// over the other L - 2 modes.
__host__ __device__ __forceinline__ uint64_t bh_orbit_of_class(const SectorDev& S, const int64_t (*G)[DMAX + 1],
                                                               int i, int j, int M, int64_t u) {
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

// The same for a global orbit number t (classes in increasing M).
__host__ __device__ __forceinline__ uint64_t bh_orbit(const SectorDev& S, const int64_t (*G)[DMAX + 1], int i, int j,
                                                      int64_t t, int& M) {
  M = 0;
  while (M < S.N && t >= S.bh2_off[M + 1]) ++M;
  return bh_orbit_of_class(S, G, i, j, M, t - S.bh2_off[M]);
}

template <class T>
__device__ __forceinline__ BhIdxT<T> bh_idx_of(const SectorDev& S, const T (*G)[DMAX + 1], int i, int j,
                                               uint64_t w0) {
  BhIdxT<T> h;
  h.w0 = w0;
  h.wR0 = bh_suffix(w0, S.L);
  h.r0 = bh_rank(w0, S.L, S.N, G);
  h.i = i;
  h.j = j;
  h.L = S.L;
  h.G = G;
  return h;
}

}  // namespace cvq

namespace cvq {

// ------------------------------------------------------------ one block

// Forward: psi[x_k] <- sum_l U_kl psi[x_l].  Reverse: accumulate the gradient
// term sum_k F_k Re(cp z_k), z_k = conj(lam_k) psi_{k+1} - lam_{k+1} conj(psi_k)
// (the tridiagonal generator A[k][k+1] = cp F_k, A[k+1][k] = -conj(cp) F_k),
// then psi <- U^dag psi and lam <- U^dag lam.
template <bool ADJ, bool REALU, bool CACHE, class IDX>
__device__ __forceinline__ void apply_block(const int b, const cdf* __restrict__ Ub, const int2* __restrict__ mem,
                                            const float2* __restrict__ F, const float cpr, const float cpi,
                                            const IDX& idx, const cdf* src, cdf* dst, cdf* lam, cdf* stg,
                                            int64_t* sx, dfacc& gacc) {
  const int tid = threadIdx.x;
  // sector index of member l: cached in shared memory (CACHE) or recomputed
  auto X = [&](int l) -> int64_t { return CACHE ? sx[l * NTHREADS + tid] : idx(mem[l]); };
#pragma unroll 4
  for (int l = 0; l < b; ++l) {
    const int64_t x = idx(mem[l]);
    if (CACHE) sx[l * NTHREADS + tid] = x;
    stg[l * NTHREADS + tid] = src[x];
  }
  if (!ADJ) {
    for (int k = 0; k < b; ++k) {
      dfacc ar, ai;
      acc_zero(ar);
      acc_zero(ai);
      for (int l = 0; l < b; ++l) cmac_cb<REALU, false>(ar, ai, Ub[k * b + l], stg[l * NTHREADS + tid], (k ^ l) & 1);
      dst[X(k)] = make_cdf(acc_get(ar), acc_get(ai));
    }
    return;
  }
  if (b > 1) {
    cdf lk = lam[X(0)];
    for (int k = 0; k + 1 < b; ++k) {
      const cdf lk1 = lam[X(k + 1)];
      const cdf pk = stg[k * NTHREADS + tid], pk1 = stg[(k + 1) * NTHREADS + tid];
      const df Fk = df_make(F[k].x, F[k].y);
      if (cpr != 0.f) {  // Re z_k
        dfacc z;
        acc_zero(z);
        acc_mac(z, re_of(lk), re_of(pk1));
        acc_mac(z, im_of(lk), im_of(pk1));
        acc_mac(z, df_neg(re_of(lk1)), re_of(pk));
        acc_mac(z, df_neg(im_of(lk1)), im_of(pk));
        const df zr = acc_get(z);
        acc_mac(gacc, Fk, df_make(zr.h * cpr, zr.l * cpr));
      }
      if (cpi != 0.f) {  // -Im z_k
        dfacc z;
        acc_zero(z);
        acc_mac(z, re_of(lk), im_of(pk1));
        acc_mac(z, df_neg(im_of(lk)), re_of(pk1));
        acc_mac(z, df_neg(im_of(lk1)), re_of(pk));
        acc_mac(z, re_of(lk1), im_of(pk));
        const df zi = acc_get(z);
        acc_mac(gacc, Fk, df_make(-zi.h * cpi, -zi.l * cpi));
      }
      lk = lk1;
    }
  }
  for (int k = 0; k < b; ++k) {  // psi <- U^dag psi
    dfacc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
    for (int l = 0; l < b; ++l) cmac_cb<REALU, true>(ar, ai, Ub[l * b + k], stg[l * NTHREADS + tid], (k ^ l) & 1);
    dst[X(k)] = make_cdf(acc_get(ar), acc_get(ai));
  }
#pragma unroll 4
  for (int l = 0; l < b; ++l) stg[l * NTHREADS + tid] = lam[X(l)];
  for (int k = 0; k < b; ++k) {  // lam <- U^dag lam
    dfacc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
    for (int l = 0; l < b; ++l) cmac_cb<REALU, true>(ar, ai, Ub[l * b + k], stg[l * NTHREADS + tid], (k ^ l) & 1);
    lam[X(k)] = make_cdf(acc_get(ar), acc_get(ai));
  }
}

// ------------------------------------------------------------ gate pieces

// Shared-memory carve-out of one gate: its block unitaries, block list,
// members, generator factors (reverse only), then the per-thread staging
// columns of amplitudes and sector indices.
struct GateSmem {
  cdf* U;
  BlockDesc* B;
  int2* M;
  float2* F;
  cdf* stg;
  int64_t* sx;
};

__device__ __forceinline__ GateSmem gate_smem(char* smem, const TypeDesc& t) {
  GateSmem m;
  m.U = reinterpret_cast<cdf*>(smem);
  m.B = reinterpret_cast<BlockDesc*>(m.U + t.nu);
  m.M = reinterpret_cast<int2*>(m.B + t.nblocks);
  m.F = reinterpret_cast<float2*>(m.M + DMAX * DMAX);
  m.stg = reinterpret_cast<cdf*>(smem + gate_tables_bytes(t));
  m.sx = reinterpret_cast<int64_t*>(m.stg + (size_t)t.bmax * NTHREADS);
  return m;
}

// Copies one gate's tables into shared memory (the caller synchronises).
template <bool ADJ>
__device__ __forceinline__ void stage_gate(const GateSmem& m, const TypeDesc& t, const cdf* U, const PoolDev& P) {
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) m.U[e] = U[e];
  for (int e = threadIdx.x; e < t.nblocks; e += blockDim.x) m.B[e] = P.blk[t.blk_base + e];
  for (int e = threadIdx.x; e < t.nmem; e += blockDim.x) m.M[e] = P.mem[t.mem_base + e];
  if (ADJ)
    for (int e = threadIdx.x; e < t.nf; e += blockDim.x) m.F[e] = P.F[t.f_base + e];
}

// Kitaev chain: orbits it = first, first + step, ... < end of the gate on
// modes (gi, gj) (gj < 0: single-mode).
template <bool ADJ, bool REALU>
__device__ __forceinline__ void bkc_gate_range(const SectorDev& S, int gi, int gj, const TypeDesc& t,
                                               const GateSmem& m, int64_t first, int64_t end, int64_t step,
                                               const cdf* src, cdf* dst, cdf* lam, dfacc& gacc) {
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  const int64_t items = bkc_items(S, gj >= 0 ? 2 : 1);
  BkcIdx idx;
  idx.si = S.stride[gi];
  idx.sj = (gj >= 0) ? S.stride[gj] : 0;
  for (int64_t it = first; it < end; it += step) {
    int cls;
    bkc_orbit(S, gi, gj, it, items, idx.f0, cls);
    for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
      const BlockDesc bd = m.B[bi];
      if (bd.bext < 2) continue;  // zero generator: identity, no gradient term
      apply_block<ADJ, REALU, false>(bd.size, m.U + bd.u_off, m.M + bd.mem_off, m.F + bd.f_off, cpr, cpi, idx, src,
                                     dst, lam, m.stg, m.sx, gacc);
    }
  }
}

// Bose-Hubbard: one equal-work chunk (class M, orbits [u0, u1)) of the
// two-mode gate on (gi, gj); each thread takes a contiguous run of the
// chunk's orbits and steps from one outer composition to the next instead of
// unranking every orbit.
template <bool ADJ, bool REALU>
__device__ __forceinline__ void bh_gate_chunk(const SectorDev& S, const int32_t (*Gs)[DMAX + 1], int gi, int gj,
                                              const TypeDesc& t, const GateSmem& m, int4 ch, const cdf* src,
                                              cdf* dst, cdf* lam, dfacc& gacc) {
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  const int lo = min(gi, gj), hi = max(gi, gj);
  const int M = ch.x;
  const int run = (ch.z - ch.y + NTHREADS - 1) / NTHREADS;
  int u = ch.y + threadIdx.x * run;
  const int uend = min(u + run, ch.z);
  if (u >= uend) return;
  uint64_t wo = bh_unrank<int32_t>(u, S.L - 2, S.N - M, Gs);
  for (;;) {
    const uint64_t w0 = spread2(wo, lo, hi) | ((uint64_t)M << (4 * gj));
    const BhIdxT<int32_t> idx = bh_idx_of<int32_t>(S, Gs, gi, gj, w0);
    for (int bi = t.class_off[M]; bi < t.class_off[M + 1]; ++bi) {
      const BlockDesc bd = m.B[bi];
      if (bd.bext < 2) continue;  // zero generator: identity, no gradient term
      apply_block<ADJ, REALU, true>(bd.size, m.U + bd.u_off, m.M + bd.mem_off, m.F + bd.f_off, cpr, cpi, idx, src,
                                    dst, lam, m.stg, m.sx, gacc);
    }
    if (++u >= uend) break;
    comp_next(wo, S.L - 2);
  }
}

// Bose-Hubbard: every orbit t = first, first + step, ... < end of the
// two-mode gate on (gi, gj), classes in increasing pair occupation M, each
// orbit unranked on its own (for sectors small enough that one pass of
// threads covers them, where the chunk schedule would leave most threads of
// a CTA idle).
template <bool ADJ, bool REALU>
__device__ __forceinline__ void bh_gate_orbits(const SectorDev& S, const int64_t (*G)[DMAX + 1], int gi, int gj,
                                               const TypeDesc& t, const GateSmem& m, int64_t first, int64_t end,
                                               int64_t step, const cdf* src, cdf* dst, cdf* lam, dfacc& gacc) {
  const float cpr = (float)t.cp_re, cpi = (float)t.cp_im;
  for (int64_t u = first; u < end; u += step) {
    int M;
    const uint64_t w0 = bh_orbit(S, G, gi, gj, u, M);
    const BhIdx idx = bh_idx_of<int64_t>(S, G, gi, gj, w0);
    for (int bi = t.class_off[M]; bi < t.class_off[M + 1]; ++bi) {
      const BlockDesc bd = m.B[bi];
      if (bd.bext < 2) continue;  // zero generator: identity, no gradient term
      apply_block<ADJ, REALU, true>(bd.size, m.U + bd.u_off, m.M + bd.mem_off, m.F + bd.f_off, cpr, cpi, idx, src,
                                    dst, lam, m.stg, m.sx, gacc);
    }
  }
}

// U_g = (W V) exp(i theta Lambda) (W V)^dag for every block of one gate,
// formed in FP64 by the calling CTA and stored as df complex.  Every
// generator here has phases that are multiples of pi/2 and a zero-diagonal
// tridiagonal block, so exp(theta A) has purely real entries (real
// generator) or real entries at even k - l and imaginary ones at odd k - l;
// the other component is zero up to rounding and is set to zero.
// One block bi of one gate (the calling CTA): U = P (W V) e^{i theta Lambda}
// (W V)^dag P over the block's members, and when Dg is given its theta
// derivative D = P (W V) (i Lambda) e^{i theta Lambda} (W V)^dag P.  P keeps
// the members of the (possibly extended) chain; blocks whose chain is a
// single member are the identity and are never read.
__device__ __forceinline__ void build_block_unitary(const TypeDesc& t, double th, const PoolDev& P, cdf* Ug, int bi,
                                                    double2* ph, cdf* Dg = nullptr) {
  if (bi >= t.nblocks) return;
  const BlockDesc bd = P.blk[t.blk_base + bi];
  const int b = bd.size, be = bd.bext;
  if (be < 2) return;
  for (int q = threadIdx.x; q < be; q += blockDim.x) {
    double s, c;
    sincos(th * P.lam[t.lam_base + bd.ev_off + q], &s, &c);
    ph[q] = make_double2(c, s);
  }
  __syncthreads();
  const double2* Vb = reinterpret_cast<const double2*>(P.V) + t.v_base + bd.v_off;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int k = e / b, l = e - k * b;
    double re = 0.0, im = 0.0, dre = 0.0, dim_ = 0.0;
    for (int q = 0; q < be; ++q) {
      const double2 vk = Vb[k * be + q], vl = Vb[l * be + q], p = ph[q];
      const double xr = vk.x * p.x - vk.y * p.y, xi = vk.x * p.y + vk.y * p.x;  // vk p
      const double ur = xr * vl.x + xi * vl.y, ui = xi * vl.x - xr * vl.y;       // * conj(vl)
      re += ur;
      im += ui;
      if (Dg) {  // times i lambda_q
        const double lq = P.lam[t.lam_base + bd.ev_off + q];
        dre -= lq * ui;
        dim_ += lq * ur;
      }
    }
    // Generators here have phases that are multiples of pi/2 on a bipartite
    // chain, so U is real (real generator) or real at even k - l and
    // imaginary at odd k - l; the other component is rounding and is zeroed.
    if (t.realu || ((k - l) & 1) == 0) im = 0.0;
    else re = 0.0;
    Ug[bd.u_off + e] = make_cdf(df_from_double(re), df_from_double(im));
    if (Dg) Dg[bd.u_off + e] = make_cdf(df_from_double(dre), df_from_double(dim_));
  }
}

// ------------------------------------------------------------ kernel

template <int KIND, bool ADJ, bool REALU>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_gate_block(const __grid_constant__ SectorDev S, const __grid_constant__ GateArg g, PoolDev P, const cdf* src,
                 cdf* dst, cdf* lam, double* partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int32_t Gs[LMAX][DMAX + 1];  // BH ranks fit in 32 bits for L, D <= 16
  if (KIND == CVQ_BH) load_G(Gs, S);
  const TypeDesc& t = g.t;
  const GateSmem m = gate_smem(smem, t);
  stage_gate<ADJ>(m, t, g.U, P);
  __syncthreads();
  const int j = t.single ? -1 : g.j;
  dfacc gacc;
  acc_zero(gacc);
  if (KIND == CVQ_BKC) {
    bkc_gate_range<ADJ, REALU>(S, g.i, j, t, m, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                               bkc_items(S, t.single ? 1 : 2), (int64_t)gridDim.x * blockDim.x, src, dst, lam, gacc);
  } else {
    for (int c = blockIdx.x; c < t.nchunks; c += gridDim.x)
      bh_gate_chunk<ADJ, REALU>(S, Gs, g.i, j, t, m, P.chunks[t.chunk_base + c], src, dst, lam, gacc);
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
