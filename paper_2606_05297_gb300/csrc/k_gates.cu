// k_gates.cu -- gate engine: per-call block unitaries, forward gate
// application exp(theta A) psi (Sec. IV.B, O_r = exp(theta_r A_r)) and the
// fused reverse step of the adjoint gradient.
//
// A gate acts block-diagonally: with every mode other than the gate's fixed
// (an "orbit"), the generator couples only the occupation pairs (a, b) of the
// gate's modes that are joined by its move, so each orbit splits into small
// blocks.  One thread owns one orbit (Kitaev chain) or one orbit of a fixed
// pair occupation M (Bose-Hubbard), reads its block amplitudes once,
// multiplies them by the b x b block unitary staged in shared memory and
// writes them back in place.  Diagonal gates (K, R, CK, n(n-1)) are a
// streaming phase multiply.
#include "cvq_internal.cuh"

namespace cvq {

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double block_sum(double v) {
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
  return v;  // valid in thread 0
}

// ------------------------------------------------------------ build

// U_g = Vt exp(i theta Lambda) Vt^dag for every block of every gate g of the
// call (one CTA per gate); diagonal gates get the table e^{i theta f}.
__global__ void k_build(const __grid_constant__ BuildArgs a, const TypeDesc* __restrict__ types, PoolDev P,
                        double2* __restrict__ U) {
  const int g = blockIdx.x;
  if (g >= a.n) return;
  const TypeDesc& t = types[a.type_of[g]];
  const double th = a.theta[g];
  double2* Ug = U + (size_t)g * a.ustride;
  if (t.diag) {
    for (int f = threadIdx.x; f < PHASE_TABLE; f += blockDim.x) {
      double s, c;
      sincos(th * (double)f, &s, &c);
      Ug[f] = make_double2(c, s);
    }
    return;
  }
  __shared__ double2 ph[BMAX];
  for (int bi = 0; bi < t.nblocks; ++bi) {
    const BlockDesc bd = P.blk[t.blk_base + bi];
    const int b = bd.size;
    if (threadIdx.x < b) {
      double s, c;
      sincos(th * P.lam[t.lam_base + bd.ev_off + threadIdx.x], &s, &c);
      ph[threadIdx.x] = make_double2(c, s);
    }
    __syncthreads();
    const double2* Vb = reinterpret_cast<const double2*>(P.V) + t.v_base + bd.u_off;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int k = e / b, l = e - k * b;
      double re = 0.0, im = 0.0;
      for (int m = 0; m < b; ++m) {
        const double2 vk = Vb[k * b + m], vl = Vb[l * b + m], p = ph[m];
        // vk * p * conj(vl)
        const double xr = vk.x * p.x - vk.y * p.y, xi = vk.x * p.y + vk.y * p.x;
        re += xr * vl.x + xi * vl.y;
        im += xi * vl.x - xr * vl.y;
      }
      Ug[bd.u_off + e] = make_double2(re, im);
    }
    __syncthreads();
  }
}

cudaError_t launch_build_gates(const BuildArgs& a, const TypeDesc*, const TypeDesc* types_dev, PoolDev P, double2* U,
                               cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_build<<<a.n, 128, 0, st>>>(a, types_dev, P, U);
  return cudaGetLastError();
}

// ------------------------------------------------------------ block math

struct BkcIdx {  // member (a, b) of an orbit with base f0: (f0 + a s_i + b s_j) >> 1
  int64_t f0, si, sj;
  __device__ __forceinline__ int64_t operator()(int2 m) const { return (f0 + m.x * si + m.y * sj) >> 1; }
};

struct BhIdx {   // member (a, b): rank of the base tuple with n_i = a, n_j = b
  uint64_t w0;
  int i, j, L, N;
  const int64_t (*G)[DMAX + 1];
  __device__ __forceinline__ int64_t operator()(int2 m) const {
    uint64_t w = w0 | ((uint64_t)m.x << (4 * i));
    if (j >= 0) w |= (uint64_t)m.y << (4 * j);
    return bh_rank(w, L, N, G);
  }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

template <int B, class IDX>
__device__ __forceinline__ void block_fwd(const double2* __restrict__ Ub, const int2* __restrict__ mem, const IDX& idx,
                                          const double2* src, double2* dst) {
  int64_t x[B];
  double2 in[B];
#pragma unroll
  for (int l = 0; l < B; ++l) {
    x[l] = idx(mem[l]);
    in[l] = src[x[l]];
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int l = 0; l < B; ++l) {
      const double2 u = Ub[k * B + l];
      re = fma(u.x, in[l].x, re);
      re = fma(-u.y, in[l].y, re);
      im = fma(u.x, in[l].y, im);
      im = fma(u.y, in[l].x, im);
    }
    dst[x[k]] = make_double2(re, im);
  }
}

// Reverse step for one block: accumulate Re sum_k conj(lam_k) (A psi)_k with the
// tridiagonal generator, then psi <- U^dag psi and lam <- U^dag lam.
template <int B, class IDX>
__device__ __forceinline__ void block_adj(const double2* __restrict__ Ub, const int2* __restrict__ mem,
                                          const double* __restrict__ F, double2 cp, const IDX& idx, double2* psi,
                                          double2* lam, double& gacc) {
  int64_t x[B];
  double2 ps[B], la[B];
#pragma unroll
  for (int l = 0; l < B; ++l) {
    x[l] = idx(mem[l]);
    ps[l] = psi[x[l]];
    la[l] = lam[x[l]];
  }
  const double2 cm = make_double2(-cp.x, cp.y);  // -conj(c_plus)
#pragma unroll
  for (int k = 0; k < B; ++k) {
    double2 ap = make_double2(0.0, 0.0);
    if (k + 1 < B) {
      const double2 t = cmul(cp, ps[k + 1]);
      ap.x = fma(F[k], t.x, ap.x);
      ap.y = fma(F[k], t.y, ap.y);
    }
    if (k > 0) {
      const double2 t = cmul(cm, ps[k - 1]);
      ap.x = fma(F[k - 1], t.x, ap.x);
      ap.y = fma(F[k - 1], t.y, ap.y);
    }
    gacc = fma(la[k].x, ap.x, gacc);
    gacc = fma(la[k].y, ap.y, gacc);
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    double pr = 0.0, pi = 0.0, lr = 0.0, li = 0.0;
#pragma unroll
    for (int l = 0; l < B; ++l) {
      const double2 u = Ub[l * B + k];  // conj(U_lk)
      pr = fma(u.x, ps[l].x, pr); pr = fma(u.y, ps[l].y, pr);
      pi = fma(u.x, ps[l].y, pi); pi = fma(-u.y, ps[l].x, pi);
      lr = fma(u.x, la[l].x, lr); lr = fma(u.y, la[l].y, lr);
      li = fma(u.x, la[l].y, li); li = fma(-u.y, la[l].x, li);
    }
    psi[x[k]] = make_double2(pr, pi);
    lam[x[k]] = make_double2(lr, li);
  }
}

#define CVQ_BLOCK_SWITCH(B, CALL)            \
  switch (B) {                               \
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
    default: break;                          \
  }

// ------------------------------------------------------------ orbit enumeration

// Kitaev chain: number of orbits of a gate on `nm` modes (1 or 2).  Orbits are
// split in two halves by the parity class q of the gate modes' occupation sum;
// within a half, the lowest-stride outer mode absorbs the parity constraint so
// consecutive threads touch consecutive amplitudes.
__device__ __forceinline__ int64_t bkc_items(const SectorDev& S, int nm) {
  int64_t n = 1;
  for (int r = 0; r < S.L - nm; ++r) n *= S.D;
  return n;  // = 1 when no outer mode exists
}

__device__ __forceinline__ void bkc_orbit(const SectorDev& S, int i, int j, int64_t t, int64_t items, int64_t& f0,
                                          int& q) {
  const int nm = (j >= 0) ? 2 : 1;
  if (S.L == nm) {  // no outer mode: one orbit, class fixed by the sector parity
    f0 = 0;
    q = S.parity;
    return;
  }
  const int64_t halfn = items / 2;
  q = (t >= halfn) ? 1 : 0;
  int64_t u = t - q * halfn;
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

// Bose-Hubbard two-mode orbit t: class M (= n_i + n_j) and base tuple with
// zeros at i and j.
__device__ __forceinline__ uint64_t bh_orbit(const SectorDev& S, const int64_t (*G)[DMAX + 1], int i, int j,
                                             int64_t t, int& M) {
  M = 0;
  while (M < S.N && t >= S.bh2_off[M + 1]) ++M;
  const int64_t u = t - S.bh2_off[M];
  const uint64_t wo = bh_unrank(u, S.L - 2, S.N - M, G);
  uint64_t w = 0;
  int k = 0;
  for (int r = 0; r < S.L; ++r) {
    if (r == i || r == j) continue;
    w |= (uint64_t)occ_get(wo, k) << (4 * r);
    ++k;
  }
  return w;
}

// ------------------------------------------------------------ kernels

struct GateSmem {
  double2* U;
  int2* mem;
  double* F;
  BlockDesc* blk;
};

__device__ __forceinline__ GateSmem stage_gate(const GateArg& g, PoolDev P, bool needF, char* smem) {
  GateSmem s;
  const TypeDesc& t = g.t;
  s.U = reinterpret_cast<double2*>(smem);
  s.blk = reinterpret_cast<BlockDesc*>(s.U + t.nu);
  // members and F follow the block table
  int nmem = 0, nf = 0;
  for (int bi = 0; bi < t.nblocks; ++bi) {
    const BlockDesc bd = P.blk[t.blk_base + bi];
    nmem = max(nmem, bd.mem_off + bd.size);
    nf = max(nf, bd.f_off + bd.size - 1);
  }
  s.mem = reinterpret_cast<int2*>(s.blk + t.nblocks);
  s.F = reinterpret_cast<double*>(s.mem + nmem + (nmem & 1));
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) s.U[e] = g.U[e];
  for (int e = threadIdx.x; e < t.nblocks; e += blockDim.x) s.blk[e] = P.blk[t.blk_base + e];
  for (int e = threadIdx.x; e < nmem; e += blockDim.x) s.mem[e] = P.mem[t.mem_base + e];
  if (needF)
    for (int e = threadIdx.x; e < nf; e += blockDim.x) s.F[e] = P.F[t.f_base + e];
  __syncthreads();
  return s;
}

template <int KIND, bool ADJ>
__global__ void __launch_bounds__(NTHREADS) k_gate_block(const __grid_constant__ SectorDev S, const __grid_constant__ GateArg g,
                                                         PoolDev P, const double2* src, double2* dst, double2* lam,
                                                         double* partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  const GateSmem sm = stage_gate(g, P, ADJ, smem);
  const TypeDesc& t = g.t;
  const double2 cp = make_double2(t.cp_re, t.cp_im);
  double gacc = 0.0;
  const int nm = t.single ? 1 : 2;
  const int j = t.single ? -1 : g.j;
  int64_t items;
  if (KIND == CVQ_BKC) items = bkc_items(S, nm);
  else items = S.bh2_off[S.N + 1];
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
      hidx.i = g.i; hidx.j = j; hidx.L = S.L; hidx.N = S.N; hidx.G = Gs;
    }
    for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
      const BlockDesc bd = sm.blk[bi];
      const double2* Ub = sm.U + bd.u_off;
      const int2* mem = sm.mem + bd.mem_off;
      if (KIND == CVQ_BKC) {
        if (ADJ) { CVQ_BLOCK_SWITCH(bd.size, (block_adj<BB>(Ub, mem, sm.F + bd.f_off, cp, bidx, dst, lam, gacc))) }
        else { CVQ_BLOCK_SWITCH(bd.size, (block_fwd<BB>(Ub, mem, bidx, src, dst))) }
      } else {
        if (ADJ) { CVQ_BLOCK_SWITCH(bd.size, (block_adj<BB>(Ub, mem, sm.F + bd.f_off, cp, hidx, dst, lam, gacc))) }
        else { CVQ_BLOCK_SWITCH(bd.size, (block_fwd<BB>(Ub, mem, hidx, src, dst))) }
      }
    }
  }
  if (ADJ) {
    const double s = block_sum(gacc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// Diagonal gates: psi[x] *= e^{i theta f(n(x))}.  Adjoint: accumulate
// Re conj(lam) (i f psi) and multiply both by e^{-i theta f}.
template <int KIND, bool ADJ>
__global__ void __launch_bounds__(NTHREADS) k_gate_diag(const __grid_constant__ SectorDev S, const __grid_constant__ GateArg g,
                                                        const double2* src, double2* dst, double2* lam, double* partial) {
  __shared__ double2 ph[PHASE_TABLE];
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < PHASE_TABLE; e += blockDim.x) ph[e] = g.U[e];
  __syncthreads();
  const int dg = g.t.diag;
  double gacc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, S.L, S.N, Gs);
    const int ni = occ_get(w, g.i);
    int f;
    if (dg == 1) f = ni * ni;
    else if (dg == 2) f = ni * (ni - 1);
    else if (dg == 3) f = ni;
    else f = ni * occ_get(w, g.j);
    const double2 p = ph[f];
    if (!ADJ) {
      dst[x] = cmul(p, src[x]);
    } else {
      const double2 ps = dst[x], la = lam[x];
      // Re(conj(la) * i f ps) = f * (la.x * (-ps.y) + la.y * ps.x)
      gacc = fma((double)f, fma(la.y, ps.x, -la.x * ps.y), gacc);
      const double2 pc = make_double2(p.x, -p.y);
      dst[x] = cmul(pc, ps);
      lam[x] = cmul(pc, la);
    }
  }
  if (ADJ) {
    const double s = block_sum(gacc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

static size_t gate_smem_bytes(const TypeDesc& t) {
  // U, block table, members (<= D^2 + pad), F
  return (size_t)t.nu * sizeof(double2) + (size_t)t.nblocks * sizeof(BlockDesc) +
         (size_t)(DMAX * DMAX + 2) * sizeof(int2) + (size_t)(DMAX * DMAX) * sizeof(double);
}

template <bool ADJ>
static cudaError_t launch_gate_impl(const SectorDev& S, const GateArg& g, PoolDev P, const double2* src, double2* dst,
                                    double2* lam, double* partial, cudaStream_t st) {
  const int grid = NBLK;
  if (g.t.diag) {
    if (S.kind == CVQ_BH) k_gate_diag<CVQ_BH, ADJ><<<grid, NTHREADS, 0, st>>>(S, g, src, dst, lam, partial);
    else k_gate_diag<CVQ_BKC, ADJ><<<grid, NTHREADS, 0, st>>>(S, g, src, dst, lam, partial);
    return cudaGetLastError();
  }
  const size_t sm = gate_smem_bytes(g.t);
  // The largest gate table: a two-mode gate at cutoff 16 has at most
  // 2 * (1^2 + ... + 15^2) + 16^2 = 2736 block entries and at most 64 blocks.
  constexpr int kMaxNu = 2816, kMaxBlocks = 64;
  if (g.t.nu > kMaxNu || g.t.nblocks > kMaxBlocks) return cudaErrorInvalidValue;
  static bool attr_set = false;  // one opt-in to the largest dynamic shared memory a gate can need
  if (!attr_set) {
    const int mx = (int)(kMaxNu * sizeof(double2) + kMaxBlocks * sizeof(BlockDesc) + (DMAX * DMAX + 2) * sizeof(int2) +
                         DMAX * DMAX * sizeof(double));
    cudaFuncSetAttribute(k_gate_block<CVQ_BH, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_gate_block<CVQ_BKC, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr_set = true;
  }
  if (S.kind == CVQ_BH) k_gate_block<CVQ_BH, ADJ><<<grid, NTHREADS, sm, st>>>(S, g, P, src, dst, lam, partial);
  else k_gate_block<CVQ_BKC, ADJ><<<grid, NTHREADS, sm, st>>>(S, g, P, src, dst, lam, partial);
  return cudaGetLastError();
}

cudaError_t launch_gate(const SectorDev& S, const GateArg& g, PoolDev P, const double2* src, double2* dst,
                        cudaStream_t st) {
  return launch_gate_impl<false>(S, g, P, src, dst, nullptr, nullptr, st);
}

cudaError_t launch_gate_adjoint(const SectorDev& S, const GateArg& g, PoolDev P, double2* psi, double2* lam,
                                double* partial, cudaStream_t st) {
  return launch_gate_impl<true>(S, g, P, psi, psi, lam, partial, st);
}

}  // namespace cvq

namespace cvq {

// ------------------------------------------------------------ diagonal runs

template <int KIND, bool ADJ>
__global__ void __launch_bounds__(NTHREADS) k_diag_run(const __grid_constant__ SectorDev S, const __grid_constant__ DiagRunArg a,
                                                       const double2* src, double2* dst, double2* lam, double* partial) {
  __shared__ int64_t Gs[LMAX][DMAX + 1];
  __shared__ double ang[LMAX][DMAX];
  if (KIND == CVQ_BH) load_G(Gs, S);
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) ang[e / DMAX][e % DMAX] = a.ang[e / DMAX][e % DMAX];
  __syncthreads();
  double acc[MAX_RUN];
#pragma unroll
  for (int k = 0; k < MAX_RUN; ++k) acc[k] = 0.0;
  const int L = S.L;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < S.dim; x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = (KIND == CVQ_BKC) ? bkc_unrank(x, S) : bh_unrank(x, L, S.N, Gs);
    double phi = 0.0;
    for (int r = 0; r < L; ++r) phi += ang[r][occ_get(w, r)];
    for (int p = 0; p < a.npair; ++p) phi = fma(a.pth[p], (double)(occ_get(w, a.pi[p]) * occ_get(w, a.pj[p])), phi);
    double sn, cs;
    sincos(phi, &sn, &cs);
    if (!ADJ) {
      const double2 v = src[x];
      dst[x] = make_double2(fma(cs, v.x, -sn * v.y), fma(cs, v.y, sn * v.x));
    } else {
      const double2 ps = dst[x], la = lam[x];
      // Re(conj(la) * i f ps) = -f * Im(conj(la) ps)
      const double c = fma(la.y, ps.x, -la.x * ps.y);
#pragma unroll
      for (int k = 0; k < MAX_RUN; ++k) {
        if (k < a.m) {
          const int ni = occ_get(w, a.gi[k]);
          const int dg = a.diag[k];
          const int f = (dg == 1) ? ni * ni : (dg == 2) ? ni * (ni - 1) : (dg == 3) ? ni : ni * occ_get(w, a.gj[k]);
          acc[k] = fma((double)f, c, acc[k]);
        }
      }
      dst[x] = make_double2(fma(cs, ps.x, sn * ps.y), fma(cs, ps.y, -sn * ps.x));
      lam[x] = make_double2(fma(cs, la.x, sn * la.y), fma(cs, la.y, -sn * la.x));
    }
  }
  if (ADJ) {
#pragma unroll
    for (int k = 0; k < MAX_RUN; ++k) {
      if (k < a.m) {
        const double s = block_sum(acc[k]);
        if (threadIdx.x == 0) partial[(size_t)k * NBLK + blockIdx.x] = s;
      }
    }
  }
}

cudaError_t launch_diag_run(const SectorDev& S, const DiagRunArg& a, const double2* src, double2* dst, double2* lam,
                            double* partial, bool adjoint, cudaStream_t st) {
  if (S.kind == CVQ_BH) {
    if (adjoint) k_diag_run<CVQ_BH, true><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
    else k_diag_run<CVQ_BH, false><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
  } else {
    if (adjoint) k_diag_run<CVQ_BKC, true><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
    else k_diag_run<CVQ_BKC, false><<<NBLK, NTHREADS, 0, st>>>(S, a, src, dst, lam, partial);
  }
  return cudaGetLastError();
}

}  // namespace cvq
