// cvq_internal.cuh -- device-side sector description, indexers and kernel
// launchers shared by the CUDA translation units of libcvq.so.
//
// Occupation tuples (n_0..n_{L-1}) travel through the kernels packed four bits
// per mode in one uint64 (L <= 16, D <= 16), so that no kernel needs a
// dynamically indexed per-thread array.  States inside a call are stored as
// double-float complex numbers (df.cuh); the C ABI's complex128 buffers are
// converted at the entry and exit of a call.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cvq.h"
#include "df.cuh"

namespace cvq {

constexpr int LMAX = 16;
constexpr int DMAX = 16;
constexpr int BMAX = 16;          // largest block of a gate (<= D)
constexpr int MAX_BEXT = 64;      // longest chain of a block's eigendecomposition (projected pools)
constexpr int MAX_CLASSES = 17;   // BH: total pair occupation M = 0..N (N <= 15); BKC: 2 parities
constexpr int MAX_GATES = 512;    // ansatz length per call and pool size
constexpr int NTHREADS = 256;
constexpr int NBLK = 152 * 4;     // fixed grid: 4 CTAs per SM on the 152 SMs of a GB300
constexpr int PHASE_TABLE = 256;  // complex entries reserved per gate (>= D^2)

// ------------------------------------------------------------------ sector

// Tables too large for kernel parameters; device-resident, staged into shared
// memory by the kernels that index them per thread.
struct SectorTabs {
  int64_t G[LMAX][DMAX + 1];        // BH: G[p][R] = C(R + p, p)
  float2 diagE[LMAX][DMAX];         // df: nn1 n(n-1) + n2 n^2 + n1 n, per site and occupation
  float2 P[4][DMAX][DMAX];          // df: sqrt factors of the H moves (+1,-1) (-1,+1) (+1,+1) (-1,-1) on (n_r, n_s)
  float2 sq[DMAX][5];               // df: sqrt(max(n,n+e)!/min(n,n+e)!) for e = -2..2
  float2 hop[LMAX], pair[LMAX];     // df bond coefficients
};

struct SectorDev {
  int kind, L, N, D, parity, periodic, nb, half;   // half = d / 2 (BKC)
  int div32;                            // BKC with dim < 2^31: unrank by multiply-high divisions
  uint32_t m_half, m_d;                 // their multipliers and shifts (set_bkc_div)
  int s_half, s_d;
  int64_t dim;
  int64_t stride[LMAX];                 // BKC: d^(L-1-r)
  int64_t bh2_off[MAX_CLASSES + 1];     // BH two-mode gate work items of class M start at bh2_off[M]
  const SectorTabs* tab;                // device copy
};

__host__ __device__ __forceinline__ int occ_get(uint64_t w, int r) { return (int)((w >> (4 * r)) & 15ull); }
__host__ __device__ __forceinline__ uint64_t occ_shift(uint64_t w, int r, int delta) {
  return w + (uint64_t)((int64_t)delta * (int64_t)(1ull << (4 * r)));
}

// Lexicographic rank of a composition of N (combinatorial number system):
// rank = sum_{k < L-1} G[L-1-k][R_k] - G[L-1-k][R_{k+1}],  R_k = n_k + ... + n_{L-1}.
// T is the table's integer type (int32 suffices for L, D <= 16: C(30, 15) < 2^31).
template <class T>
__host__ __device__ __forceinline__ T bh_rank(uint64_t w, int L, int N, const T (*G)[DMAX + 1]) {
  T r = 0;
  int R = N;
  for (int k = 0; k < L - 1; ++k) {
    const int n = occ_get(w, k);
    r += G[L - 1 - k][R] - G[L - 1 - k][R - n];
    R -= n;
  }
  return r;
}

// Suffix sums R_k = n_k + ... + n_{L-1}, packed like the occupations.
__host__ __device__ __forceinline__ uint64_t bh_suffix(uint64_t w, int L) {
  uint64_t s = 0;
  int R = 0;
  for (int k = L - 1; k >= 0; --k) {
    R += occ_get(w, k);
    s |= (uint64_t)R << (4 * k);
  }
  return s;
}

// Rank change when w is moved by (+dr on mode r, -dr on mode s): only the terms
// of positions min(r,s)..max(r,s) change; wR holds the suffix sums of w.
template <class T>
__host__ __device__ __forceinline__ T bh_move_delta(uint64_t w, uint64_t wR, int r, int s, int dr, int L,
                                                   const T (*G)[DMAX + 1]) {
  int lo = r, hi = s, dlo = dr;
  if (s < r) { lo = s; hi = r; dlo = -dr; }
  T d = 0;
  const int top = (hi < L - 1) ? hi : L - 2;
  for (int k = lo; k <= top; ++k) {
    const int p = L - 1 - k;
    const int R = occ_get(wR, k), n = occ_get(w, k);
    const int Rn = (k == lo) ? R : R - dlo;
    const int nn = (k == lo) ? n + dlo : (k == hi) ? n - dlo : n;
    d += (G[p][Rn] - G[p][Rn - nn]) - (G[p][R] - G[p][R - n]);
  }
  return d;
}

// Rank change of the hop x -> x + e_r - e_{r+1} on a chain of L modes holding
// N bosons when the suffix sum R_{r+1} = n_{r+1} + ... + n_{L-1} equals Q:
// only the terms of positions r and r+1 change, and within them the parts
// that involve n_r and n_{r+1} cancel (0 outside 0 <= r <= L-2, 1 <= Q <= N).
template <class T>
__host__ __device__ __forceinline__ T bh_hop_delta(const T (*G)[DMAX + 1], int L, int N, int r, int Q) {
  if (r < 0 || r > L - 2 || Q < 1 || Q > N) return 0;
  const int p = L - 1 - r;
  T d = G[p][Q] - G[p][Q - 1];
  if (r + 1 <= L - 2) d += G[p - 1][Q - 1] - G[p - 1][Q];
  return d;
}

// Inverse of bh_rank for a chain of Lc modes holding Nc bosons; the tuple is
// written to consecutive nibbles starting at nibble 0, its suffix sums to *wR.
template <class T>
__host__ __device__ __forceinline__ uint64_t bh_unrank(T x, int Lc, int Nc, const T (*G)[DMAX + 1],
                                                       uint64_t* wR = nullptr) {
  uint64_t w = 0, sR = 0;
  int R = Nc;
  for (int k = 0; k < Lc - 1; ++k) {
    const int p = Lc - 1 - k;
    const T base = G[p][R];
    int n = 0;
    while (n < R && x >= base - G[p][R - n - 1]) ++n;
    x -= base - G[p][R - n];
    w |= (uint64_t)n << (4 * k);
    sR |= (uint64_t)R << (4 * k);
    R -= n;
  }
  if (Lc > 0) {
    w |= (uint64_t)R << (4 * (Lc - 1));
    sR |= (uint64_t)R << (4 * (Lc - 1));
  }
  if (wR) *wR = sR;
  return w;
}

// Next composition in lexicographic order (same number of parts and sum),
// packed in nibbles 0..Lc-1; false if w is the last one.  The rightmost part
// p < Lc-1 with a nonzero sum after it grows by one and the parts after it
// become (0, ..., 0, that sum - 1).
__host__ __device__ __forceinline__ bool comp_next(uint64_t& w, int Lc) {
  int S = 0, p;
  for (p = Lc - 2; p >= 0; --p) {
    S += occ_get(w, p + 1);
    if (S > 0) break;
  }
  if (p < 0) return false;
  w &= (4 * (p + 1) >= 64) ? ~0ull : ((1ull << (4 * (p + 1))) - 1);
  w += 1ull << (4 * p);
  w |= (uint64_t)(S - 1) << (4 * (Lc - 1));
  return true;
}

// Bose-Hubbard sector indices [x0, x1) visited by the warps of a grid, each
// tuple stepped to rather than unranked: the range is cut into chunks of 32 R
// consecutive indices (R <= WALK_RMAX, odd), warp w of the grid taking chunks
// w, w + nw, ...  In a chunk, lane l unranks index base + l R and steps R - 1
// times to the next composition in lexicographic order (the order of the
// ranks), leaving the tuples in the warp's part of wbuf (32 WALK_RMAX
// entries per warp of the CTA); the warp then visits indices base + l + 32 i,
// so its amplitude accesses stay coalesced while one index in R is unranked.
// f(x, w) is called once for every index.
constexpr int WALK_RMAX = 9;

__host__ __device__ __forceinline__ int walk_r(int64_t n, int64_t nwarps) {
  if (n <= 0) return 1;
  const int64_t per = (n + 32 * nwarps - 1) / (32 * nwarps);  // indices per lane over all passes
  const int64_t passes = (per + WALK_RMAX - 1) / WALK_RMAX;
  const int r = (int)((per + passes - 1) / passes);
  return (r & 1) ? r : r + 1;  // odd: the lanes' buffer writes fall on distinct bank pairs
}

// The warps taking part are warp = 0 .. nw - 1 (bh_walk: every warp of the
// grid; bh_walk_cta: the warps of one CTA, for a range of its own).
template <class T, class F>
__device__ __forceinline__ void bh_walk_warps(const SectorDev& S, const T (*G)[DMAX + 1], uint64_t* wbuf, int64_t x0,
                                              int64_t x1, int64_t warp, int64_t nw, F&& f) {
  const int lane = threadIdx.x & 31;
  const int R = walk_r(x1 - x0, nw);
  const int64_t ch = 32 * (int64_t)R;
  uint64_t* buf = wbuf + (threadIdx.x >> 5) * (32 * WALK_RMAX);
  for (int64_t base = x0 + warp * ch; base < x1; base += nw * ch) {  // uniform over the warp
    const int64_t xs = base + (int64_t)lane * R;
    if (xs < x1) {
      uint64_t w = bh_unrank<T>((T)xs, S.L, S.N, G);
      buf[lane * R] = w;
      const int n = (int)((x1 - xs < R) ? x1 - xs : R);
      for (int i = 1; i < n; ++i) {
        comp_next(w, S.L);
        buf[lane * R + i] = w;
      }
    }
    __syncwarp();
    for (int i = 0; i < R; ++i) {
      const int64_t x = base + lane + 32 * i;
      if (x < x1) f(x, buf[lane + 32 * i]);
    }
    __syncwarp();
  }
}

template <class T, class F>
__device__ __forceinline__ void bh_walk(const SectorDev& S, const T (*G)[DMAX + 1], uint64_t* wbuf, int64_t x0,
                                        int64_t x1, F&& f) {
  bh_walk_warps(S, G, wbuf, x0, x1, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                ((int64_t)gridDim.x * blockDim.x) >> 5, f);
}

template <class T, class F>
__device__ __forceinline__ void bh_walk_cta(const SectorDev& S, const T (*G)[DMAX + 1], uint64_t* wbuf, int64_t x0,
                                            int64_t x1, F&& f) {
  bh_walk_warps(S, G, wbuf, x0, x1, threadIdx.x >> 5, blockDim.x >> 5, f);
}

// Insert two empty nibbles at modes lo < hi: the packed tuple of the other
// L - 2 modes becomes a full tuple with n_lo = n_hi = 0.
__host__ __device__ __forceinline__ uint64_t spread2(uint64_t wo, int lo, int hi) {
  const uint64_t m1 = (lo == 0) ? 0ull : ((1ull << (4 * lo)) - 1);
  const int mid = hi - lo - 1;
  const uint64_t m2 = (mid <= 0) ? 0ull : ((1ull << (4 * mid)) - 1);
  uint64_t w = wo & m1;
  w |= ((wo >> (4 * lo)) & m2) << (4 * (lo + 1));
  if (hi + 1 < 16) w |= (wo >> (4 * (hi - 1))) << (4 * (hi + 1));
  return w;
}

// n / q for 0 <= n < 2^31 and 1 <= q <= 2^31 with one 32 x 32 -> 64 bit
// multiply: with l = ceil(log2 q) and m = ceil(2^(31+l) / q) < 2^32, the
// quotient is (n m) >> (31 + l) (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994: the error m q - 2^(31+l) is
// below q <= 2^l, so n times it stays below 2^(31+l)).
__host__ __device__ __forceinline__ uint32_t div_by_mul(uint32_t n, uint32_t m, int s) {
  return (uint32_t)(((uint64_t)n * m) >> s);
}

__host__ __device__ __forceinline__ void div_magic(uint32_t q, uint32_t* m, int* s) {
  int l = 0;
  while ((1ull << l) < q) ++l;
  *s = 31 + l;
  *m = (uint32_t)(((1ull << (31 + l)) + q - 1) / q);
}

// The division constants of a Kitaev-chain sector (every caller that fills a
// SectorDev by hand calls this after setting D, half and dim).
__host__ __device__ __forceinline__ void set_bkc_div(SectorDev& S) {
  S.div32 = (S.kind == CVQ_BKC && S.dim > 0 && S.dim <= 0x7fffffffll) ? 1 : 0;
  if (!S.div32) return;
  div_magic((uint32_t)S.half, &S.m_half, &S.s_half);
  div_magic((uint32_t)S.D, &S.m_d, &S.s_d);
}

// Kitaev chain, even d: index = floor(f / 2), f = sum_r n_r d^(L-1-r).
__host__ __device__ __forceinline__ uint64_t bkc_unrank(int64_t x, const SectorDev& S) {
  const int L = S.L, d = S.D;
  uint64_t w = 0;
  int par = 0, lo;
  if (S.div32) {  // every quantity below fits 31 bits
    uint32_t hi = div_by_mul((uint32_t)x, S.m_half, S.s_half);
    lo = (int)((uint32_t)x - hi * (uint32_t)S.half);
    for (int k = L - 2; k >= 0; --k) {
      const uint32_t q = div_by_mul(hi, S.m_d, S.s_d);
      const int n = (int)(hi - q * (uint32_t)d);
      hi = q;
      w |= (uint64_t)n << (4 * k);
      par += n;
    }
  } else {
    int64_t hi = x / S.half;
    lo = (int)(x - hi * S.half);
    for (int k = L - 2; k >= 0; --k) {
      const int64_t q = hi / d;
      const int n = (int)(hi - q * d);
      hi = q;
      w |= (uint64_t)n << (4 * k);
      par += n;
    }
  }
  const int nl = 2 * lo + ((S.parity - par) & 1);
  w |= (uint64_t)nl << (4 * (L - 1));
  return w;
}

// ------------------------------------------------------------------ pool

// A Hermitian generator block of a gate type (Sec. IV.B): the members are
// occupation pairs (a, b) of modes (i, j) joined by the generator's move,
// ordered along it.  Within a block the anti-Hermitian generator is
// tridiagonal, A[k][k+1] = c_plus * F[k], A[k+1][k] = -conj(c_plus) * F[k],
// and exp(theta A) = W V exp(i theta Lambda) V^T W^dag with W = diag(omega^k).
struct BlockDesc {
  int size;     // members
  int mem_off;  // into members[]
  int u_off;    // complex offset of the size x size block within a gate's U
  int f_off;    // into F[] (size - 1 entries)
  int ev_off;   // into lam[] (bext entries)
  int bext;     // length of the chain the eigendecomposition is of: size, or the chain extended to the
                // inner cutoff of a projected pool (the members are a contiguous segment of it)
  int v_off;    // complex offset into V[] of the size x bext rows of the members
  int pad;
};

struct TypeDesc {
  int type, phase, single, diag;   // single: one-mode generator; diag: diagonal in the Fock basis
  int di, dj;                      // the generator's move (a, b) -> (a + di, b + dj)
  int nclass;
  int nblocks, nu, bmax;           // blocks, complex entries of one gate's U, largest block
  int realu;                       // c_plus real: A and exp(theta A) are real
  int nmem, nf;                    // members and generator factors of all blocks
  int chunk_base, nchunks;         // BH: equal-work schedule of (class, orbit range) chunks
  int class_off[MAX_CLASSES + 1];  // blocks of class c are blk[class_off[c] .. class_off[c+1])
  double cp_re, cp_im;             // c_plus
  double om_re, om_im;             // omega
  int blk_base, mem_base, f_base, v_base, lam_base;  // offsets of this type's tables in the pool arrays
};

struct PoolDev {
  const int4* chunks;  // BH: (class M, first orbit, end orbit, 0)
  const BlockDesc* blk;
  const int2* mem;
  const float2* F;     // df tridiagonal factors
  const double* V;     // complex W V, row-major per block
  const double* lam;
};

// Tiled block gates.  For one gate structure (modes, move) the sector indices
// of every block of two or more members are listed in a table, orbit group by
// orbit group.  Orbits of one class ("region": same block structure) are cut
// into tiles of G whole orbits, G = T / (members per orbit), T = TILE_T x S
// slots (S slots per thread of a CTA), so that a tile holds every amplitude of
// its orbits and neighbouring amplitudes are loaded by the same tile.  Within
// a tile the blocks of one class ("sub-block" c of the region, size b_c) take
// b_c G consecutive slots from off_c, member-major: slot off_c + a G + k is
// member a of the block of orbit k.  Unused slots hold -1.  Large sectors take
// S = TILE_S_LARGE, so that each thread keeps several loads in flight; smaller
// ones S = 1, so that every CTA gets work (two slots on the 1.35M-amplitude
// Bose-Hubbard sector were 17 % slower than one).
constexpr int TILE_T = NTHREADS;
constexpr int TILE_S_LARGE = 4;
constexpr int64_t TILE_LARGE_DIM = 1 << 22;
constexpr int TILE_MAX_SUB = 32;  // block classes of one orbit class
struct TileSub {
  int b, off;            // block size, first slot within the tile
  int u_off, f_off;      // the class's unitary (within a gate's U) and generator factors (within the type's F)
  int bi, pad;           // block index within the type's list (table build only)
};
struct TileRegion {
  int G, count;          // orbits per tile, orbits in the region
  int sub0, nsub;        // its sub-blocks: subs[sub0 .. sub0 + nsub)
  int cls, pad;          // orbit class (table build only)
  int64_t tile0;         // first tile of the region
};
struct TileMap {
  const int* idx;           // ntiles x (TILE_T x slots) sector indices; null: the gate has no table
  const TileRegion* reg;    // nreg regions, in tile order
  const TileSub* sub;       // nsub sub-blocks of all regions
  int nreg, nsub, slots;    // slots: S, the tile slots per thread
  int64_t ntiles;
};

// Everything a gate kernel needs about one gate of an ansatz.
struct GateArg {
  int i, j;              // modes
  TypeDesc t;            // structure of the generator
  const cdf* U;          // this gate's block unitaries (t.nu entries, df complex)
  TileMap tm;            // tiled index table of the gate's structure (may be empty)
};

// Shared memory of a block-gate kernel: the gate tables (block unitaries,
// block descriptors, members, generator factors) followed by each thread's
// staging columns for bmax amplitudes and bmax sector indices.
__host__ __device__ __forceinline__ size_t gate_tables_bytes(const TypeDesc& t) {
  const size_t b = (size_t)t.nu * sizeof(cdf) + (size_t)t.nblocks * sizeof(BlockDesc) +
                   (size_t)(DMAX * DMAX) * sizeof(int2) + (size_t)(DMAX * DMAX) * sizeof(float2);
  return (b + 15) & ~(size_t)15;
}

// Bose-Hubbard kernels also cache the members' sector indices (costly to
// recompute); Kitaev-chain indices are recomputed from the orbit base.
__host__ __device__ __forceinline__ size_t gate_smem_bytes(const TypeDesc& t, int kind) {
  return gate_tables_bytes(t) +
         (size_t)NTHREADS * t.bmax * (sizeof(cdf) + (kind == CVQ_BH ? sizeof(int64_t) : 0));
}

// Shared tables of the projected reverse step: unitaries, derivatives, blocks, members.
__host__ __device__ __forceinline__ size_t proj_tables_bytes(const TypeDesc& t) {
  const size_t b = 2 * (size_t)t.nu * sizeof(cdf) + (size_t)t.nblocks * sizeof(BlockDesc) + (size_t)t.nmem * sizeof(int2);
  return (b + 15) & ~(size_t)15;
}

// Per-call list of gates for the unitary build kernel (passed by value).
struct BuildArgs {
  int n;
  int maxblk;            // most blocks of any gate of the call (grid y)
  cdf* D;                // projected pools: theta derivatives of the blocks (same layout as U), else null
  int ustride;           // complex entries reserved per gate
  int type_of[MAX_GATES];
  double theta[MAX_GATES];
};

// A run of consecutive diagonal gates (they commute) applied in one pass:
// psi[x] *= prod_r T[r][n_r] * prod_p TP[p][n_{pi[p]} D + n_{pj[p]}], the
// tables holding exp(i sum_k theta_k f_k(n)) per mode and exp(i theta_p n_i n_j)
// per cross-Kerr gate (built on the host in FP64, passed by value).  The
// reverse pass forms every gradient of the run from the same (psi, lambda).
constexpr int MAX_RUN = 32, MAX_RUN_PAIRS = 4;
// Gradient accumulators of one diagonal-run reverse pass: 8, or 24 for runs of
// more than 8 gates (a warm-start layer's Kerr and rotation gates on every
// mode), whose kernel then runs two CTAs per SM; gates beyond that take
// gradient-only passes.
constexpr int DIAG_ACC = 8, DIAG_ACC_LONG = 24;
__host__ __device__ constexpr int diag_run_acc(int m) { return m > DIAG_ACC ? DIAG_ACC_LONG : DIAG_ACC; }
struct DiagRunArg {
  int m, npair;
  int diag[MAX_RUN], gi[MAX_RUN], gj[MAX_RUN];   // per gate: f type (1..4) and modes
  int pi[MAX_RUN_PAIRS], pj[MAX_RUN_PAIRS];
  int nact, act[LMAX];                            // modes with a single-mode gate (T[r] is not all ones)
  cdf T[LMAX][DMAX];
  cdf TP[MAX_RUN_PAIRS][DMAX * DMAX];
};

// ------------------------------------------------------------- batched engine

constexpr int BATCH_RUN = 8;  // diagonal gates per run in the batched engine

enum BItemKind { BI_TODF = 0, BI_GATE = 1, BI_DIAG = 2, BI_APPLYH = 3, BI_TILE = 4 };  // BI_TILE: a range of gate tiles

// One instance of a batch: its sector, pool tables and device buffers.
struct BInst {
  SectorDev S;
  PoolDev P;
  const GateArg* ops;   // per pool operator (modes and generator structure)
  cdf *psi, *lam, *U;   // df state, adjoint state, block unitaries (n_max x ustride)
  const double2* psi0;  // reference state (complex128)
  int ustride, ids_off, theta_off;
  int seg0, nseg;       // the instance's segments in the plan (nseg = -1: left out)
};

// One segment of one instance's ansatz: a block gate (m = 1) or a run of m
// diagonal gates; the run's gate list uses the field names of DiagRunArg.
struct BSeg {
  int inst, k0, m, isdiag, npair;
  int diag[BATCH_RUN], gi[BATCH_RUN], gj[BATCH_RUN];
  int pi[MAX_RUN_PAIRS], pj[MAX_RUN_PAIRS];
  int nact, act[LMAX];  // modes with a single-mode gate of the run
};

// One work item: a range [a, b) of chunks (BH gate), orbits (BKC gate) or
// sector indices (everything else) of one segment or instance; its partial
// sums go to partial[slot ...].
struct BItem {
  int kind, inst, seg, slot;
  int64_t a, b;
};

// One output of the final reduction.
struct BRed {
  int inst, out, is_energy, slot0, count, stride;
};

// Batched screen: one instance's distinct ladder shifts and diagonal
// functions (ranges of the plan's descriptor array).  Its work items each
// leave 2 nsh + ndg partial sums (Re and Im of Z per shift, then one per
// diagonal function), reduced into rows zrow.. of the z buffer.
struct BScreen {
  int sh_off, nsh, dg_off, ndg;
};
// One screened element: g = 2 [Re(cp Z_sp) - Re(conj(cp) Z_sn)], or 2 D with D
// in row d (the instance's diagonal rows follow its 2 nsh shift rows).
struct BScreenOut {
  int inst, zrow, out, isdg, sp, sn, d, pad;
  double2 cp;
};

cudaError_t launch_batch_build(const BInst* insts, const int2* gates, int ngates, int maxblk, const int* ids,
                               const double* theta, const int* active, cudaStream_t st);
cudaError_t launch_batch_layer(int kind, bool adj, int grid, size_t smem, const BInst* insts, const BSeg* segs,
                               const BItem* items, int nitems, int* counter, const int* ids, const double* theta,
                               const int* active, double* partial, cudaStream_t st);
cudaError_t set_batch_smem_limit(int bytes);
// A layer of block-gate tile ranges only (BI_TILE items), 5 CTAs per SM.
cudaError_t launch_batch_tile_layer(bool adj, int grid, size_t smem, const BInst* insts, const BSeg* segs,
                                    const BItem* items, int nitems, int* counter, const int* ids, const int* active,
                                    double* partial, cudaStream_t st);
cudaError_t set_batch_tile_smem_limit(int bytes);
cudaError_t launch_batch_reduce(const BRed* red, int n, const double* partial, const int* active, double* E,
                                double* grad, cudaStream_t st);
// Batches whose sectors all fit in shared memory: one CTA per instance runs
// the whole evaluation with the states in shared memory.  Mode 0: energy and
// gradient into E and grad; mode 1: the forward sweep and lambda = H psi
// only, both written to the instance's global psi and lambda buffers (the
// batched screen reads them).
size_t batch_small_smem(size_t tab_bytes, int seg_cap, int64_t dim_max);
cudaError_t launch_batch_small(int kind, int mode, int n_inst, size_t tab_bytes, int seg_cap, size_t smem_total,
                               const BInst* insts, const BSeg* segs, const int* ids, const double* theta,
                               const int* active, double* E, double* grad, cudaStream_t st);
cudaError_t set_batch_small_smem_limit(int bytes);
cudaError_t launch_batch_screen(int kind, int grid, const BInst* insts, const BItem* items, int nitems, int* counter,
                                const int* active, const BScreen* screens, const int4* desc, double* partial,
                                cudaStream_t st);
cudaError_t launch_batch_screen_out(const BScreenOut* outs, int n, const double* z, const int* active, double* grad,
                                    cudaStream_t st);

// Pool indices screened by one launch (passed by value).
struct SubsetArg {
  int n;
  int idx[MAX_GATES];
};

// The distinct ladder shifts and diagonal functions of a screened subset.
constexpr int SCREEN_CHUNK = 8, MAX_SHIFTS = 2 * MAX_GATES, MAX_DIAGF = 256;
struct ScreenArg {
  int nsh, ndg;
  int4 sh[MAX_SHIFTS];  // (i, di, j, dj); j < 0 for a single-mode move
  int4 dg[MAX_DIAGF];   // (f type 1..4 as TypeDesc::diag, i, j, 0)
};

// Per screened element: e = (1 diagonal / 0 shift pair, plus-shift or
// diagonal index, minus-shift index, 0) and c_plus.
struct ScreenMap {
  int n;
  int4 e[MAX_GATES];
  double2 cp[MAX_GATES];
};

// ------------------------------------------------------------- launchers
// All launchers enqueue on `stream` and return the launch status.  States
// (cdf*) are df complex; the C ABI's complex128 buffers go through
// launch_to_df / launch_from_df.

cudaError_t launch_to_df(int64_t dim, const double2* src, cdf* dst, cudaStream_t st);
cudaError_t launch_from_df(int64_t dim, const cdf* src, double2* dst, cudaStream_t st);
cudaError_t launch_apply_H(const SectorDev& S, const cdf* psi, cdf* sigma, double* partial, cudaStream_t st);
cudaError_t launch_reduce(const double* partial, int nred, int nblk, double scale, double* out, cudaStream_t st);
// Gradient rows 0..n-1 of partial (x 2) into grad and energy row n into E.
cudaError_t launch_reduce_eg(const double* partial, int n, int nblk, double* E, double* grad, cudaStream_t st);
cudaError_t launch_build_gates(const BuildArgs& a, const TypeDesc* types_dev, PoolDev P, cdf* U, cudaStream_t st);
cudaError_t launch_gate(const SectorDev& S, const GateArg& g, PoolDev P, const cdf* src, cdf* dst, cudaStream_t st);
// Tiled gates: the table of one gate structure, and the in-place forward gate
// and reverse step that read it (k_tile.cu).
cudaError_t launch_tile_build(const SectorDev& S, int i, int j, const TypeDesc& t, PoolDev P, const TileRegion* reg_dev,
                              const TileSub* sub_dev, int nreg, int64_t max_count, int tile_slots, int* idx, int* bad,
                              cudaStream_t st);
// store (forward, may be NULL): each output amplitude also written there in
// slot order (ntiles x TILE_T x slots entries).
cudaError_t launch_tile_gate(const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial, bool adjoint,
                             cudaStream_t st, cdf* store = nullptr);
// The reverse step with psi at the gate's output read from store (as written
// by the forward gate): the gradient term and lambda <- U^dag lambda only.
cudaError_t launch_tile_gate_stored(const GateArg& g, PoolDev P, const cdf* store, cdf* lam, double* partial,
                                    cudaStream_t st);
cudaError_t launch_gate_adjoint(const SectorDev& S, const GateArg& g, PoolDev P, cdf* psi, cdf* lam, double* partial,
                                cudaStream_t st);
// Gradient-only pass over up to DIAG_GRAD_ACC gates of a diagonal run (their
// f type and modes): the gates of a run beyond the reverse pass's DIAG_ACC,
// so that a run of up to DIAG_ACC + DIAG_GRAD_ACC gates (a warm-start layer's
// Kerr and rotation gates on every mode) takes one extra pass.
constexpr int DIAG_GRAD_ACC = 16;
struct DiagGradArg {
  int m;
  int diag[DIAG_GRAD_ACC], gi[DIAG_GRAD_ACC], gj[DIAG_GRAD_ACC];
};
cudaError_t launch_diag_grad(const SectorDev& S, const DiagGradArg& a, const cdf* psi, const cdf* lam, double* partial,
                             cudaStream_t st);
// keep_psi (reverse only): dst holds the stored output state of the run,
// which is read and left unchanged; only lam is multiplied.
cudaError_t launch_diag_run(const SectorDev& S, const DiagRunArg& a, const cdf* src, cdf* dst, cdf* lam,
                            double* partial, bool adjoint, cudaStream_t st, bool keep_psi = false);
cudaError_t launch_dot_re(int64_t dim, const cdf* a, const cdf* b, double* partial, cudaStream_t st);
cudaError_t launch_scale_inv_sqrt(int64_t dim, cdf* v, const double* n2, cudaStream_t st);
cudaError_t launch_gate_proj_adj(const SectorDev& S, const GateArg& g, const cdf* D, PoolDev P, const cdf* prev,
                                 const cdf* cur, cdf* lam, const double* rdot, const double* n2, double* partial,
                                 cudaStream_t st);
// CTAs of the screen (at most NBLK): its partials are rows of screen_grid(S) slots.
int screen_grid(const SectorDev& S);
cudaError_t launch_screen(const SectorDev& S, const ScreenArg& a, const cdf* psi, const cdf* sigma, double* partial,
                          cudaStream_t st);
cudaError_t launch_screen_epilogue(const ScreenMap& m, int nsh, const double* z, double* grad, cudaStream_t st);
// State features (<n_r>, <n_r^2>, <a_i^dag a_j>) as (2L + 2 npairs) rows of partials.
cudaError_t launch_features(const SectorDev& S, const double2* psi, const int* pi, const int* pj, int npairs,
                            double* partial, cudaStream_t st);
// Lanczos on complex128 vectors: w <- w - alpha v - beta_prev v_prev with
// partial sums of ||w||^2, then v_next = w / ||w||.
cudaError_t launch_lanczos_update(const SectorDev& S, const double2* v_prev, const double2* v, double2* w,
                                  const double* alpha, const double* beta_prev, double* partial, cudaStream_t st);
cudaError_t launch_lanczos_scale(const SectorDev& S, const double2* w, double2* v_next, const double* partial,
                                 double* beta, cudaStream_t st);

// ------------------------------------------------------------- shared device helpers

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

// CTA sums of m <= N values per thread with two barriers in all, where N calls
// of block_sum take 2 N: each warp reduces every value with block_sum's
// shuffle tree, then thread k adds the eight warps' sums of value k in the
// order of block_sum's second tree (lanes 8..31 of that tree hold zeros, and
// adding zero is exact), so each result equals block_sum's bit for bit.
// val(k) gives value k; it is evaluated for k < m only.  Returns the sum of
// value k in thread k < min(m, N), 0 elsewhere.
template <int N, class V>
__device__ __forceinline__ double block_sums(V&& val, int m) {
  static_assert(NTHREADS == 256, "the cross-warp order below is block_sum's for eight warps");
  __shared__ double red[N][NTHREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // an earlier call's threads may still read red
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k < m) {
      double x = val(k);
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) red[k][warp] = x;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x >= min(m, N)) return 0.0;
  const double* r = red[threadIdx.x];
  return ((r[0] + r[4]) + (r[2] + r[6])) + ((r[1] + r[5]) + (r[3] + r[7]));
}

template <class T>
__device__ __forceinline__ void load_G(T (*Gs)[DMAX + 1], const SectorDev& S) {
  const int64_t* src = &S.tab->G[0][0];
  T* dst = &Gs[0][0];
  for (int t = threadIdx.x; t < LMAX * (DMAX + 1); t += blockDim.x) dst[t] = (T)src[t];
}

}  // namespace cvq
