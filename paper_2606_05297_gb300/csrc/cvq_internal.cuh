// cvq_internal.cuh -- device-side sector description, indexers and kernel
// launchers shared by the CUDA translation units of libcvq.so.
//
// Occupation tuples (n_0..n_{L-1}) travel through the kernels packed four bits
// per mode in one uint64 (L <= 16, D <= 16), so that no kernel needs a
// dynamically indexed per-thread array.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cvq.h"

namespace cvq {

constexpr int LMAX = 16;
constexpr int DMAX = 16;
constexpr int BMAX = 16;          // largest block of a gate (<= D)
constexpr int MAX_CLASSES = 17;   // BH: total pair occupation M = 0..N (N <= 15); BKC: 2 parities
constexpr int MAX_GATES = 512;    // ansatz length per call and pool size
constexpr int NTHREADS = 256;
constexpr int NBLK = 152 * 4;     // fixed grid: 4 CTAs per SM on the 152 SMs of a GB300
constexpr int PHASE_TABLE = 256;  // diagonal gates: e^{i theta f}, f = 0..(D-1)^2 <= 225

// ------------------------------------------------------------------ sector

struct SectorDev {
  int kind, L, N, D, parity, periodic, nb, half;   // half = d / 2 (BKC)
  int64_t dim;
  int64_t stride[LMAX];                 // BKC: d^(L-1-r)
  int64_t G[LMAX][DMAX + 1];            // BH: G[p][R] = C(R + p, p)
  int64_t bh2_off[MAX_CLASSES + 1];     // BH two-mode gate work items of class M start at bh2_off[M]
  double hop[LMAX], pair[LMAX], nn1[LMAX], n2[LMAX], n1[LMAX];
  double sqf[DMAX][5];                  // sqrt(max(n,n+e)! / min(n,n+e)!) for e = -2..2
};

__device__ __forceinline__ int occ_get(uint64_t w, int r) { return (int)((w >> (4 * r)) & 15ull); }
__device__ __forceinline__ uint64_t occ_shift(uint64_t w, int r, int delta) {
  return w + (uint64_t)((int64_t)delta * (int64_t)(1ull << (4 * r)));
}

// Lexicographic rank of a composition of N (combinatorial number system):
// rank = sum_{k < L-1} G[L-1-k][R_k] - G[L-1-k][R_{k+1}],  R_k = n_k + ... + n_{L-1}.
__device__ __forceinline__ int64_t bh_rank(uint64_t w, int L, int N, const int64_t (*G)[DMAX + 1]) {
  int64_t r = 0;
  int R = N;
  for (int k = 0; k < L - 1; ++k) {
    int n = occ_get(w, k);
    r += G[L - 1 - k][R] - G[L - 1 - k][R - n];
    R -= n;
  }
  return r;
}

// Inverse of bh_rank for a chain of Lc modes holding Nc bosons; the tuple is
// written to consecutive nibbles starting at nibble 0.
__device__ __forceinline__ uint64_t bh_unrank(int64_t x, int Lc, int Nc, const int64_t (*G)[DMAX + 1]) {
  uint64_t w = 0;
  int R = Nc;
  for (int k = 0; k < Lc - 1; ++k) {
    const int p = Lc - 1 - k;
    const int64_t base = G[p][R];
    int n = 0;
    while (n < R && x >= base - G[p][R - n - 1]) ++n;
    x -= base - G[p][R - n];
    w |= (uint64_t)n << (4 * k);
    R -= n;
  }
  if (Lc > 0) w |= (uint64_t)R << (4 * (Lc - 1));
  return w;
}

// Kitaev chain, even d: index = floor(f / 2), f = sum_r n_r d^(L-1-r).
__device__ __forceinline__ uint64_t bkc_unrank(int64_t x, const SectorDev& S) {
  const int L = S.L, d = S.D;
  int64_t hi = x / S.half;
  const int lo = (int)(x - hi * S.half);
  uint64_t w = 0;
  int par = 0;
  for (int k = L - 2; k >= 0; --k) {
    const int64_t q = hi / d;
    const int n = (int)(hi - q * d);
    hi = q;
    w |= (uint64_t)n << (4 * k);
    par += n;
  }
  const int nl = 2 * lo + ((S.parity - par) & 1);
  w |= (uint64_t)nl << (4 * (L - 1));
  return w;
}

__device__ __forceinline__ int64_t bkc_full(uint64_t w, const SectorDev& S) {
  int64_t f = 0;
  for (int r = 0; r < S.L; ++r) f += (int64_t)occ_get(w, r) * S.stride[r];
  return f;
}

// Copy the binomial table into shared memory (BH kernels).
__device__ __forceinline__ void load_G(int64_t (*Gs)[DMAX + 1], const SectorDev& S) {
  for (int t = threadIdx.x; t < LMAX * (DMAX + 1); t += blockDim.x) Gs[t / (DMAX + 1)][t % (DMAX + 1)] = S.G[t / (DMAX + 1)][t % (DMAX + 1)];
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
  int ev_off;   // into lam[] (size entries); V shares u_off layout in V[]
  int pad[3];
};

struct TypeDesc {
  int type, phase, single, diag;   // single: one-mode generator; diag: diagonal in the Fock basis
  int di, dj;                      // the generator's move (a, b) -> (a + di, b + dj)
  int nclass;
  int nblocks, nu, bmax;           // blocks, complex entries of one gate's U, largest block
  int class_off[MAX_CLASSES + 1];  // blocks of class c are blk[class_off[c] .. class_off[c+1])
  double cp_re, cp_im;             // c_plus
  double om_re, om_im;             // omega
  int blk_base, mem_base, f_base, v_base, lam_base;  // offsets of this type's tables in the pool arrays
};

struct PoolDev {
  const BlockDesc* blk;
  const int2* mem;
  const double* F;
  const double* V;
  const double* lam;
};

// Everything a gate kernel needs about one gate of an ansatz.
struct GateArg {
  int i, j;              // modes
  TypeDesc t;            // structure of the generator
  const double2* U;      // this gate's block unitaries (t.nu entries) or phase table (diagonal)
};

// Per-call list of gates for the unitary build kernel (passed by value).
struct BuildArgs {
  int n;
  int ustride;           // complex entries reserved per gate
  int type_of[MAX_GATES];
  int op_i[MAX_GATES], op_j[MAX_GATES];
  double theta[MAX_GATES];
};

// ------------------------------------------------------------- launchers
// All launchers enqueue on `stream` and return the launch status.

cudaError_t launch_apply_H(const SectorDev& S, const double2* psi, double2* sigma, double* partial, cudaStream_t st);
cudaError_t launch_reduce(const double* partial, int nred, int nblk, double scale, double* out, cudaStream_t st);
cudaError_t launch_build_gates(const BuildArgs& a, const TypeDesc* types_host, const TypeDesc* types_dev, PoolDev P,
                               double2* U, cudaStream_t st);
cudaError_t launch_gate(const SectorDev& S, const GateArg& g, PoolDev P, const double2* src, double2* dst,
                        cudaStream_t st);
cudaError_t launch_gate_adjoint(const SectorDev& S, const GateArg& g, PoolDev P, double2* psi, double2* lam,
                                double* partial, cudaStream_t st);
// A run of consecutive diagonal gates (they commute) applied in one pass:
// psi[x] *= exp(i phi(x)),  phi = sum_r ang[r][n_r] + sum_p pth[p] n_{pi[p]} n_{pj[p]}.
// The reverse pass forms every gradient of the run from the same (psi, lambda).
constexpr int MAX_RUN = 32, MAX_RUN_PAIRS = 8;
struct DiagRunArg {
  int m, npair;
  int diag[MAX_RUN], gi[MAX_RUN], gj[MAX_RUN];   // per gate: f type (1..4) and modes
  int pi[MAX_RUN_PAIRS], pj[MAX_RUN_PAIRS];
  double pth[MAX_RUN_PAIRS];
  double ang[LMAX][DMAX];                        // single-mode angles per occupation
};

cudaError_t launch_diag_run(const SectorDev& S, const DiagRunArg& a, const double2* src, double2* dst, double2* lam,
                            double* partial, bool adjoint, cudaStream_t st);

// Pool indices screened by one launch (passed by value).
struct SubsetArg {
  int n;
  int idx[MAX_GATES];
};

cudaError_t launch_screen(const SectorDev& S, const GateArg* pool_ops, const SubsetArg& sub, const double2* psi,
                          const double2* sigma, double* partial, cudaStream_t st);
// Lanczos: w <- w - alpha v - beta_prev v_prev with partial sums of ||w||^2,
// then v_next = w / ||w||.
cudaError_t launch_lanczos_update(const SectorDev& S, const double2* v_prev, const double2* v, double2* w,
                                  const double* alpha, const double* beta_prev, double* partial, cudaStream_t st);
cudaError_t launch_lanczos_scale(const SectorDev& S, const double2* w, double2* v_next, const double* partial,
                                 double* beta, cudaStream_t st);

}  // namespace cvq
