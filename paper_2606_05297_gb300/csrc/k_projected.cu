// k_projected.cu -- kernels of the projected-gate sweep (Sec. V.A): gates
// whose matrix elements are those of the untruncated gate kept inside the
// cutoff, with the state renormalised after every such gate.
//
// Forward, each block gate is the ordinary block kernel (its blocks hold the
// projected unitary) followed by the squared norm (k_dot_re) and a rescale.
// Reverse, with every forward state kept, one pass per gate forms
//   mu = (lambda - Re<psi_k|lambda> psi_k) / N_k,
//   g_k += Re <mu| D psi_{k-1}>   (D: theta derivative of the projected blocks),
//   lambda <- U^dag mu,
// orbit by orbit on the Kitaev-chain sector (the only sector a cutoff cuts).
#include "cvq_internal.cuh"
#include "k_diag_impl.cuh"
#include "k_gate_impl.cuh"

namespace cvq {

// partial[b] = Re sum_x conj(a[x]) b[x] over the CTA's grid-stride share (df sums).
__global__ void __launch_bounds__(NTHREADS) k_dot_re(int64_t dim, const cdf* __restrict__ a, const cdf* __restrict__ b,
                                                     double* __restrict__ partial) {
  dfacc acc;
  acc_zero(acc);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    const cdf u = a[x], v = b[x];
    acc_mac(acc, re_of(u), re_of(v));
    acc_mac(acc, im_of(u), im_of(v));
  }
  const double s = block_sum(acc_to_double(acc));
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// v <- v / sqrt(n2[0])
__global__ void __launch_bounds__(NTHREADS) k_scale_inv_sqrt(int64_t dim, cdf* __restrict__ v,
                                                             const double* __restrict__ n2) {
  const df f = df_from_double(1.0 / sqrt(n2[0]));
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
    const cdf u = v[x];
    v[x] = make_cdf(df_mul(re_of(u), f), df_mul(im_of(u), f));
  }
}

// One block of the reverse projected step (members staged in this thread's
// shared-memory column).
template <bool REALU>
__device__ __forceinline__ void proj_block(const int b, const cdf* __restrict__ Ub, const cdf* __restrict__ Db,
                                           const int2* __restrict__ mem, const BkcIdx& idx, const cdf* prev,
                                           const cdf* cur, cdf* lam, df r, df invN, cdf* stg, dfacc& gacc) {
  const int tid = threadIdx.x;
  for (int l = 0; l < b; ++l) stg[l * NTHREADS + tid] = prev[idx(mem[l])];
  auto mu_of = [&](int64_t x) -> cdf {
    const cdf la = lam[x], ps = cur[x];
    const df mr = df_mul(df_add(re_of(la), df_neg(df_mul(r, re_of(ps)))), invN);
    const df mi = df_mul(df_add(im_of(la), df_neg(df_mul(r, im_of(ps)))), invN);
    return make_cdf(mr, mi);
  };
  for (int k = 0; k < b; ++k) {
    dfacc dr, di;  // (D psi_{k-1})_k
    acc_zero(dr);
    acc_zero(di);
    for (int l = 0; l < b; ++l) cmac_full(dr, di, Db[k * b + l], stg[l * NTHREADS + tid]);
    const cdf mu = mu_of(idx(mem[k]));
    acc_mac(gacc, re_of(mu), acc_get(dr));
    acc_mac(gacc, im_of(mu), acc_get(di));
  }
  for (int l = 0; l < b; ++l) stg[l * NTHREADS + tid] = mu_of(idx(mem[l]));
  for (int k = 0; k < b; ++k) {  // lambda <- U^dag mu
    dfacc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
    for (int l = 0; l < b; ++l) cmac_cb<REALU, true>(ar, ai, Ub[l * b + k], stg[l * NTHREADS + tid], (k ^ l) & 1);
    lam[idx(mem[k])] = make_cdf(acc_get(ar), acc_get(ai));
  }
}

template <bool REALU>
__global__ void __launch_bounds__(NTHREADS)
    k_gate_proj_adj(const __grid_constant__ SectorDev S, const __grid_constant__ GateArg g, const cdf* __restrict__ Dg,
                    PoolDev P, const cdf* prev, const cdf* cur, cdf* lam, const double* __restrict__ rdot,
                    const double* __restrict__ n2, double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  const TypeDesc& t = g.t;
  cdf* sU = reinterpret_cast<cdf*>(smem);
  cdf* sD = sU + t.nu;
  BlockDesc* sB = reinterpret_cast<BlockDesc*>(sD + t.nu);
  int2* sM = reinterpret_cast<int2*>(sB + t.nblocks);
  cdf* stg = reinterpret_cast<cdf*>(smem + proj_tables_bytes(t));
  for (int e = threadIdx.x; e < t.nu; e += blockDim.x) {
    sU[e] = g.U[e];
    sD[e] = Dg[e];
  }
  for (int e = threadIdx.x; e < t.nblocks; e += blockDim.x) sB[e] = P.blk[t.blk_base + e];
  for (int e = threadIdx.x; e < t.nmem; e += blockDim.x) sM[e] = P.mem[t.mem_base + e];
  __syncthreads();
  const df r = df_from_double(rdot[0]), invN = df_from_double(1.0 / sqrt(n2[0]));
  const int j = t.single ? -1 : g.j;
  const int64_t items = bkc_items(S, t.single ? 1 : 2);
  BkcIdx idx;
  idx.si = S.stride[g.i];
  idx.sj = (j >= 0) ? S.stride[j] : 0;
  dfacc gacc;
  acc_zero(gacc);
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (int64_t)gridDim.x * blockDim.x) {
    int cls;
    bkc_orbit(S, g.i, j, it, items, idx.f0, cls);
    for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
      const BlockDesc bd = sB[bi];
      if (bd.bext < 2) {  // identity and no gradient term, but lambda still becomes mu
        const int64_t x = idx(sM[bd.mem_off]);
        const cdf la = lam[x], ps = cur[x];
        lam[x] = make_cdf(df_mul(df_add(re_of(la), df_neg(df_mul(r, re_of(ps)))), invN),
                          df_mul(df_add(im_of(la), df_neg(df_mul(r, im_of(ps)))), invN));
        continue;
      }
      proj_block<REALU>(bd.size, sU + bd.u_off, sD + bd.u_off, sM + bd.mem_off, idx, prev, cur, lam, r, invN, stg,
                        gacc);
    }
  }
  const double s = block_sum(acc_to_double(gacc));
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t launch_dot_re(int64_t dim, const cdf* a, const cdf* b, double* partial, cudaStream_t st) {
  k_dot_re<<<NBLK, NTHREADS, 0, st>>>(dim, a, b, partial);
  return cudaGetLastError();
}

cudaError_t launch_scale_inv_sqrt(int64_t dim, cdf* v, const double* n2, cudaStream_t st) {
  k_scale_inv_sqrt<<<NBLK, NTHREADS, 0, st>>>(dim, v, n2);
  return cudaGetLastError();
}

cudaError_t launch_gate_proj_adj(const SectorDev& S, const GateArg& g, const cdf* D, PoolDev P, const cdf* prev,
                                 const cdf* cur, cdf* lam, const double* rdot, const double* n2, double* partial,
                                 cudaStream_t st) {
  if (S.kind != CVQ_BKC || g.t.diag) return cudaErrorInvalidValue;
  const size_t sm = proj_tables_bytes(g.t) + (size_t)NTHREADS * g.t.bmax * sizeof(cdf);
  constexpr int kMaxSmem = 200 * 1024;
  if (sm > (size_t)kMaxSmem) return cudaErrorInvalidValue;
  static const bool attr_set = [] {  // once, also when several host threads launch
    cudaFuncSetAttribute(k_gate_proj_adj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_gate_proj_adj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    return true;
  }();
  (void)attr_set;
  if (g.t.realu) k_gate_proj_adj<true><<<NBLK, NTHREADS, sm, st>>>(S, g, D, P, prev, cur, lam, rdot, n2, partial);
  else k_gate_proj_adj<false><<<NBLK, NTHREADS, sm, st>>>(S, g, D, P, prev, cur, lam, rdot, n2, partial);
  return cudaGetLastError();
}

}  // namespace cvq
