// k_batch.cu -- batched engine: the energy and adjoint gradient of many
// Hamiltonian instances (sectors of uneven size, each with its own pool and
// ansatz) evaluated together, as in a U/J sweep.
//
// One evaluation is a fixed sequence of layers: the conversion of every
// instance's reference state, one layer per ansatz segment (block gate, or
// run of diagonal gates) forward, the matvec lambda = H psi with the energy,
// one layer per segment in reverse with the gradient partials, and a
// fixed-order reduction.  Each layer is one persistent launch (a fixed grid
// of CTAs) that pulls (instance, tile) work items from a device counter, so
// small and large instances share the GPU within a layer; the layers follow
// one another on the stream, which orders them without any in-kernel wait.
// The host captures the whole sequence in a CUDA graph once per ansatz
// structure and replays it for every theta.
//
// Work items are disjoint ranges of one segment of one instance (block gates
// of pools with tile tables: ranges of the gate's tiles; other BH gates:
// ranges of the pool type's equal-work chunks; everything else: ranges of
// sector indices or orbits).  Each item leaves its partial sums in its own
// slots, so every result is independent of which CTA ran which item.
#include "cvq_internal.cuh"
#include "k_diag_impl.cuh"
#include "k_gate_impl.cuh"
#include "k_ham_impl.cuh"
#include "k_tile_impl.cuh"

namespace cvq {

__global__ void __launch_bounds__(128) k_batch_build(const BInst* __restrict__ insts, const int2* __restrict__ gates,
                                                     int ngates, const int* __restrict__ ids,
                                                     const double* __restrict__ theta, const int* __restrict__ active) {
  const int g = blockIdx.x;
  if (g >= ngates) return;
  const int2 ik = gates[g];
  if (!active[ik.x]) return;
  const BInst& I = insts[ik.x];
  const int op = ids[I.ids_off + ik.y];
  const TypeDesc& t = I.ops[op].t;
  if (t.diag) return;
  __shared__ double2 ph[MAX_BEXT];
  build_block_unitary(t, theta[I.theta_off + ik.y], I.P, I.U + (size_t)ik.y * I.ustride, blockIdx.y, ph);
}

// Shared state of one layer CTA.
struct BShared {
  SectorDev S;
  TypeDesc t;
  TileMap tm;
  BSeg seg;
  int item;
  int gi, gj;
};

__device__ __forceinline__ void copy_words(void* dst, const void* src, int bytes) {
  int* d = reinterpret_cast<int*>(dst);
  const int* s = reinterpret_cast<const int*>(src);
  for (int e = threadIdx.x; e < bytes / 4; e += blockDim.x) d[e] = s[e];
}

// Phase tables of a diagonal run from theta, in FP64 (as the single-instance
// path builds them on the host).
__device__ __forceinline__ void diag_tables(const BSeg& sg, const SectorDev& S, const double* th, cdf (*T)[DMAX],
                                            cdf (*TP)[DMAX * DMAX]) {
  const int D = S.D;
  for (int e = threadIdx.x; e < LMAX * DMAX; e += blockDim.x) {
    const int r = e / DMAX, n = e % DMAX;
    double ang = 0.0;
    for (int q = 0; q < sg.m; ++q) {
      const int dg = sg.diag[q];
      if (dg == 4 || sg.gi[q] != r) continue;
      const int f = (dg == 1) ? n * n : (dg == 2) ? n * (n - 1) : n;
      ang += th[q] * (double)f;
    }
    double s, c;
    sincos(ang, &s, &c);
    T[r][n] = make_cdf(df_from_double(c), df_from_double(s));
  }
  int p = 0;
  for (int q = 0; q < sg.m; ++q) {
    if (sg.diag[q] != 4) continue;
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
      const int u = e / D, v = e % D;
      double s, c;
      sincos(th[q] * (double)(u * v), &s, &c);
      TP[p][e] = make_cdf(df_from_double(c), df_from_double(s));
    }
    ++p;
  }
}

// One layer: items [0, nitems) of the layer's list, claimed in order from *counter.
template <int KIND, bool ADJ>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_batch_layer(const BInst* __restrict__ insts, const BSeg* __restrict__ segs, const BItem* __restrict__ items,
                  int nitems, int* counter, const int* __restrict__ ids, const double* __restrict__ theta,
                  const int* __restrict__ active, double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ BShared sh;
  __shared__ int64_t G64[LMAX][DMAX + 1];
  __shared__ int32_t G32[LMAX][DMAX + 1];
  // Bose-Hubbard matvec and diagonal-run items: the CTA's warps walk the
  // item's range (bh_walk_cta) with their tuple buffer in dynamic shared
  // memory after the item's tables (batch_walk_offset), and bond hops take
  // their rank changes from Dp
  __shared__ int32_t Dp[(KIND == CVQ_BH) ? LMAX : 1][DMAX + 1];
  uint64_t* wbuf = reinterpret_cast<uint64_t*>(smem + batch_walk_offset());
  for (;;) {
    if (threadIdx.x == 0) sh.item = atomicAdd(counter, 1);
    __syncthreads();
    const int k = sh.item;
    if (k >= nitems) break;
    const BItem it = items[k];
    if (!active[it.inst]) {  // instance paused for this evaluation: skip the item
      __syncthreads();
      continue;
    }
    const BInst& I = insts[it.inst];
    copy_words(&sh.S, &I.S, sizeof(SectorDev));
    if (it.kind != BI_TODF && it.kind != BI_APPLYH) copy_words(&sh.seg, &segs[it.seg], sizeof(BSeg));
    __syncthreads();
    const SectorDev& S = sh.S;
    if (KIND == CVQ_BH) {
      load_G(G64, S);
      load_G(G32, S);
    }
    if (it.kind == BI_TODF) {
      __syncthreads();
      for (int64_t x = it.a + threadIdx.x; x < it.b; x += NTHREADS) {
        const double2 v = I.psi0[x];
        I.psi[x] = make_cdf(df_from_double(v.x), df_from_double(v.y));
      }
    } else if (it.kind == BI_APPLYH) {
      HSmem& H = *reinterpret_cast<HSmem*>(smem);
      load_htabs(H, S);
      __syncthreads();
      dfacc eacc;
      acc_zero(eacc);
      if (KIND == CVQ_BH) {
        load_dhop(Dp, G64, S);
        __syncthreads();
        bh_walk_cta(S, G64, wbuf, it.a, it.b,
                    [&](int64_t x, uint64_t w) { apply_H_one<KIND>(S, G64, Dp, H, I.psi, I.lam, x, w, eacc); });
      } else {
        apply_H_range<KIND>(S, G64, H, I.psi, I.lam, it.a + threadIdx.x, it.b, NTHREADS, eacc);
      }
      const double s = block_sum(acc_to_double(eacc));
      if (threadIdx.x == 0) partial[it.slot] = s;
    } else if (it.kind == BI_DIAG) {
      cdf(*T)[DMAX] = reinterpret_cast<cdf(*)[DMAX]>(smem);
      cdf(*TP)[DMAX * DMAX] = reinterpret_cast<cdf(*)[DMAX * DMAX]>(smem + sizeof(cdf) * LMAX * DMAX);
      const BSeg& sg = sh.seg;
      diag_tables(sg, S, theta + I.theta_off + sg.k0, T, TP);
      __syncthreads();
      dfacc acc[BATCH_RUN];
#pragma unroll
      for (int q = 0; q < BATCH_RUN; ++q) acc_zero(acc[q]);
      if (KIND == CVQ_BH)
        bh_walk_cta(S, G64, wbuf, it.a, it.b, [&](int64_t x, uint64_t w) {
          diag_run_one<ADJ, BATCH_RUN>(S, T, TP, sg, I.psi, I.psi, I.lam, x, w, acc);
        });
      else
        diag_run_range<KIND, ADJ, BATCH_RUN>(S, G64, T, TP, sg, I.psi, I.psi, I.lam, it.a + threadIdx.x, it.b,
                                             NTHREADS, acc);
      if (ADJ) {
        const double s = block_sums<BATCH_RUN>([&](int q) { return acc_to_double(acc[q]); }, sg.m);
        if ((int)threadIdx.x < min(sg.m, BATCH_RUN)) partial[it.slot + threadIdx.x] = s;
      }
    } else if (it.kind == BI_TILE) {  // tiles [a, b) of a block gate
      const GateArg& ga = I.ops[ids[I.ids_off + segs[it.seg].k0]];
      copy_words(&sh.t, &ga.t, sizeof(TypeDesc));
      copy_words(&sh.tm, &ga.tm, sizeof(TileMap));
      __syncthreads();
      const cdf* U = I.U + (size_t)sh.seg.k0 * I.ustride;
      dfacc gacc;
      acc_zero(gacc);
      // one slot per thread (the plan gives tiles of more slots to the orbit kernels)
      if (sh.t.realu) tile_gate_range<ADJ, true, 1>(sh.t, sh.tm, U, I.P, it.a, it.b, 1, I.psi, I.lam, nullptr, smem, gacc);
      else tile_gate_range<ADJ, false, 1>(sh.t, sh.tm, U, I.P, it.a, it.b, 1, I.psi, I.lam, nullptr, smem, gacc);
      if (ADJ) {
        const double s = block_sum(acc_to_double(gacc));
        if (threadIdx.x == 0) partial[it.slot] = s;
      }
    } else {  // BI_GATE
      if (threadIdx.x == 0) {
        const GateArg& ga = I.ops[ids[I.ids_off + sh.seg.k0]];
        sh.gi = ga.i;
        sh.gj = ga.t.single ? -1 : ga.j;
      }
      copy_words(&sh.t, &I.ops[ids[I.ids_off + segs[it.seg].k0]].t, sizeof(TypeDesc));
      __syncthreads();
      const TypeDesc& t = sh.t;
      const GateSmem m = gate_smem(smem, t);
      stage_gate<ADJ>(m, t, I.U + (size_t)sh.seg.k0 * I.ustride, I.P);
      __syncthreads();
      dfacc gacc;
      acc_zero(gacc);
      if (KIND == CVQ_BKC) {
        if (t.realu)
          bkc_gate_range<ADJ, true>(S, sh.gi, sh.gj, t, m, it.a + threadIdx.x, it.b, NTHREADS, I.psi, I.psi, I.lam,
                                    gacc);
        else
          bkc_gate_range<ADJ, false>(S, sh.gi, sh.gj, t, m, it.a + threadIdx.x, it.b, NTHREADS, I.psi, I.psi, I.lam,
                                     gacc);
      } else {
        for (int64_t c = it.a; c < it.b; ++c) {
          const int4 ch = I.P.chunks[t.chunk_base + c];
          if (t.realu) bh_gate_chunk<ADJ, true>(S, G32, sh.gi, sh.gj, t, m, ch, I.psi, I.psi, I.lam, gacc);
          else bh_gate_chunk<ADJ, false>(S, G32, sh.gi, sh.gj, t, m, ch, I.psi, I.psi, I.lam, gacc);
        }
      }
      if (ADJ) {
        const double s = block_sum(acc_to_double(gacc));
        if (threadIdx.x == 0) partial[it.slot] = s;
      }
    }
    __syncthreads();  // the shared tables and item number are reused by the next item
  }
}

// A layer whose items are all tile ranges of block gates: the same loop as
// k_batch_layer's BI_TILE items, with only the tile code's registers, so five
// CTAs fit on an SM (the generic layer kernel, which also holds the orbit and
// diagonal-run code, fits two).
template <bool ADJ>
__global__ void __launch_bounds__(NTHREADS, 5)
    k_batch_tile_layer(const BInst* __restrict__ insts, const BSeg* __restrict__ segs, const BItem* __restrict__ items,
                       int nitems, int* counter, const int* __restrict__ ids, const int* __restrict__ active,
                       double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ TypeDesc t;
  __shared__ TileMap tm;
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int k = item;
    if (k >= nitems) break;
    const BItem it = items[k];
    if (!active[it.inst]) {  // instance paused for this evaluation: skip the item
      __syncthreads();
      continue;
    }
    const BInst& I = insts[it.inst];
    const int k0 = segs[it.seg].k0;
    const GateArg& ga = I.ops[ids[I.ids_off + k0]];
    copy_words(&t, &ga.t, sizeof(TypeDesc));
    copy_words(&tm, &ga.tm, sizeof(TileMap));
    __syncthreads();
    const cdf* U = I.U + (size_t)k0 * I.ustride;
    dfacc gacc;
    acc_zero(gacc);
    if (t.realu) tile_gate_range<ADJ, true, 1>(t, tm, U, I.P, it.a, it.b, 1, I.psi, I.lam, nullptr, smem, gacc);
    else tile_gate_range<ADJ, false, 1>(t, tm, U, I.P, it.a, it.b, 1, I.psi, I.lam, nullptr, smem, gacc);
    if (ADJ) {
      const double s = block_sum(acc_to_double(gacc));
      if (threadIdx.x == 0) partial[it.slot] = s;
    }
    __syncthreads();  // the shared tables and item number are reused by the next item
  }
}

cudaError_t launch_batch_tile_layer(bool adj, int grid, size_t smem, const BInst* insts, const BSeg* segs,
                                    const BItem* items, int nitems, int* counter, const int* ids, const int* active,
                                    double* partial, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (adj) k_batch_tile_layer<true><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, active, partial);
  else k_batch_tile_layer<false><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, active, partial);
  return cudaGetLastError();
}

cudaError_t set_batch_tile_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_tile_layer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_tile_layer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

// out = scale * sum of `count` partials from slot0 with `stride`, in order.
__global__ void k_batch_reduce(const BRed* __restrict__ red, int n, const double* __restrict__ partial,
                               const int* __restrict__ active, double* __restrict__ E, double* __restrict__ grad) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const BRed d = red[r];
  if (!active[d.inst]) return;
  double v = 0.0;
  for (int q = 0; q < d.count; ++q) v += partial[(size_t)d.slot0 + (size_t)q * d.stride];
  if (d.is_energy) E[d.out] = v;
  else grad[d.out] = 2.0 * v;
}

// The screen layer of the batched screen: items [0, nitems) claimed in order
// from *counter, each a range of one instance's sector, with that instance's
// sigma = H psi in its lambda buffer.
template <int KIND>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_batch_screen(const BInst* __restrict__ insts, const BItem* __restrict__ items, int nitems, int* counter,
                   const int* __restrict__ active, const BScreen* __restrict__ screens, const int4* __restrict__ desc,
                   double* __restrict__ partial) {
  __shared__ SectorDev S;
  __shared__ int item;
  __shared__ int64_t G64[LMAX][DMAX + 1];
  __shared__ float2 sq[DMAX][5];
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int k = item;
    if (k >= nitems) break;
    const BItem it = items[k];
    if (!active[it.inst]) {
      __syncthreads();
      continue;
    }
    const BInst& I = insts[it.inst];
    copy_words(&S, &I.S, sizeof(SectorDev));
    __syncthreads();
    if (KIND == CVQ_BH) load_G(G64, S);
    for (int e = threadIdx.x; e < DMAX * 5; e += blockDim.x) (&sq[0][0])[e] = (&S.tab->sq[0][0])[e];
    __syncthreads();
    const BScreen sc = screens[it.inst];
    const int nc_sh = (sc.nsh + SCREEN_CHUNK - 1) / SCREEN_CHUNK, nc_dg = (sc.ndg + SCREEN_CHUNK - 1) / SCREEN_CHUNK;
    for (int c = 0; c < nc_sh + nc_dg; ++c) {
      const bool isdg = c >= nc_sh;
      const int base = (isdg ? c - nc_sh : c) * SCREEN_CHUNK;
      const int cnt = min(SCREEN_CHUNK, (isdg ? sc.ndg : sc.nsh) - base);
      dfacc zr[SCREEN_CHUNK], zi[SCREEN_CHUNK];
      screen_chunk<KIND>(S, G64, sq, isdg, desc + (isdg ? sc.dg_off : sc.sh_off) + base, cnt, I.psi, I.lam,
                         it.a + threadIdx.x, it.b, NTHREADS, zr, zi);
      // one reduction for the chunk, laid out as in k_screen
      const int m = isdg ? cnt : 2 * cnt, q = threadIdx.x;
      const double s = block_sums<2 * SCREEN_CHUNK>(
          [&](int k) {
            return acc_to_double(isdg ? zr[k & (SCREEN_CHUNK - 1)] : ((k & 1) ? zi[k >> 1] : zr[k >> 1]));
          },
          m);
      if (q < m) partial[(size_t)it.slot + (isdg ? 2 * sc.nsh + base + q : 2 * base + q)] = s;
    }
    __syncthreads();  // S and the item number are reused by the next item
  }
}

__global__ void k_batch_screen_out(const BScreenOut* __restrict__ outs, int n, const double* __restrict__ z,
                                   const int* __restrict__ active, double* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const BScreenOut o = outs[k];
  if (!active[o.inst]) return;
  const double* zz = z + o.zrow;
  if (o.isdg) {
    grad[o.out] = 2.0 * zz[o.d];
  } else {
    const double pr = zz[2 * o.sp], pi = zz[2 * o.sp + 1], mr = zz[2 * o.sn], mi = zz[2 * o.sn + 1];
    grad[o.out] = 2.0 * ((o.cp.x * pr - o.cp.y * pi) - (o.cp.x * mr + o.cp.y * mi));
  }
}

cudaError_t launch_batch_screen(int kind, int grid, const BInst* insts, const BItem* items, int nitems, int* counter,
                                const int* active, const BScreen* screens, const int4* desc, double* partial,
                                cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (kind == CVQ_BH) k_batch_screen<CVQ_BH><<<grid, NTHREADS, 0, st>>>(insts, items, nitems, counter, active, screens, desc, partial);
  else k_batch_screen<CVQ_BKC><<<grid, NTHREADS, 0, st>>>(insts, items, nitems, counter, active, screens, desc, partial);
  return cudaGetLastError();
}

cudaError_t launch_batch_screen_out(const BScreenOut* outs, int n, const double* z, const int* active, double* grad,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_batch_screen_out<<<(n + 127) / 128, 128, 0, st>>>(outs, n, z, active, grad);
  return cudaGetLastError();
}

// One CTA per instance: the instance's whole evaluation with psi and lambda
// in shared memory (the sector must fit; the host checks).  Every segment's
// descriptor and generator structure is copied into shared memory once, at
// the start, so a segment only waits for its gate tables (staged in front of
// the states) before it runs.  Every partial sum of the instance lives in
// this CTA, so energies and gradients are written directly (2 x the
// fixed-order CTA sum for the gradients).
// Shared layout: [tables: tab_bytes][BSeg x seg_cap][TypeDesc x seg_cap][gi, gj x seg_cap][psi][lambda].
__host__ __device__ __forceinline__ size_t small_meta_bytes(int seg_cap) {
  const size_t b = (size_t)seg_cap * (sizeof(BSeg) + sizeof(TypeDesc) + sizeof(int2));
  return (b + 255) & ~(size_t)255;
}

template <int KIND>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_batch_small(int mode, size_t tab_bytes, int seg_cap, const BInst* __restrict__ insts,
                  const BSeg* __restrict__ segs, const int* __restrict__ ids, const double* __restrict__ theta,
                  const int* __restrict__ active, double* __restrict__ E, double* __restrict__ grad) {
  extern __shared__ __align__(16) char smem[];
  __shared__ SectorDev S;
  __shared__ int64_t G64[LMAX][DMAX + 1];
  __shared__ int32_t G32[LMAX][DMAX + 1];
  const int i = blockIdx.x;
  if (!active[i]) return;
  const BInst& I = insts[i];
  const int nseg = I.nseg;
  if (nseg < 0 || nseg > seg_cap) return;  // left out (the host sizes seg_cap for every instance)
  BSeg* sg_all = reinterpret_cast<BSeg*>(smem + tab_bytes);
  TypeDesc* td_all = reinterpret_cast<TypeDesc*>(sg_all + seg_cap);
  int2* ij_all = reinterpret_cast<int2*>(td_all + seg_cap);
  cdf* psi = reinterpret_cast<cdf*>(smem + tab_bytes + small_meta_bytes(seg_cap));
  const int64_t dim = I.S.dim;
  cdf* lam = psi + dim;
  copy_words(&S, &I.S, sizeof(SectorDev));
  copy_words(sg_all, segs + I.seg0, (int)(sizeof(BSeg) * nseg));
  for (int64_t x = threadIdx.x; x < dim; x += NTHREADS) {
    const double2 v = I.psi0[x];
    psi[x] = make_cdf(df_from_double(v.x), df_from_double(v.y));
  }
  __syncthreads();
  if (KIND == CVQ_BH) {
    load_G(G64, S);
    load_G(G32, S);
  }
  // generator structure and modes of every block-gate segment, fetched together
  for (int k = 0; k < nseg; ++k) {
    if (sg_all[k].isdiag) continue;
    const GateArg& ga = I.ops[ids[I.ids_off + sg_all[k].k0]];
    copy_words(&td_all[k], &ga.t, sizeof(TypeDesc));
    if (threadIdx.x == 0) ij_all[k] = make_int2(ga.i, ga.t.single ? -1 : ga.j);
  }
  __syncthreads();
  auto segment = [&](int k, bool adj) {
    const BSeg& sg = sg_all[k];
    if (sg.isdiag) {
      cdf(*T)[DMAX] = reinterpret_cast<cdf(*)[DMAX]>(smem);
      cdf(*TP)[DMAX * DMAX] = reinterpret_cast<cdf(*)[DMAX * DMAX]>(smem + sizeof(cdf) * LMAX * DMAX);
      diag_tables(sg, S, theta + I.theta_off + sg.k0, T, TP);
      __syncthreads();
      dfacc acc[BATCH_RUN];
#pragma unroll
      for (int q = 0; q < BATCH_RUN; ++q) acc_zero(acc[q]);
      if (adj) diag_run_range<KIND, true, BATCH_RUN>(S, G64, T, TP, sg, psi, psi, lam, threadIdx.x, dim, NTHREADS, acc);
      else diag_run_range<KIND, false, BATCH_RUN>(S, G64, T, TP, sg, psi, psi, lam, threadIdx.x, dim, NTHREADS, acc);
      if (adj) {
        const double s = block_sums<BATCH_RUN>([&](int q) { return acc_to_double(acc[q]); }, sg.m);
        if ((int)threadIdx.x < min(sg.m, BATCH_RUN)) grad[I.theta_off + sg.k0 + threadIdx.x] = 2.0 * s;
      }
    } else {
      const TypeDesc& t = td_all[k];
      const int gi = ij_all[k].x, gj = ij_all[k].y;
      const GateSmem m = gate_smem(smem, t);
      if (adj) stage_gate<true>(m, t, I.U + (size_t)sg.k0 * I.ustride, I.P);
      else stage_gate<false>(m, t, I.U + (size_t)sg.k0 * I.ustride, I.P);
      __syncthreads();
      dfacc gacc;
      acc_zero(gacc);
      if (KIND == CVQ_BKC) {
        const int64_t items = bkc_items(S, t.single ? 1 : 2);
        if (adj) {
          if (t.realu) bkc_gate_range<true, true>(S, gi, gj, t, m, threadIdx.x, items, NTHREADS, psi, psi, lam, gacc);
          else bkc_gate_range<true, false>(S, gi, gj, t, m, threadIdx.x, items, NTHREADS, psi, psi, lam, gacc);
        } else {
          if (t.realu) bkc_gate_range<false, true>(S, gi, gj, t, m, threadIdx.x, items, NTHREADS, psi, psi, lam, gacc);
          else bkc_gate_range<false, false>(S, gi, gj, t, m, threadIdx.x, items, NTHREADS, psi, psi, lam, gacc);
        }
      } else {  // every orbit of every class at once: one pass of the CTA for small sectors
        const int64_t norb = S.bh2_off[S.N + 1];
        if (adj) {
          if (t.realu) bh_gate_orbits<true, true>(S, G64, gi, gj, t, m, threadIdx.x, norb, NTHREADS, psi, psi, lam, gacc);
          else bh_gate_orbits<true, false>(S, G64, gi, gj, t, m, threadIdx.x, norb, NTHREADS, psi, psi, lam, gacc);
        } else {
          if (t.realu) bh_gate_orbits<false, true>(S, G64, gi, gj, t, m, threadIdx.x, norb, NTHREADS, psi, psi, lam, gacc);
          else bh_gate_orbits<false, false>(S, G64, gi, gj, t, m, threadIdx.x, norb, NTHREADS, psi, psi, lam, gacc);
        }
      }
      if (adj) {
        const double s = block_sum(acc_to_double(gacc));
        if (threadIdx.x == 0) grad[I.theta_off + sg.k0] = 2.0 * s;
      }
    }
    __syncthreads();  // the state is complete and the shared tables are free again
  };
  for (int k = 0; k < nseg; ++k) segment(k, false);
  {
    HSmem& H = *reinterpret_cast<HSmem*>(smem);
    load_htabs(H, S);
    __syncthreads();
    dfacc eacc;
    acc_zero(eacc);
    apply_H_range<KIND>(S, G64, H, psi, lam, threadIdx.x, dim, NTHREADS, eacc);
    const double s = block_sum(acc_to_double(eacc));
    if (threadIdx.x == 0 && mode == 0) E[i] = s;
    __syncthreads();
  }
  if (mode == 1) {  // the forward state and H psi for the screen layer
    for (int64_t x = threadIdx.x; x < dim; x += NTHREADS) {
      I.psi[x] = psi[x];
      I.lam[x] = lam[x];
    }
    return;
  }
  for (int k = nseg - 1; k >= 0; --k) segment(k, true);
}

size_t batch_small_smem(size_t tab_bytes, int seg_cap, int64_t dim_max) {
  return tab_bytes + small_meta_bytes(seg_cap) + 2 * sizeof(cdf) * (size_t)dim_max;
}

cudaError_t launch_batch_small(int kind, int mode, int n_inst, size_t tab_bytes, int seg_cap, size_t smem_total,
                               const BInst* insts, const BSeg* segs, const int* ids, const double* theta,
                               const int* active, double* E, double* grad, cudaStream_t st) {
  if (n_inst <= 0) return cudaSuccess;
  if (kind == CVQ_BH)
    k_batch_small<CVQ_BH><<<n_inst, NTHREADS, smem_total, st>>>(mode, tab_bytes, seg_cap, insts, segs, ids, theta,
                                                               active, E, grad);
  else
    k_batch_small<CVQ_BKC><<<n_inst, NTHREADS, smem_total, st>>>(mode, tab_bytes, seg_cap, insts, segs, ids, theta,
                                                                active, E, grad);
  return cudaGetLastError();
}

cudaError_t set_batch_small_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_small<CVQ_BH>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_small<CVQ_BKC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_batch_build(const BInst* insts, const int2* gates, int ngates, int maxblk, const int* ids,
                               const double* theta, const int* active, cudaStream_t st) {
  if (ngates <= 0 || maxblk <= 0) return cudaSuccess;
  k_batch_build<<<dim3(ngates, maxblk), 128, 0, st>>>(insts, gates, ngates, ids, theta, active);
  return cudaGetLastError();
}

cudaError_t launch_batch_layer(int kind, bool adj, int grid, size_t smem, const BInst* insts, const BSeg* segs,
                               const BItem* items, int nitems, int* counter, const int* ids, const double* theta,
                               const int* active, double* partial, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (kind == CVQ_BH) {
    if (adj) k_batch_layer<CVQ_BH, true><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, theta, active, partial);
    else k_batch_layer<CVQ_BH, false><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, theta, active, partial);
  } else {
    if (adj) k_batch_layer<CVQ_BKC, true><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, theta, active, partial);
    else k_batch_layer<CVQ_BKC, false><<<grid, NTHREADS, smem, st>>>(insts, segs, items, nitems, counter, ids, theta, active, partial);
  }
  return cudaGetLastError();
}

cudaError_t set_batch_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_batch_layer<CVQ_BH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_layer<CVQ_BH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_layer<CVQ_BKC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_layer<CVQ_BKC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_batch_reduce(const BRed* red, int n, const double* partial, const int* active, double* E,
                                double* grad, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_batch_reduce<<<(n + 127) / 128, 128, 0, st>>>(red, n, partial, active, E, grad);
  return cudaGetLastError();
}

}  // namespace cvq
