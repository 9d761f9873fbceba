// k_mlp.cu -- the learned proposal's scorer: a 32 -> 256 -> 256 -> 1 ReLU MLP
// with bf16 weights and fp32 accumulation, its backward pass, a listwise
// softmax cross-entropy, and Adam.
//
// One forward over a pool of ~200 operators is ~15 MFLOP.  The two 256 x 256
// contractions (hidden layer forward, its transpose and its weight gradient
// backward) run on the tensor cores (mma.sync, bf16 operands, fp32 sums); the
// 32-wide input layer, the biases and the output layer stay on the CUDA
// cores, with weight copies laid out so that consecutive threads read
// consecutive bf16 values.  Every reduction (over hidden units or over rows)
// runs in a fixed order, so results are deterministic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <cstdio>
#include <new>
#include <vector>

#include "cvq_internal.cuh"

namespace cvq {

int internal_fail(int code, const char* msg);
int internal_prof_mlp_begin(cudaStream_t st, double bytes, double flops);
void internal_prof_end(int idx, cudaStream_t st);

constexpr int MF = 32, MH = 256;  // input width, hidden width
constexpr int O_W1 = 0, O_B1 = O_W1 + MH * MF, O_W2 = O_B1 + MH, O_B2 = O_W2 + MH * MH, O_W3 = O_B2 + MH,
              O_B3 = O_W3 + MH, NPARAM = O_B3 + 1;

typedef __nv_bfloat16 bf16;

struct MlpDev {
  float *P, *G, *Am, *Av;          // master parameters, gradients, Adam moments
  bf16 *W1T, *W2, *W2T, *W3;       // bf16 copies: W1T[f][u], W2[v][u], W2T[u][v], w3[v]
  float *H1, *H2, *dH1, *dH2;      // activations and their gradients, max_rows x MH
};

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

// Gradient of one parameter other than W2 (p outside [O_W2, O_B2)) as a sum
// over rows in row order.
__device__ __forceinline__ void param_grad(const MlpDev& m, const float* __restrict__ X, int rows,
                                           const float* __restrict__ ds, int p) {
  float g = 0.f;
  if (p < O_B1) {  // W1[u][f] = sum_r dH1[r][u] x[r][f]
    const int u = p / MF, f = p % MF;
    for (int r = 0; r < rows; ++r) g = fmaf(m.dH1[(size_t)r * MH + u], X[(size_t)r * MF + f], g);
  } else if (p < O_W2) {
    const int u = p - O_B1;
    for (int r = 0; r < rows; ++r) g += m.dH1[(size_t)r * MH + u];
  } else if (p < O_W3) {
    const int v = p - O_B2;
    for (int r = 0; r < rows; ++r) g += m.dH2[(size_t)r * MH + v];
  } else if (p < O_B3) {  // w3[v] = sum_r ds[r] h2[r][v]
    const int v = p - O_W3;
    for (int r = 0; r < rows; ++r) g = fmaf(ds[r], m.H2[(size_t)r * MH + v], g);
  } else {
    for (int r = 0; r < rows; ++r) g += ds[r];
  }
  m.G[p] = g;
}

// ------------------------------------------------------------ tensor-core layers
//
// The two 256 x 256 products (the hidden layer forward, and its transpose and
// weight gradient backward) run on the tensor cores with
// mma.sync.m16n8k16 (bf16 operands, fp32 accumulation).  The weights are
// bf16 already; an fp32 activation a is split into two bf16 numbers
// a_hi = bf16(a), a_lo = bf16(a - a_hi), whose sum is within 2^-18 |a| of a,
// and both halves are multiplied (the weight gradient, whose two operands
// are activations, takes hi*hi + hi*lo + lo*hi).  Each output still sums
// its terms in a fixed order, so results are deterministic.

constexpr int TC_ROWS = 16;            // rows of one forward / backward CTA (the MMA's M)
constexpr int TC_PAD = 8;              // bf16 padding per shared row: conflict-free fragment loads

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_bf16(float x, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragment (16 x 16, row major) of rows 0..15, columns k0..k0+15 of a
// shared [16][MH + TC_PAD] bf16 array.
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const bf16 (*A)[MH + TC_PAD], int k0) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
  a[0] = ld_pair(&A[g][k0 + 2 * t]);
  a[1] = ld_pair(&A[g + 8][k0 + 2 * t]);
  a[2] = ld_pair(&A[g][k0 + 2 * t + 8]);
  a[3] = ld_pair(&A[g + 8][k0 + 2 * t + 8]);
}

// out[r][n] = sum_k A[r][k] B[n][k] for the 16 rows of A (hi and lo halves)
// and this warp's 32 columns n0..n0+31; Bt is row n, column k (k contiguous).
__device__ __forceinline__ void mma_rows_x_256(float (&c)[4][4], const bf16 (*Ah)[MH + TC_PAD],
                                               const bf16 (*Al)[MH + TC_PAD], const bf16* __restrict__ Bt, int n0) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
#pragma unroll 4
  for (int k0 = 0; k0 < MH; k0 += 16) {
    uint32_t ah[4], al[4];
    frag_a(ah, Ah, k0);
    frag_a(al, Al, k0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bf16* bp = Bt + (size_t)(n0 + 8 * j + g) * MH + k0 + 2 * t;
      const uint32_t b0 = ld_pair(bp), b1 = ld_pair(bp + 8);
      mma_bf16(c[j], ah, b0, b1);
      mma_bf16(c[j], al, b0, b1);
    }
  }
}

// Rows r0..r0+15: h1 = relu(W1 x + b1) on the CUDA cores (K = 32), then
// h2 = relu(W2 h1 + b2) on the tensor cores, s = w3 . h2 + b3.
__global__ void __launch_bounds__(MH) k_mlp_fwd_tc(MlpDev m, const float* __restrict__ X, int rows,
                                                   float* __restrict__ out) {
  __shared__ float xs[TC_ROWS][MF];
  __shared__ __align__(16) bf16 Ah[TC_ROWS][MH + TC_PAD], Al[TC_ROWS][MH + TC_PAD];
  __shared__ float red[TC_ROWS][MH / 32];
  const int r0 = blockIdx.x * TC_ROWS, u = threadIdx.x;
  for (int e = u; e < TC_ROWS * MF; e += MH) {
    const int r = e / MF, f = e % MF;
    xs[r][f] = (r0 + r < rows) ? X[(size_t)(r0 + r) * MF + f] : 0.f;
  }
  __syncthreads();
  float acc[TC_ROWS];
  const float b1 = bf(__float2bfloat16_rn(m.P[O_B1 + u]));
#pragma unroll
  for (int r = 0; r < TC_ROWS; ++r) acc[r] = b1;
  for (int f = 0; f < MF; ++f) {
    const float w = bf(m.W1T[f * MH + u]);
#pragma unroll
    for (int r = 0; r < TC_ROWS; ++r) acc[r] = fmaf(xs[r][f], w, acc[r]);
  }
#pragma unroll
  for (int r = 0; r < TC_ROWS; ++r) {
    const float h = (r0 + r < rows) ? fmaxf(acc[r], 0.f) : 0.f;
    if (r0 + r < rows) m.H1[(size_t)(r0 + r) * MH + u] = h;
    split_bf16(h, Ah[r][u], Al[r][u]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int n0 = 32 * warp;
  float c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + 8 * j + 2 * t;
    const float b20 = bf(__float2bfloat16_rn(m.P[O_B2 + n])), b21 = bf(__float2bfloat16_rn(m.P[O_B2 + n + 1]));
    c[j][0] = b20;
    c[j][1] = b21;
    c[j][2] = b20;
    c[j][3] = b21;
  }
  mma_rows_x_256(c, Ah, Al, m.W2, n0);
  float s0 = 0.f, s1 = 0.f;  // score terms of rows g and g + 8
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + 8 * j + 2 * t;
    const float w30 = bf(m.W3[n]), w31 = bf(m.W3[n + 1]);
    const float h00 = fmaxf(c[j][0], 0.f), h01 = fmaxf(c[j][1], 0.f);
    const float h10 = fmaxf(c[j][2], 0.f), h11 = fmaxf(c[j][3], 0.f);
    if (r0 + g < rows) {
      m.H2[(size_t)(r0 + g) * MH + n] = h00;
      m.H2[(size_t)(r0 + g) * MH + n + 1] = h01;
    }
    if (r0 + g + 8 < rows) {
      m.H2[(size_t)(r0 + g + 8) * MH + n] = h10;
      m.H2[(size_t)(r0 + g + 8) * MH + n + 1] = h11;
    }
    s0 = fmaf(h01, w31, fmaf(h00, w30, s0));
    s1 = fmaf(h11, w31, fmaf(h10, w30, s1));
  }
  // the four lanes of a row group hold the row's terms of this warp's 32 columns
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  if (t == 0) {
    red[g][warp] = s0;
    red[g + 8][warp] = s1;
  }
  __syncthreads();
  if (u < TC_ROWS && r0 + u < rows) {
    float sc = bf(__float2bfloat16_rn(m.P[O_B3]));
    for (int w = 0; w < MH / 32; ++w) sc += red[u][w];
    out[r0 + u] = sc;
  }
}

// Rows r0..r0+15: dH2 = ds w3 [h2 > 0] on the CUDA cores, then
// dH1 = (W2^T dH2) [h1 > 0] on the tensor cores.
__global__ void __launch_bounds__(MH) k_mlp_bwd_rows_tc(MlpDev m, int rows, const float* __restrict__ ds) {
  __shared__ __align__(16) bf16 Ah[TC_ROWS][MH + TC_PAD], Al[TC_ROWS][MH + TC_PAD];
  const int r0 = blockIdx.x * TC_ROWS, v = threadIdx.x;
  const float w3 = bf(m.W3[v]);
#pragma unroll
  for (int r = 0; r < TC_ROWS; ++r) {
    float gv = 0.f;
    if (r0 + r < rows) {
      gv = (m.H2[(size_t)(r0 + r) * MH + v] > 0.f) ? ds[r0 + r] * w3 : 0.f;
      m.dH2[(size_t)(r0 + r) * MH + v] = gv;
    }
    split_bf16(gv, Ah[r][v], Al[r][v]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int n0 = 32 * warp;
  float c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[j][q] = 0.f;
  mma_rows_x_256(c, Ah, Al, m.W2T, n0);  // B[k = v][n = u] = W2[v][u], stored n-major as W2T[u][v]
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + 8 * j + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + g + 8 * h;
      if (r >= rows) continue;
      const float* H1 = m.H1 + (size_t)r * MH;
      m.dH1[(size_t)r * MH + n] = (H1[n] > 0.f) ? c[j][2 * h] : 0.f;
      m.dH1[(size_t)r * MH + n + 1] = (H1[n + 1] > 0.f) ? c[j][2 * h + 1] : 0.f;
    }
  }
}

// dW2[v][u] = sum_r dH2[r][v] H1[r][u] on the tensor cores: each CTA one
// 64 x 64 output tile, rows taken 16 at a time in order.
// CTAs past the 16 tiles compute every other parameter's gradient on the CUDA
// cores (one thread per parameter), so the whole weight gradient is one launch.
constexpr int DW_T = 64, DW_TILES = (MH / DW_T) * (MH / DW_T);
constexpr int DW_OTHER = O_W2 + (NPARAM - O_B2);  // parameters outside W2
__global__ void __launch_bounds__(MH) k_mlp_dw2_tc(MlpDev m, const float* __restrict__ X, int rows,
                                                   const float* __restrict__ ds) {
  if (blockIdx.x >= DW_TILES) {
    const int q = (blockIdx.x - DW_TILES) * blockDim.x + threadIdx.x;
    if (q < DW_OTHER) param_grad(m, X, rows, ds, q < O_W2 ? q : q - O_W2 + O_B2);
    return;
  }
  __shared__ __align__(16) bf16 Ah[DW_T][16 + TC_PAD], Al[DW_T][16 + TC_PAD];  // [v][r]
  __shared__ __align__(16) bf16 Bh[DW_T][16 + TC_PAD], Bl[DW_T][16 + TC_PAD];  // [u][r]
  const int v0 = (blockIdx.x / (MH / DW_T)) * DW_T, u0 = (blockIdx.x % (MH / DW_T)) * DW_T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 16, wn = (warp & 1) * 32;  // warp tile: 16 v x 32 u
  float c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[j][q] = 0.f;
  for (int rb = 0; rb < rows; rb += 16) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * DW_T; e += blockDim.x) {
      const int r = e / DW_T, x = e % DW_T;
      const bool ok = rb + r < rows;
      const float a = ok ? m.dH2[(size_t)(rb + r) * MH + v0 + x] : 0.f;
      const float b = ok ? m.H1[(size_t)(rb + r) * MH + u0 + x] : 0.f;
      split_bf16(a, Ah[x][r], Al[x][r]);
      split_bf16(b, Bh[x][r], Bl[x][r]);
    }
    __syncthreads();
    uint32_t ah[4], al[4];
    ah[0] = ld_pair(&Ah[wm + g][2 * t]);
    ah[1] = ld_pair(&Ah[wm + g + 8][2 * t]);
    ah[2] = ld_pair(&Ah[wm + g][2 * t + 8]);
    ah[3] = ld_pair(&Ah[wm + g + 8][2 * t + 8]);
    al[0] = ld_pair(&Al[wm + g][2 * t]);
    al[1] = ld_pair(&Al[wm + g + 8][2 * t]);
    al[2] = ld_pair(&Al[wm + g][2 * t + 8]);
    al[3] = ld_pair(&Al[wm + g + 8][2 * t + 8]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = wn + 8 * j + g;
      const uint32_t bh0 = ld_pair(&Bh[n][2 * t]), bh1 = ld_pair(&Bh[n][2 * t + 8]);
      const uint32_t bl0 = ld_pair(&Bl[n][2 * t]), bl1 = ld_pair(&Bl[n][2 * t + 8]);
      mma_bf16(c[j], ah, bh0, bh1);
      mma_bf16(c[j], ah, bl0, bl1);
      mma_bf16(c[j], al, bh0, bh1);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int u = u0 + wn + 8 * j + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = v0 + wm + g + 8 * h;
      m.G[O_W2 + v * MH + u] = c[j][2 * h];
      m.G[O_W2 + v * MH + u + 1] = c[j][2 * h + 1];
    }
  }
}

// Adam on the master weights, then the bf16 copies.
__global__ void __launch_bounds__(MH) k_mlp_adam(MlpDev m, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float g = m.G[p];
  const float a = 0.9f * m.Am[p] + 0.1f * g;
  const float b = 0.999f * m.Av[p] + 0.001f * g * g;
  m.Am[p] = a;
  m.Av[p] = b;
  m.P[p] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

__global__ void __launch_bounds__(MH) k_mlp_refresh(MlpDev m) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const bf16 w = __float2bfloat16_rn(m.P[p]);
  if (p < O_B1) {
    const int u = p / MF, f = p % MF;
    m.W1T[f * MH + u] = w;
  } else if (p >= O_W2 && p < O_B2) {
    const int q = p - O_W2, v = q / MH, u = q % MH;
    m.W2[v * MH + u] = w;
    m.W2T[u * MH + v] = w;
  } else if (p >= O_W3 && p < O_B3) {
    m.W3[p - O_W3] = w;
  }
}

// One CTA per list: softmax of the scores, dscores = softmax - p, loss = -sum p log softmax.
__global__ void __launch_bounds__(MH) k_listwise(const float* __restrict__ s, const float* __restrict__ t,
                                                 const int* __restrict__ off, float* __restrict__ ds,
                                                 float* __restrict__ loss) {
  __shared__ float red[MH / 32];
  __shared__ float bc;
  const int l = blockIdx.x, a = off[l], n = off[l + 1] - a;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto reduce = [&](float v, bool mx) -> float {
    for (int o = 16; o > 0; o >>= 1) {
      const float w = __shfl_down_sync(0xffffffffu, v, o);
      v = mx ? fmaxf(v, w) : v + w;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float r = red[0];
      for (int w = 1; w < MH / 32; ++w) r = mx ? fmaxf(r, red[w]) : r + red[w];
      bc = r;
    }
    __syncthreads();
    return bc;
  };
  float mx = -INFINITY;
  for (int k = threadIdx.x; k < n; k += MH) mx = fmaxf(mx, s[a + k]);
  mx = reduce(mx, true);
  float se = 0.f;
  for (int k = threadIdx.x; k < n; k += MH) se += expf(s[a + k] - mx);
  se = reduce(se, false);
  const float lse = mx + logf(se);
  float lo = 0.f;
  for (int k = threadIdx.x; k < n; k += MH) {
    const float p = t[a + k];
    ds[a + k] = expf(s[a + k] - lse) - p;
    lo -= p * (s[a + k] - lse);
  }
  lo = reduce(lo, false);
  if (threadIdx.x == 0) loss[l] = lo;
}

}  // namespace cvq

// ------------------------------------------------------------------ host side

using namespace cvq;

struct cvq_mlp {
  int device = 0, max_rows = 0, last_rows = -1;
  void* blob = nullptr;
  MlpDev d{};
};

namespace {

// splitmix64 (Steele, Lea and Flood, 2014) and the Box-Muller transform.
struct InitRng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u = uniform(), v = uniform();
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
  }
};

int cuda_err(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  const int code = cvq_status_from_cuda((int)e);
  return internal_fail(code == CVQ_OK ? CVQ_ECUDA : code, buf);
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

int refresh(cvq_mlp* m, cudaStream_t st) {
  k_mlp_refresh<<<(NPARAM + MH - 1) / MH, MH, 0, st>>>(m->d);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "mlp refresh");
}

int on_device(const cvq_mlp* m) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev != m->device) return internal_fail(CVQ_EINVAL, "model lives on another device");
  return CVQ_OK;
}

}  // namespace

extern "C" int cvq_mlp_create(int in_dim, int hidden, int max_rows, uint64_t seed, cvq_mlp** out) {
  if (!out) return internal_fail(CVQ_EINVAL, "null argument");
  *out = nullptr;
  if (in_dim != MF || hidden != MH) return internal_fail(CVQ_EINVAL, "the scorer is built for 32 inputs and 256 hidden units");
  if (max_rows < 1 || max_rows > (1 << 20)) return internal_fail(CVQ_EINVAL, "max_rows outside [1, 2^20]");
  cvq_mlp* m = new (std::nothrow) cvq_mlp;
  if (!m) return internal_fail(CVQ_ENOMEM, "host allocation");
  m->max_rows = max_rows;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) { delete m; return cuda_err(e, "cudaGetDevice"); }
  const size_t fp = a256(sizeof(float) * NPARAM);
  const size_t w1 = a256(sizeof(bf16) * MF * MH), w2 = a256(sizeof(bf16) * MH * MH), w3 = a256(sizeof(bf16) * MH);
  const size_t act = a256(sizeof(float) * (size_t)max_rows * MH);
  const size_t total = 4 * fp + w1 + 2 * w2 + w3 + 4 * act;
  e = cudaMalloc(&m->blob, total);
  if (e != cudaSuccess) { delete m; return internal_fail(CVQ_ENOMEM, "cudaMalloc of the scorer"); }
  char* b = (char*)m->blob;
  m->d.P = (float*)b; b += fp;
  m->d.G = (float*)b; b += fp;
  m->d.Am = (float*)b; b += fp;
  m->d.Av = (float*)b; b += fp;
  m->d.W1T = (bf16*)b; b += w1;
  m->d.W2 = (bf16*)b; b += w2;
  m->d.W2T = (bf16*)b; b += w2;
  m->d.W3 = (bf16*)b; b += w3;
  m->d.H1 = (float*)b; b += act;
  m->d.H2 = (float*)b; b += act;
  m->d.dH1 = (float*)b; b += act;
  m->d.dH2 = (float*)b;
  // He initialisation for the ReLU layers, variance 1/fan_in for the output; zero biases.
  std::vector<float> P(NPARAM, 0.f);
  InitRng rng{seed};
  for (int k = 0; k < MH * MF; ++k) P[O_W1 + k] = (float)(rng.normal() * std::sqrt(2.0 / MF));
  for (int k = 0; k < MH * MH; ++k) P[O_W2 + k] = (float)(rng.normal() * std::sqrt(2.0 / MH));
  for (int k = 0; k < MH; ++k) P[O_W3 + k] = (float)(rng.normal() * std::sqrt(1.0 / MH));
  const int rc = cvq_mlp_set(m, P.data(), P.size());
  if (rc) { cvq_mlp_destroy(m); return rc; }
  *out = m;
  return CVQ_OK;
}

extern "C" void cvq_mlp_destroy(cvq_mlp* m) {
  if (!m) return;
  if (m->blob) cudaFree(m->blob);
  delete m;
}

extern "C" int cvq_mlp_set(cvq_mlp* m, const float* host, size_t n) {
  if (!m || !host) return internal_fail(CVQ_EINVAL, "null argument");
  if (n != (size_t)NPARAM) return internal_fail(CVQ_EINVAL, "parameter vector must hold 74497 floats");
  if (int rc = on_device(m)) return rc;
  cudaError_t e = cudaMemcpy(m->d.P, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(e, "copy parameters");
  e = cudaMemset(m->d.G, 0, 3 * a256(sizeof(float) * NPARAM));  // G, Am, Av are contiguous
  if (e != cudaSuccess) return cuda_err(e, "zero moments");
  if (int rc = refresh(m, 0)) return rc;
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "synchronise");
}

extern "C" int cvq_mlp_get(const cvq_mlp* m, int which, float* host, size_t n) {
  if (!m || !host) return internal_fail(CVQ_EINVAL, "null argument");
  if (which != 0 && which != 1) return internal_fail(CVQ_EINVAL, "which must be 0 (parameters) or 1 (gradients)");
  if (n != (size_t)NPARAM) return internal_fail(CVQ_EINVAL, "parameter vector must hold 74497 floats");
  if (int rc = on_device(m)) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(e, "synchronise");
  e = cudaMemcpy(host, which ? m->d.G : m->d.P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "copy parameters");
}

extern "C" int cvq_mlp_forward(cvq_mlp* m, const float* X_dev, int rows, float* scores_dev, void* stream) {
  if (!m || (rows > 0 && (!X_dev || !scores_dev))) return internal_fail(CVQ_EINVAL, "null argument");
  if (rows < 0 || rows > m->max_rows) return internal_fail(CVQ_EINVAL, "rows outside [0, max_rows]");
  m->last_rows = rows;
  if (rows == 0) return CVQ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const double fl = 2.0 * rows * (MF * MH + MH * MH + MH);
  const double by = 2.0 * (MF * MH + MH * MH + MH) + 4.0 * rows * (MF + 1 + 2 * MH);
  const int pi = internal_prof_mlp_begin(st, by, fl);
  k_mlp_fwd_tc<<<(rows + TC_ROWS - 1) / TC_ROWS, MH, 0, st>>>(m->d, X_dev, rows, scores_dev);
  internal_prof_end(pi, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "mlp forward");
}

extern "C" int cvq_mlp_backward(cvq_mlp* m, const float* X_dev, int rows, const float* dscores_dev, void* stream) {
  if (!m || (rows > 0 && (!X_dev || !dscores_dev))) return internal_fail(CVQ_EINVAL, "null argument");
  if (rows != m->last_rows) return internal_fail(CVQ_EINVAL, "backward needs the rows of the last forward call");
  cudaStream_t st = (cudaStream_t)stream;
  if (rows > 0) {
    const int pi = internal_prof_mlp_begin(st, 2.0 * MH * MH + 4.0 * rows * (1 + 4 * MH), 2.0 * rows * MH * MH);
    k_mlp_bwd_rows_tc<<<(rows + TC_ROWS - 1) / TC_ROWS, MH, 0, st>>>(m->d, rows, dscores_dev);
    internal_prof_end(pi, st);
  }
  {
    const int pi = internal_prof_mlp_begin(st, 4.0 * NPARAM + 4.0 * rows * (MF + 1 + 4 * MH),
                                           2.0 * rows * (MF * MH + MH * MH + MH));
    k_mlp_dw2_tc<<<DW_TILES + (DW_OTHER + MH - 1) / MH, MH, 0, st>>>(m->d, X_dev, rows, dscores_dev);
    internal_prof_end(pi, st);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "mlp backward");
}

extern "C" int cvq_mlp_listwise_loss(const float* scores_dev, const float* targets_dev, const int* list_off_dev,
                                     int nlists, float* dscores_dev, float* loss_dev, void* stream) {
  if (nlists < 0 || nlists > (1 << 20)) return internal_fail(CVQ_EINVAL, "nlists outside [0, 2^20]");
  if (nlists == 0) return CVQ_OK;
  if (!scores_dev || !targets_dev || !list_off_dev || !dscores_dev || !loss_dev)
    return internal_fail(CVQ_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  k_listwise<<<nlists, MH, 0, st>>>(scores_dev, targets_dev, list_off_dev, dscores_dev, loss_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CVQ_OK : cuda_err(e, "listwise loss");
}

extern "C" int cvq_mlp_adam_step(cvq_mlp* m, float lr, int t, void* stream) {
  if (!m) return internal_fail(CVQ_EINVAL, "null argument");
  if (t < 1 || !(lr >= 0.f) || !std::isfinite(lr)) return internal_fail(CVQ_EINVAL, "need t >= 1 and a finite lr >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const float c1 = (float)(1.0 - std::pow(0.9, t)), c2 = (float)(1.0 - std::pow(0.999, t));
  const int pi = internal_prof_mlp_begin(st, 4.0 * 7 * NPARAM, 10.0 * NPARAM);
  k_mlp_adam<<<(NPARAM + MH - 1) / MH, MH, 0, st>>>(m->d, lr, c1, c2);
  internal_prof_end(pi, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "adam");
  return refresh(m, st);
}
