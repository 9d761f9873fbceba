// api.cu -- the C-ABI of libcvq.so (include/cvq.h): sector indexer and
// Hamiltonian tables, pool builder with per-block eigendecompositions, and the
// entry points that enqueue the kernels.
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "cvq_internal.cuh"

using namespace cvq;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Errors after which the context is unusable (every later CUDA call of the
// process fails): device-side faults and their relatives.
static bool sticky_cuda_error(cudaError_t e) {
  switch (e) {
    case cudaErrorIllegalAddress:
    case cudaErrorLaunchFailure:
    case cudaErrorIllegalInstruction:
    case cudaErrorMisalignedAddress:
    case cudaErrorInvalidAddressSpace:
    case cudaErrorInvalidPc:
    case cudaErrorHardwareStackError:
    case cudaErrorAssert:
    case cudaErrorLaunchTimeout:
    case cudaErrorECCUncorrectable:
    case cudaErrorContextIsDestroyed:
      return true;
    default:
      return false;
  }
}

extern "C" int cvq_status_from_cuda(int cuda_error) {
  const cudaError_t e = (cudaError_t)cuda_error;
  if (e == cudaSuccess) return CVQ_OK;
  if (e == cudaErrorMemoryAllocation) return CVQ_ENOMEM;
  return sticky_cuda_error(e) ? CVQ_EDEVICE : CVQ_ECUDA;
}

static int cuda_fail(cudaError_t e, const char* what) {
  const int code = cvq_status_from_cuda((int)e);
  return fail(code == CVQ_OK ? CVQ_ECUDA : code, "%s: %s", what, cudaGetErrorString(e));
}

#define CVQ_CUDA(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

extern "C" const char* cvq_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ profiling

enum KernelKind {
  KK_APPLY_H, KK_SCREEN, KK_GATE, KK_GATE_DIAG, KK_ADJ, KK_ADJ_DIAG, KK_BUILD, KK_REDUCE, KK_LANCZOS, KK_CONVERT,
  KK_FEATURES, KK_MLP, KK_COUNT
};
static const char* const kKindName[KK_COUNT] = {"apply_H", "screen", "gate_block", "gate_diag", "adjoint_block",
                                                "adjoint_diag", "build_unitaries", "reduce", "lanczos", "convert",
                                                "features", "mlp"};

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double bytes, flops;
};

static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};  // read without the lock on every launch
static std::vector<ProfRec> g_prof;
static size_t g_prof_n = 0;
static int g_prof_every = 1;                 // time one launch in this many of each kind
static int64_t g_prof_count[KK_COUNT];       // every launch while timing is on
static int64_t g_prof_timed[KK_COUNT];       // of which timed with an event pair
static double g_prof_bytes[KK_COUNT], g_prof_flops[KK_COUNT];

// Brackets one launch with an event pair on its stream while timing is on.
struct ProfScope {
  int idx = -1;
  cudaStream_t st;
  ProfScope(int kind, cudaStream_t s, double bytes, double flops) : st(s) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    g_prof_bytes[kind] += bytes;
    g_prof_flops[kind] += flops;
    if (g_prof_count[kind]++ % g_prof_every != 0 || g_prof_n >= g_prof.size()) return;
    ++g_prof_timed[kind];
    idx = (int)g_prof_n++;
    g_prof[idx].kind = kind;
    g_prof[idx].bytes = bytes;
    g_prof[idx].flops = flops;
    cudaEventRecord(g_prof[idx].a, st);
  }
  ~ProfScope() {
    if (idx >= 0) cudaEventRecord(g_prof[idx].b, st);
  }
};

extern "C" int cvq_profile_start(int capacity) {
  if (capacity <= 0 || capacity > (1 << 22)) return fail(CVQ_EINVAL, "capacity %d outside [1, 2^22]", capacity);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof.size() < (size_t)capacity) {
    size_t old = g_prof.size();
    g_prof.resize(capacity);
    for (size_t k = old; k < g_prof.size(); ++k) {
      cudaError_t e1 = cudaEventCreate(&g_prof[k].a), e2 = cudaEventCreate(&g_prof[k].b);
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        g_prof.resize(k);
        return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaEventCreate");
      }
    }
  }
  g_prof_n = 0;
  memset(g_prof_count, 0, sizeof g_prof_count);
  memset(g_prof_timed, 0, sizeof g_prof_timed);
  memset(g_prof_bytes, 0, sizeof g_prof_bytes);
  memset(g_prof_flops, 0, sizeof g_prof_flops);
  g_prof_on = true;
  return CVQ_OK;
}

extern "C" int cvq_profile_sample(int every) {
  if (every < 1) return fail(CVQ_EINVAL, "every must be >= 1");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_every = every;
  return CVQ_OK;
}

extern "C" int cvq_profile_stop(cvq_kernel_stat* out, int max_out, int* n_out) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = false;
  cvq_kernel_stat acc[KK_COUNT];
  memset(acc, 0, sizeof acc);
  for (size_t k = 0; k < g_prof_n; ++k) {
    const ProfRec& r = g_prof[k];
    CVQ_CUDA(cudaEventSynchronize(r.b), "cudaEventSynchronize");
    float ms = 0.f;
    CVQ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    acc[r.kind].ms += ms;
  }
  for (int k = 0; k < KK_COUNT; ++k) {  // every launch counts; the timed ones stand for their kind
    acc[k].launches = g_prof_count[k];
    if (g_prof_timed[k] > 0) acc[k].ms *= (double)g_prof_count[k] / (double)g_prof_timed[k];
    acc[k].bytes = g_prof_bytes[k];
    acc[k].flops = g_prof_flops[k];
  }
  g_prof_n = 0;
  int n = 0;
  for (int k = 0; k < KK_COUNT; ++k) {
    if (!acc[k].launches) continue;
    if (out && n < max_out) {
      out[n] = acc[k];
      snprintf(out[n].name, sizeof out[n].name, "%s", kKindName[k]);
    }
    ++n;
  }
  if (n_out) *n_out = std::min(n, max_out);
  return CVQ_OK;
}

// ------------------------------------------------------------------ objects

struct cvq_sector {
  SectorDev S;
  SectorTabs tabs;               // host copy of the device tables
  SectorTabs* tabs_dev = nullptr;
  double hop[LMAX], pair[LMAX];  // bond coefficients (FP64, host side)
  int device;
};

struct cvq_pool {
  const cvq_sector* sec;
  int K;
  std::vector<TypeDesc> types;   // distinct (type, phase) generators
  std::vector<int> op_type, op_i, op_j;
  TypeDesc* types_dev = nullptr;
  GateArg* ops_dev = nullptr;    // one per pool element (screen)
  void* blob = nullptr;          // device tables
  PoolDev P{};
  int ustride = PHASE_TABLE;     // complex entries per gate in a call's U buffer
  std::vector<int> blk_size;     // host copy of every block's size (costs)
  int dc = 0;                    // > 0: projected gates with this inner cutoff
  void* tile_blob = nullptr;     // index tables of the tiled gates (one per distinct gate structure)
  std::vector<TileMap> op_tiles; // per pool element (empty map for diagonal generators)
};

static int64_t binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

static int64_t fact_ratio(int lo, int hi) {  // hi! / lo!
  int64_t r = 1;
  for (int v = lo + 1; v <= hi; ++v) r *= v;
  return r;
}

// Round-to-nearest split of a double into a df pair (hi + lo).
static float2 split_df(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// ------------------------------------------------------------------ sector

extern "C" int cvq_init_sector(const cvq_model* m, cvq_sector** out) {
  if (!m || !out) return fail(CVQ_EINVAL, "null argument");
  *out = nullptr;
  const int L = m->L;
  if (L < 1 || L > LMAX) return fail(CVQ_EINVAL, "L = %d outside [1, %d]", L, LMAX);
  if (m->periodic && L < 2) return fail(CVQ_EINVAL, "periodic chain needs L >= 2");
  if (m->kind != CVQ_BH && m->kind != CVQ_BKC) return fail(CVQ_EINVAL, "unknown model kind %d", m->kind);
  cvq_sector* s = new (std::nothrow) cvq_sector;
  if (!s) return fail(CVQ_ENOMEM, "host allocation");
  SectorDev& S = s->S;
  SectorTabs& T = s->tabs;
  memset(&S, 0, sizeof S);
  memset(&T, 0, sizeof T);
  memset(s->hop, 0, sizeof s->hop);
  memset(s->pair, 0, sizeof s->pair);
  S.kind = m->kind;
  S.L = L;
  S.periodic = m->periodic ? 1 : 0;
  S.nb = m->periodic ? L : L - 1;
  int rc = CVQ_OK;
  if (m->kind == CVQ_BH) {
    if (m->N < 0 || m->N + 1 > DMAX) rc = fail(CVQ_EINVAL, "BH needs 0 <= N <= %d", DMAX - 1);
    S.N = m->N;
    S.D = m->N + 1;
    if (m->pair)
      for (int b = 0; b < S.nb; ++b)
        if (m->pair[b] != 0.0) rc = fail(CVQ_EINVAL, "pairing term breaks the fixed-N sector");
    S.dim = binom(S.N + L - 1, L - 1);
  } else {
    if (m->d < 2 || m->d > DMAX || (m->d & 1)) {
      rc = fail(CVQ_EINVAL, "BKC needs even d in [2, %d]", DMAX);
    } else {
      S.D = m->d;
      S.half = m->d / 2;
      S.parity = m->parity & 1;
      int64_t full = 1;
      for (int r = L - 1; r >= 0 && !rc; --r) {
        S.stride[r] = full;
        if (full > ((int64_t)1 << 42) / m->d) rc = fail(CVQ_EINVAL, "sector dimension above 2^40");
        full *= m->d;
      }
      S.dim = full / 2;
    }
  }
  if (!rc && S.dim > ((int64_t)1 << 40)) rc = fail(CVQ_EINVAL, "sector dimension above 2^40");
  if (!rc) set_bkc_div(S);
  if (rc) {
    delete s;
    return rc;
  }
  for (int p = 0; p < LMAX; ++p)
    for (int R = 0; R <= DMAX; ++R) T.G[p][R] = binom(R + p, p);
  if (S.kind == CVQ_BH) {
    // two-mode gate work items: classes M = n_i + n_j = 0..N, each holding the
    // compositions of N - M into the other L - 2 modes
    int64_t acc = 0;
    for (int M = 0; M <= S.N; ++M) {
      S.bh2_off[M] = acc;
      if (L >= 3) acc += binom(S.N - M + L - 3, L - 3);
      else if (L == 2) acc += (M == S.N) ? 1 : 0;
    }
    S.bh2_off[S.N + 1] = acc;
    for (int M = S.N + 2; M <= MAX_CLASSES; ++M) S.bh2_off[M] = acc;
  }
  for (int b = 0; b < S.nb; ++b) {
    s->hop[b] = m->hop ? m->hop[b] : 0.0;
    s->pair[b] = m->pair ? m->pair[b] : 0.0;
    T.hop[b] = split_df(s->hop[b]);
    T.pair[b] = split_df(s->pair[b]);
  }
  for (int r = 0; r < L; ++r) {
    const double c2 = m->onsite_nn1 ? m->onsite_nn1[r] : 0.0;
    const double cq = m->onsite_n2 ? m->onsite_n2[r] : 0.0;
    const double c1 = m->onsite_n ? m->onsite_n[r] : 0.0;
    for (int n = 0; n < S.D; ++n) T.diagE[r][n] = split_df(c2 * n * (n - 1) + cq * n * n + c1 * n);
  }
  for (int n = 0; n < DMAX; ++n) {
    for (int e = -2; e <= 2; ++e) {
      const int t = n + e;
      T.sq[n][e + 2] = (t < 0 || t >= S.D) ? make_float2(0.f, 0.f)
                                             : split_df(std::sqrt((double)fact_ratio(std::min(n, t), std::max(n, t))));
    }
    for (int q = 0; q < DMAX; ++q) {
      T.P[0][n][q] = split_df(std::sqrt((double)(n + 1) * q));
      T.P[1][n][q] = split_df(std::sqrt((double)n * (q + 1)));
      T.P[2][n][q] = split_df(std::sqrt((double)(n + 1) * (q + 1)));
      T.P[3][n][q] = split_df(std::sqrt((double)n * q));
    }
  }
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->tabs_dev, sizeof(SectorTabs));
  if (e == cudaSuccess) e = cudaMemcpy(s->tabs_dev, &T, sizeof(SectorTabs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (s->tabs_dev) cudaFree(s->tabs_dev);
    delete s;
    return cuda_fail(e, "sector tables");
  }
  S.tab = s->tabs_dev;
  *out = s;
  return CVQ_OK;
}

extern "C" int cvq_sector_dim(const cvq_sector* s, int64_t* dim) {
  if (!s || !dim) return fail(CVQ_EINVAL, "null argument");
  *dim = s->S.dim;
  return CVQ_OK;
}

extern "C" int cvq_sector_index(const cvq_sector* s, const int* occ, int64_t* index) {
  if (!s || !occ || !index) return fail(CVQ_EINVAL, "null argument");
  const SectorDev& S = s->S;
  int tot = 0;
  for (int r = 0; r < S.L; ++r) {
    if (occ[r] < 0 || occ[r] >= S.D) return fail(CVQ_EINVAL, "occupation %d of mode %d outside [0, %d)", occ[r], r, S.D);
    tot += occ[r];
  }
  if (S.kind == CVQ_BH) {
    if (tot != S.N) return fail(CVQ_EINVAL, "occupations sum to %d, sector has N = %d", tot, S.N);
    int64_t rk = 0;
    int R = S.N;
    for (int k = 0; k < S.L - 1; ++k) {
      rk += s->tabs.G[S.L - 1 - k][R] - s->tabs.G[S.L - 1 - k][R - occ[k]];
      R -= occ[k];
    }
    *index = rk;
  } else {
    if ((tot & 1) != S.parity) return fail(CVQ_EINVAL, "occupation parity differs from the sector's");
    int64_t f = 0;
    for (int r = 0; r < S.L; ++r) f += occ[r] * S.stride[r];
    *index = f >> 1;
  }
  return CVQ_OK;
}

extern "C" void cvq_destroy_sector(cvq_sector* s) {
  if (!s) return;
  if (s->tabs_dev) cudaFree(s->tabs_dev);
  delete s;
}

// ------------------------------------------------------------------ pool

// Eigen-decomposition of a real symmetric matrix by cyclic Jacobi rotations:
// A = V diag(w) V^T, V column m = eigenvector m.  A is overwritten.
static void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& V, std::vector<double>& w) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        const double a = A[(size_t)p * n + q];
        tot += a * a;
        if (p != q) off += a * a;
      }
    if (off <= 1e-34 * (tot > 0 ? tot : 1.0)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        // rotation angle phi with tan(2 phi) = 2 a_pq / (a_qq - a_pp); t = tan(phi), smaller root
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

struct PoolBuild {
  std::vector<int4> chunks;
  std::vector<BlockDesc> blk;
  std::vector<int2> mem;
  std::vector<float2> F;
  std::vector<double> V, lam;
};

static std::complex<double> ipow(int p) {
  static const std::complex<double> t[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
  return t[((p % 4) + 4) % 4];
}

// Build the block tables of one (type, phase) generator in sector S.
// dc > 0: projected gates (Sec. V.A): every block's chain is extended past the
// cutoff up to occupations dc - 1 and the eigendecomposition is of that chain;
// the members inside the cutoff are a contiguous segment of it.
static int build_type(const SectorDev& S, int type, int phase, PoolBuild& pb, TypeDesc& t, int dc = 0) {
  memset(&t, 0, sizeof t);
  t.type = type;
  t.phase = phase & 3;
  const std::complex<double> e = ipow(phase);
  std::complex<double> cp(1, 0);
  switch (type) {
    case CVQ_OP_HOP: t.di = 1; t.dj = -1; cp = e; break;
    case CVQ_OP_SQ2: t.di = 1; t.dj = 1; cp = e; break;
    case CVQ_OP_SQ1: t.di = 2; t.dj = 0; t.single = 1; cp = 0.5 * std::conj(e); break;
    case CVQ_OP_PAIRHOP: t.di = 2; t.dj = -2; cp = e; break;
    case CVQ_OP_KERR: t.single = 1; t.diag = 1; break;
    case CVQ_OP_NN1: t.single = 1; t.diag = 2; break;
    case CVQ_OP_ROT: t.single = 1; t.diag = 3; break;
    case CVQ_OP_XKERR: t.diag = 4; break;
    default: return fail(CVQ_EINVAL, "unknown op type %d", type);
  }
  if (S.kind == CVQ_BH && (type == CVQ_OP_SQ2 || type == CVQ_OP_SQ1))
    return fail(CVQ_EINVAL, "op type %d breaks the fixed-N sector", type);
  t.cp_re = cp.real();
  t.cp_im = cp.imag();
  t.realu = (cp.imag() == 0.0) ? 1 : 0;
  if (t.diag) return CVQ_OK;
  const double acp = std::abs(cp);
  const std::complex<double> om = std::complex<double>(0, 1) * std::conj(cp) / acp;
  t.om_re = om.real();
  t.om_im = om.imag();
  t.blk_base = (int)pb.blk.size();
  t.mem_base = (int)pb.mem.size();
  t.f_base = (int)pb.F.size();
  t.v_base = (int)pb.V.size() / 2;
  t.lam_base = (int)pb.lam.size();
  const int D = S.D;
  t.nclass = (S.kind == CVQ_BH) ? S.N + 1 : 2;
  auto allowed_c = [&](int cls, int a, int b, int cut) -> bool {
    if (a < 0 || a >= cut) return false;
    if (t.single) return b == 0 && (a & 1) == cls;
    if (b < 0 || b >= cut) return false;
    if (S.kind == CVQ_BH) return a + b == cls;
    return ((a + b) & 1) == cls;
  };
  auto allowed = [&](int cls, int a, int b) -> bool { return allowed_c(cls, a, b, D); };
  const int cut_ext = dc > 0 ? dc : D;
  int nu = 0, nmem = 0, nf = 0, nlam = 0, nv = 0;
  for (int cls = 0; cls < t.nclass; ++cls) {
    t.class_off[cls] = (int)pb.blk.size() - t.blk_base;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < (t.single ? 1 : D); ++b) {
        if (!allowed(cls, a, b) || allowed(cls, a - t.di, b - t.dj)) continue;
        std::vector<std::pair<int, int>> ch;
        for (int x = a, y = b; allowed(cls, x, y); x += t.di, y += t.dj) ch.push_back({x, y});
        const int n = (int)ch.size();
        if (n > BMAX) return fail(CVQ_EINVAL, "block of size %d exceeds %d", n, BMAX);
        // the chain the eigendecomposition is of: the block itself, or extended to the inner cutoff
        std::vector<std::pair<int, int>> ex;
        int x0 = a, y0 = b;
        while (allowed_c(cls, x0 - t.di, y0 - t.dj, cut_ext)) {
          x0 -= t.di;
          y0 -= t.dj;
        }
        for (int x = x0, y = y0; allowed_c(cls, x, y, cut_ext); x += t.di, y += t.dj) ex.push_back({x, y});
        const int ne = (int)ex.size();
        int off = 0;
        while (off < ne && ex[off] != ch[0]) ++off;
        if (ne > MAX_BEXT || off + n > ne) return fail(CVQ_EINVAL, "extended chain of %d members exceeds %d", ne, MAX_BEXT);
        BlockDesc bd;
        memset(&bd, 0, sizeof bd);
        bd.size = n;
        bd.bext = ne;
        bd.mem_off = nmem;
        bd.u_off = nu;
        bd.v_off = nv;
        bd.f_off = nf;
        bd.ev_off = nlam;
        auto factor = [&](const std::pair<int, int>& p0, const std::pair<int, int>& p1) {
          double fk = (double)fact_ratio(std::min(p0.first, p1.first), std::max(p0.first, p1.first));
          if (!t.single) fk *= (double)fact_ratio(std::min(p0.second, p1.second), std::max(p0.second, p1.second));
          return std::sqrt(fk);
        };
        for (int k = 0; k + 1 < n; ++k) pb.F.push_back(split_df(factor(ch[k], ch[k + 1])));
        std::vector<double> T((size_t)ne * ne, 0.0), Vr, w;
        for (int k = 0; k + 1 < ne; ++k) T[(size_t)k * ne + k + 1] = T[(size_t)(k + 1) * ne + k] = acp * factor(ex[k], ex[k + 1]);
        if (ne > 1) {
          jacobi_eigen(T, ne, Vr, w);
        } else {
          Vr.assign(1, 1.0);
          w.assign(1, 0.0);
        }
        // rows of the members (chain positions off .. off + n - 1) of W V, W = diag(om^k)
        std::complex<double> omk(1, 0);
        for (int k = 0; k < off; ++k) omk *= om;
        for (int k = off; k < off + n; ++k) {
          for (int m = 0; m < ne; ++m) {
            const std::complex<double> v = omk * Vr[(size_t)k * ne + m];
            pb.V.push_back(v.real());
            pb.V.push_back(v.imag());
          }
          omk *= om;
        }
        for (int m = 0; m < ne; ++m) pb.lam.push_back(w[m]);
        for (auto& pr : ch) pb.mem.push_back(make_int2(pr.first, pr.second));
        pb.blk.push_back(bd);
        nu += n * n;
        nv += n * ne;
        nmem += n;
        nf += n - 1;
        nlam += ne;
        t.bmax = std::max(t.bmax, n);
      }
  }
  t.class_off[t.nclass] = (int)pb.blk.size() - t.blk_base;
  t.nblocks = t.class_off[t.nclass];
  t.nu = nu;
  t.nmem = nmem;
  t.nf = nf;
  if (S.kind == CVQ_BH) {
    // Equal-work schedule: orbits of class M cost about 24 + sum_blocks (b^2 + 4 b)
    // units; classes are cut into chunks of about total / (4 NBLK) units so that
    // every CTA gets a similar share and each chunk has a single block structure.
    // A chunk holds a multiple of NTHREADS orbits (all but a class's last), so
    // every thread of the CTA gets the same run of orbits.
    std::vector<double> w(t.nclass, 24.0);
    double total = 0.0;
    for (int M = 0; M < t.nclass; ++M) {
      for (int bi = t.class_off[M]; bi < t.class_off[M + 1]; ++bi) {
        const int b = pb.blk[t.blk_base + bi].size;
        w[M] += (double)b * b + 4.0 * b;
      }
      total += w[M] * (double)(S.bh2_off[M + 1] - S.bh2_off[M]);
    }
    const double target = std::max(total / (4.0 * NBLK), 1.0);
    t.chunk_base = (int)pb.chunks.size();
    for (int M = 0; M < t.nclass; ++M) {
      int bm = 0;
      for (int bi = t.class_off[M]; bi < t.class_off[M + 1]; ++bi) bm = std::max(bm, pb.blk[t.blk_base + bi].bext);
      if (bm < 2) continue;  // only one-member blocks: the gate is the identity on this class
      const int64_t cnt = S.bh2_off[M + 1] - S.bh2_off[M];
      if (cnt > INT32_MAX) return fail(CVQ_EINVAL, "too many orbits in one class");
      const int64_t per = NTHREADS * std::max<int64_t>(1, std::llround(target / (w[M] * NTHREADS)));
      for (int64_t u0 = 0; u0 < cnt; u0 += per)
        pb.chunks.push_back(make_int4(M, (int)u0, (int)std::min(cnt, u0 + per), 0));
    }
    t.nchunks = (int)pb.chunks.size() - t.chunk_base;
  }
  return CVQ_OK;
}

static int set_pool(const cvq_sector* s, const cvq_op* ops, int K, int dc, cvq_pool** out);

// Index tables of the tiled gates (k_tile.cu): one per distinct gate
// structure (modes, move) of the pool's block generators.  Each region is one
// orbit class; its tiles hold G whole orbits each (every block of two or more
// members of those orbits), G = T / (members per orbit).  Synchronises.
static int build_tiles(cvq_pool* p, const PoolBuild& pb) {
  const SectorDev& S = p->sec->S;
  struct Plan {
    int type, i, j;
    std::vector<TileRegion> reg;
    std::vector<TileSub> sub;
    int64_t ntiles = 0, max_count = 0;
    size_t idx_off = 0, reg_off = 0, sub_off = 0;
  };
  std::vector<Plan> plans;
  std::map<std::array<int, 7>, int> where;
  const int slots = (S.dim >= TILE_LARGE_DIM) ? TILE_S_LARGE : 1;
  const int T = TILE_T * slots;
  std::vector<int> plan_of(p->K, -1);
  auto orbits = [&](const TypeDesc& t, int cls) -> int64_t {
    if (S.kind == CVQ_BH) return S.bh2_off[cls + 1] - S.bh2_off[cls];
    const int nm = t.single ? 1 : 2;
    if (S.L == nm) return cls == S.parity ? 1 : 0;
    int64_t items = 1;
    for (int r = 0; r < S.L - nm; ++r) items *= S.D;
    return items / 2;
  };
  for (int k = 0; k < p->K; ++k) {
    const TypeDesc& t = p->types[p->op_type[k]];
    if (t.diag) continue;
    const std::array<int, 7> key = {p->op_i[k], p->op_j[k], t.di, t.dj, t.single, t.nblocks, t.nu};
    auto it = where.find(key);
    if (it != where.end()) {
      plan_of[k] = it->second;
      continue;
    }
    Plan pl;
    pl.type = p->op_type[k];
    pl.i = p->op_i[k];
    pl.j = p->op_j[k];
    for (int cls = 0; cls < t.nclass; ++cls) {
      const int64_t cnt = orbits(t, cls);
      if (cnt <= 0) continue;
      if (cnt > INT32_MAX) return fail(CVQ_EINVAL, "too many orbits in one class for the tiled gates");
      TileRegion R;
      memset(&R, 0, sizeof R);
      R.sub0 = (int)pl.sub.size();
      int per_orbit = 0;
      for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
        const BlockDesc& bd = pb.blk[t.blk_base + bi];
        if (bd.size < 2) continue;  // zero generator: identity
        TileSub u;
        memset(&u, 0, sizeof u);
        u.b = bd.size;
        u.u_off = bd.u_off;
        u.f_off = bd.f_off;
        u.bi = bi;
        pl.sub.push_back(u);
        per_orbit += bd.size;
      }
      R.nsub = (int)pl.sub.size() - R.sub0;
      if (R.nsub == 0) continue;
      if (R.nsub > TILE_MAX_SUB || per_orbit > T)
        return fail(CVQ_EINVAL, "an orbit of %d members in %d blocks does not fit a tile", per_orbit, R.nsub);
      R.G = T / per_orbit;
      int off = 0;
      for (int c = R.sub0; c < R.sub0 + R.nsub; ++c) {
        pl.sub[c].off = off;
        off += pl.sub[c].b * R.G;
      }
      R.count = (int)cnt;
      R.cls = cls;
      R.tile0 = pl.ntiles;
      pl.ntiles += (cnt + R.G - 1) / R.G;
      pl.max_count = std::max(pl.max_count, cnt);
      pl.reg.push_back(R);
    }
    if (pl.sub.size() > 64) return fail(CVQ_EINVAL, "%zu block classes exceed the tiled gates' 64", pl.sub.size());
    if (pl.ntiles * T > (int64_t)INT32_MAX)  // the gate kernels address tables and stored slots with 32-bit offsets
      return fail(CVQ_EINVAL, "a gate table of %lld slots exceeds 2^31 - 1", (long long)(pl.ntiles * T));
    where[key] = (int)plans.size();
    plan_of[k] = (int)plans.size();
    plans.push_back(std::move(pl));
  }
  p->op_tiles.assign(p->K, TileMap{nullptr, nullptr, nullptr, 0, 0, 0, 0});
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t total = 0;
  for (auto& pl : plans) {
    pl.idx_off = total;
    total = a256(total + (size_t)pl.ntiles * T * sizeof(int));
    pl.reg_off = total;
    total = a256(total + pl.reg.size() * sizeof(TileRegion));
    pl.sub_off = total;
    total = a256(total + pl.sub.size() * sizeof(TileSub));
  }
  if (total == 0) return CVQ_OK;
  const size_t o_bad = total;  // count of member indices outside [0, dim) (must stay 0)
  total += 256;
  cudaError_t e = cudaMalloc(&p->tile_blob, total);
  if (e != cudaSuccess) return fail(CVQ_ENOMEM, "cudaMalloc(%zu) for the gate tables: %s", total, cudaGetErrorString(e));
  char* base = (char*)p->tile_blob;
  int* bad = (int*)(base + o_bad);
  if ((e = cudaMemset(bad, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "gate table build");
  for (auto& pl : plans) {
    int* idx = (int*)(base + pl.idx_off);
    TileRegion* reg = (TileRegion*)(base + pl.reg_off);
    TileSub* sub = (TileSub*)(base + pl.sub_off);
    if ((e = cudaMemset(idx, 0xFF, (size_t)pl.ntiles * T * sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(reg, pl.reg.data(), pl.reg.size() * sizeof(TileRegion), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sub, pl.sub.data(), pl.sub.size() * sizeof(TileSub), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = launch_tile_build(S, pl.i, pl.j, p->types[pl.type], p->P, reg, sub, (int)pl.reg.size(), pl.max_count,
                               slots, idx, bad, 0)) != cudaSuccess)
      return cuda_fail(e, "gate table build");
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "gate table build");
  int nbad = 0;
  if ((e = cudaMemcpy(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "gate table build");
  if (nbad) return fail(CVQ_EINVAL, "gate table build produced %d indices outside the sector", nbad);
  for (int k = 0; k < p->K; ++k) {
    if (plan_of[k] < 0) continue;
    const Plan& pl = plans[plan_of[k]];
    p->op_tiles[k] = TileMap{(const int*)(base + pl.idx_off), (const TileRegion*)(base + pl.reg_off),
                             (const TileSub*)(base + pl.sub_off), (int)pl.reg.size(), (int)pl.sub.size(), slots,
                             pl.ntiles};
  }
  return CVQ_OK;
}

extern "C" int cvq_set_pool(const cvq_sector* s, const cvq_op* ops, int K, cvq_pool** out) {
  return set_pool(s, ops, K, 0, out);
}

extern "C" int cvq_set_pool_projected(const cvq_sector* s, const cvq_op* ops, int K, int inner_cutoff,
                                      cvq_pool** out) {
  if (!s) return fail(CVQ_EINVAL, "null argument");
  if (s->S.kind != CVQ_BKC) return fail(CVQ_EINVAL, "projected gates apply to Kitaev-chain sectors (BH is not cut)");
  if (inner_cutoff < s->S.D || inner_cutoff > MAX_BEXT)
    return fail(CVQ_EINVAL, "inner cutoff %d outside [d = %d, %d]", inner_cutoff, s->S.D, MAX_BEXT);
  return set_pool(s, ops, K, inner_cutoff, out);
}

static int set_pool(const cvq_sector* s, const cvq_op* ops, int K, int dc, cvq_pool** out) {
  if (!s || !out || (K > 0 && !ops)) return fail(CVQ_EINVAL, "null argument");
  *out = nullptr;
  if (K < 0 || K > MAX_GATES) return fail(CVQ_EINVAL, "pool size %d outside [0, %d]", K, MAX_GATES);
  const SectorDev& S = s->S;
  cvq_pool* p = new (std::nothrow) cvq_pool;
  if (!p) return fail(CVQ_ENOMEM, "host allocation");
  p->sec = s;
  p->K = K;
  p->dc = dc;
  PoolBuild pb;
  std::map<std::pair<int, int>, int> seen;
  for (int k = 0; k < K; ++k) {
    const cvq_op& o = ops[k];
    const bool single = (o.type == CVQ_OP_SQ1 || o.type == CVQ_OP_KERR || o.type == CVQ_OP_NN1 || o.type == CVQ_OP_ROT);
    if (o.i < 0 || o.i >= S.L || (!single && (o.j < 0 || o.j >= S.L || o.j == o.i))) {
      delete p;
      return fail(CVQ_EINVAL, "pool element %d has bad modes (%d, %d)", k, o.i, o.j);
    }
    const bool diag = (o.type >= CVQ_OP_KERR);
    const auto key = std::make_pair(o.type, diag ? 0 : (o.phase & 3));
    auto it = seen.find(key);
    int ti;
    if (it == seen.end()) {
      TypeDesc t;
      const int rc = build_type(S, o.type, key.second, pb, t, dc);
      if (rc) { delete p; return rc; }
      ti = (int)p->types.size();
      p->types.push_back(t);
      seen[key] = ti;
    } else {
      ti = it->second;
    }
    p->op_type.push_back(ti);
    p->op_i.push_back(o.i);
    p->op_j.push_back(single ? -1 : o.j);
  }
  for (auto& t : p->types) p->ustride = std::max(p->ustride, t.nu);
  for (auto& b : pb.blk) p->blk_size.push_back(b.size);
  p->ustride = (p->ustride + 15) & ~15;
  // device tables: types, ops, blocks, members, F, V, lam in one allocation
  const size_t nT = p->types.size();
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_chunks = 0;
  const size_t o_types = al(o_chunks + pb.chunks.size() * sizeof(int4));
  const size_t o_ops = al(o_types + nT * sizeof(TypeDesc));
  const size_t o_blk = al(o_ops + (size_t)K * sizeof(GateArg));
  const size_t o_mem = al(o_blk + pb.blk.size() * sizeof(BlockDesc));
  const size_t o_F = al(o_mem + pb.mem.size() * sizeof(int2));
  const size_t o_V = al(o_F + pb.F.size() * sizeof(float2));
  const size_t o_lam = al(o_V + pb.V.size() * sizeof(double));
  const size_t total = al(o_lam + pb.lam.size() * sizeof(double)) + 256;
  cudaError_t e = cudaMalloc(&p->blob, total);
  if (e != cudaSuccess) { delete p; return fail(CVQ_ENOMEM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e)); }
  char* base = (char*)p->blob;
  p->P.chunks = (const int4*)(base + o_chunks);
  p->types_dev = (TypeDesc*)(base + o_types);
  p->ops_dev = (GateArg*)(base + o_ops);
  p->P.blk = (const BlockDesc*)(base + o_blk);
  p->P.mem = (const int2*)(base + o_mem);
  p->P.F = (const float2*)(base + o_F);
  p->P.V = (const double*)(base + o_V);
  p->P.lam = (const double*)(base + o_lam);
  std::vector<GateArg> ga(K);
  for (int k = 0; k < K; ++k) {
    memset(&ga[k], 0, sizeof(GateArg));
    ga[k].i = p->op_i[k];
    ga[k].j = p->op_j[k];
    ga[k].t = p->types[p->op_type[k]];
    ga[k].U = nullptr;
  }
  auto up = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    return n ? cudaMemcpy(base + off, src, n, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  if ((e = up(o_chunks, pb.chunks.data(), pb.chunks.size() * sizeof(int4))) != cudaSuccess ||
      (e = up(o_types, p->types.data(), nT * sizeof(TypeDesc))) != cudaSuccess ||
      (e = up(o_ops, ga.data(), (size_t)K * sizeof(GateArg))) != cudaSuccess ||
      (e = up(o_blk, pb.blk.data(), pb.blk.size() * sizeof(BlockDesc))) != cudaSuccess ||
      (e = up(o_mem, pb.mem.data(), pb.mem.size() * sizeof(int2))) != cudaSuccess ||
      (e = up(o_F, pb.F.data(), pb.F.size() * sizeof(float2))) != cudaSuccess ||
      (e = up(o_V, pb.V.data(), pb.V.size() * sizeof(double))) != cudaSuccess ||
      (e = up(o_lam, pb.lam.data(), pb.lam.size() * sizeof(double))) != cudaSuccess) {
    cudaFree(p->blob);
    delete p;
    return cuda_fail(e, "pool upload");
  }
  // Tiled gates need int32 sector indices; projected pools keep the orbit
  // kernels.  The tables are built from the pool tables uploaded above.
  if (dc == 0 && S.dim <= (int64_t)INT32_MAX) {
    int rc = build_tiles(p, pb);
    if (rc == CVQ_OK) {  // the device op table carries each operator's tiles (batched engine)
      for (int k = 0; k < K; ++k) ga[k].tm = p->op_tiles[k];
      e = up(o_ops, ga.data(), (size_t)K * sizeof(GateArg));
      if (e != cudaSuccess) rc = cuda_fail(e, "op table upload");
    }
    if (rc) {
      if (p->tile_blob) cudaFree(p->tile_blob);
      cudaFree(p->blob);
      delete p;
      return rc;
    }
  }
  *out = p;
  return CVQ_OK;
}

extern "C" void cvq_destroy_pool(cvq_pool* p) {
  if (!p) return;
  if (p->blob) cudaFree(p->blob);
  if (p->tile_blob) cudaFree(p->tile_blob);
  delete p;
}

// ------------------------------------------------------------------ workspace

struct Layout {
  size_t psi, lam, U, partial, z, total;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// psi and lambda (df states, 16 B per amplitude), per-call block unitaries
// (n x ustride df complex), reduction partials ((max(n, 5K) + 1) x NBLK: the
// screen keeps two rows per distinct shift, at most 2K of them, and one per
// diagonal function), and the screen's reduced shift sums (5K + 1).
static Layout layout(const cvq_sector* s, const cvq_pool* p, int n_max) {
  Layout l;
  const size_t dim = (size_t)s->S.dim;
  const int K = p ? p->K : 0;
  const int ust = p ? p->ustride : PHASE_TABLE;
  const int nred = std::max(std::max(n_max, 5 * K), 1) + 1;
  l.psi = 0;
  l.lam = al256(l.psi + dim * sizeof(cdf));
  l.U = al256(l.lam + dim * sizeof(cdf));
  l.partial = al256(l.U + (size_t)std::max(n_max, 0) * ust * sizeof(cdf));
  l.z = al256(l.partial + (size_t)nred * NBLK * sizeof(double));
  l.total = al256(l.z + (size_t)(5 * K + 1) * sizeof(double));
  return l;
}

extern "C" int cvq_workspace_bytes(const cvq_sector* s, const cvq_pool* p, int n_max, size_t* bytes) {
  if (!s || !bytes) return fail(CVQ_EINVAL, "null argument");
  if (n_max < 0 || n_max > MAX_GATES) return fail(CVQ_EINVAL, "n_max %d outside [0, %d]", n_max, MAX_GATES);
  *bytes = layout(s, p, n_max).total;
  return CVQ_OK;
}

static int check_ws(const cvq_sector* s, const cvq_pool* p, int n, void* ws, size_t wsb, Layout& l) {
  if (!ws) return fail(CVQ_EINVAL, "workspace is NULL");
  if ((uintptr_t)ws & 255) return fail(CVQ_EINVAL, "workspace not 256-byte aligned");
  l = layout(s, p, n);
  if (wsb < l.total) return fail(CVQ_EINVAL, "workspace of %zu bytes, %zu needed", wsb, l.total);
  return CVQ_OK;
}

// ------------------------------------------------------------------ costs

// Algorithmic bytes and flops of one application of pool element op: every
// amplitude read and written once; a complex multiply-add = 8 flops.  Block
// gates: b^2 complex MACs per block (forward); the reverse step applies U^dag
// to psi and lambda (2 b^2) and forms the tridiagonal A psi and its overlap
// with lambda (3 b - 2).  Diagonal gates: 1 (forward) or 3 (reverse) per amplitude.
struct OpCost {
  double fb, ff, ab, af;
  double amps;  // amplitudes the gate changes
  double af_stored;  // reverse step with psi read from the stored forward states (no U^dag psi)
};

static OpCost op_cost(const cvq_sector* s, const cvq_pool* p, int op) {
  const SectorDev& S = s->S;
  const TypeDesc& t = p->types[p->op_type[op]];
  OpCost c;
  const double dim = (double)S.dim;
  c.fb = 32.0 * dim;
  c.ab = 64.0 * dim;
  c.amps = dim;
  if (t.diag) {
    c.ff = 8.0 * dim;
    c.af = 24.0 * dim;
    c.af_stored = 16.0 * dim;
    return c;
  }
  // Blocks of one member have a zero generator: the gate is the identity there
  // and the kernels skip them, so they count neither bytes nor flops.
  double ff = 0.0, af = 0.0, afs = 0.0, amps = 0.0;
  for (int cls = 0; cls < t.nclass; ++cls) {
    double orbits;
    if (S.kind == CVQ_BH) {
      orbits = (double)(S.bh2_off[cls + 1] - S.bh2_off[cls]);
    } else {
      const int nm = t.single ? 1 : 2;
      double items = 1.0;
      for (int r = 0; r < S.L - nm; ++r) items *= S.D;
      orbits = (S.L == nm) ? (cls == S.parity ? 1.0 : 0.0) : items / 2.0;
    }
    double bf = 0.0, baf = 0.0, bafs = 0.0;
    for (int bi = t.class_off[cls]; bi < t.class_off[cls + 1]; ++bi) {
      const int b = p->blk_size[t.blk_base + bi];
      if (b < 2) continue;
      bf += 8.0 * b * b;
      baf += 8.0 * (2.0 * b * b + 3.0 * b - 2.0);
      bafs += 8.0 * (1.0 * b * b + 3.0 * b - 2.0);
      amps += orbits * b;
    }
    ff += orbits * bf;
    af += orbits * baf;
    afs += orbits * bafs;
  }
  c.fb = 32.0 * amps;
  c.ab = 64.0 * amps;
  c.amps = amps;
  c.ff = ff;
  c.af = af;
  c.af_stored = afs;
  return c;
}

extern "C" int cvq_op_cost(const cvq_sector* s, const cvq_pool* p, int op, double* fwd_bytes, double* fwd_flops,
                           double* adj_bytes, double* adj_flops) {
  if (!s || !p || p->sec != s) return fail(CVQ_EINVAL, "bad sector / pool");
  if (op < 0 || op >= p->K) return fail(CVQ_EINVAL, "op %d outside the pool", op);
  const OpCost c = op_cost(s, p, op);
  if (fwd_bytes) *fwd_bytes = c.fb;
  if (fwd_flops) *fwd_flops = c.ff;
  if (adj_bytes) *adj_bytes = c.ab;
  if (adj_flops) *adj_flops = c.af;
  return CVQ_OK;
}

// sigma = H psi: every amplitude read and written once; per amplitude the
// diagonal term (4 flops) and the energy term (4), and 4 flops per
// off-diagonal matrix element (real coefficient x complex amplitude).
static void apply_H_cost(const cvq_sector* s, double& bytes, double& flops) {
  const SectorDev& S = s->S;
  const double dim = (double)S.dim;
  bytes = 32.0 * dim;
  double offd = 0.0;
  for (int b = 0; b < S.nb; ++b) {
    // fraction of sector states where a move (+1, -1) (resp. (+1, +1), (-1, -1)) stays in range
    double fh, fp = 0.0;
    if (S.kind == CVQ_BH) {
      fh = (S.N >= 1) ? (double)s->tabs.G[S.L - 1][S.N - 1] / dim : 0.0;  // n_s >= 1: compositions of N - 1
    } else {
      const double q = (double)(S.D - 1) / S.D;
      fh = q * q;
      fp = q * q;
    }
    if (s->hop[b] != 0.0) offd += 2.0 * fh * dim;
    if (s->pair[b] != 0.0) offd += 2.0 * fp * dim;
  }
  flops = 8.0 * dim + 4.0 * offd;
}

// ------------------------------------------------------------------ calls

static int to_df(const cvq_sector* s, const cvq_c128* src, cdf* dst, cudaStream_t st) {
  ProfScope ps(KK_CONVERT, st, 32.0 * (double)s->S.dim, 0.0);
  CVQ_CUDA(launch_to_df(s->S.dim, (const double2*)src, dst, st), "to df");
  return CVQ_OK;
}

static int from_df(const cvq_sector* s, const cdf* src, cvq_c128* dst, cudaStream_t st) {
  ProfScope ps(KK_CONVERT, st, 32.0 * (double)s->S.dim, 0.0);
  CVQ_CUDA(launch_from_df(s->S.dim, src, (double2*)dst, st), "from df");
  return CVQ_OK;
}

static int run_apply_H(const cvq_sector* s, const cdf* psi, cdf* sigma, double* partial, cudaStream_t st) {
  double hb, hf;
  apply_H_cost(s, hb, hf);
  ProfScope ps(KK_APPLY_H, st, hb, hf);
  CVQ_CUDA(launch_apply_H(s->S, psi, sigma, partial, st), "apply_H");
  return CVQ_OK;
}

extern "C" int cvq_apply_H(const cvq_sector* s, const cvq_c128* psi, cvq_c128* sigma, double* energy_dev, void* ws,
                           size_t wsb, void* stream) {
  if (!s || !psi || !sigma) return fail(CVQ_EINVAL, "null argument");
  if ((const void*)psi == (const void*)sigma) return fail(CVQ_EINVAL, "psi and sigma must not alias");
  Layout l;
  if (int rc = check_ws(s, nullptr, 0, ws, wsb, l)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cdf* vpsi = (cdf*)((char*)ws + l.psi);
  cdf* vsig = (cdf*)((char*)ws + l.lam);
  double* partial = (double*)((char*)ws + l.partial);
  if (int rc = to_df(s, psi, vpsi, st)) return rc;
  if (int rc = run_apply_H(s, vpsi, vsig, energy_dev ? partial : nullptr, st)) return rc;
  if (int rc = from_df(s, vsig, sigma, st)) return rc;
  if (energy_dev) {
    ProfScope ps(KK_REDUCE, st, 8.0 * NBLK, NBLK);
    CVQ_CUDA(launch_reduce(partial, 1, NBLK, 1.0, energy_dev, st), "reduce");
  }
  return CVQ_OK;
}

// The screen of the pool indices in sub: its distinct ladder shifts
// (canonical: lower mode first) and diagonal functions, and per screened
// element the rows of Z it combines.
static int screen_plan(const cvq_pool* p, const SubsetArg& sub, ScreenArg& sa, ScreenMap& sm) {
  sa.nsh = sa.ndg = 0;
  sm.n = sub.n;
  std::map<std::array<int, 4>, int> shift_id, diag_id;
  auto shift = [&](int i, int di, int j, int dj) {
    if (j >= 0 && j < i) {
      std::swap(i, j);
      std::swap(di, dj);
    }
    if (j < 0) dj = 0;
    const std::array<int, 4> key{i, di, j, dj};
    auto it = shift_id.find(key);
    if (it != shift_id.end()) return it->second;
    sa.sh[sa.nsh] = make_int4(i, di, j, dj);
    shift_id[key] = sa.nsh;
    return sa.nsh++;
  };
  for (int k = 0; k < sub.n; ++k) {
    const int op = sub.idx[k];
    const TypeDesc& t = p->types[p->op_type[op]];
    const int i = p->op_i[op], j = t.single ? -1 : p->op_j[op];
    sm.cp[k] = make_double2(t.cp_re, t.cp_im);
    if (t.diag) {
      const std::array<int, 4> key{t.diag, i, t.diag == 4 ? j : -1, 0};
      auto it = diag_id.find(key);
      int d;
      if (it != diag_id.end()) {
        d = it->second;
      } else {
        if (sa.ndg == MAX_DIAGF) return fail(CVQ_EINVAL, "more than %d distinct diagonal generators", MAX_DIAGF);
        d = sa.ndg++;
        sa.dg[d] = make_int4(key[0], key[1], key[2], 0);
        diag_id[key] = d;
      }
      sm.e[k] = make_int4(1, d, 0, 0);
    } else {
      const int sp = shift(i, t.di, j, t.dj), sn = shift(i, -t.di, j, -t.dj);
      sm.e[k] = make_int4(0, sp, sn, 0);
    }
  }
  return CVQ_OK;
}

// Checked subset (NULL: the whole pool) into sub.
static int screen_subset(const cvq_pool* p, const int* subset, int n_subset, SubsetArg& sub) {
  if (subset) {
    if (n_subset < 0 || n_subset > p->K) return fail(CVQ_EINVAL, "n_subset %d outside [0, K=%d]", n_subset, p->K);
    for (int k = 0; k < n_subset; ++k) {
      if (subset[k] < 0 || subset[k] >= p->K) return fail(CVQ_EINVAL, "subset[%d] = %d outside the pool", k, subset[k]);
      sub.idx[k] = subset[k];
    }
    sub.n = n_subset;
  } else {
    sub.n = p->K;
    for (int k = 0; k < p->K; ++k) sub.idx[k] = k;
  }
  return CVQ_OK;
}

extern "C" int cvq_screen_pool(const cvq_sector* s, const cvq_pool* p, const cvq_c128* psi, const int* subset,
                               int n_subset, double* grad_dev, void* ws, size_t wsb, void* stream) {
  if (!s || !p || !psi || !grad_dev) return fail(CVQ_EINVAL, "null argument");
  if (p->sec != s) return fail(CVQ_EINVAL, "pool belongs to another sector");
  SubsetArg sub;
  if (int rc = screen_subset(p, subset, n_subset, sub)) return rc;
  static thread_local ScreenArg sa;
  static thread_local ScreenMap sm;
  if (int rc = screen_plan(p, sub, sa, sm)) return rc;
  Layout l;
  if (int rc = check_ws(s, p, 0, ws, wsb, l)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cdf* vpsi = (cdf*)((char*)ws + l.psi);
  cdf* vsig = (cdf*)((char*)ws + l.lam);
  double* partial = (double*)((char*)ws + l.partial);
  double* z = (double*)((char*)ws + l.z);
  if (int rc = to_df(s, psi, vpsi, st)) return rc;
  if (int rc = run_apply_H(s, vpsi, vsig, nullptr, st)) return rc;
  const int rows = 2 * sa.nsh + sa.ndg;
  {
    // per chunk of shifts one pass over sigma, and per shift one neighbour read of psi
    const double dim = (double)s->S.dim;
    const int chunks = (sa.nsh + SCREEN_CHUNK - 1) / SCREEN_CHUNK + (sa.ndg + SCREEN_CHUNK - 1) / SCREEN_CHUNK;
    const double fl = dim * (48.0 * sa.nsh + 8.0 * sa.ndg);
    ProfScope ps(KK_SCREEN, st, 16.0 * dim * (chunks + sa.nsh + (sa.ndg ? 1 : 0)), fl);
    CVQ_CUDA(launch_screen(s->S, sa, vpsi, vsig, partial, st), "screen");
  }
  {
    const int nb = screen_grid(s->S);
    ProfScope ps(KK_REDUCE, st, 8.0 * nb * rows, (double)nb * rows);
    CVQ_CUDA(launch_reduce(partial, rows, nb, 1.0, z, st), "reduce");
  }
  CVQ_CUDA(launch_screen_epilogue(sm, sa.nsh, z, grad_dev, st), "screen epilogue");
  return CVQ_OK;
}

static int prepare_gates(const cvq_sector*, const cvq_pool* p, const int* op_ids, const double* theta, int n, cdf* U,
                         cudaStream_t st, cdf* D = nullptr) {
  if (n < 0 || n > MAX_GATES) return fail(CVQ_EINVAL, "ansatz length %d outside [0, %d]", n, MAX_GATES);
  if (n > 0 && (!op_ids || !theta)) return fail(CVQ_EINVAL, "null op_ids / theta");
  BuildArgs a;
  a.n = n;
  a.maxblk = 0;
  a.D = D;
  a.ustride = p->ustride;
  for (int k = 0; k < n; ++k) {
    if (op_ids[k] < 0 || op_ids[k] >= p->K) return fail(CVQ_EINVAL, "op_ids[%d] = %d outside the pool", k, op_ids[k]);
    if (!std::isfinite(theta[k])) return fail(CVQ_EINVAL, "theta[%d] is not finite", k);
    a.type_of[k] = p->op_type[op_ids[k]];
    a.theta[k] = theta[k];
    if (!p->types[a.type_of[k]].diag) a.maxblk = std::max(a.maxblk, p->types[a.type_of[k]].nblocks);
  }
  ProfScope ps(KK_BUILD, st, 0.0, 0.0);
  CVQ_CUDA(launch_build_gates(a, p->types_dev, p->P, U, st), "build gates");
  return CVQ_OK;
}

static GateArg gate_arg(const cvq_pool* p, int op, const cdf* U) {
  GateArg g;
  g.i = p->op_i[op];
  g.j = p->op_j[op];
  g.t = p->types[p->op_type[op]];
  g.U = U;
  g.tm = p->op_tiles.empty() ? TileMap{nullptr, nullptr, nullptr, 0, 0, 0, 0} : p->op_tiles[op];
  return g;
}

// The ansatz as launch segments: each block gate alone, and maximal runs of
// consecutive diagonal gates (they commute) fused into one pass.
struct Seg {
  int k0, m;
  bool diag;
};

static std::vector<Seg> segments(const cvq_pool* p, const int* ids, int n) {
  std::vector<Seg> v;
  int k = 0;
  while (k < n) {
    if (!p->types[p->op_type[ids[k]]].diag) {
      v.push_back({k, 1, false});
      ++k;
      continue;
    }
    int m = 0, npair = 0;
    while (k + m < n && m < MAX_RUN) {
      const TypeDesc& t = p->types[p->op_type[ids[k + m]]];
      if (!t.diag) break;
      if (t.diag == 4) {
        if (npair == MAX_RUN_PAIRS) break;
        ++npair;
      }
      ++m;
    }
    v.push_back({k, m, true});
    k += m;
  }
  return v;
}

static float4 cdf_of(double re, double im) {
  const float2 a = split_df(re), b = split_df(im);
  return make_float4(a.x, a.y, b.x, b.y);
}

// Phase tables of a diagonal run: per mode and occupation
// exp(i sum_k theta_k f_k(n)) over the run's single-mode gates on that mode,
// and exp(i theta_p n_i n_j) for each cross-Kerr gate.  FP64 on the host.
static void diag_run_arg(const cvq_sector* s, const cvq_pool* p, const int* ids, const double* theta, const Seg& g,
                         DiagRunArg& a) {
  memset(&a, 0, sizeof a);
  a.m = g.m;
  double ang[LMAX][DMAX];
  memset(ang, 0, sizeof ang);
  const int D = s->S.D;
  for (int q = 0; q < g.m; ++q) {
    const int op = ids[g.k0 + q];
    const TypeDesc& t = p->types[p->op_type[op]];
    const double th = theta[g.k0 + q];
    a.diag[q] = t.diag;
    a.gi[q] = p->op_i[op];
    a.gj[q] = p->op_j[op];
    if (t.diag == 4) {
      const int pp = a.npair++;
      a.pi[pp] = p->op_i[op];
      a.pj[pp] = p->op_j[op];
      for (int u = 0; u < D; ++u)
        for (int v = 0; v < D; ++v) a.TP[pp][u * D + v] = cdf_of(std::cos(th * u * v), std::sin(th * u * v));
    } else {
      for (int nn = 0; nn < D; ++nn) {
        const int f = (t.diag == 1) ? nn * nn : (t.diag == 2) ? nn * (nn - 1) : nn;
        ang[a.gi[q]][nn] += th * (double)f;
      }
    }
  }
  for (int r = 0; r < LMAX; ++r)
    for (int nn = 0; nn < DMAX; ++nn) a.T[r][nn] = cdf_of(std::cos(ang[r][nn]), std::sin(ang[r][nn]));
  bool on[LMAX] = {};
  for (int q = 0; q < g.m; ++q)
    if (a.diag[q] != 4) on[a.gi[q]] = true;
  a.nact = 0;
  for (int r = 0; r < s->S.L; ++r)
    if (on[r]) a.act[a.nact++] = r;
}

// Checkpointed forward states: before the first segment whose first gate index
// reaches j * every (j = 1, 2, ...), psi is copied to slot j - 1 of buf.
struct Ckpt {
  cdf* buf = nullptr;
  int every = 0;
  std::vector<int> seg_of;  // segment index at which each slot was taken
};

// Stored forward states: for every segment of the ansatz, what the reverse
// sweep needs of psi at the segment's output, so that it does not recompute
// psi by undoing the gates: the output amplitudes of a tiled block gate in
// table-slot order (only those the gate changes; its gradient term and its
// U^dag lambda need no others), the whole state after a diagonal run or an
// untiled block gate.  Slot si starts at off[si] bytes into buf.
struct Stored {
  cdf* buf = nullptr;
  std::vector<size_t> off;
};

static size_t stored_seg_bytes(const cvq_sector* s, const cvq_pool* p, const int* ids, const Seg& g) {
  if (!g.diag && !p->op_tiles.empty() && p->op_tiles[ids[g.k0]].idx) {
    const TileMap& tm = p->op_tiles[ids[g.k0]];
    return al256((size_t)tm.ntiles * TILE_T * tm.slots * sizeof(cdf));
  }
  return al256((size_t)s->S.dim * sizeof(cdf));
}

// U_n ... U_1 applied in place to the df state psi.
static int forward_sweep(const cvq_sector* s, const cvq_pool* p, const int* ids, const double* theta, int n,
                         const cdf* U, cdf* psi, cudaStream_t st, Ckpt* ck = nullptr, const Stored* sv = nullptr) {
  const double dim = (double)s->S.dim;
  const std::vector<Seg> segs = segments(p, ids, n);
  for (size_t si = 0; si < segs.size(); ++si) {
    const Seg& g = segs[si];
    if (ck && si > 0 && g.k0 >= (int)(ck->seg_of.size() + 1) * ck->every) {
      CVQ_CUDA(cudaMemcpyAsync(ck->buf + ck->seg_of.size() * (size_t)s->S.dim, psi, sizeof(cdf) * (size_t)s->S.dim,
                               cudaMemcpyDeviceToDevice, st), "checkpoint copy");
      ck->seg_of.push_back((int)si);
    }
    if (g.diag) {
      DiagRunArg a;
      diag_run_arg(s, p, ids, theta, g, a);
      {
        ProfScope ps(KK_GATE_DIAG, st, 32.0 * dim, dim * (8.0 * s->S.L + 8.0 * a.npair));
        CVQ_CUDA(launch_diag_run(s->S, a, psi, psi, nullptr, nullptr, false, st), "diagonal run");
      }
      if (sv)
        CVQ_CUDA(cudaMemcpyAsync((char*)sv->buf + sv->off[si], psi, sizeof(cdf) * (size_t)s->S.dim,
                                 cudaMemcpyDeviceToDevice, st), "stored state copy");
    } else {
      const GateArg ga = gate_arg(p, ids[g.k0], U + (size_t)g.k0 * p->ustride);
      const OpCost c = op_cost(s, p, ids[g.k0]);
      if (sv && ga.tm.idx) {
        ProfScope ps(KK_GATE, st, c.fb + 16.0 * (double)c.amps, c.ff);
        CVQ_CUDA(launch_tile_gate(ga, p->P, psi, nullptr, nullptr, false, st, (cdf*)((char*)sv->buf + sv->off[si])),
                 "gate");
        continue;
      }
      {
        ProfScope ps(KK_GATE, st, c.fb, c.ff);
        CVQ_CUDA(launch_gate(s->S, ga, p->P, psi, psi, st), "gate");
      }
      if (sv)
        CVQ_CUDA(cudaMemcpyAsync((char*)sv->buf + sv->off[si], psi, sizeof(cdf) * (size_t)s->S.dim,
                                 cudaMemcpyDeviceToDevice, st), "stored state copy");
    }
  }
  return CVQ_OK;
}

extern "C" int cvq_apply_ansatz(const cvq_sector* s, const cvq_pool* p, const int* op_ids, const double* theta, int n,
                                const cvq_c128* psi0, cvq_c128* psi_out, void* ws, size_t wsb, void* stream) {
  if (!s || !p || !psi0 || !psi_out) return fail(CVQ_EINVAL, "null argument");
  if (p->dc) return fail(CVQ_EINVAL, "a projected pool needs cvq_apply_ansatz_projected");
  if (p->sec != s) return fail(CVQ_EINVAL, "pool belongs to another sector");
  Layout l;
  if (int rc = check_ws(s, p, n, ws, wsb, l)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cdf* psi = (cdf*)((char*)ws + l.psi);
  cdf* U = (cdf*)((char*)ws + l.U);
  if (int rc = prepare_gates(s, p, op_ids, theta, n, U, st)) return rc;
  if (int rc = to_df(s, psi0, psi, st)) return rc;
  if (int rc = forward_sweep(s, p, op_ids, theta, n, U, psi, st)) return rc;
  return from_df(s, psi, psi_out, st);
}

static int energy_and_grad(const cvq_sector* s, const cvq_pool* p, const int* op_ids, const double* theta, int n,
                           const cvq_c128* psi0, double* E_dev, double* grad_dev, void* ws, size_t wsb,
                           void* stream, Ckpt* ck, const Stored* sv = nullptr);

// Byte offsets of the stored-state slots of an ansatz (one per segment).
static int stored_layout(const cvq_sector* s, const cvq_pool* p, const int* op_ids, int n, std::vector<size_t>& off,
                         size_t& total) {
  if (n < 0 || n > MAX_GATES) return fail(CVQ_EINVAL, "ansatz length %d outside [0, %d]", n, MAX_GATES);
  if (n > 0 && !op_ids) return fail(CVQ_EINVAL, "null op_ids");
  for (int k = 0; k < n; ++k)
    if (op_ids[k] < 0 || op_ids[k] >= p->K) return fail(CVQ_EINVAL, "op_ids[%d] = %d outside the pool", k, op_ids[k]);
  off.clear();
  total = 0;
  for (const Seg& g : segments(p, op_ids, n)) {
    off.push_back(total);
    total += stored_seg_bytes(s, p, op_ids, g);
  }
  return CVQ_OK;
}

extern "C" int cvq_stored_states_bytes(const cvq_sector* s, const cvq_pool* p, const int* op_ids, int n,
                                       size_t* bytes) {
  if (!s || !p || !bytes) return fail(CVQ_EINVAL, "null argument");
  if (p->dc) return fail(CVQ_EINVAL, "a projected pool keeps its states with cvq_projected_states_bytes");
  std::vector<size_t> off;
  return stored_layout(s, p, op_ids, n, off, *bytes);
}

extern "C" int cvq_energy_and_grad_stored(const cvq_sector* s, const cvq_pool* p, const int* op_ids,
                                          const double* theta, int n, const cvq_c128* psi0, double* E_dev,
                                          double* grad_dev, void* states, size_t states_bytes, void* ws, size_t wsb,
                                          void* stream) {
  if (!s || !p) return fail(CVQ_EINVAL, "null argument");
  if (p->dc) return fail(CVQ_EINVAL, "a projected pool needs cvq_energy_and_grad_projected");
  Stored sv;
  size_t need = 0;
  if (int rc = stored_layout(s, p, op_ids, n, sv.off, need)) return rc;
  if (need > 0 && (!states || ((uintptr_t)states & 255)))
    return fail(CVQ_EINVAL, "stored-state buffer NULL or not 256-byte aligned");
  if (states_bytes < need) return fail(CVQ_EINVAL, "stored-state buffer of %zu bytes, %zu needed", states_bytes, need);
  sv.buf = (cdf*)states;
  return energy_and_grad(s, p, op_ids, theta, n, psi0, E_dev, grad_dev, ws, wsb, stream, nullptr, &sv);
}

extern "C" int cvq_energy_and_grad(const cvq_sector* s, const cvq_pool* p, const int* op_ids, const double* theta,
                                   int n, const cvq_c128* psi0, double* E_dev, double* grad_dev, void* ws, size_t wsb,
                                   void* stream) {
  return energy_and_grad(s, p, op_ids, theta, n, psi0, E_dev, grad_dev, ws, wsb, stream, nullptr);
}

extern "C" int cvq_checkpoint_bytes(const cvq_sector* s, int n, int every, size_t* bytes) {
  if (!s || !bytes) return fail(CVQ_EINVAL, "null argument");
  if (n < 0 || n > MAX_GATES || every < 1) return fail(CVQ_EINVAL, "need 0 <= n <= %d and every >= 1", MAX_GATES);
  *bytes = (size_t)(n > 0 ? (n - 1) / every : 0) * (size_t)s->S.dim * sizeof(cdf);
  return CVQ_OK;
}

extern "C" int cvq_energy_and_grad_ckpt(const cvq_sector* s, const cvq_pool* p, const int* op_ids,
                                        const double* theta, int n, const cvq_c128* psi0, double* E_dev,
                                        double* grad_dev, int every, void* ckpt, size_t ckpt_bytes, void* ws,
                                        size_t wsb, void* stream) {
  size_t need = 0;
  if (int rc = cvq_checkpoint_bytes(s, n, every, &need)) return rc;
  if (need > 0 && (!ckpt || ((uintptr_t)ckpt & 255))) return fail(CVQ_EINVAL, "checkpoint buffer NULL or not 256-byte aligned");
  if (ckpt_bytes < need) return fail(CVQ_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", ckpt_bytes, need);
  Ckpt ck;
  ck.buf = (cdf*)ckpt;
  ck.every = every;
  return energy_and_grad(s, p, op_ids, theta, n, psi0, E_dev, grad_dev, ws, wsb, stream, &ck);
}

static int energy_and_grad(const cvq_sector* s, const cvq_pool* p, const int* op_ids, const double* theta, int n,
                           const cvq_c128* psi0, double* E_dev, double* grad_dev, void* ws, size_t wsb,
                           void* stream, Ckpt* ck, const Stored* sv) {
  if (!s || !p || !psi0 || !E_dev || (n > 0 && !grad_dev)) return fail(CVQ_EINVAL, "null argument");
  if (p->dc) return fail(CVQ_EINVAL, "a projected pool needs cvq_energy_and_grad_projected");
  if (p->sec != s) return fail(CVQ_EINVAL, "pool belongs to another sector");
  Layout l;
  if (int rc = check_ws(s, p, n, ws, wsb, l)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cdf* psi = (cdf*)((char*)ws + l.psi);
  cdf* lam = (cdf*)((char*)ws + l.lam);
  cdf* U = (cdf*)((char*)ws + l.U);
  double* partial = (double*)((char*)ws + l.partial);
  if (int rc = prepare_gates(s, p, op_ids, theta, n, U, st)) return rc;
  if (int rc = to_df(s, psi0, psi, st)) return rc;
  if (int rc = forward_sweep(s, p, op_ids, theta, n, U, psi, st, ck, sv)) return rc;
  double* pE = partial + (size_t)n * NBLK;  // reduced with the gradient rows at the end
  if (int rc = run_apply_H(s, psi, lam, pE, st)) return rc;
  const std::vector<Seg> segs = segments(p, op_ids, n);
  const double dim = (double)s->S.dim;
  int slot = ck ? (int)ck->seg_of.size() - 1 : -1;
  for (int si = (int)segs.size() - 1; si >= 0; --si) {
    const Seg& g = segs[si];
    // stored output state of this segment (whole state, or a tiled gate's slots)
    cdf* sto = sv ? (cdf*)((char*)sv->buf + sv->off[si]) : nullptr;
    if (g.diag) {
      DiagRunArg a;
      diag_run_arg(s, p, op_ids, theta, g, a);
      cdf* pst = sto ? sto : psi;  // psi at the run's output
      // gradients of the gates past the reverse pass's accumulators, at the run's output state, before the reverse pass undoes the phases
      for (int q0 = diag_run_acc(g.m); q0 < g.m; q0 += DIAG_GRAD_ACC) {
        DiagGradArg ga;
        memset(&ga, 0, sizeof ga);
        ga.m = std::min(DIAG_GRAD_ACC, g.m - q0);
        for (int q = 0; q < ga.m; ++q) {
          ga.diag[q] = a.diag[q0 + q];
          ga.gi[q] = a.gi[q0 + q];
          ga.gj[q] = a.gj[q0 + q];
        }
        ProfScope ps(KK_ADJ_DIAG, st, 32.0 * dim, dim * (16.0 + 4.0 * ga.m));
        CVQ_CUDA(launch_diag_grad(s->S, ga, pst, lam, partial + (size_t)(g.k0 + q0) * NBLK, st), "diagonal-run gradients");
      }
      ProfScope ps(KK_ADJ_DIAG, st, sto ? 48.0 * dim : 64.0 * dim,
                   dim * (8.0 * s->S.L + 8.0 * a.npair + 24.0 + 4.0 * std::min(g.m, diag_run_acc(g.m))));
      CVQ_CUDA(launch_diag_run(s->S, a, pst, pst, lam, partial + (size_t)g.k0 * NBLK, true, st, sto != nullptr),
               "adjoint diagonal run");
    } else {
      const GateArg ga = gate_arg(p, op_ids[g.k0], U + (size_t)g.k0 * p->ustride);
      const OpCost c = op_cost(s, p, op_ids[g.k0]);
      if (sto && ga.tm.idx) {  // psi from the stored slots, lambda only
        ProfScope ps(KK_ADJ, st, 48.0 * c.amps, c.af_stored);
        CVQ_CUDA(launch_tile_gate_stored(ga, p->P, sto, lam, partial + (size_t)g.k0 * NBLK, st), "adjoint gate");
        continue;
      }
      if (sto)  // untiled gate: the stored state replaces the working one, which the gate then undoes
        CVQ_CUDA(cudaMemcpyAsync(psi, sto, sizeof(cdf) * (size_t)s->S.dim, cudaMemcpyDeviceToDevice, st),
                 "stored state restore");
      ProfScope ps(KK_ADJ, st, c.ab, c.af);
      CVQ_CUDA(launch_gate_adjoint(s->S, ga, p->P, psi, lam, partial + (size_t)g.k0 * NBLK, st), "adjoint gate");
    }
    if (slot >= 0 && ck->seg_of[slot] == si) {  // psi is now the state before segment si: restore the stored copy
      CVQ_CUDA(cudaMemcpyAsync(psi, ck->buf + (size_t)slot * (size_t)s->S.dim, sizeof(cdf) * (size_t)s->S.dim,
                               cudaMemcpyDeviceToDevice, st), "checkpoint restore");
      --slot;
    }
  }
  {
    ProfScope ps(KK_REDUCE, st, 8.0 * NBLK * (n + 1), (double)NBLK * (n + 1));
    CVQ_CUDA(launch_reduce_eg(partial, n, NBLK, E_dev, grad_dev, st), "reduce E and grad");
  }
  return CVQ_OK;
}

// ------------------------------------------------------------------ projected gates (Sec. V.A)

// Caller buffer of the projected sweep: one df state per segment boundary
// (nseg + 1), the theta derivatives of the block unitaries (n x ustride), and
// per segment the squared norm before renormalising plus one scratch dot.
struct ProjLayout {
  size_t slots, D, n2, r, total;
  int nseg;
};

static ProjLayout proj_layout(const cvq_sector* s, const cvq_pool* p, int nseg, int n) {
  ProjLayout l;
  l.nseg = nseg;
  const size_t st = al256((size_t)s->S.dim * sizeof(cdf));
  l.slots = 0;
  l.D = (size_t)(nseg + 1) * st;
  l.n2 = al256(l.D + (size_t)std::max(n, 1) * p->ustride * sizeof(cdf));
  l.r = al256(l.n2 + (size_t)std::max(nseg, 1) * sizeof(double));
  l.total = al256(l.r + sizeof(double));
  return l;
}

extern "C" int cvq_projected_states_bytes(const cvq_sector* s, const cvq_pool* p, const int* op_ids, int n,
                                          size_t* bytes) {
  if (!s || !p || !bytes || (n > 0 && !op_ids)) return fail(CVQ_EINVAL, "null argument");
  if (n < 0 || n > MAX_GATES) return fail(CVQ_EINVAL, "ansatz length %d outside [0, %d]", n, MAX_GATES);
  for (int k = 0; k < n; ++k)
    if (op_ids[k] < 0 || op_ids[k] >= p->K) return fail(CVQ_EINVAL, "op_ids[%d] = %d outside the pool", k, op_ids[k]);
  *bytes = proj_layout(s, p, (int)segments(p, op_ids, n).size(), n).total;
  return CVQ_OK;
}

// Forward projected sweep into the state slots; returns the segments.
static int proj_forward(const cvq_sector* s, const cvq_pool* p, const int* ids, const double* theta, int n,
                        const cvq_c128* psi0, char* sb, const ProjLayout& pl, const cdf* U, double* partial,
                        std::vector<Seg>& segs, cudaStream_t st) {
  const size_t stride = al256((size_t)s->S.dim * sizeof(cdf));
  auto slot = [&](int k) { return (cdf*)(sb + pl.slots + (size_t)k * stride); };
  double* n2 = (double*)(sb + pl.n2);
  const double dim = (double)s->S.dim;
  segs = segments(p, ids, n);
  if (int rc = to_df(s, psi0, slot(0), st)) return rc;
  for (size_t si = 0; si < segs.size(); ++si) {
    const Seg& g = segs[si];
    cdf* psi = slot((int)si + 1);
    CVQ_CUDA(cudaMemcpyAsync(psi, slot((int)si), sizeof(cdf) * (size_t)s->S.dim, cudaMemcpyDeviceToDevice, st),
             "copy state");
    if (g.diag) {
      DiagRunArg a;
      diag_run_arg(s, p, ids, theta, g, a);
      ProfScope ps(KK_GATE_DIAG, st, 32.0 * dim, dim * (8.0 * s->S.L + 8.0 * a.npair));
      CVQ_CUDA(launch_diag_run(s->S, a, psi, psi, nullptr, nullptr, false, st), "diagonal run");
    } else {
      const GateArg ga = gate_arg(p, ids[g.k0], U + (size_t)g.k0 * p->ustride);
      {
        const OpCost c = op_cost(s, p, ids[g.k0]);
        ProfScope ps(KK_GATE, st, c.fb, c.ff);
        CVQ_CUDA(launch_gate(s->S, ga, p->P, psi, psi, st), "projected gate");
      }
      CVQ_CUDA(launch_dot_re(s->S.dim, psi, psi, partial, st), "norm");
      CVQ_CUDA(launch_reduce(partial, 1, NBLK, 1.0, n2 + si, st), "reduce norm");
      CVQ_CUDA(launch_scale_inv_sqrt(s->S.dim, psi, n2 + si, st), "renormalise");
    }
  }
  return CVQ_OK;
}

static int proj_prepare(const cvq_sector* s, const cvq_pool* p, const int* op_ids, const double* theta, int n,
                        void* ws, size_t wsb, void* states, size_t states_bytes, Layout& l, ProjLayout& pl,
                        cudaStream_t st) {
  if (!p->dc) return fail(CVQ_EINVAL, "the pool was not built with cvq_set_pool_projected");
  if (p->sec != s) return fail(CVQ_EINVAL, "pool belongs to another sector");
  if (int rc = check_ws(s, p, n, ws, wsb, l)) return rc;
  size_t need = 0;
  if (int rc = cvq_projected_states_bytes(s, p, op_ids, n, &need)) return rc;
  if (!states || ((uintptr_t)states & 255)) return fail(CVQ_EINVAL, "state buffer NULL or not 256-byte aligned");
  if (states_bytes < need) return fail(CVQ_EINVAL, "state buffer of %zu bytes, %zu needed", states_bytes, need);
  pl = proj_layout(s, p, (int)segments(p, op_ids, n).size(), n);
  cdf* U = (cdf*)((char*)ws + l.U);
  return prepare_gates(s, p, op_ids, theta, n, U, st, (cdf*)((char*)states + pl.D));
}

extern "C" int cvq_apply_ansatz_projected(const cvq_sector* s, const cvq_pool* p, const int* op_ids,
                                          const double* theta, int n, const cvq_c128* psi0, cvq_c128* psi_out,
                                          void* states, size_t states_bytes, void* ws, size_t wsb, void* stream) {
  if (!s || !p || !psi0 || !psi_out) return fail(CVQ_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  Layout l;
  ProjLayout pl;
  if (int rc = proj_prepare(s, p, op_ids, theta, n, ws, wsb, states, states_bytes, l, pl, st)) return rc;
  std::vector<Seg> segs;
  if (int rc = proj_forward(s, p, op_ids, theta, n, psi0, (char*)states, pl, (cdf*)((char*)ws + l.U),
                            (double*)((char*)ws + l.partial), segs, st))
    return rc;
  const size_t stride = al256((size_t)s->S.dim * sizeof(cdf));
  return from_df(s, (const cdf*)((char*)states + (size_t)segs.size() * stride), psi_out, st);
}

extern "C" int cvq_energy_and_grad_projected(const cvq_sector* s, const cvq_pool* p, const int* op_ids,
                                             const double* theta, int n, const cvq_c128* psi0, double* E_dev,
                                             double* grad_dev, void* states, size_t states_bytes, void* ws,
                                             size_t wsb, void* stream) {
  if (!s || !p || !psi0 || !E_dev || (n > 0 && !grad_dev)) return fail(CVQ_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  Layout l;
  ProjLayout pl;
  if (int rc = proj_prepare(s, p, op_ids, theta, n, ws, wsb, states, states_bytes, l, pl, st)) return rc;
  char* sb = (char*)states;
  cdf* U = (cdf*)((char*)ws + l.U);
  const cdf* D = (const cdf*)(sb + pl.D);
  cdf* lam = (cdf*)((char*)ws + l.lam);
  double* partial = (double*)((char*)ws + l.partial);
  std::vector<Seg> segs;
  if (int rc = proj_forward(s, p, op_ids, theta, n, psi0, sb, pl, U, partial, segs, st)) return rc;
  const size_t stride = al256((size_t)s->S.dim * sizeof(cdf));
  auto slot = [&](int k) { return (cdf*)(sb + pl.slots + (size_t)k * stride); };
  double* n2 = (double*)(sb + pl.n2);
  double* rdot = (double*)(sb + pl.r);
  const int ns = (int)segs.size();
  double* pE = partial + (size_t)n * NBLK;
  if (int rc = run_apply_H(s, slot(ns), lam, pE, st)) return rc;
  CVQ_CUDA(launch_reduce(pE, 1, NBLK, 1.0, E_dev, st), "reduce E");
  const double dim = (double)s->S.dim;
  for (int si = ns - 1; si >= 0; --si) {
    const Seg& g = segs[si];
    if (g.diag) {  // unitary: the plain reverse step on psi_k (slot si + 1, consumed)
      DiagRunArg a;
      diag_run_arg(s, p, op_ids, theta, g, a);
      cdf* psi = slot(si + 1);
      for (int q0 = diag_run_acc(g.m); q0 < g.m; q0 += DIAG_GRAD_ACC) {
        DiagGradArg ga;
        memset(&ga, 0, sizeof ga);
        ga.m = std::min(DIAG_GRAD_ACC, g.m - q0);
        for (int q = 0; q < ga.m; ++q) {
          ga.diag[q] = a.diag[q0 + q];
          ga.gi[q] = a.gi[q0 + q];
          ga.gj[q] = a.gj[q0 + q];
        }
        CVQ_CUDA(launch_diag_grad(s->S, ga, psi, lam, partial + (size_t)(g.k0 + q0) * NBLK, st), "diagonal-run gradients");
      }
      ProfScope ps(KK_ADJ_DIAG, st, 64.0 * dim, dim * (8.0 * s->S.L + 8.0 * a.npair + 24.0));
      CVQ_CUDA(launch_diag_run(s->S, a, psi, psi, lam, partial + (size_t)g.k0 * NBLK, true, st), "adjoint diagonal run");
    } else {
      CVQ_CUDA(launch_dot_re(s->S.dim, slot(si + 1), lam, partial + (size_t)g.k0 * NBLK, st), "Re <psi_k|lambda>");
      CVQ_CUDA(launch_reduce(partial + (size_t)g.k0 * NBLK, 1, NBLK, 1.0, rdot, st), "reduce dot");
      const GateArg ga = gate_arg(p, op_ids[g.k0], U + (size_t)g.k0 * p->ustride);
      const OpCost c = op_cost(s, p, op_ids[g.k0]);
      ProfScope ps(KK_ADJ, st, c.ab + 16.0 * dim, c.af);
      CVQ_CUDA(launch_gate_proj_adj(s->S, ga, D + (size_t)g.k0 * p->ustride, p->P, slot(si), slot(si + 1), lam, rdot,
                                    n2 + si, partial + (size_t)g.k0 * NBLK, st),
               "projected reverse step");
    }
  }
  if (n > 0) CVQ_CUDA(launch_reduce(partial, n, NBLK, 2.0, grad_dev, st), "reduce grad");
  return CVQ_OK;
}

extern "C" int cvq_lanczos_step(const cvq_sector* s, const cvq_c128* v_prev, const cvq_c128* v, cvq_c128* w,
                                cvq_c128* v_next, const double* alpha_dev, const double* beta_prev_dev, double* beta_dev,
                                void* ws, size_t wsb, void* stream) {
  if (!s || !v_prev || !v || !w || !v_next || !alpha_dev || !beta_prev_dev || !beta_dev)
    return fail(CVQ_EINVAL, "null argument");
  if ((const void*)w == (const void*)v || (const void*)v_next == (const void*)v || (const void*)v_next == (const void*)w)
    return fail(CVQ_EINVAL, "w, v and v_next must be distinct");
  Layout l;
  if (int rc = check_ws(s, nullptr, 0, ws, wsb, l)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double* partial = (double*)((char*)ws + l.partial);
  const double dim = (double)s->S.dim;
  {
    ProfScope ps(KK_LANCZOS, st, 64.0 * dim, 16.0 * dim);
    CVQ_CUDA(launch_lanczos_update(s->S, (const double2*)v_prev, (const double2*)v, (double2*)w, alpha_dev,
                                   beta_prev_dev, partial, st), "lanczos update");
  }
  {
    ProfScope ps(KK_LANCZOS, st, 32.0 * dim, 2.0 * dim);
    CVQ_CUDA(launch_lanczos_scale(s->S, (const double2*)w, (double2*)v_next, partial, beta_dev, st), "lanczos scale");
  }
  return CVQ_OK;
}

// ------------------------------------------------------------------ internal accessors
// Used by translation units that add entry points of their own (k_noalloc.cu)
// without reaching into these structures directly.

namespace cvq {

const SectorDev* internal_sector(const cvq_sector* s) { return s ? &s->S : nullptr; }

const GateArg* internal_pool_ops(const cvq_pool* p, const cvq_sector** sec, int* K) {
  if (!p) return nullptr;
  if (sec) *sec = p->sec;
  if (K) *K = p->K;
  return p->ops_dev;
}

int internal_fail(int code, const char* msg) { return fail(code, "%s", msg); }

// The screen plan of a pool subset (NULL: the whole pool), for the batched screen.
int internal_screen_plan(const cvq_pool* p, const int* subset, int n_subset, ScreenArg* sa, ScreenMap* sm) {
  if (!p || !sa || !sm) return fail(CVQ_EINVAL, "null argument");
  SubsetArg sub;
  if (int rc = screen_subset(p, subset, n_subset, sub)) return rc;
  return screen_plan(p, sub, *sa, *sm);
}

// Host-side view of a pool for the batched engine.
int internal_pool_host(const cvq_pool* p, const cvq_sector** sec, const TypeDesc** types, int* ntypes,
                       const int** op_type, const int** op_i, const int** op_j, int* K, PoolDev* P, int* ustride,
                       const GateArg** ops_dev, const TileMap** op_tiles) {
  if (!p) return fail(CVQ_EINVAL, "null pool");
  *op_tiles = p->op_tiles.empty() ? nullptr : p->op_tiles.data();
  *sec = p->sec;
  *types = p->types.data();
  *ntypes = (int)p->types.size();
  *op_type = p->op_type.data();
  *op_i = p->op_i.data();
  *op_j = p->op_j.data();
  *K = p->K;
  *P = p->P;
  *ustride = p->ustride;
  *ops_dev = p->ops_dev;
  return CVQ_OK;
}

int internal_sector_device(const cvq_sector* s) { return s ? s->device : -1; }

// Event-pair timing for launches made outside this file (the scorer MLP).
int internal_prof_mlp_begin(cudaStream_t st, double bytes, double flops) {
  if (!g_prof_on) return -1;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  g_prof_bytes[KK_MLP] += bytes;
  g_prof_flops[KK_MLP] += flops;
  if (g_prof_count[KK_MLP]++ % g_prof_every != 0 || g_prof_n >= g_prof.size()) return -1;
  ++g_prof_timed[KK_MLP];
  const int idx = (int)g_prof_n++;
  g_prof[idx].kind = KK_MLP;
  g_prof[idx].bytes = bytes;
  g_prof[idx].flops = flops;
  cudaEventRecord(g_prof[idx].a, st);
  return idx;
}

void internal_prof_end(int idx, cudaStream_t st) {
  if (idx >= 0) cudaEventRecord(g_prof[idx].b, st);
}

}  // namespace cvq

// ------------------------------------------------------------------ features

extern "C" int cvq_features_workspace_bytes(const cvq_sector* s, int npairs, size_t* bytes) {
  if (!s || !bytes) return fail(CVQ_EINVAL, "null argument");
  if (npairs < 0 || npairs > 240) return fail(CVQ_EINVAL, "npairs %d outside [0, 240]", npairs);
  *bytes = al256((size_t)(2 * s->S.L + 2 * npairs) * NBLK * sizeof(double));
  return CVQ_OK;
}

extern "C" int cvq_features(const cvq_sector* s, const cvq_c128* psi, const int* pair_i, const int* pair_j,
                            int npairs, double* out_dev, void* ws, size_t wsb, void* stream) {
  if (!s || !psi || !out_dev || (npairs > 0 && (!pair_i || !pair_j))) return fail(CVQ_EINVAL, "null argument");
  size_t need = 0;
  if (int rc = cvq_features_workspace_bytes(s, npairs, &need)) return rc;
  if (!ws || ((uintptr_t)ws & 255)) return fail(CVQ_EINVAL, "workspace NULL or not 256-byte aligned");
  if (wsb < need) return fail(CVQ_EINVAL, "workspace of %zu bytes, %zu needed", wsb, need);
  for (int p = 0; p < npairs; ++p)
    if (pair_i[p] < 0 || pair_i[p] >= s->S.L || pair_j[p] < 0 || pair_j[p] >= s->S.L || pair_i[p] == pair_j[p])
      return fail(CVQ_EINVAL, "feature pair %d = (%d, %d) invalid", p, pair_i[p], pair_j[p]);
  cudaStream_t st = (cudaStream_t)stream;
  double* partial = (double*)ws;
  const int rows = 2 * s->S.L + 2 * npairs;
  {
    ProfScope ps(KK_FEATURES, st, 16.0 * (double)s->S.dim * (1 + npairs), (double)s->S.dim * (4.0 * s->S.L + 8.0 * npairs));
    CVQ_CUDA(launch_features(s->S, (const double2*)psi, pair_i, pair_j, npairs, partial, st), "features");
  }
  {
    ProfScope ps(KK_REDUCE, st, 8.0 * NBLK * rows, (double)NBLK * rows);
    CVQ_CUDA(launch_reduce(partial, rows, NBLK, 1.0, out_dev, st), "reduce features");
  }
  return CVQ_OK;
}
