// Host-only exhaustive check of the sector indexers and orbit enumerations of
// libcvq (compiled by tests/test_index_host.py with nvcc, run on the CPU).
//
// For small Bose-Hubbard and Kitaev-chain sectors it enumerates every tuple in
// lexicographic order (mode 0 most significant) and checks:
//   * rank/unrank round trips and suffix sums;
//   * the rank change of every number-conserving move (bh_move_delta) and of
//     the bond hops of the matvec (bh_hop_delta);
//   * for every two-mode and single-mode gate, that the orbits of the gate
//     kernels, with every member allowed by the orbit's class, cover each
//     sector index exactly once.
#include <cstdio>
#include <cstring>
#include <vector>

#include "cvq_internal.cuh"
#include "k_gate_impl.cuh"

using namespace cvq;

static int64_t binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

static int failures = 0;
#define CHECK(c, ...)                 \
  do {                                \
    if (!(c)) {                       \
      if (failures < 20) {            \
        printf("FAIL %s:%d ", __FILE__, __LINE__); \
        printf(__VA_ARGS__);          \
        printf("\n");                 \
      }                               \
      ++failures;                     \
    }                                 \
  } while (0)

static void enum_tuples(int L, int D, std::vector<std::vector<int>>& out, std::vector<int>& cur, int pos,
                        bool (*keep)(const std::vector<int>&, int), int arg) {
  if (pos == L) {
    if (keep(cur, arg)) out.push_back(cur);
    return;
  }
  for (int v = 0; v < D; ++v) {
    cur[pos] = v;
    enum_tuples(L, D, out, cur, pos + 1, keep, arg);
  }
}

static bool keep_sum(const std::vector<int>& t, int N) {
  int s = 0;
  for (int v : t) s += v;
  return s == N;
}
static bool keep_par(const std::vector<int>& t, int p) {
  int s = 0;
  for (int v : t) s += v;
  return (s & 1) == p;
}

static uint64_t pack(const std::vector<int>& t) {
  uint64_t w = 0;
  for (size_t r = 0; r < t.size(); ++r) w |= (uint64_t)t[r] << (4 * r);
  return w;
}

static void check_bh(int L, int N) {
  SectorDev S;
  memset(&S, 0, sizeof S);
  S.kind = CVQ_BH;
  S.L = L;
  S.N = N;
  S.D = N + 1;
  S.dim = binom(N + L - 1, L - 1);
  int64_t G[LMAX][DMAX + 1];
  for (int p = 0; p < LMAX; ++p)
    for (int R = 0; R <= DMAX; ++R) G[p][R] = binom(R + p, p);
  int64_t acc = 0;
  for (int M = 0; M <= N; ++M) {
    S.bh2_off[M] = acc;
    if (L >= 3) acc += binom(N - M + L - 3, L - 3);
    else if (L == 2) acc += (M == N) ? 1 : 0;
  }
  for (int M = N + 1; M <= MAX_CLASSES; ++M) S.bh2_off[M] = acc;
  std::vector<std::vector<int>> tup;
  std::vector<int> cur(L);
  enum_tuples(L, N + 1, tup, cur, 0, keep_sum, N);
  CHECK((int64_t)tup.size() == S.dim, "BH L=%d N=%d dim", L, N);
  for (int64_t x = 0; x < S.dim; ++x) {
    const uint64_t w = pack(tup[x]);
    CHECK(bh_rank(w, L, N, G) == x, "rank L=%d N=%d x=%lld", L, N, (long long)x);
    uint64_t wR = 0;
    CHECK(bh_unrank(x, L, N, G, &wR) == w, "unrank L=%d N=%d x=%lld", L, N, (long long)x);
    CHECK(wR == bh_suffix(w, L), "suffix L=%d N=%d", L, N);
    for (int r = 0; r < L; ++r)
      for (int s = 0; s < L; ++s) {
        if (r == s) continue;
        for (int dr = -2; dr <= 2; ++dr) {
          if (!dr) continue;
          std::vector<int> t = tup[x];
          t[r] += dr;
          t[s] -= dr;
          if (t[r] < 0 || t[s] < 0) continue;
          const int64_t y = bh_rank(pack(t), L, N, G);
          CHECK(x + bh_move_delta(w, wR, r, s, dr, L, G) == y, "move L=%d N=%d r=%d s=%d dr=%d", L, N, r, s, dr);
        }
      }
    // hops along the bonds (r, r+1) from the tables of the matvec
    for (int r = 0; r + 1 < L; ++r) {
      const int Q = occ_get(wR, r + 1);
      std::vector<int> t = tup[x];
      if (t[r + 1] >= 1) {
        t[r] += 1;
        t[r + 1] -= 1;
        CHECK(x + bh_hop_delta(G, L, N, r, Q) == bh_rank(pack(t), L, N, G), "hop L=%d N=%d r=%d", L, N, r);
      }
      t = tup[x];
      if (t[r] >= 1) {
        t[r] -= 1;
        t[r + 1] += 1;
        CHECK(x - bh_hop_delta(G, L, N, r, Q + 1) == bh_rank(pack(t), L, N, G), "reverse hop L=%d N=%d r=%d", L, N, r);
      }
    }
  }
  // lexicographic successor of compositions, and the nibble spread used by the gate kernels
  for (int Lc = 0; Lc <= L; ++Lc) {
    for (int R = 0; R <= N; ++R) {
      std::vector<std::vector<int>> c;
      std::vector<int> cc(Lc);
      if (Lc > 0) enum_tuples(Lc, N + 1, c, cc, 0, keep_sum, R);
      if (Lc == 0 && R != 0) continue;
      if (Lc == 0) c.push_back({});
      uint64_t w = bh_unrank<int64_t>(0, Lc, R, G);
      for (size_t k = 0; k < c.size(); ++k) {
        CHECK(w == pack(c[k]), "comp order Lc=%d R=%d k=%zu", Lc, R, k);
        const bool more = comp_next(w, Lc);
        CHECK(more == (k + 1 < c.size()), "comp_next end Lc=%d R=%d", Lc, R);
      }
    }
  }
  for (int lo = 0; lo < L; ++lo)
    for (int hi = lo + 1; hi < L; ++hi) {
      std::vector<int> o(L - 2);
      for (int k = 0; k < L - 2; ++k) o[k] = (k * 7 + 3) % (N + 1);
      std::vector<int> full;
      int k = 0;
      for (int r = 0; r < L; ++r) full.push_back((r == lo || r == hi) ? 0 : o[k++]);
      CHECK(spread2(pack(o), lo, hi) == pack(full), "spread2 L=%d lo=%d hi=%d", L, lo, hi);
    }
  // two-mode gate orbits: every index covered once
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      if (i == j || L < 2) continue;
      std::vector<int> seen(S.dim, 0);
      for (int64_t it = 0; it < S.bh2_off[N + 1]; ++it) {
        int M;
        BhIdx idx;
        idx.w0 = bh_orbit(S, G, i, j, it, M);
        idx.wR0 = bh_suffix(idx.w0, L);
        idx.r0 = bh_rank(idx.w0, L, N, G);
        idx.i = i;
        idx.j = j;
        idx.L = L;
        idx.G = G;
        for (int a = 0; a <= M; ++a) {
          const int64_t y = idx(make_int2(a, M - a));
          CHECK(y >= 0 && y < S.dim, "BH orbit index out of range");
          if (y >= 0 && y < S.dim) seen[y]++;
        }
      }
      for (int64_t x = 0; x < S.dim; ++x) CHECK(seen[x] == 1, "BH orbit cover L=%d N=%d i=%d j=%d x=%lld", L, N, i, j,
                                                 (long long)x);
    }
}

// n / q by multiply-high against plain division: every divisor of a sector
// (1..16), the ends of the range, and a pseudo-random sweep of [0, 2^31).
static void check_div() {
  for (uint32_t q = 1; q <= 16; ++q) {
    uint32_t m;
    int sh;
    div_magic(q, &m, &sh);
    const uint32_t edge[] = {0u, 1u, q - 1, q, q + 1, 0x7fffffffu, 0x7ffffffeu, 0x40000000u, 0x3fffffffu};
    for (uint32_t n : edge) CHECK(div_by_mul(n, m, sh) == n / q, "div q=%u n=%u", q, n);
    uint64_t z = 0x9E3779B97F4A7C15ull * q;
    for (int k = 0; k < 200000; ++k) {
      z ^= z << 13;
      z ^= z >> 7;
      z ^= z << 17;
      const uint32_t n = (uint32_t)(z & 0x7fffffffu);
      CHECK(div_by_mul(n, m, sh) == n / q, "div q=%u n=%u", q, n);
    }
  }
}

static void check_bkc(int L, int d, int parity) {
  SectorDev S;
  memset(&S, 0, sizeof S);
  S.kind = CVQ_BKC;
  S.L = L;
  S.D = d;
  S.half = d / 2;
  S.parity = parity;
  int64_t full = 1;
  for (int r = L - 1; r >= 0; --r) {
    S.stride[r] = full;
    full *= d;
  }
  S.dim = full / 2;
  std::vector<std::vector<int>> tup;
  std::vector<int> cur(L);
  enum_tuples(L, d, tup, cur, 0, keep_par, parity);
  CHECK((int64_t)tup.size() == S.dim, "BKC dim");
  // the 64-bit division path, then the multiply-high path the kernels take
  for (int64_t x = 0; x < S.dim; ++x) CHECK(bkc_unrank(x, S) == pack(tup[x]), "bkc unrank L=%d d=%d", L, d);
  set_bkc_div(S);
  CHECK(S.div32 == 1, "BKC small sector takes the 32-bit division");
  for (int64_t x = 0; x < S.dim; ++x)
    CHECK(bkc_unrank(x, S) == pack(tup[x]), "bkc unrank (multiply-high) L=%d d=%d", L, d);
  // gate orbits (two-mode and single-mode): every index covered once
  for (int i = 0; i < L; ++i)
    for (int j = -1; j < L; ++j) {
      if (i == j) continue;
      const int nm = (j >= 0) ? 2 : 1;
      std::vector<int> seen(S.dim, 0);
      const int64_t items = bkc_items(S, nm);
      for (int64_t it = 0; it < items; ++it) {
        int q;
        BkcIdx idx;
        bkc_orbit(S, i, j, it, items, idx.f0, q);
        idx.si = S.stride[i];
        idx.sj = (j >= 0) ? S.stride[j] : 0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < (j >= 0 ? d : 1); ++b) {
            if (((a + b) & 1) != q) continue;
            const int64_t y = idx(make_int2(a, b));
            CHECK(y >= 0 && y < S.dim, "BKC orbit index out of range");
            if (y < 0 || y >= S.dim) continue;
            seen[y]++;
            std::vector<int> t = tup[y];
            CHECK(t[i] == a && (j < 0 || t[j] == b), "BKC member occupation");
          }
      }
      for (int64_t x = 0; x < S.dim; ++x) CHECK(seen[x] == 1, "BKC orbit cover L=%d d=%d i=%d j=%d", L, d, i, j);
    }
}

// Runs of the warp walk: odd, at most WALK_RMAX, and enough passes of
// 32 R indices per warp to cover the range.
static void check_walk() {
  const int64_t nws[] = {1, 7, 4864};
  for (int64_t nw : nws)
    for (int64_t n = 1; n < 3000000; n = n * 3 + 1) {
      const int R = walk_r(n, nw);
      CHECK(R >= 1 && R <= WALK_RMAX && (R & 1), "walk_r(%lld, %lld) = %d", (long long)n, (long long)nw, R);
      const int64_t per = (n + 32 * nw - 1) / (32 * nw);
      CHECK(R * ((per + R - 1) / R) >= per, "walk cover");
    }
}

int main() {
  const int bh[][2] = {{2, 3}, {3, 1}, {3, 4}, {4, 4}, {5, 3}, {5, 6}, {6, 5}};
  for (auto& c : bh) check_bh(c[0], c[1]);
  const int bkc[][3] = {{1, 4, 0}, {1, 6, 1}, {2, 2, 0}, {2, 4, 1}, {3, 4, 0}, {3, 6, 1}, {4, 4, 0}, {4, 2, 1}};
  for (auto& c : bkc) check_bkc(c[0], c[1], c[2]);
  check_div();
  check_walk();
  printf("%s (%d failures)\n", failures ? "FAILED" : "OK", failures);
  return failures ? 1 : 0;
}
