/*
 * cvq_oracle.c -- plain, slow FP64 CPU oracle for the CV-ADAPT-VQE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code, header, table or helper with the CUDA library in
 * paper_2606_05297_gb300/csrc, and the product path never calls it.
 *
 * What it computes, with the passage each step follows (arXiv 2606.05297):
 *
 *   - Fock truncation and ladder action (Sec. II.A):
 *       a|n> = sqrt(n)|n-1>,  a^dag|n> = sqrt(n+1)|n+1>,  a^dag|D-1> = 0 (truncated).
 *   - Symmetry sectors: fixed total boson number N for Bose-Hubbard
 *     (Sec. III.A, [N_tot, H_BH] = 0) and fixed global parity for the bosonic
 *     Kitaev chain (Sec. III.B, P = (-1)^N_tot).  The sector is enumerated by
 *     brute force in lexicographic order (mode 0 most significant) and looked
 *     up by binary search over the sorted tuple keys -- deliberately not the
 *     combinatorial rank the GPU path uses.
 *   - Every operator (Hamiltonian terms, pool generators A_r) is a sum of
 *     coefficient x ladder-operator strings, applied literally by the ladder
 *     rules above.  The strings themselves are built in oracle/operators.py
 *     from Eqs. (BoseHubbard), (BosonicKitaevChain), (BosonicKitaevChain_Kerr)
 *     and the gate definitions of Sec. II.B.
 *   - exp(theta A) psi (Sec. IV.B, O_r = exp(theta_r A_r)): Taylor series on the
 *     vector with scaling -- never the block structure the GPU path exploits.
 *   - Energy E = <psi|H|psi> (Sec. IV.A/B).
 *   - Pool gradient, Eq. (grad): g_r = <psi|[H, A_r]|psi>, evaluated literally
 *     as <psi|H A_r psi> - <psi|A_r H psi>.
 *   - Ansatz gradient dE/dtheta_k for E = <psi_n|H|psi_n>,
 *     psi_k = exp(theta_k A_k) psi_{k-1}: all forward states are stored, then
 *     dE/dtheta_k = 2 Re <lambda_k| A_k psi_k>,
 *     lambda_n = H psi_n,  lambda_{k-1} = exp(-theta_k A_k) lambda_k.
 *
 * Complex numbers are C99 double complex (interleaved re, im), which matches
 * numpy complex128 memory.
 */
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ sector */

typedef struct {
    int kind;      /* 0: Bose-Hubbard fixed N, 1: Kitaev chain fixed parity */
    int L;         /* number of modes (sites) */
    int N;         /* BH: total boson number */
    int D;         /* local Fock cutoff: N+1 for BH (exact, Sec. III.A), d for BKC */
    int parity;    /* BKC: 0 even, 1 odd */
    int64_t dim;
    uint64_t *key; /* key = sum_r n_r D^(L-1-r); increasing = lexicographic order */
    int64_t cap;
} orc_sector;

static int tuple_in_sector(const orc_sector *s, const int *n) {
    int tot = 0;
    for (int r = 0; r < s->L; ++r) {
        if (n[r] < 0 || n[r] >= s->D) return 0;
        tot += n[r];
    }
    if (s->kind == 0) return tot == s->N;
    return (tot & 1) == s->parity;
}

static uint64_t tuple_key(const orc_sector *s, const int *n) {
    uint64_t k = 0;
    for (int r = 0; r < s->L; ++r) k = k * (uint64_t)s->D + (uint64_t)n[r];
    return k;
}

static void key_tuple(const orc_sector *s, uint64_t k, int *n) {
    for (int r = s->L - 1; r >= 0; --r) {
        n[r] = (int)(k % (uint64_t)s->D);
        k /= (uint64_t)s->D;
    }
}

/* Depth-first enumeration over modes 0..L-1 with values 0..D-1 in increasing
 * order, so tuples come out in lexicographic order.  The only pruning is the
 * BH running-sum bound (partial sum may not exceed N). */
static int enum_rec(orc_sector *s, int *n, int pos, int partial) {
    if (pos == s->L) {
        if (!tuple_in_sector(s, n)) return 0;
        if (s->dim == s->cap) {
            int64_t nc = s->cap ? 2 * s->cap : 1024;
            uint64_t *nk = (uint64_t *)realloc(s->key, (size_t)nc * sizeof(uint64_t));
            if (!nk) return -1;
            s->key = nk;
            s->cap = nc;
        }
        s->key[s->dim++] = tuple_key(s, n);
        return 0;
    }
    for (int v = 0; v < s->D; ++v) {
        if (s->kind == 0 && partial + v > s->N) break;
        n[pos] = v;
        if (enum_rec(s, n, pos + 1, partial + v)) return -1;
    }
    return 0;
}

int orc_sector_new(int kind, int L, int N, int d, int parity, void **out, int64_t *dim) {
    if (L < 1 || L > 24) return 1;
    orc_sector *s = (orc_sector *)calloc(1, sizeof(orc_sector));
    if (!s) return 2;
    s->kind = kind;
    s->L = L;
    s->N = N;
    s->D = (kind == 0) ? N + 1 : d;
    s->parity = parity & 1;
    if (s->D < 1 || (kind == 0 && N < 0)) { free(s); return 1; }
    /* keys must fit in 64 bits: D^L < 2^63 */
    double bits = (double)L * log2((double)(s->D > 1 ? s->D : 2));
    if (bits > 62.5) { free(s); return 1; }
    int n[32];
    if (enum_rec(s, n, 0, 0)) { free(s->key); free(s); return 2; }
    *out = s;
    *dim = s->dim;
    return 0;
}

void orc_sector_free(void *h) {
    orc_sector *s = (orc_sector *)h;
    if (!s) return;
    free(s->key);
    free(s);
}

/* Index of tuple n in the sector, or -1 if it is not a member. */
static int64_t sector_find(const orc_sector *s, const int *n) {
    if (!tuple_in_sector(s, n)) return -1;
    uint64_t k = tuple_key(s, n);
    int64_t lo = 0, hi = s->dim - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (s->key[mid] == k) return mid;
        if (s->key[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int64_t orc_sector_index(void *h, const int *n) { return sector_find((orc_sector *)h, n); }

void orc_sector_tuples(void *h, int *out) {
    orc_sector *s = (orc_sector *)h;
    for (int64_t x = 0; x < s->dim; ++x) key_tuple(s, s->key[x], out + x * s->L);
}

/* ---------------------------------------------------------------- operators */

/* One ladder string c * o_0 o_1 ... o_{m-1}, written as in the paper: the
 * rightmost factor acts first.  dag = 1 is a^dag, dag = 0 is a. */
#define ORC_MAXF 4
typedef struct {
    cplx c;
    int m;
    int mode[ORC_MAXF];
    int dag[ORC_MAXF];
} orc_string;

typedef struct {
    int ns;
    orc_string *s;
} orc_op;

/* coef: 2*ns doubles (re, im); fac: ns * ORC_MAXF * 2 ints (mode, dag), mode < 0 = unused. */
int orc_op_new(int ns, const double *coef, const int *fac, void **out) {
    orc_op *o = (orc_op *)calloc(1, sizeof(orc_op));
    if (!o) return 2;
    o->ns = ns;
    o->s = (orc_string *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(orc_string));
    if (!o->s) { free(o); return 2; }
    for (int t = 0; t < ns; ++t) {
        o->s[t].c = coef[2 * t] + I * coef[2 * t + 1];
        int m = 0;
        for (int f = 0; f < ORC_MAXF; ++f) {
            int mode = fac[(t * ORC_MAXF + f) * 2], dag = fac[(t * ORC_MAXF + f) * 2 + 1];
            if (mode < 0) continue;
            o->s[t].mode[m] = mode;
            o->s[t].dag[m] = dag;
            ++m;
        }
        o->s[t].m = m;
    }
    *out = o;
    return 0;
}

void orc_op_free(void *h) {
    orc_op *o = (orc_op *)h;
    if (!o) return;
    free(o->s);
    free(o);
}

/* Apply one ladder string to the basis ket |n> in place.  Returns the real
 * factor, or 0 when the ket is annihilated (a|0> = 0, truncated a^dag|D-1> = 0). */
static double string_on_ket(const orc_sector *s, const orc_string *st, int *n) {
    double f = 1.0;
    for (int q = st->m - 1; q >= 0; --q) {
        int r = st->mode[q];
        if (st->dag[q]) {
            if (n[r] + 1 >= s->D) return 0.0;
            f *= sqrt((double)(n[r] + 1));
            n[r] += 1;
        } else {
            if (n[r] == 0) return 0.0;
            f *= sqrt((double)n[r]);
            n[r] -= 1;
        }
    }
    return f;
}

/* out = O in, by applying every string to every basis ket (scatter form).
 * Strings are taken one after another; for one string the map |x> -> |y> is
 * a fixed shift of the occupations, so distinct kets never meet in one y and
 * the kets of a string can be spread over OpenMP threads without a race.
 * Each out[y] thus sums its terms in string order.  Returns 3 if some string
 * maps a sector state out of the sector (the operator does not respect the
 * symmetry). */
#define ORC_PAR_MIN 32768  /* smaller sectors run on one thread */
int orc_apply(void *sh, void *oh, const cplx *in, cplx *out) {
    const orc_sector *s = (const orc_sector *)sh;
    const orc_op *o = (const orc_op *)oh;
    int err = 0;
    memset(out, 0, (size_t)s->dim * sizeof(cplx));
    for (int t = 0; t < o->ns; ++t) {
#pragma omp parallel for schedule(static) if (s->dim >= ORC_PAR_MIN)
        for (int64_t x = 0; x < s->dim; ++x) {
            int n[32];
            if (in[x] == 0.0) continue;
            key_tuple(s, s->key[x], n);
            double f = string_on_ket(s, &o->s[t], n);
            if (f == 0.0) continue;
            int64_t y = sector_find(s, n);
            if (y < 0) {
#pragma omp atomic write
                err = 3;
                continue;
            }
            out[y] += o->s[t].c * f * in[x];
        }
        if (err) return err;
    }
    return 0;
}

/* Selected rows of O in: out[i] = (O in)[rows[i]].  For a ladder string T the
 * matrix element <y|T|x> is the real factor of T^dag|y> = f|x>, so each row is
 * a gather through the adjoint string (reversed order, dagger flipped). */
int orc_apply_rows(void *sh, void *oh, const cplx *in, const int64_t *rows, int64_t nrows, cplx *out) {
    const orc_sector *s = (const orc_sector *)sh;
    const orc_op *o = (const orc_op *)oh;
    int err = 0;
#pragma omp parallel for schedule(static) if (nrows >= ORC_PAR_MIN)
    for (int64_t i = 0; i < nrows; ++i) {
        int n[32];
        cplx acc = 0.0;
        for (int t = 0; t < o->ns; ++t) {
            const orc_string *st = &o->s[t];
            orc_string adj;
            adj.m = st->m;
            adj.c = conj(st->c);
            for (int q = 0; q < st->m; ++q) {
                adj.mode[q] = st->mode[st->m - 1 - q];
                adj.dag[q] = !st->dag[st->m - 1 - q];
            }
            key_tuple(s, s->key[rows[i]], n);
            double f = string_on_ket(s, &adj, n);
            if (f == 0.0) continue;
            int64_t x = sector_find(s, n);
            if (x < 0) {
#pragma omp atomic write
                err = 3;
                break;
            }
            acc += st->c * f * in[x];
        }
        out[i] = acc;
    }
    return err;
}

/* Upper bound on ||O||_2 for anti-Hermitian or Hermitian O: the largest
 * column sum of |O| (for such O the 1- and inf-norms agree and bound the
 * 2-norm). */
double orc_norm_bound(void *sh, void *oh) {
    const orc_sector *s = (const orc_sector *)sh;
    const orc_op *o = (const orc_op *)oh;
    double best = 0.0;
#pragma omp parallel for schedule(static) reduction(max : best) if (s->dim >= ORC_PAR_MIN)
    for (int64_t x = 0; x < s->dim; ++x) {
        int n[32];
        double col = 0.0;
        for (int t = 0; t < o->ns; ++t) {
            key_tuple(s, s->key[x], n);
            double f = string_on_ket(s, &o->s[t], n);
            col += cabs(o->s[t].c) * f;
        }
        if (col > best) best = col;
    }
    return best;
}

static double vec_norm(const cplx *v, int64_t dim) {
    double a = 0.0;
    for (int64_t x = 0; x < dim; ++x) a += creal(v[x]) * creal(v[x]) + cimag(v[x]) * cimag(v[x]);
    return sqrt(a);
}

static cplx vec_dot(const cplx *a, const cplx *b, int64_t dim) { /* <a|b> */
    cplx acc = 0.0;
    for (int64_t x = 0; x < dim; ++x) acc += conj(a[x]) * b[x];
    return acc;
}

/* out = exp(theta A) in.  Taylor series sum_k (h A)^k / k! applied to the
 * vector, in s sub-steps of h = theta / s with |h| * bound <= 1/2; each
 * sub-step is summed until the term norm drops below 1e-18 * ||v||.
 * in and out may alias. */
int orc_expm_apply(void *sh, void *oh, double theta, const cplx *in, cplx *out) {
    const orc_sector *s = (const orc_sector *)sh;
    int64_t dim = s->dim;
    double bound = orc_norm_bound(sh, oh);
    int steps = (int)ceil(fabs(theta) * bound / 0.5);
    if (steps < 1) steps = 1;
    double h = theta / steps;
    cplx *v = (cplx *)malloc((size_t)dim * sizeof(cplx));
    cplx *term = (cplx *)malloc((size_t)dim * sizeof(cplx));
    cplx *tmp = (cplx *)malloc((size_t)dim * sizeof(cplx));
    if (!v || !term || !tmp) { free(v); free(term); free(tmp); return 2; }
    memcpy(v, in, (size_t)dim * sizeof(cplx));
    for (int st = 0; st < steps; ++st) {
        memcpy(term, v, (size_t)dim * sizeof(cplx));
        double vn = vec_norm(v, dim);
        for (int k = 1; k <= 200; ++k) {
            int rc = orc_apply(sh, oh, term, tmp);
            if (rc) { free(v); free(term); free(tmp); return rc; }
            double tn = 0.0;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
            for (int64_t x = 0; x < dim; ++x) {
                term[x] = tmp[x] * (h / k);
                v[x] += term[x];
            }
            tn = vec_norm(term, dim);
            if (tn <= 1e-18 * (vn > 0 ? vn : 1.0)) break;
        }
    }
    memcpy(out, v, (size_t)dim * sizeof(cplx));
    free(v); free(term); free(tmp);
    return 0;
}

/* E = Re <psi|H|psi>, and <psi|psi>. */
int orc_energy(void *sh, void *hh, const cplx *psi, double *E, double *norm2) {
    const orc_sector *s = (const orc_sector *)sh;
    cplx *hp = (cplx *)malloc((size_t)s->dim * sizeof(cplx));
    if (!hp) return 2;
    int rc = orc_apply(sh, hh, psi, hp);
    if (!rc) {
        *E = creal(vec_dot(psi, hp, s->dim));
        if (norm2) *norm2 = creal(vec_dot(psi, psi, s->dim));
    }
    free(hp);
    return rc;
}

/* Eq. (grad): g_r = <psi|[H, A_r]|psi> = <psi|H A_r psi> - <psi|A_r H psi>.
 * gim receives the imaginary parts (zero up to rounding for anti-Hermitian
 * A_r and Hermitian H), for checking. */
int orc_screen(void *sh, void *hh, int K, void **ops, const cplx *psi, double *g, double *gim) {
    const orc_sector *s = (const orc_sector *)sh;
    int64_t dim = s->dim;
    cplx *hpsi = (cplx *)malloc((size_t)dim * sizeof(cplx));
    if (!hpsi) return 2;
    int rc = orc_apply(sh, hh, psi, hpsi);
    if (rc) { free(hpsi); return rc; }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        cplx *apsi = (cplx *)malloc((size_t)dim * sizeof(cplx));
        cplx *t = (cplx *)malloc((size_t)dim * sizeof(cplx));
        if (!apsi || !t) { err = 2; free(apsi); free(t); continue; }
        int r1 = orc_apply(sh, ops[k], psi, apsi);   /* A psi */
        int r2 = orc_apply(sh, hh, apsi, t);         /* H A psi */
        cplx first = vec_dot(psi, t, dim);
        int r3 = orc_apply(sh, ops[k], hpsi, t);     /* A H psi */
        cplx second = vec_dot(psi, t, dim);
        if (r1 || r2 || r3) err = 3;
        cplx gk = first - second;
        g[k] = creal(gk);
        if (gim) gim[k] = cimag(gk);
        free(apsi);
        free(t);
    }
    free(hpsi);
    return err;
}

/* psi_out = U_n ... U_1 psi0,  U_k = exp(theta_k A_k). */
int orc_apply_ansatz(void *sh, int n, void **ops, const double *theta, const cplx *psi0, cplx *psi_out) {
    const orc_sector *s = (const orc_sector *)sh;
    memcpy(psi_out, psi0, (size_t)s->dim * sizeof(cplx));
    for (int k = 0; k < n; ++k) {
        int rc = orc_expm_apply(sh, ops[k], theta[k], psi_out, psi_out);
        if (rc) return rc;
    }
    return 0;
}

/* E(theta) = <psi_n|H|psi_n> and dE/dtheta_k for k = 1..n (stored forward
 * states, lambda swept backwards with exp(-theta_k A_k)). */
int orc_energy_and_grad(void *sh, void *hh, int n, void **ops, const double *theta, const cplx *psi0,
                        double *E, double *grad) {
    const orc_sector *s = (const orc_sector *)sh;
    int64_t dim = s->dim;
    cplx *states = (cplx *)malloc((size_t)(n + 1) * (size_t)dim * sizeof(cplx));
    cplx *lam = (cplx *)malloc((size_t)dim * sizeof(cplx));
    cplx *t = (cplx *)malloc((size_t)dim * sizeof(cplx));
    if (!states || !lam || !t) { free(states); free(lam); free(t); return 2; }
    int rc = 0;
    memcpy(states, psi0, (size_t)dim * sizeof(cplx));
    for (int k = 0; k < n && !rc; ++k)
        rc = orc_expm_apply(sh, ops[k], theta[k], states + (size_t)k * dim, states + (size_t)(k + 1) * dim);
    if (!rc) rc = orc_apply(sh, hh, states + (size_t)n * dim, lam);
    if (!rc) *E = creal(vec_dot(states + (size_t)n * dim, lam, dim));
    for (int k = n - 1; k >= 0 && !rc; --k) {
        rc = orc_apply(sh, ops[k], states + (size_t)(k + 1) * dim, t);   /* A_k psi_k */
        if (rc) break;
        grad[k] = 2.0 * creal(vec_dot(lam, t, dim));
        if (k > 0) rc = orc_expm_apply(sh, ops[k], -theta[k], lam, lam);
    }
    free(states); free(lam); free(t);
    return rc;
}

/* Plain inner products and norms for the Python side. */
void orc_dot(const cplx *a, const cplx *b, int64_t dim, double *re, double *im) {
    cplx z = vec_dot(a, b, dim);
    *re = creal(z);
    *im = cimag(z);
}

/* Threads used by the parallel loops (the CPU baseline times 1 and all). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
