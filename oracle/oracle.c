/*
 * Reference oracle for Gaussian-boson-sampling output probabilities.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code with the CUDA library.
 *
 * Every routine is the plain definition or the plain published algorithm,
 * written for a reader to check by eye, in double-double ("dd") arithmetic
 * unless its name ends in _f64:
 *
 *   orc_build_B       B = U diag(t) U^T, t_i = tanh r_i (Sec. 2.3, W = U U^T;
 *                     per-mode squeezing as in the Gaussian-state formula the
 *                     paper cites for Eq. ProOri)
 *   orc_haf_pm        Hafnian by the perfect-matching sum of Eq. HafMatch,
 *                     expanded along one index as in Appendix A
 *   orc_haf_subset    Hafnian by the 2^{n/2}-subset power-trace sum of
 *                     Bjorklund, Gupt and Quesada (the O(n^3 2^{n/2}) method the
 *                     paper cites in Sec. 2.3), traces by repeated products
 *   orc_per_ryser     permanent by Ryser's inclusion-exclusion formula
 *   orc_prob          p(s) = |Haf(B_x)|^2 / (prod_j s_j! prod_i cosh r_i)
 *                     (Eq. ProOri with per-mode r; W_x gather of Sec. 3.2)
 *
 * Complex matrices are passed as interleaved (re, im) doubles, row-major.
 * dd results are returned as 4 doubles: re.hi, re.lo, im.hi, im.lo.
 *
 * Double-double arithmetic: Knuth's two-sum, Dekker's fast two-sum and the
 * FMA-based exact product, as published; compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* double-double                                                             */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

static dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}
static dd fast_two_sum(double a, double b) { /* requires |a| >= |b| or a == 0 */
  double s = a + b;
  double e = b - (s - a);
  dd r = {s, e};
  return r;
}
static dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  dd r = {p, e};
  return r;
}
static dd dd_from(double a) { dd r = {a, 0.0}; return r; }
static dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
static dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  p.lo += x.hi * y.lo + x.lo * y.hi;
  return fast_two_sum(p.hi, p.lo);
}
static dd dd_div_d(dd x, double d) { /* x / d for a double d */
  double q1 = x.hi / d;
  dd p = two_prod(q1, d);
  double r = ((x.hi - p.hi) - p.lo) + x.lo;
  double q2 = r / d;
  return fast_two_sum(q1, q2);
}
static double dd_to_d(dd x) { return x.hi + x.lo; }

static cdd cdd_zero(void) { cdd z = {{0, 0}, {0, 0}}; return z; }
static cdd cdd_from(double re, double im) { cdd z = {dd_from(re), dd_from(im)}; return z; }
static cdd cdd_add(cdd a, cdd b) { cdd z = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return z; }
static cdd cdd_sub(cdd a, cdd b) { cdd z = {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; return z; }
static cdd cdd_mul(cdd a, cdd b) {
  cdd z;
  z.re = dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
  z.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
  return z;
}
static cdd cdd_scale_d(cdd a, double s) { /* a * s, s a double */
  cdd z = {dd_mul(a.re, dd_from(s)), dd_mul(a.im, dd_from(s))};
  return z;
}
static cdd cdd_div_d(cdd a, double d) { cdd z = {dd_div_d(a.re, d), dd_div_d(a.im, d)}; return z; }
static double cdd_abs(cdd a) { return hypot(dd_to_d(a.re), dd_to_d(a.im)); }
static void cdd_store(cdd a, double* out4) {
  out4[0] = a.re.hi; out4[1] = a.re.lo; out4[2] = a.im.hi; out4[3] = a.im.lo;
}

/* plain double complex */
typedef struct { double re, im; } cd;
static cd cd_add(cd a, cd b) { cd z = {a.re + b.re, a.im + b.im}; return z; }
static cd cd_mul(cd a, cd b) { cd z = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return z; }

/* ------------------------------------------------------------------------ */
/* Kernel matrix B = U diag(t) U^T                                           */
/* ------------------------------------------------------------------------ */
/* U: m*m interleaved complex, row-major. t: m doubles. B_out: m*m entries of
 * 4 doubles (re.hi, re.lo, im.hi, im.lo). B[i][j] = sum_k U[i][k] t_k U[j][k]. */
void orc_build_B(int m, const double* U, const double* t, double* B_out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < m; i++) {
    for (int j = 0; j < m; j++) {
      cdd acc = cdd_zero();
      for (int k = 0; k < m; k++) {
        cdd uik = cdd_from(U[2 * (i * m + k)], U[2 * (i * m + k) + 1]);
        cdd ujk = cdd_from(U[2 * (j * m + k)], U[2 * (j * m + k) + 1]);
        acc = cdd_add(acc, cdd_scale_d(cdd_mul(uik, ujk), t[k]));
      }
      cdd_store(acc, B_out + 4 * ((size_t)i * m + j));
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Hafnian by perfect matchings (Eq. HafMatch; expansion of Appendix A)      */
/* ------------------------------------------------------------------------ */
/* Haf over the index set `mask` (bit i set = index i still unmatched): match
 * the lowest remaining index with every other remaining index u and recurse. */
static cdd haf_pm_rec(int n, const cdd* A, uint32_t mask) {
  if (mask == 0) return cdd_from(1.0, 0.0);
  int i = __builtin_ctz(mask);
  uint32_t rest = mask & ~(1u << i);
  cdd acc = cdd_zero();
  for (int u = 0; u < n; u++) {
    if (!(rest & (1u << u))) continue;
    cdd sub = haf_pm_rec(n, A, rest & ~(1u << u));
    acc = cdd_add(acc, cdd_mul(A[i * n + u], sub));
  }
  return acc;
}

static cdd* load_cdd(int n, const double* A) {
  cdd* M = (cdd*)malloc(sizeof(cdd) * (size_t)(n > 0 ? n * n : 1));
  for (int i = 0; i < n * n; i++) M[i] = cdd_from(A[2 * i], A[2 * i + 1]);
  return M;
}

static cdd haf_pm_cdd(int n, const cdd* A) {
  if (n % 2) return cdd_zero();
  if (n == 0) return cdd_from(1.0, 0.0);
  uint32_t all = (n == 32) ? 0xffffffffu : ((1u << n) - 1u);
  return haf_pm_rec(n, A, all);
}

/* A: n*n interleaved complex doubles. out4: dd complex. */
void orc_haf_pm(int n, const double* A, double* out4) {
  cdd* M = load_cdd(n, A);
  cdd_store(haf_pm_cdd(n, M), out4);
  free(M);
}

/* ------------------------------------------------------------------------ */
/* Hafnian by the subset power-trace sum (Bjorklund, Gupt, Quesada 2018)     */
/* ------------------------------------------------------------------------ */
/* For n = 2h, pair P_i = {2i, 2i+1} (0-based). For S a subset of the h pairs:
 *   A_S   rows/cols of A in the pairs of S (in increasing order),
 *   X     the permutation that swaps the two members of every pair,
 *   f(M)  = [lambda^h] exp( sum_{k=1..h} tr(M^k) lambda^k / (2k) ),
 *   Haf(A) = sum_S (-1)^{h-|S|} f(X A_S).
 * tr(M^k) by repeated products M^k = M^{k-1} M; the exponential's power series
 * by e_0 = 1, e_k = (1/(2k)) sum_{j=1..k} tr(M^j) e_{k-j}.
 * kappa accumulates sum_S |f(X A_S)|. */
static cdd subset_term_cdd(int h, const cdd* A, int n, uint32_t S, cdd* M, cdd* P, cdd* Q,
                           cdd* tr, cdd* e) {
  int idx[64];
  int N = 0;
  for (int i = 0; i < h; i++)
    if (S & (1u << i)) { idx[N++] = 2 * i; idx[N++] = 2 * i + 1; }
  /* M = X A_S: row a of M is row X(a) of A_S; X swaps 2t <-> 2t+1. */
  for (int a = 0; a < N; a++) {
    int ra = idx[a ^ 1];
    for (int b = 0; b < N; b++) M[a * N + b] = A[ra * n + idx[b]];
  }
  memcpy(P, M, sizeof(cdd) * (size_t)N * N);
  for (int k = 1; k <= h; k++) {
    if (k > 1) { /* P <- P M */
      for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
          cdd acc = cdd_zero();
          for (int c = 0; c < N; c++) acc = cdd_add(acc, cdd_mul(P[a * N + c], M[c * N + b]));
          Q[a * N + b] = acc;
        }
      memcpy(P, Q, sizeof(cdd) * (size_t)N * N);
    }
    cdd t = cdd_zero();
    for (int a = 0; a < N; a++) t = cdd_add(t, P[a * N + a]);
    tr[k] = t;
  }
  e[0] = cdd_from(1.0, 0.0);
  for (int k = 1; k <= h; k++) {
    cdd acc = cdd_zero();
    for (int j = 1; j <= k; j++) acc = cdd_add(acc, cdd_mul(tr[j], e[k - j]));
    e[k] = cdd_div_d(acc, 2.0 * k);
  }
  return e[h];
}

#define ORC_CHUNKS 256

static cdd haf_subset_cdd(int n, const cdd* A, double* kappa_out) {
  if (n % 2) { if (kappa_out) *kappa_out = 0.0; return cdd_zero(); }
  if (n == 0) { if (kappa_out) *kappa_out = 1.0; return cdd_from(1.0, 0.0); }
  int h = n / 2;
  uint64_t total = 1ull << h;
  int nch = total < ORC_CHUNKS ? (int)total : ORC_CHUNKS;
  cdd part[ORC_CHUNKS];
  double kpart[ORC_CHUNKS];
  /* fixed chunking, partial sums added in chunk order: deterministic */
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < nch; c++) {
    uint64_t lo = total * (uint64_t)c / nch, hi = total * (uint64_t)(c + 1) / nch;
    cdd* buf = (cdd*)malloc(sizeof(cdd) * (3 * (size_t)n * n + 2 * (h + 1)));
    cdd *M = buf, *P = M + n * n, *Q = P + n * n, *tr = Q + n * n, *e = tr + h + 1;
    cdd acc = cdd_zero();
    double kacc = 0.0;
    for (uint64_t S = lo; S < hi; S++) {
      int s = __builtin_popcountll(S);
      if (s == 0) continue; /* f = [lambda^h] 1 = 0 for h >= 1 */
      cdd f = subset_term_cdd(h, A, n, (uint32_t)S, M, P, Q, tr, e);
      kacc += cdd_abs(f);
      acc = ((h - s) % 2) ? cdd_sub(acc, f) : cdd_add(acc, f);
    }
    part[c] = acc;
    kpart[c] = kacc;
    free(buf);
  }
  cdd haf = cdd_zero();
  double K = 0.0;
  for (int c = 0; c < nch; c++) { haf = cdd_add(haf, part[c]); K += kpart[c]; }
  if (kappa_out) *kappa_out = K;
  return haf;
}

/* A: n*n interleaved complex. out4: dd complex Hafnian. kappa_sum: sum_S |f|. */
void orc_haf_subset(int n, const double* A, double* out4, double* kappa_sum) {
  cdd* M = load_cdd(n, A);
  cdd_store(haf_subset_cdd(n, M, kappa_sum), out4);
  free(M);
}

/* Same algorithm in plain double precision (the CPU baseline). out2: re, im. */
static cd subset_term_f64(int h, const cd* A, int n, uint32_t S, cd* M, cd* P, cd* Q, cd* tr,
                          cd* e) {
  int idx[64];
  int N = 0;
  for (int i = 0; i < h; i++)
    if (S & (1u << i)) { idx[N++] = 2 * i; idx[N++] = 2 * i + 1; }
  for (int a = 0; a < N; a++) {
    int ra = idx[a ^ 1];
    for (int b = 0; b < N; b++) M[a * N + b] = A[ra * n + idx[b]];
  }
  memcpy(P, M, sizeof(cd) * (size_t)N * N);
  for (int k = 1; k <= h; k++) {
    if (k > 1) {
      for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
          cd acc = {0, 0};
          for (int c = 0; c < N; c++) acc = cd_add(acc, cd_mul(P[a * N + c], M[c * N + b]));
          Q[a * N + b] = acc;
        }
      memcpy(P, Q, sizeof(cd) * (size_t)N * N);
    }
    cd t = {0, 0};
    for (int a = 0; a < N; a++) t = cd_add(t, P[a * N + a]);
    tr[k] = t;
  }
  e[0].re = 1.0; e[0].im = 0.0;
  for (int k = 1; k <= h; k++) {
    cd acc = {0, 0};
    for (int j = 1; j <= k; j++) acc = cd_add(acc, cd_mul(tr[j], e[k - j]));
    e[k].re = acc.re / (2.0 * k);
    e[k].im = acc.im / (2.0 * k);
  }
  return e[h];
}

static cd haf_subset_f64_serial(int n, const cd* A) {
  cd haf = {0, 0};
  if (n % 2) return haf;
  if (n == 0) { haf.re = 1.0; return haf; }
  int h = n / 2;
  cd* buf = (cd*)malloc(sizeof(cd) * (3 * (size_t)n * n + 2 * (h + 1)));
  cd *M = buf, *P = M + n * n, *Q = P + n * n, *tr = Q + n * n, *e = tr + h + 1;
  for (uint64_t S = 1; S < (1ull << h); S++) {
    int s = __builtin_popcountll(S);
    cd f = subset_term_f64(h, A, n, (uint32_t)S, M, P, Q, tr, e);
    if ((h - s) % 2) { haf.re -= f.re; haf.im -= f.im; }
    else { haf.re += f.re; haf.im += f.im; }
  }
  free(buf);
  return haf;
}

void orc_haf_subset_f64(int n, const double* A, double* out2) {
  cd* M = (cd*)malloc(sizeof(cd) * (size_t)(n > 0 ? n * n : 1));
  for (int i = 0; i < n * n; i++) { M[i].re = A[2 * i]; M[i].im = A[2 * i + 1]; }
  cd r = haf_subset_f64_serial(n, M);
  out2[0] = r.re; out2[1] = r.im;
  free(M);
}

/* ------------------------------------------------------------------------ */
/* Permanent by Ryser's formula                                              */
/* ------------------------------------------------------------------------ */
/* Per(C) = (-1)^k sum_{T subset [k]} (-1)^{|T|} prod_i sum_{j in T} C_ij */
void orc_per_ryser(int k, const double* C, double* out4) {
  cdd* M = load_cdd(k, C);
  cdd per = cdd_zero();
  for (uint64_t T = 1; T < (1ull << k); T++) {
    cdd prod = cdd_from(1.0, 0.0);
    for (int i = 0; i < k; i++) {
      cdd rs = cdd_zero();
      for (int j = 0; j < k; j++)
        if (T & (1ull << j)) rs = cdd_add(rs, M[i * k + j]);
      prod = cdd_mul(prod, rs);
    }
    int sgn = ((k - __builtin_popcountll(T)) % 2) ? -1 : 1;
    per = sgn > 0 ? cdd_add(per, prod) : cdd_sub(per, prod);
  }
  if (k == 0) per = cdd_from(1.0, 0.0);
  cdd_store(per, out4);
  free(M);
}

/* ------------------------------------------------------------------------ */
/* Output probabilities                                                      */
/* ------------------------------------------------------------------------ */
/* Bdd: m*m dd-complex kernel matrix from orc_build_B (4 doubles per entry).
 * idx: concatenated 0-based mode lists, in any order (Appendix B: the order
 * of x does not change Haf(W_x)); n[b], offs[b] (start of pattern b in idx).
 * log_norm = sum_i log cosh r_i. method 0 = subset sum, 1 = perfect
 * matchings. zero_diag != 0: W_x(i, i) is set to 0 before the sum (no perfect
 * matching uses V(i, i), Eq. HafMatch, so Haf is unchanged; the subset sum's
 * individual terms, and so kappa_sum, are not). Outputs per pattern: p, log p
 * (-inf when Haf = 0), Haf (dd, 4 doubles), kappa_sum (subset method; 0 for
 * matchings). Patterns run in parallel; each pattern's own sum is computed
 * serially inside. */
void orc_prob(int m, const double* Bdd, const int* idx, const int* n, const long* offs, int batch,
              double log_norm, int method, int zero_diag, double* p_out, double* logp_out,
              double* haf_out, double* kappa_out) {
  /* patterns in parallel when there are enough of them; otherwise each
   * pattern's subset sum runs its fixed chunks in parallel (same arithmetic
   * either way: the chunked sum below) */
#ifdef _OPENMP
  int outer = batch >= omp_get_max_threads();
#else
  int outer = 1;
#endif
#pragma omp parallel for schedule(dynamic, 1) if (outer)
  for (int b = 0; b < batch; b++) {
    int nb = n[b];
    const int* x = idx + offs[b];
    cdd* W = (cdd*)malloc(sizeof(cdd) * (size_t)(nb > 0 ? nb * nb : 1));
    /* W_x(i, j) = B(x_i, x_j) (Sec. 3.2) */
    for (int i = 0; i < nb; i++)
      for (int j = 0; j < nb; j++) {
        const double* e = Bdd + 4 * ((size_t)x[i] * m + x[j]);
        cdd v = {{e[0], e[1]}, {e[2], e[3]}};
        W[i * nb + j] = (zero_diag && i == j) ? cdd_zero() : v;
      }
    double K = 0.0;
    cdd haf;
    if (method == 1) {
      haf = haf_pm_cdd(nb, W);
    } else {
      haf = haf_subset_cdd(nb, W, &K);
      if (nb == 0) K = 1.0;
    }
    /* p = |Haf|^2 / (prod_j s_j! prod_i cosh r_i), s_j the number of times
     * mode j occurs in x: sort a copy so that equal modes are adjacent, then
     * sum log s_j! over the runs. */
    int xs[64];
    for (int i = 0; i < nb; i++) {
      int v = x[i], k = i;
      while (k > 0 && xs[k - 1] > v) { xs[k] = xs[k - 1]; k--; }
      xs[k] = v;
    }
    double log_fact = 0.0;
    int run = 1;
    for (int i = 1; i <= nb; i++) {
      if (i < nb && xs[i] == xs[i - 1]) { run++; continue; }
      if (nb > 0)
        for (int k = 2; k <= run; k++) log_fact += log((double)k);
      run = 1;
    }
    dd a2 = dd_add(dd_mul(haf.re, haf.re), dd_mul(haf.im, haf.im));
    double mod2 = dd_to_d(a2);
    double logp = (mod2 > 0.0) ? log(a2.hi) + log1p(a2.lo / a2.hi) - log_fact - log_norm : -INFINITY;
    p_out[b] = (mod2 > 0.0) ? exp(logp) : 0.0;
    logp_out[b] = logp;
    cdd_store(haf, haf_out + 4 * b);
    kappa_out[b] = K;
    free(W);
  }
}

/* Hafnians of a batch of explicit matrices, FP64 subset sum, patterns in
 * parallel: the timed CPU baseline. A: concatenated n_b*n_b interleaved complex
 * matrices at offs[b] (in complex elements). out: 2 doubles per matrix. */
void orc_haf_batch_f64(const double* A, const int* n, const long* offs, int batch, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < batch; b++) {
    int nb = n[b];
    const double* a = A + 2 * offs[b];
    cd* M = (cd*)malloc(sizeof(cd) * (size_t)(nb > 0 ? nb * nb : 1));
    for (int i = 0; i < nb * nb; i++) { M[i].re = a[2 * i]; M[i].im = a[2 * i + 1]; }
    cd r = haf_subset_f64_serial(nb, M);
    out[2 * b] = r.re; out[2 * b + 1] = r.im;
    free(M);
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads used by later parallel loops (timing only; no effect on results,
   which are per pattern). */
void orc_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
