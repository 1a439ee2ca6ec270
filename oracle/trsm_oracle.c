/*
 * Plain FP64 CPU oracle for the selective diagonal-block-inversion TRSM of
 * Wicky, Solomonik & Hoefler, "Communication-Avoiding Parallel Algorithms for
 * Solving Triangular Systems of Linear Equations" (arXiv:1612.01855).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file: only the tests, the smoke check and the bench's
 * CPU-baseline leg use it.  It shares no code, header or constant with the
 * CUDA library.
 *
 * Conventions (all functions):
 *   - matrices are column-major, element (i, j) of M with leading dimension ld
 *     is M[j*ld + i];
 *   - L is n x n lower-triangular (only the lower triangle, diagonal included,
 *     is read); B, X are n x k dense;
 *   - every loop is a plain triple loop in the order the paper (or the
 *     textbook definition) states, with no blocking and no reordering;
 *   - build with -ffp-contract=off so that a*b+c is rounded twice, the
 *     canonical IEEE reading (the explicit fma() in the double-double
 *     routine is the one intended exception).
 *
 * Return value: 0 on success, -1 on a bad argument, -2 on a zero diagonal
 * entry (the paper is silent on singular L; see the design notes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, ld, i, j) ((M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* A deliberate-mistake switch for the pin-strength tests: when nonzero, one
 * plausible error is planted in the arithmetic below (see oracle/__init__.py
 * for the list).  It is 0 in every real use. */
static int g_mutation = 0;
void oracle_set_mutation(int m) { g_mutation = m; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Forward substitution (Section 1, L X = B; textbook column sweep).
 *   x_j = (b_j - sum_{l<j} L_jl x_l) / L_jj,  the sum taken in increasing l.
 * The column sweep below subtracts L_jl x_l from b_j as soon as x_l is known,
 * which performs exactly these subtractions in exactly this order.  The
 * columns of X are independent (Section 2.3.4, the independent split), so
 * they are distributed over OpenMP threads. */
static int subst_one_column(int64_t n, const double* L, int64_t ldl,
                            double* w /* in: b, out: x */) {
  for (int64_t l = 0; l < n; ++l) {
    double d = AT(L, ldl, l, l);
    if (d == 0.0) return -2;
    double xl = w[l] / d;
    w[l] = xl;
    int64_t jstart = l + 1;
    if (g_mutation == 3) jstart = l + 2;            /* planted: drops a term */
    for (int64_t j = jstart; j < n; ++j) w[j] -= AT(L, ldl, j, l) * xl;
  }
  return 0;
}

int oracle_forward_subst(int64_t n, int64_t k, const double* L, int64_t ldl,
                         const double* B, int64_t ldb, double* X, int64_t ldx) {
  if (n < 0 || k < 0 || ldl < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) ||
      ldx < (n > 0 ? n : 1))
    return -1;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : status)
  for (int64_t c = 0; c < k; ++c) {
    double* w = X + (size_t)c * (size_t)ldx;
    const double* b = B + (size_t)c * (size_t)ldb;
    if (w != b) memcpy(w, b, sizeof(double) * (size_t)n);
    int s = subst_one_column(n, L, ldl, w);
    if (s < status) status = s;
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Inverse by definition: column j of L^-1 solves L y = e_j. */
int oracle_tri_inv_columns(int64_t m, const double* L, int64_t ldl,
                           double* Linv, int64_t ldinv) {
  if (m < 0 || ldl < (m > 0 ? m : 1) || ldinv < (m > 0 ? m : 1)) return -1;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : status)
  for (int64_t j = 0; j < m; ++j) {
    double* y = Linv + (size_t)j * (size_t)ldinv;
    for (int64_t i = 0; i < m; ++i) y[i] = (i == j) ? 1.0 : 0.0;
    int s = subst_one_column(m, L, ldl, y);
    if (s < status) status = s;
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Recursive triangular inversion, Algorithm RecTriInv (Section 5.1):
 *   L = [L11 0; L21 L22],  L^-1 = [L11^-1 0; L21^-1 L22^-1] with
 *   L'21 = -(L22^-1 * L21)        (the first multiply),
 *   L21^-1 = L'21 * L11^-1        (the second multiply),
 * the two half inversions being independent.  The split is h = floor(m/2)
 * rows on top.  The base case ("sequential inversion" in the paper, which
 * names no method) is the inverse by definition above, used when m <= base.
 * Linv receives the full m x m inverse, its upper triangle set to zero. */
static int rec_tri_inv(int64_t m, const double* L, int64_t ldl, double* Linv,
                       int64_t ldinv, int64_t base) {
  if (m <= base || m <= 1) return oracle_tri_inv_columns(m, L, ldl, Linv, ldinv);
  int64_t h = m / 2, r = m - h;
  const double* L11 = L;
  const double* L21 = L + h;
  const double* L22 = L + (size_t)h * (size_t)ldl + h;
  double* I11 = Linv;
  double* I21 = Linv + h;
  double* I22 = Linv + (size_t)h * (size_t)ldinv + h;
  int s = rec_tri_inv(h, L11, ldl, I11, ldinv, base);
  if (s) return s;
  s = rec_tri_inv(r, L22, ldl, I22, ldinv, base);
  if (s) return s;
  /* upper-right block of the inverse is zero */
  for (int64_t j = h; j < m; ++j)
    for (int64_t i = 0; i < h; ++i) AT(Linv, ldinv, i, j) = 0.0;
  /* T = -(L22^-1 * L21), r x h */
  double* T = (double*)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1) * (size_t)(h > 0 ? h : 1));
  if (!T) return -3;
  for (int64_t j = 0; j < h; ++j)
    for (int64_t i = 0; i < r; ++i) {
      double acc = 0.0;
      for (int64_t t = 0; t < r; ++t) {
        double a = (g_mutation == 2) ? AT(I22, ldinv, t, i) : AT(I22, ldinv, i, t); /* planted: transposed operand */
        acc += a * AT(L21, ldl, t, j);
      }
      AT(T, r, i, j) = (g_mutation == 1) ? acc : -acc;            /* planted: lost sign */
    }
  /* L21^-1 = T * L11^-1, r x h */
  for (int64_t j = 0; j < h; ++j)
    for (int64_t i = 0; i < r; ++i) {
      double acc = 0.0;
      for (int64_t t = 0; t < h; ++t) acc += AT(T, r, i, t) * AT(I11, ldinv, t, j);
      AT(I21, ldinv, i, j) = acc;
    }
  free(T);
  return 0;
}

int oracle_rec_tri_inv(int64_t m, const double* L, int64_t ldl, double* Linv,
                       int64_t ldinv, int64_t base) {
  if (m < 0 || ldl < (m > 0 ? m : 1) || ldinv < (m > 0 ? m : 1) || base < 1) return -1;
  return rec_tri_inv(m, L, ldl, Linv, ldinv, base);
}

/* ------------------------------------------------------------------------ */
/* Algorithm Diagonal-Inverter (Section 6.1): L~ equals L except that each
 * diagonal block L(S_b, S_b), S_b = [b*n0, min((b+1)*n0, n)), is replaced by
 * its inverse computed with RecTriInv.  Off the block diagonal L~ keeps L's
 * entries (the update of Section 6.2 reads them there); the upper triangle of
 * Lt is written as zero.  When n0 does not divide n the last block is short. */
int oracle_diagonal_inverter(int64_t n, int64_t n0, const double* L, int64_t ldl,
                             double* Lt, int64_t ldt, int64_t base) {
  if (n < 0 || n0 < 1 || ldl < (n > 0 ? n : 1) || ldt < (n > 0 ? n : 1) || base < 1) return -1;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(Lt, ldt, i, j) = (i >= j) ? AT(L, ldl, i, j) : 0.0;
  for (int64_t s0 = 0; s0 < n; s0 += n0) {
    int64_t m = (n - s0 < n0) ? (n - s0) : n0;
    const double* Lb = L + (size_t)s0 * (size_t)ldl + s0;
    double* Tb = Lt + (size_t)s0 * (size_t)ldt + s0;
    int s = rec_tri_inv(m, Lb, ldl, Tb, ldt, base);
    if (s) return s;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm It-Inv-TRSM (Section 6.2), on one processor, in the paper's
 * right-looking order.  With S_i = [i*n0, (i+1)*n0) and T_i = [i*n0, n):
 *   for i = 0 .. N-1:
 *     X(S_i)        = L~(S_i, S_i) * B(S_i)            (the solve)
 *     Bbar(T_{i+1}) += L~(T_{i+1}, S_i) * X(S_i)        (the update)
 *     B(S_{i+1})    -= Bbar(S_{i+1})                    (the local subtract)
 * The work array Bbar starts at zero; B is copied, never modified.
 * counts (may be NULL) receives the multiply-adds performed by
 *   counts[0]: the solve (structurally nonzero entries of L~(S_i,S_i) only),
 *   counts[1]: the update,
 * so that 2*counts[1] and 2*counts[0] can be compared with the paper's
 * F_Upd and F_Solve (Sections 7.3 and 7.2). */
int oracle_it_inv_trsm(int64_t n, int64_t k, int64_t n0, const double* L, int64_t ldl,
                       const double* B, int64_t ldb, double* X, int64_t ldx,
                       int64_t base, int64_t* counts) {
  if (n < 0 || k < 0 || n0 < 1 || ldl < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) ||
      ldx < (n > 0 ? n : 1) || base < 1)
    return -1;
  if (counts) { counts[0] = 0; counts[1] = 0; }
  if (n == 0 || k == 0) return 0;
  size_t nn = (size_t)n;
  double* Lt = (double*)malloc(sizeof(double) * nn * nn);
  double* Bw = (double*)malloc(sizeof(double) * nn * (size_t)k);
  double* Bbar = (double*)calloc(nn * (size_t)k, sizeof(double));
  if (!Lt || !Bw || !Bbar) { free(Lt); free(Bw); free(Bbar); return -3; }
  int s = oracle_diagonal_inverter(n, n0, L, ldl, Lt, n, base);
  if (s) { free(Lt); free(Bw); free(Bbar); return s; }
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < n; ++r) AT(Bw, n, r, c) = AT(B, ldb, r, c);
  int64_t cnt_solve = 0, cnt_upd = 0;
  for (int64_t s0 = 0; s0 < n; s0 += n0) {
    int64_t m = (n - s0 < n0) ? (n - s0) : n0; /* |S_i| */
    int64_t t0 = s0 + m;                         /* first row of T_{i+1} */
    /* X(S_i) = L~(S_i,S_i) B(S_i); the block is lower-triangular */
    for (int64_t c = 0; c < k; ++c)
      for (int64_t r = 0; r < m; ++r) {
        double acc = 0.0;
        for (int64_t t = 0; t <= r; ++t) acc += AT(Lt, n, s0 + r, s0 + t) * AT(Bw, n, s0 + t, c);
        AT(X, ldx, s0 + r, c) = acc;
      }
    cnt_solve += k * (m * (m + 1) / 2);
    /* Bbar(T_{i+1}) += L~(T_{i+1}, S_i) X(S_i) */
    for (int64_t c = 0; c < k; ++c)
      for (int64_t r = t0; r < n; ++r) {
        double acc = 0.0;
        for (int64_t t = 0; t < m; ++t) acc += AT(Lt, n, r, s0 + t) * AT(X, ldx, s0 + t, c);
        AT(Bbar, n, r, c) += acc;
      }
    cnt_upd += k * (n - t0) * m;
    /* B(S_{i+1}) -= Bbar(S_{i+1}) */
    int64_t m1 = (n - t0 < n0) ? (n - t0) : n0;
    for (int64_t c = 0; c < k; ++c)
      for (int64_t r = t0; r < t0 + m1; ++r) AT(Bw, n, r, c) -= AT(Bbar, n, r, c);
  }
  if (counts) { counts[0] = cnt_solve; counts[1] = cnt_upd; }
  free(Lt); free(Bw); free(Bbar);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm Rec-TRSM (Section 4), sequential form: for n <= n0 solve by
 * substitution; otherwise split L = [L11 0; L21 L22] at h = floor(n/2) and
 *   X1 = Rec-TRSM(L11, B1);  B2' = B2 - L21 X1;  X2 = Rec-TRSM(L22, B2'). */
static int rec_trsm(int64_t n, int64_t k, const double* L, int64_t ldl, double* W,
                    int64_t ldw, int64_t n0) {
  if (n <= n0 || n <= 1) {
    for (int64_t c = 0; c < k; ++c) {
      int s = subst_one_column(n, L, ldl, W + (size_t)c * (size_t)ldw);
      if (s) return s;
    }
    return 0;
  }
  int64_t h = n / 2, r = n - h;
  int s = rec_trsm(h, k, L, ldl, W, ldw, n0);
  if (s) return s;
  const double* L21 = L + h;
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < r; ++i) {
      double acc = 0.0;
      for (int64_t t = 0; t < h; ++t) acc += AT(L21, ldl, i, t) * AT(W, ldw, t, c);
      AT(W, ldw, h + i, c) -= acc;
    }
  return rec_trsm(r, k, L + (size_t)h * (size_t)ldl + h, ldl, W + h, ldw, n0);
}

int oracle_rec_trsm(int64_t n, int64_t k, int64_t n0, const double* L, int64_t ldl,
                    const double* B, int64_t ldb, double* X, int64_t ldx) {
  if (n < 0 || k < 0 || n0 < 1 || ldl < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) ||
      ldx < (n > 0 ? n : 1))
    return -1;
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < n; ++r) AT(X, ldx, r, c) = AT(B, ldb, r, c);
  return rec_trsm(n, k, L, ldl, X, ldx, n0);
}

/* ------------------------------------------------------------------------ */
/* Double-double forward substitution, for forward-error statements that need
 * more than FP64.  Error-free transformations:
 *   TwoSum   (Knuth, TAOCP vol. 2, 4.2.2):  s = a+b, e = (a-(s-bb)) + (b-bb),
 *            bb = s-a;
 *   TwoProd  (via fused multiply-add):      p = a*b, e = fma(a, b, -p).
 * A double-double value is an unevaluated sum hi + lo with |lo| <= ulp(hi)/2.
 * The substitution order is the one of oracle_forward_subst. */
static inline void two_sum(double a, double b, double* s, double* e) {
  double ss = a + b;
  double bb = ss - a;
  *e = (a - (ss - bb)) + (b - bb);
  *s = ss;
}
static inline void two_prod(double a, double b, double* p, double* e) {
  double pp = a * b;
  *e = fma(a, b, -pp);
  *p = pp;
}
/* (ah,al) + (bh,bl), renormalised */
static inline void dd_add(double ah, double al, double bh, double bl, double* ch, double* cl) {
  double s, e;
  two_sum(ah, bh, &s, &e);
  e += al + bl;
  two_sum(s, e, ch, cl);
}
/* d * (xh,xl) for a double d */
static inline void dd_mul_d(double xh, double xl, double d, double* ph, double* pl) {
  double p, e;
  two_prod(xh, d, &p, &e);
  e += xl * d;
  two_sum(p, e, ph, pl);
}
/* (sh,sl) / d for a double d: q1 = sh/d, remainder r = s - q1*d exactly
 * in double-double, q2 = r/d. */
static inline void dd_div_d(double sh, double sl, double d, double* qh, double* ql) {
  double q1 = sh / d;
  double p, e;
  two_prod(q1, d, &p, &e);
  double rh, rl;
  dd_add(sh, sl, -p, -e, &rh, &rl);
  double q2 = (rh + rl) / d;
  two_sum(q1, q2, qh, ql);
}

int oracle_forward_subst_dd(int64_t n, int64_t k, const double* L, int64_t ldl,
                            const double* B, int64_t ldb, double* Xhi, double* Xlo,
                            int64_t ldx) {
  if (n < 0 || k < 0 || ldl < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) ||
      ldx < (n > 0 ? n : 1))
    return -1;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : status)
  for (int64_t c = 0; c < k; ++c) {
    double* wh = Xhi + (size_t)c * (size_t)ldx;
    double* wl = Xlo + (size_t)c * (size_t)ldx;
    int st = 0;
    for (int64_t r = 0; r < n; ++r) { wh[r] = AT(B, ldb, r, c); wl[r] = 0.0; }
    for (int64_t l = 0; l < n; ++l) {
      double d = AT(L, ldl, l, l);
      if (d == 0.0) { st = -2; break; }
      double xh, xl;
      dd_div_d(wh[l], wl[l], d, &xh, &xl);
      wh[l] = xh; wl[l] = xl;
      for (int64_t j = l + 1; j < n; ++j) {
        double ph, pl;
        dd_mul_d(xh, xl, AT(L, ldl, j, l), &ph, &pl);
        dd_add(wh[j], wl[j], -ph, -pl, &wh[j], &wl[j]);
      }
    }
    if (st < status) status = st;
  }
  return status;
}
