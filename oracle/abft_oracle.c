/*
 * abft_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of Huang-Abraham
 * algorithm-based fault-tolerant matrix multiplication as used by Bosilca,
 * Delmas, Dongarra and Langou, "Algorithmic Based Fault Tolerance Applied to
 * High Performance Computing" (2008).  It is the correctness authority for
 * the CUDA library: the tests, the smoke check and the benchmark's CPU
 * baseline are the only code allowed to load it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Every loop below is the textbook definition of the quantity it computes,
 * summed in increasing index order, in IEEE binary64 with round-to-nearest
 * (built with -ffp-contract=off so no multiply-add is fused).  OpenMP only
 * splits independent outputs across threads; no sum is reordered.
 *
 * Notation (paper section 2.2, Eq. (1)):  C = A B with A m-by-k, B k-by-n,
 * all row-major with leading dimensions in elements.  A gains checksum rows
 * C_C^T A, B gains checksum columns B C_R, and the product of the encoded
 * operands is the full-checksum matrix (AB)_F.
 *
 *  - verify blocks: rows are cut into blocks of vb_r rows (the last one may be
 *    shorter), columns into blocks of vb_c columns.  Per block there is one
 *    unweighted checksum (weights e = 1) and one weighted checksum with
 *    weights w_t = (t+1) * 2^-ceil(log2 vb), t = 0 .. vb-1 the index inside
 *    the block.  The power-of-two scale is exact and only keeps the weighted
 *    sums in range; the ratio of weighted to unweighted residual, multiplied
 *    back by 2^ceil(log2 vb), is the 1-based position of a single error.
 *  - erasure grid: when p > 0 the rows form p block-rows of bs = m/p rows and
 *    the columns q block-columns of n/q columns.  A gains bs extra rows
 *    S_A = sum_I A_I (C_C = [I; I; ...; I], section 2.1 with all a_i = 1), so
 *    the product carries S = S_A B = sum_I C_I, from which one lost block of
 *    a block column is rebuilt (section 2.1, section 3.3 "T_checksum").
 *
 * Parity status of each function is stated at the function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_VERSION 1

/* report kinds */
#define K_CORRECTED 1
#define K_NONFINITE 2
#define K_UNCORRECTABLE 3
#define K_RECOVERED 4

/* status codes */
#define ST_OK 0
#define ST_INVALID (-1)
#define ST_UNCORRECTABLE 1

int oracle_version(void) { return ORACLE_VERSION; }

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* e = ceil(log2(vb)), vb >= 1 */
static int ceil_log2(int64_t vb) {
  int e = 0;
  while (((int64_t)1 << e) < vb) ++e;
  return e;
}

/* Weight of position t (0-based) inside a verify block of nominal size vb. */
double oracle_weight(int64_t t, int64_t vb) {
  return ldexp((double)(t + 1), -ceil_log2(vb));
}

/* ------------------------------------------------------------------------ */
/* GEMM: C = A B, the plain definition C_ij = sum_l A_il B_lj (Eq. (1)).
 * Every C_ij is accumulated from 0 by adding the products A_il B_lj in
 * increasing l; the loops visit l before j only so that B is read row by row
 * (each element's sum is the same sequence of roundings as the i-j-l order).
 * Pinned by: numpy's product (library special case), exact integer inputs,
 * identity and rank-one closed forms, the residual check of section 4.3. */
void oracle_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* C, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double* c = C + i * ldc;
    for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
    for (int64_t l = 0; l < k; ++l) {
      const double a = A[i * lda + l];
      const double* b = B + l * ldb;
      for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
    }
  }
}

/* Threads of the GEMM loop above (OpenMP): the number it runs on, and a way to
 * set it -- a process whose environment limits OpenMP to one thread (one of
 * several processes launched together) may use the host's cores when it is the
 * only one working.  Neither is part of the method. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Coefficient c_{l,I} of block row I in block checksum l of a p-block grid
 * (section 2.1: f checksums with f independent weight vectors recover f lost
 * blocks; the paper draws them at random so that every f-by-f minor is
 * nonsingular).  Here: Vandermonde weights c_{l,I} = x_I^l with distinct
 * nodes x_I = (2I + 1 - p) / 2^e, 2^e > p, symmetric about 0 -- every
 * f-by-f minor of a Vandermonde matrix with distinct nodes is nonsingular,
 * the dyadic values are exact in binary32 and binary64, and centred nodes
 * keep the systems of neighbouring blocks better conditioned than nodes in
 * (0, 1).  l = 0 is the plain sum (c = 1). */
double oracle_block_coef(int64_t l, int64_t I, int64_t p) {
  int e = 0;
  while (((int64_t)1 << e) <= p) ++e;
  double x = ldexp((double)(2 * I + 1 - p), -e), c = 1.0;
  for (int64_t t = 0; t < l; ++t) c *= x;
  return c;
}

/* Encode A (section 2.1 and the left operand of Eq. (1)).
 * acs has (2*nvb + f*bs) rows of k values, nvb = ceil(m/vb), bs = m/p (0 if
 * p == 0):
 *   row 2I           : e^T A_I                     (unweighted column checksum of block I)
 *   row 2I+1         : w^T A_I                     (weighted column checksum of block I)
 *   row 2nvb+l*bs+t  : sum_I c_{l,I} A[I*bs+t]     (block checksum rows S^(l), l < f)
 * Pinned by: hand-worked golden values and exact integer invariants
 * e^T C = (e^T A) B, S^(l) B = sum_I c_{l,I} C_I. */
void oracle_encode_A(int64_t m, int64_t k, const double* A, int64_t lda, int64_t vb, int64_t p,
                     int64_t f, double* acs) {
  int64_t nvb = ceil_div(m, vb);
  for (int64_t I = 0; I < nvb; ++I) {
    int64_t i0 = I * vb, i1 = (i0 + vb < m) ? i0 + vb : m;
    for (int64_t l = 0; l < k; ++l) {
      double se = 0.0, sw = 0.0;
      for (int64_t i = i0; i < i1; ++i) {
        se += A[i * lda + l];
        sw += oracle_weight(i - i0, vb) * A[i * lda + l];
      }
      acs[(2 * I) * k + l] = se;
      acs[(2 * I + 1) * k + l] = sw;
    }
  }
  if (p > 0) {
    int64_t bs = m / p;
    if (f < 1) f = 1;
    for (int64_t c = 0; c < f; ++c)
      for (int64_t t = 0; t < bs; ++t)
        for (int64_t l = 0; l < k; ++l) {
          double s = 0.0;
          for (int64_t I = 0; I < p; ++I) s += oracle_block_coef(c, I, p) * A[(I * bs + t) * lda + l];
          acs[(2 * nvb + c * bs + t) * k + l] = s;
        }
  }
}

/* Encode B (the right operand of Eq. (1)): bcs is k-by-(2*nvb), nvb =
 * ceil(n/vb); column 2J is B_J e and column 2J+1 is B_J w. */
void oracle_encode_B(int64_t k, int64_t n, const double* B, int64_t ldb, int64_t vb, double* bcs) {
  int64_t nvb = ceil_div(n, vb);
  for (int64_t l = 0; l < k; ++l)
    for (int64_t J = 0; J < nvb; ++J) {
      int64_t j0 = J * vb, j1 = (j0 + vb < n) ? j0 + vb : n;
      double se = 0.0, sw = 0.0;
      for (int64_t j = j0; j < j1; ++j) {
        se += B[l * ldb + j];
        sw += oracle_weight(j - j0, vb) * B[l * ldb + j];
      }
      bcs[l * (2 * nvb) + 2 * J] = se;
      bcs[l * (2 * nvb) + 2 * J + 1] = sw;
    }
}

/* ------------------------------------------------------------------------ */
/* Norms feeding the detection thresholds (the paper only says rounding in
 * floating-point checksums is of the order of the method's own rounding,
 * section 2.1; the bound built from them is this library's reading of it).
 *   nrow[i]         = ||A_{i,:}||_2
 *   nblk[4I+0]      = sqrt( sum_{i in I} ||A_{i,:}||^2 )        (= ||A_I||_F)
 *   nblk[4I+1]      = sqrt( sum_{i in I} w_{i-I0}^2 ||A_{i,:}||^2 )
 *   nblk[4I+2]      = || e^T A_I ||_2      (the stored checksum row)
 *   nblk[4I+3]      = || w^T A_I ||_2
 * Pinned by numpy norms of explicitly formed vectors. */
void oracle_norms_A(int64_t m, int64_t k, const double* A, int64_t lda, int64_t vb, double* nrow,
                    double* nblk) {
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t l = 0; l < k; ++l) s += A[i * lda + l] * A[i * lda + l];
    nrow[i] = sqrt(s);
  }
  int64_t nvb = ceil_div(m, vb);
  for (int64_t I = 0; I < nvb; ++I) {
    int64_t i0 = I * vb, i1 = (i0 + vb < m) ? i0 + vb : m;
    double f0 = 0.0, f1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      double w = oracle_weight(i - i0, vb);
      f0 += nrow[i] * nrow[i];
      f1 += (w * nrow[i]) * (w * nrow[i]);
    }
    for (int64_t l = 0; l < k; ++l) {
      double se = 0.0, sw = 0.0;
      for (int64_t i = i0; i < i1; ++i) {
        double a = A[i * lda + l];
        se += a;
        sw += oracle_weight(i - i0, vb) * a;
      }
      q2 += se * se;
      q3 += sw * sw;
    }
    nblk[4 * I + 0] = sqrt(f0);
    nblk[4 * I + 1] = sqrt(f1);
    nblk[4 * I + 2] = sqrt(q2);
    nblk[4 * I + 3] = sqrt(q3);
  }
}

/* Column analog for B: ncol[j] = ||B_{:,j}||_2; per column block J
 * sqrt(sum_{j in J} ||B_{:,j}||^2), sqrt(sum w^2 ||B_{:,j}||^2), and the norms
 * of the stored checksum columns B_J e, B_J w (vectors of length k). */
void oracle_norms_B(int64_t k, int64_t n, const double* B, int64_t ldb, int64_t vb, double* ncol,
                    double* nblk) {
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t l = 0; l < k; ++l) s += B[l * ldb + j] * B[l * ldb + j];
    ncol[j] = sqrt(s);
  }
  int64_t nvb = ceil_div(n, vb);
  for (int64_t J = 0; J < nvb; ++J) {
    int64_t j0 = J * vb, j1 = (j0 + vb < n) ? j0 + vb : n;
    double f0 = 0.0, f1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
      double w = oracle_weight(j - j0, vb);
      f0 += ncol[j] * ncol[j];
      f1 += (w * ncol[j]) * (w * ncol[j]);
    }
    for (int64_t l = 0; l < k; ++l) {
      double se = 0.0, sw = 0.0;
      for (int64_t j = j0; j < j1; ++j) {
        double b = B[l * ldb + j];
        se += b;
        sw += oracle_weight(j - j0, vb) * b;
      }
      q2 += se * se;
      q3 += sw * sw;
    }
    nblk[4 * J + 0] = sqrt(f0);
    nblk[4 * J + 1] = sqrt(f1);
    nblk[4 * J + 2] = sqrt(q2);
    nblk[4 * J + 3] = sqrt(q3);
  }
}

/* ------------------------------------------------------------------------ */
/* Configuration of a verify call. */
typedef struct {
  int64_t m, n, k;
  int64_t vb_r, vb_c; /* verify block sizes */
  int64_t p, q;       /* erasure grid, p = 0: none */
  double u_acc;       /* unit roundoff of the product's accumulation */
  double u_sum;       /* unit roundoff of the observed block sums */
  double u_enc;       /* unit roundoff of the checksum encoding sums */
  double u_c;         /* rounding of C's storage format relative to the accumulator */
  double u_cs;        /* relative representation error of the checksum operand */
  double s;           /* safety factor */
  int32_t round_f32;  /* corrected values are rounded to binary32 */
  int32_t f;          /* block checksum rows of the erasure grid (0 means 1) */
  /* Chained calls: bounds of the carried checksums' deviation from the sums
   * of the stored operand (see oracle_carry_rows); NULL when not chained. */
  const double* car_a; /* 2 per row verify block: unweighted, weighted */
  const double* car_b; /* 2 per column verify block */
} oracle_cfg;

typedef struct {
  int32_t row, col, kind, side; /* side: 0 column check, 1 row check, 2 block */
  double delta, r_e, r_w;
} oracle_fault;

/* Thresholds: a bound on |residual| for fault-free data under a
 * probabilistic rounding model -- a sum of n rounded terms errs by about
 * sqrt(n) u times the magnitude of its terms, and the independent errors of
 * the elements of a verify block add in quadrature -- with Cauchy-Schwarz
 * for the magnitudes.  For the column check of verify block I and column j:
 *   tau_e = s * ||B_j|| * (f1 * ||A_I||_F + f2 * ||e^T A_I||)
 *   tau_w = s * ||B_j|| * (f1 * ||diag(w) A_I||_F + f2 * ||w^T A_I||)
 *   f1 = sqrt(k) u_acc + sqrt(vb) (u_sum + u_enc) + u_c
 *   f2 = sqrt(k) u_acc + u_cs
 * (f1: accumulation of the block's elements, their block sum, the checksum
 * encoding and C's storage; f2: the checksum row's own product and its
 * representation).  The row check is the transposed formula.  The formula is
 * a reading of section 2.1; it is pinned by hand-worked values on a small
 * integer case, by the rigorous worst-case rounding bound of each residual
 * (every fault-free residual lies inside it and the threshold never exceeds
 * it), by the rounding model's predicted size of fault-free residuals for
 * N(0,1) data (the largest sits at a predictable fraction of the threshold),
 * and by exact integer data leaving residual 0. */
static void factors(const oracle_cfg* c, int64_t vb, double* f1, double* f2) {
  *f1 = sqrt((double)c->k) * c->u_acc + sqrt((double)vb) * (c->u_sum + c->u_enc) + c->u_c;
  *f2 = sqrt((double)c->k) * c->u_acc + c->u_cs;
}

/* In a chained call the threshold gains the carried deviation (car2: the two
 * bounds of the line's verify block, NULL when not chained):
 *   tau_e = s * ||B_j|| * (f1 * ||A_I||_F + f2 * ||e^T A_I|| + car_e(I)). */
static void taus(const oracle_cfg* c, int64_t vb, double nvec, const double* nb4,
                 const double* car2, double* te, double* tw) {
  double f1, f2;
  factors(c, vb, &f1, &f2);
  double ce = car2 ? car2[0] : 0.0, cw = car2 ? car2[1] : 0.0;
  *te = c->s * nvec * (f1 * nb4[0] + f2 * nb4[2] + ce);
  *tw = c->s * nvec * (f1 * nb4[1] + f2 * nb4[3] + cw);
}

static const double* car_col(const oracle_cfg* c, int64_t I) {
  return c->car_a ? &c->car_a[2 * I] : NULL;
}
static const double* car_row(const oracle_cfg* c, int64_t J) {
  return c->car_b ? &c->car_b[2 * J] : NULL;
}

/* The four thresholds that apply to element (i, j): those of its column line
 * (tau_e, tau_w) and of its row line (tau_e, tau_w), in that order. */
void oracle_thresholds_at(const oracle_cfg* c, const double* nArow, const double* nAblk,
                          const double* nBcol, const double* nBblk, int64_t i, int64_t j,
                          double* out4) {
  int64_t I = i / c->vb_r, J = j / c->vb_c;
  taus(c, c->vb_r, nBcol[j], &nAblk[4 * I], car_col(c, I), &out4[0], &out4[1]);
  taus(c, c->vb_c, nArow[i], &nBblk[4 * J], car_row(c, J), &out4[2], &out4[3]);
}

/* Does the line of rows [i0, i1) x columns [j0, j1) touch an erased block? */
static int touches_erased(const oracle_cfg* c, const int32_t* erased, int32_t n_erased, int64_t i0,
                          int64_t i1, int64_t j0, int64_t j1) {
  if (c->p <= 0 || n_erased <= 0) return 0;
  int64_t bs = c->m / c->p, bc = c->n / c->q;
  for (int32_t t = 0; t < n_erased; ++t) {
    int64_t r0 = erased[2 * t] * bs, c0 = erased[2 * t + 1] * bc;
    if (i0 < r0 + bs && r0 < i1 && j0 < c0 + bc && c0 < j1) return 1;
  }
  return 0;
}

/* Column residuals (Eq. (1): the checksum rows of the product must equal the
 * checksums of its data rows):
 *   re[I*n+j] = sum_{i in I} C_ij - E[2I][j],  rw = sum w_t C_ij - E[2I+1][j]
 * plus thresholds te, tw and the count of non-finite C_ij in the line. */
void oracle_col_residuals(const oracle_cfg* c, const double* C, int64_t ldc, const double* E,
                          const double* nBcol, const double* nAblk, double* re, double* rw,
                          double* te, double* tw, int32_t* nonfin) {
  int64_t m = c->m, n = c->n, vb = c->vb_r, nvb = ceil_div(m, vb);
  for (int64_t I = 0; I < nvb; ++I) {
    int64_t i0 = I * vb, i1 = (i0 + vb < m) ? i0 + vb : m;
    for (int64_t j = 0; j < n; ++j) {
      double se = 0.0, sw = 0.0;
      int32_t nf = 0;
      for (int64_t i = i0; i < i1; ++i) {
        double x = C[i * ldc + j];
        se += x;
        sw += oracle_weight(i - i0, vb) * x;
        if (!isfinite(x)) ++nf;
      }
      re[I * n + j] = se - E[(2 * I) * n + j];
      rw[I * n + j] = sw - E[(2 * I + 1) * n + j];
      taus(c, vb, nBcol[j], &nAblk[4 * I], car_col(c, I), &te[I * n + j], &tw[I * n + j]);
      nonfin[I * n + j] = nf;
    }
  }
}

/* Row residuals: re[i*nvb+J] = sum_{j in J} C_ij - F[i][2J], rw likewise. */
void oracle_row_residuals(const oracle_cfg* c, const double* C, int64_t ldc, const double* F,
                          const double* nArow, const double* nBblk, double* re, double* rw,
                          double* te, double* tw, int32_t* nonfin) {
  int64_t m = c->m, n = c->n, vb = c->vb_c, nvb = ceil_div(n, vb);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t J = 0; J < nvb; ++J) {
      int64_t j0 = J * vb, j1 = (j0 + vb < n) ? j0 + vb : n;
      double se = 0.0, sw = 0.0;
      int32_t nf = 0;
      for (int64_t j = j0; j < j1; ++j) {
        double x = C[i * ldc + j];
        se += x;
        sw += oracle_weight(j - j0, vb) * x;
        if (!isfinite(x)) ++nf;
      }
      re[i * nvb + J] = se - F[i * (2 * nvb) + 2 * J];
      rw[i * nvb + J] = sw - F[i * (2 * nvb) + 2 * J + 1];
      taus(c, vb, nArow[i], &nBblk[4 * J], car_row(c, J), &te[i * nvb + J], &tw[i * nvb + J]);
      nonfin[i * nvb + J] = nf;
    }
}

/* flagged: not (|r_e| <= tau_e and |r_w| <= tau_w); a NaN residual fails the
 * comparison and is flagged. */
static int flagged(double re, double rw, double te, double tw) {
  return !(fabs(re) <= te && fabs(rw) <= tw);
}

/* Single-error location inside one line of `len` elements (nominal block
 * size vb) from the ratio of weighted to unweighted residual: rho =
 * 2^ceil(log2 vb) * r_w / r_e must lie within 0.25 of an integer in
 * [1, len].  Returns the 0-based offset or -1. */
static int64_t locate_ratio(double re, double rw, int64_t vb, int64_t len) {
  if (!(re != 0.0) || !isfinite(re) || !isfinite(rw)) return -1;
  double rho = ldexp(rw / re, ceil_log2(vb));
  if (!isfinite(rho)) return -1;
  double r = nearbyint(rho);
  if (!(fabs(rho - r) <= 0.25)) return -1;
  if (r < 1.0 || r > (double)len) return -1;
  return (int64_t)r - 1;
}

/* Residual of one column line (verify block I, column j) and one row line
 * (row i, verify block J); the same sums as the residual arrays above. */
static int col_line_flagged(const oracle_cfg* c, const double* C, int64_t ldc, const double* E,
                            const double* nBcol, const double* nAblk, int64_t I, int64_t j,
                            double* re, double* rw) {
  int64_t vb = c->vb_r, i0 = I * vb, i1 = (i0 + vb < c->m) ? i0 + vb : c->m;
  double se = 0.0, sw = 0.0, te, tw;
  for (int64_t i = i0; i < i1; ++i) {
    se += C[i * ldc + j];
    sw += oracle_weight(i - i0, vb) * C[i * ldc + j];
  }
  *re = se - E[(2 * I) * c->n + j];
  *rw = sw - E[(2 * I + 1) * c->n + j];
  taus(c, vb, nBcol[j], &nAblk[4 * I], car_col(c, I), &te, &tw);
  return flagged(*re, *rw, te, tw);
}

static int row_line_flagged(const oracle_cfg* c, const double* C, int64_t ldc, const double* F,
                            const double* nArow, const double* nBblk, int64_t i, int64_t J,
                            double* re, double* rw) {
  int64_t vb = c->vb_c, nvb = ceil_div(c->n, vb), j0 = J * vb, j1 = (j0 + vb < c->n) ? j0 + vb : c->n;
  double se = 0.0, sw = 0.0, te, tw;
  for (int64_t j = j0; j < j1; ++j) {
    se += C[i * ldc + j];
    sw += oracle_weight(j - j0, vb) * C[i * ldc + j];
  }
  *re = se - F[i * (2 * nvb) + 2 * J];
  *rw = sw - F[i * (2 * nvb) + 2 * J + 1];
  taus(c, vb, nArow[i], &nBblk[4 * J], car_row(c, J), &te, &tw);
  return flagged(*re, *rw, te, tw);
}

typedef struct {
  int64_t row, col;
  int kind, side;
  double r_e, r_w;
} cand_t;

static int cand_cmp(const void* a, const void* b) {
  const cand_t* x = (const cand_t*)a;
  const cand_t* y = (const cand_t*)b;
  if (x->row != y->row) return x->row < y->row ? -1 : 1;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  return 0;
}

static int fault_cmp(const void* a, const void* b) {
  const oracle_fault* x = (const oracle_fault*)a;
  const oracle_fault* y = (const oracle_fault*)b;
  if (x->row != y->row) return x->row < y->row ? -1 : 1;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  if (x->kind != y->kind) return x->kind < y->kind ? -1 : 1;
  return 0;
}

static void push_report(oracle_fault* rep, int32_t max_rep, int32_t* n, int32_t row, int32_t col,
                        int kind, int side, double delta, double re, double rw) {
  if (*n < max_rep) {
    rep[*n].row = row;
    rep[*n].col = col;
    rep[*n].kind = kind;
    rep[*n].side = side;
    rep[*n].delta = delta;
    rep[*n].r_e = re;
    rep[*n].r_w = rw;
  }
  ++*n;
}

/* ------------------------------------------------------------------------ */
/* Detect, locate and correct (section 1 and section 2.2: consistency of
 * (AB)_F "enables us to detect, localize and correct errors").  Steps, in
 * order:
 *  1. residuals of every column line (verify block I, column j) and every row
 *     line (row i, verify block J), skipping lines that touch an erased block
 *     (listed as (bi, bj) pairs of the erasure grid);
 *  2. a line is flagged when a residual exceeds its threshold or is NaN;
 *  3. each flagged line proposes a candidate: its single non-finite element
 *     when it has non-finite elements, otherwise the ratio position;
 *  4. candidates from both checks are merged (same element counted once);
 *     a flagged line holding no candidate is reported uncorrectable;
 *  5. each candidate is corrected by recomputation from a line in which it
 *     is the only candidate -- C_ij = E - sum of the other elements of its
 *     column line, or F - sum of the other elements of its row line; when it
 *     is alone in both, the line with the smaller unweighted threshold (the
 *     more accurate recomputation for lines of very different magnitude),
 *     the column line on a tie -- otherwise it is reported uncorrectable and
 *     left untouched;
 *  6. the column line and the row line of every corrected element are
 *     checked again; a line still flagged is reported uncorrectable (this
 *     catches several errors sharing lines, which the ratio cannot separate);
 *  7. the report is sorted by (row, col, kind).
 * C is modified in place.  Returns ST_OK or ST_UNCORRECTABLE; *n_rep is the
 * full number of entries (only the first max_rep are stored). */
int oracle_verify_correct(const oracle_cfg* c, double* C, int64_t ldc, const double* E,
                          const double* F, const double* nArow, const double* nAblk,
                          const double* nBcol, const double* nBblk, const int32_t* erased,
                          int32_t n_erased, oracle_fault* rep, int32_t max_rep, int32_t* n_rep) {
  int64_t m = c->m, n = c->n;
  if (m <= 0 || n <= 0 || c->vb_r <= 0 || c->vb_c <= 0) return ST_INVALID;
  if (c->p > 0 && (c->q <= 0 || m % c->p || n % c->q)) return ST_INVALID;
  int64_t nvr = ceil_div(m, c->vb_r), nvc = ceil_div(n, c->vb_c);
  size_t ncl = (size_t)(nvr * n), nrl = (size_t)(m * nvc);
  double* cre = malloc(ncl * sizeof(double));
  double* crw = malloc(ncl * sizeof(double));
  double* cte = malloc(ncl * sizeof(double));
  double* ctw = malloc(ncl * sizeof(double));
  int32_t* cnf = malloc(ncl * sizeof(int32_t));
  double* rre = malloc(nrl * sizeof(double));
  double* rrw = malloc(nrl * sizeof(double));
  double* rte = malloc(nrl * sizeof(double));
  double* rtw = malloc(nrl * sizeof(double));
  int32_t* rnf = malloc(nrl * sizeof(int32_t));
  oracle_col_residuals(c, C, ldc, E, nBcol, nAblk, cre, crw, cte, ctw, cnf);
  oracle_row_residuals(c, C, ldc, F, nArow, nBblk, rre, rrw, rte, rtw, rnf);

  /* flagged lines and their candidates */
  size_t cap = 64, nc = 0;
  cand_t* cand = malloc(cap * sizeof(cand_t));
  size_t fcap = 64, nfl = 0;
  int64_t* fl = malloc(fcap * 2 * sizeof(int64_t)); /* (side, index) */
#define PUSH_CAND(R, Cc, KIND, SIDE, RE, RW)                 \
  do {                                                       \
    if (nc == cap) {                                         \
      cap *= 2;                                              \
      cand = realloc(cand, cap * sizeof(cand_t));            \
    }                                                        \
    cand[nc].row = (R);                                      \
    cand[nc].col = (Cc);                                     \
    cand[nc].kind = (KIND);                                  \
    cand[nc].side = (SIDE);                                  \
    cand[nc].r_e = (RE);                                     \
    cand[nc].r_w = (RW);                                     \
    ++nc;                                                    \
  } while (0)
#define PUSH_FLAG(SIDE, IDX)                                 \
  do {                                                       \
    if (nfl == fcap) {                                       \
      fcap *= 2;                                             \
      fl = realloc(fl, fcap * 2 * sizeof(int64_t));          \
    }                                                        \
    fl[2 * nfl] = (SIDE);                                    \
    fl[2 * nfl + 1] = (IDX);                                 \
    ++nfl;                                                   \
  } while (0)

  for (int64_t I = 0; I < nvr; ++I) {
    int64_t i0 = I * c->vb_r, i1 = (i0 + c->vb_r < m) ? i0 + c->vb_r : m;
    for (int64_t j = 0; j < n; ++j) {
      size_t x = (size_t)(I * n + j);
      if (touches_erased(c, erased, n_erased, i0, i1, j, j + 1)) continue;
      if (!flagged(cre[x], crw[x], cte[x], ctw[x]) && cnf[x] == 0) continue;
      PUSH_FLAG(0, (int64_t)x);
      if (cnf[x] > 0) {
        if (cnf[x] == 1)
          for (int64_t i = i0; i < i1; ++i)
            if (!isfinite(C[i * ldc + j])) PUSH_CAND(i, j, K_NONFINITE, 0, cre[x], crw[x]);
      } else {
        int64_t t = locate_ratio(cre[x], crw[x], c->vb_r, i1 - i0);
        if (t >= 0) PUSH_CAND(i0 + t, j, K_CORRECTED, 0, cre[x], crw[x]);
      }
    }
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t J = 0; J < nvc; ++J) {
      int64_t j0 = J * c->vb_c, j1 = (j0 + c->vb_c < n) ? j0 + c->vb_c : n;
      size_t x = (size_t)(i * nvc + J);
      if (touches_erased(c, erased, n_erased, i, i + 1, j0, j1)) continue;
      if (!flagged(rre[x], rrw[x], rte[x], rtw[x]) && rnf[x] == 0) continue;
      PUSH_FLAG(1, (int64_t)x);
      if (rnf[x] > 0) {
        if (rnf[x] == 1)
          for (int64_t j = j0; j < j1; ++j)
            if (!isfinite(C[i * ldc + j])) PUSH_CAND(i, j, K_NONFINITE, 1, rre[x], rrw[x]);
      } else {
        int64_t t = locate_ratio(rre[x], rrw[x], c->vb_c, j1 - j0);
        if (t >= 0) PUSH_CAND(i, j0 + t, K_CORRECTED, 1, rre[x], rrw[x]);
      }
    }

  /* merge: sort by position, keep one per element (column-check entry
   * first, non-finite kind wins) */
  qsort(cand, nc, sizeof(cand_t), cand_cmp);
  size_t nu = 0;
  for (size_t t = 0; t < nc; ++t) {
    if (nu > 0 && cand[nu - 1].row == cand[t].row && cand[nu - 1].col == cand[t].col) {
      if (cand[t].kind == K_NONFINITE) cand[nu - 1].kind = K_NONFINITE;
      if (cand[t].side < cand[nu - 1].side) {
        cand[nu - 1].side = cand[t].side;
        cand[nu - 1].r_e = cand[t].r_e;
        cand[nu - 1].r_w = cand[t].r_w;
      }
      continue;
    }
    cand[nu++] = cand[t];
  }
  nc = nu;

  int32_t nr = 0;
  int status = ST_OK;
  /* flagged lines without a candidate */
  for (size_t f = 0; f < nfl; ++f) {
    int64_t side = fl[2 * f], x = fl[2 * f + 1];
    int has = 0;
    if (side == 0) {
      int64_t I = x / n, j = x % n;
      for (size_t t = 0; t < nc && !has; ++t)
        has = cand[t].col == j && cand[t].row / c->vb_r == I;
      if (!has) {
        push_report(rep, max_rep, &nr, -1, (int32_t)j, K_UNCORRECTABLE, 0, 0.0, cre[x], crw[x]);
        status = ST_UNCORRECTABLE;
      }
    } else {
      int64_t i = x / nvc, J = x % nvc;
      for (size_t t = 0; t < nc && !has; ++t)
        has = cand[t].row == i && cand[t].col / c->vb_c == J;
      if (!has) {
        push_report(rep, max_rep, &nr, (int32_t)i, -1, K_UNCORRECTABLE, 1, 0.0, rre[x], rrw[x]);
        status = ST_UNCORRECTABLE;
      }
    }
  }
  /* choose a correcting line per candidate, then correct (the choices are
   * made before any value changes; the chosen lines hold no other
   * candidate, so the corrections do not interact) */
  int* how = malloc((nc ? nc : 1) * sizeof(int));
  for (size_t t = 0; t < nc; ++t) {
    int64_t I = cand[t].row / c->vb_r, J = cand[t].col / c->vb_c;
    int ncol = 0, nrow = 0;
    for (size_t u = 0; u < nc; ++u) {
      if (cand[u].col == cand[t].col && cand[u].row / c->vb_r == I) ++ncol;
      if (cand[u].row == cand[t].row && cand[u].col / c->vb_c == J) ++nrow;
    }
    how[t] = ncol == 1 ? 0 : (nrow == 1 ? 1 : -1);
    /* alone in both lines: recompute from the line whose unweighted threshold
     * (the scale of its rounding errors) is smaller; ties take the column */
    if (ncol == 1 && nrow == 1 && rte[cand[t].row * nvc + J] < cte[I * n + cand[t].col]) how[t] = 1;
  }
  for (size_t t = 0; t < nc; ++t) {
    int64_t i = cand[t].row, j = cand[t].col;
    double old = C[i * ldc + j];
    if (how[t] < 0) {
      push_report(rep, max_rep, &nr, (int32_t)i, (int32_t)j, K_UNCORRECTABLE, cand[t].side, 0.0,
                  cand[t].r_e, cand[t].r_w);
      status = ST_UNCORRECTABLE;
      continue;
    }
    double v;
    if (how[t] == 0) {
      int64_t I = i / c->vb_r, i0 = I * c->vb_r, i1 = (i0 + c->vb_r < m) ? i0 + c->vb_r : m;
      double s = 0.0;
      for (int64_t r = i0; r < i1; ++r)
        if (r != i) s += C[r * ldc + j];
      v = E[(2 * I) * n + j] - s;
    } else {
      int64_t J = j / c->vb_c, j0 = J * c->vb_c, j1 = (j0 + c->vb_c < n) ? j0 + c->vb_c : n;
      double s = 0.0;
      for (int64_t q = j0; q < j1; ++q)
        if (q != j) s += C[i * ldc + q];
      v = F[i * (2 * nvc) + 2 * J] - s;
    }
    if (c->round_f32) v = (double)(float)v;
    C[i * ldc + j] = v;
    push_report(rep, max_rep, &nr, (int32_t)i, (int32_t)j, cand[t].kind, cand[t].side, old - v,
                cand[t].r_e, cand[t].r_w);
  }
  /* re-check the lines of the corrected elements (each line once) */
  for (size_t t = 0; t < nc; ++t) {
    if (how[t] < 0) continue;
    int64_t i = cand[t].row, j = cand[t].col, I = i / c->vb_r, J = j / c->vb_c;
    int dup_c = 0, dup_r = 0;
    for (size_t u = 0; u < t; ++u) {
      if (how[u] < 0) continue;
      if (cand[u].col == j && cand[u].row / c->vb_r == I) dup_c = 1;
      if (cand[u].row == i && cand[u].col / c->vb_c == J) dup_r = 1;
    }
    double re, rw;
    if (!dup_c && col_line_flagged(c, C, ldc, E, nBcol, nAblk, I, j, &re, &rw)) {
      push_report(rep, max_rep, &nr, -1, (int32_t)j, K_UNCORRECTABLE, 0, 0.0, re, rw);
      status = ST_UNCORRECTABLE;
    }
    if (!dup_r && row_line_flagged(c, C, ldc, F, nArow, nBblk, i, J, &re, &rw)) {
      push_report(rep, max_rep, &nr, (int32_t)i, -1, K_UNCORRECTABLE, 1, 0.0, re, rw);
      status = ST_UNCORRECTABLE;
    }
  }
  int32_t stored = nr < max_rep ? nr : max_rep;
  if (stored > 0) qsort(rep, (size_t)stored, sizeof(oracle_fault), fault_cmp);
  *n_rep = nr;

  free(how);
  free(cand);
  free(fl);
  free(cre);
  free(crw);
  free(cte);
  free(ctw);
  free(cnf);
  free(rre);
  free(rrw);
  free(rte);
  free(rtw);
  free(rnf);
#undef PUSH_CAND
#undef PUSH_FLAG
  return status;
}

/* ------------------------------------------------------------------------ */
/* Erasure recovery (section 2.1: the lost part is the checksum minus the
 * surviving parts; section 3.3: this is the paper's reduction step).  With S
 * the block checksum rows of the product (rows 2*nvb .. 2*nvb+bs-1 of E):
 *   C[bi*bs + t][j] = S[t][j] - sum_{I != bi} C[I*bs + t][j],
 * for t in [0, bs) and j in block column bj.  Afterwards the column checks
 * of the rebuilt block are recomputed; *n_flagged gets the number of its
 * column lines that still exceed their thresholds.  Pinned by exact integer
 * recovery and by re-verification. */
int oracle_recover_block(const oracle_cfg* c, double* C, int64_t ldc, const double* E,
                         const double* nBcol, const double* nAblk, int32_t bi, int32_t bj,
                         int32_t* n_flagged) {
  int64_t m = c->m, n = c->n;
  if (c->p <= 0 || c->q <= 0 || m % c->p || n % c->q) return ST_INVALID;
  int64_t bs = m / c->p, bc = n / c->q;
  if (bi < 0 || bi >= c->p || bj < 0 || bj >= c->q) return ST_INVALID;
  int64_t nvr = ceil_div(m, c->vb_r);
  const double* S = E + (2 * nvr) * n;
  for (int64_t t = 0; t < bs; ++t)
    for (int64_t j = bj * bc; j < (bj + 1) * bc; ++j) {
      double s = 0.0;
      for (int64_t I = 0; I < c->p; ++I)
        if (I != bi) s += C[(I * bs + t) * ldc + j];
      double v = S[t * n + j] - s;
      if (c->round_f32) v = (double)(float)v;
      C[(bi * bs + t) * ldc + j] = v;
    }
  /* re-verify the rebuilt block's column lines */
  int32_t nfl = 0;
  int64_t vb = c->vb_r;
  for (int64_t I = (bi * bs) / vb; I < ceil_div((bi + 1) * bs, vb); ++I) {
    for (int64_t j = bj * bc; j < (bj + 1) * bc; ++j) {
      double re, rw;
      if (col_line_flagged(c, C, ldc, E, nBcol, nAblk, I, j, &re, &rw)) ++nfl;
    }
  }
  *n_flagged = nfl;
  return nfl ? ST_UNCORRECTABLE : ST_OK;
}

/* Erasure recovery of several blocks (section 2.1: the lost parts follow from
 * the checksums and the surviving parts; with f checksums, f lost blocks of a
 * block column).  The listed blocks (bi, bj pairs) are grouped by block
 * column; for a column J with t <= f erased block rows I_1..I_t, every element
 * position (r, j) of the column's blocks solves
 *   sum_u c_{l,I_u} C[I_u*bs + r][j] = S^(l)[r][j] - sum_{I not erased} c_{l,I} C[I*bs + r][j],
 *   l = 0 .. t-1,
 * by Gaussian elimination with partial pivoting in binary64 (rounded to
 * binary32 for a binary32 C).  A column with more erasures than f is left
 * untouched and reported (ST_UNCORRECTABLE).  Then every column line of the
 * rebuilt blocks is verified again; *n_flagged counts the lines still flagged.
 * Pinned by exact recovery of every subset of up to f blocks on integer
 * data, and by the single-block case agreeing with the plain sum. */
int oracle_recover_blocks(const oracle_cfg* c, double* C, int64_t ldc, const double* E,
                          const double* nBcol, const double* nAblk, const int32_t* blocks,
                          int32_t nb, int32_t* n_flagged) {
  int64_t m = c->m, n = c->n;
  if (c->p <= 0 || c->q <= 0 || m % c->p || n % c->q || nb < 0) return ST_INVALID;
  int64_t bs = m / c->p, bc = n / c->q, f = c->f > 0 ? c->f : 1;
  for (int32_t u = 0; u < nb; ++u)
    if (blocks[2 * u] < 0 || blocks[2 * u] >= c->p || blocks[2 * u + 1] < 0 ||
        blocks[2 * u + 1] >= c->q)
      return ST_INVALID;
  int64_t nvr = ceil_div(m, c->vb_r);
  const double* S = E + (2 * nvr) * n;
  int status = ST_OK;
  int32_t nfl = 0;
  int64_t rows[8];
  for (int64_t J = 0; J < c->q; ++J) {
    int64_t t = 0;
    int dup = 0;
    for (int32_t u = 0; u < nb; ++u)
      if (blocks[2 * u + 1] == J) {
        for (int64_t v = 0; v < t && v < 8; ++v) dup |= rows[v] == blocks[2 * u];
        if (t < 8) rows[t] = blocks[2 * u];
        ++t;
      }
    if (t == 0) continue;
    if (dup || t > f || t > 8) { status = ST_UNCORRECTABLE; continue; }
    for (int64_t r = 0; r < bs; ++r)
      for (int64_t j = J * bc; j < (J + 1) * bc; ++j) {
        double M[8][9];
        for (int64_t l = 0; l < t; ++l) {
          double sum = 0.0; /* the survivors, then checksum minus their sum */
          for (int64_t I = 0; I < c->p; ++I) {
            int erased = 0;
            for (int64_t v = 0; v < t; ++v) erased |= rows[v] == I;
            if (!erased) sum += oracle_block_coef(l, I, c->p) * C[(I * bs + r) * ldc + j];
          }
          double rhs = S[(l * bs + r) * n + j] - sum;
          for (int64_t v = 0; v < t; ++v) M[l][v] = oracle_block_coef(l, rows[v], c->p);
          M[l][t] = rhs;
        }
        /* Gaussian elimination with partial pivoting */
        for (int64_t col = 0; col < t; ++col) {
          int64_t piv = col;
          for (int64_t i = col + 1; i < t; ++i)
            if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
          for (int64_t x = 0; x <= t; ++x) {
            double tmp = M[col][x];
            M[col][x] = M[piv][x];
            M[piv][x] = tmp;
          }
          for (int64_t i = col + 1; i < t; ++i) {
            double fct = M[i][col] / M[col][col];
            for (int64_t x = col; x <= t; ++x) M[i][x] -= fct * M[col][x];
          }
        }
        double x[8];
        for (int64_t i = t - 1; i >= 0; --i) {
          double v = M[i][t];
          for (int64_t y = i + 1; y < t; ++y) v -= M[i][y] * x[y];
          x[i] = v / M[i][i];
        }
        for (int64_t v = 0; v < t; ++v) {
          double val = x[v];
          if (c->round_f32) val = (double)(float)val;
          C[(rows[v] * bs + r) * ldc + j] = val;
        }
      }
    /* re-verify the rebuilt blocks' column lines */
    for (int64_t v = 0; v < t; ++v) {
      int64_t vb = c->vb_r, bi = rows[v];
      for (int64_t I = (bi * bs) / vb; I < ceil_div((bi + 1) * bs, vb); ++I)
        for (int64_t j = J * bc; j < (J + 1) * bc; ++j) {
          double re, rw;
          if (col_line_flagged(c, C, ldc, E, nBcol, nAblk, I, j, &re, &rw)) ++nfl;
        }
    }
  }
  *n_flagged = nfl;
  if (nfl) status = ST_UNCORRECTABLE;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Chained calls (section 3.2: when ABFT BLAS routines are called one after
 * the other, the checksums are not recomputed between the calls).  A product
 * whose left operand A is the output C of an earlier product takes that
 * product's expected column checksum rows E (the unweighted and weighted row
 * of every verify block, then the block checksum rows) as its encoded rows of
 * A, without reading A for them; one whose right operand B is an earlier
 * output takes that product's expected row checksum columns F as its encoded
 * columns of B.  The norms that enter the thresholds are those of the
 * operand itself (||A_I||_F, ||A_i||) and of the carried rows / columns.
 *
 * A carried row is not the sum of the stored operand rows: it carries the
 * rounding of the earlier product (and of every product before it).  The
 * reading here bounds that deviation with the same rounding model as the
 * thresholds.  The column deviation d_I(j) = E[2I][j] - sum_{i in I} C_ij of
 * the earlier product stays within its unscaled threshold
 *   |d_I(j)| <= ||B_j|| (f1 ||A_I||_F + f2 ||e^T A_I|| + car_e(I)),
 * so its largest entry is at most
 *   car'_e(I) = max_j ||B_j|| * (f1 ||A_I||_F + f2 ||e^T A_I|| + car_e(I))
 * (car_e = 0 for a freshly encoded product; the weighted row likewise with
 * diag(w) A_I, w^T A_I and car_w).  In the next product the deviation enters
 * a column residual as sum_l d_I(l) B'_lj, whose independent terms add in
 * quadrature to at most car'(I) ||B'_j||: the next threshold adds car'(I)
 * inside its bracket (taus above).  The row side is the transpose, with
 * max_i ||A_i|| of the earlier product.  The bound is a reading of section
 * 3.2, pinned by hand-worked values of a two-product chain, by the rigorous
 * worst-case bound of the deviation (the actual deviation, computed exactly,
 * lies below this bound and this bound below the worst case), by exact zero
 * residuals on integer chains and by no false flag over seeds where the
 * uncarried threshold fails. */

/* nblk[4I+2], nblk[4I+3] = norms of the carried rows acs[2I], acs[2I+1]
 * (length len, leading dimension ld). */
void oracle_norms_carried_rows(int64_t nvb, int64_t len, const double* acs, int64_t ld,
                               double* nblk) {
  for (int64_t I = 0; I < nvb; ++I)
    for (int64_t c = 0; c < 2; ++c) {
      double q = 0.0;
      for (int64_t l = 0; l < len; ++l) q += acs[(2 * I + c) * ld + l] * acs[(2 * I + c) * ld + l];
      nblk[4 * I + 2 + c] = sqrt(q);
    }
}

/* nblk[4J+2], nblk[4J+3] = norms of the carried columns bcs[:, 2J], bcs[:, 2J+1]. */
void oracle_norms_carried_cols(int64_t len, int64_t nvb, const double* bcs, int64_t ld,
                               double* nblk) {
  for (int64_t J = 0; J < nvb; ++J)
    for (int64_t c = 0; c < 2; ++c) {
      double q = 0.0;
      for (int64_t l = 0; l < len; ++l) q += bcs[l * ld + 2 * J + c] * bcs[l * ld + 2 * J + c];
      nblk[4 * J + 2 + c] = sqrt(q);
    }
}

/* Deviation bound of the column checksum rows carried out of a product with
 * configuration prev, norms nAblk / nBcol (and its own carried bound
 * prev->car_a): car_out[2I+c] as above. */
void oracle_carry_rows(const oracle_cfg* prev, const double* nAblk, const double* nBcol,
                       double* car_out) {
  double f1, f2, mx = 0.0;
  factors(prev, prev->vb_r, &f1, &f2);
  for (int64_t j = 0; j < prev->n; ++j)
    if (nBcol[j] > mx) mx = nBcol[j];
  int64_t nvb = ceil_div(prev->m, prev->vb_r);
  for (int64_t I = 0; I < nvb; ++I)
    for (int64_t c = 0; c < 2; ++c) {
      double cp = prev->car_a ? prev->car_a[2 * I + c] : 0.0;
      car_out[2 * I + c] = mx * (f1 * nAblk[4 * I + c] + f2 * nAblk[4 * I + 2 + c] + cp);
    }
}

/* The row side: deviation bound of the row checksum columns carried out of
 * a product (max_i ||A_i|| of that product, its nBblk and prev->car_b). */
void oracle_carry_cols(const oracle_cfg* prev, const double* nBblk, const double* nArow,
                       double* car_out) {
  double f1, f2, mx = 0.0;
  factors(prev, prev->vb_c, &f1, &f2);
  for (int64_t i = 0; i < prev->m; ++i)
    if (nArow[i] > mx) mx = nArow[i];
  int64_t nvb = ceil_div(prev->n, prev->vb_c);
  for (int64_t J = 0; J < nvb; ++J)
    for (int64_t c = 0; c < 2; ++c) {
      double cp = prev->car_b ? prev->car_b[2 * J + c] : 0.0;
      car_out[2 * J + c] = mx * (f1 * nBblk[4 * J + c] + f2 * nBblk[4 * J + 2 + c] + cp);
    }
}

/* ------------------------------------------------------------------------ */
/* Residual check of the stress test (section 4.3):
 *   || C x - A (B x) ||_inf / ( nmax * eps * ||C||_inf * ||x||_inf )
 * with eps = 2^-52 (binary64 machine epsilon), nmax = max(m, n, k) and
 * ||C||_inf the largest absolute row sum.  Pinned by its own behaviour: small
 * for a correct product, large after a planted error. */
double oracle_residual_check(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                             const double* B, int64_t ldb, const double* C, int64_t ldc,
                             const double* x) {
  double* bx = malloc((size_t)(k > 0 ? k : 1) * sizeof(double));
  for (int64_t l = 0; l < k; ++l) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += B[l * ldb + j] * x[j];
    bx[l] = s;
  }
  double num = 0.0, cn = 0.0, xn = 0.0;
  for (int64_t j = 0; j < n; ++j)
    if (fabs(x[j]) > xn) xn = fabs(x[j]);
  for (int64_t i = 0; i < m; ++i) {
    double cx = 0.0, abx = 0.0, rs = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      cx += C[i * ldc + j] * x[j];
      rs += fabs(C[i * ldc + j]);
    }
    for (int64_t l = 0; l < k; ++l) abx += A[i * lda + l] * bx[l];
    double d = fabs(cx - abx);
    if (!(d <= num)) num = d; /* NaN propagates */
    if (rs > cn) cn = rs;
  }
  free(bx);
  int64_t nmax = m > n ? m : n;
  if (k > nmax) nmax = k;
  double den = (double)nmax * ldexp(1.0, -52) * cn * xn;
  return den > 0 ? num / den : (num > 0 ? INFINITY : 0.0);
}

/* ------------------------------------------------------------------------ */
/* Input format decoders (plain definitions of the storage formats, so the
 * oracle works on exactly the values the GPU multiplies). */

/* bfloat16: the upper 16 bits of a binary32. */
void oracle_bf16_to_f64(const uint16_t* x, int64_t count, double* out) {
  for (int64_t t = 0; t < count; ++t) {
    uint32_t u = (uint32_t)x[t] << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    out[t] = (double)f;
  }
}

/* OCP FP8 E4M3 ("e4m3fn"): 1 sign, 4 exponent bits (bias 7), 3 mantissa
 * bits, no infinities, S.1111.111 is NaN, subnormals at exponent 0. */
double oracle_e4m3_value(uint8_t b) {
  int s = (b >> 7) & 1, e = (b >> 3) & 15, f = b & 7;
  double v;
  if (e == 15 && f == 7) return NAN;
  if (e == 0)
    v = ldexp((double)f, -9); /* f/8 * 2^(1-7) */
  else
    v = ldexp(1.0 + f / 8.0, e - 7);
  return s ? -v : v;
}

/* Dequantise a rows-by-cols E4M3 matrix with one binary32 scale per
 * blk-by-blk block (row-major scale grid of ceil(rows/blk) x ceil(cols/blk)). */
void oracle_dequant_e4m3(int64_t rows, int64_t cols, const uint8_t* q, const float* scale,
                         int64_t blk, double* out) {
  int64_t sc = ceil_div(cols, blk);
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t j = 0; j < cols; ++j)
      out[i * cols + j] = oracle_e4m3_value(q[i * cols + j]) * (double)scale[(i / blk) * sc + j / blk];
}
