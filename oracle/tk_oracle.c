/*
 * tk_oracle.c -- plain, slow, FP64 CPU oracle for randomized Tikhonov
 * regularization (Meier & Nakatsukasa, "Randomized algorithms for Tikhonov
 * regularization in Linear Least Squares").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py may load this library.  The product path (the CUDA
 * library) shares no code, header, table or helper with this file.
 *
 * Everything is double precision, row-major, written as the plain loops of the
 * definitions: no blocking, no reordering beyond what a definition states.
 * Build with -ffp-contract=off so that a*b+c is never silently fused (the
 * double-double helpers rely on it, and x86/Arm hosts then agree bit for bit
 * except inside libm's log/sin/cos).
 *
 * Sections follow the paper:
 *   problem (1.2)-(1.4) ............ ridge LLS, B = [A; sqrt(l) I], D = [A sqrt(l) I]
 *   Section 2.1.1 .................. SRTT X = sqrt(m/s) S F D, Gaussian and sparse embeddings
 *   Algorithm 1 .................... Y = XA, C = Y^T Y, R_i = chol(C + l_i I), LSQR, x = R^-1 y
 *   Algorithm 2 .................... Y = AX, C = Y Y^T, min-norm LSQR on R^-T D
 *   Section 3.1, eq. (RinvOver) .... R^-1 = l^{-1/2} (I - V S V^T)
 *   Algorithm 3, Section 3.1.2 ..... SVD of Y, sd estimate, truncation s_i
 *   LSQR (Paige & Saunders 1982) ... the inner solver the paper uses throughout
 * plus a dense reference (Householder QR, double-double refinement) for the
 * unique ridge solution x_l = (A^T A + l I)^-1 A^T b.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11) */
/* ------------------------------------------------------------------------ */
/* Round function: two 32x32->64 multiplies, xor with the other two words and
 * the round key; the key is bumped by the Weyl constants between rounds. */
static void mul32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hA, lA, hB, lB;
    mul32(0xD2511F53u, x0, &hA, &lA);
    mul32(0xCD9E8D57u, x2, &hB, &lB);
    uint32_t y0 = hB ^ x1 ^ k0;
    uint32_t y1 = lB;
    uint32_t y2 = hA ^ x3 ^ k1;
    uint32_t y3 = lA;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Draw convention: key = seed (low word, high word); counter =
 * (index low word, index high word, stream, 0).  Stream 0: Rademacher signs,
 * stream 1: row-sampling keys, stream 2: Gaussian entries, stream 4: the
 * sparse embedding's rows and signs. */
static void draw(uint64_t seed, uint64_t index, uint32_t stream, uint32_t w[4]) {
  uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), stream, 0u};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(c, k, w);
}

/* Section 2.1.1: D is a diagonal of independent random signs. d_i = -1 when
 * the low bit of word 0 is set, +1 otherwise. */
ORC_API void orc_draw_signs(uint64_t seed, int64_t mp, int8_t* d) {
  for (int64_t i = 0; i < mp; ++i) {
    uint32_t w[4];
    draw(seed, (uint64_t)i, 0u, w);
    d[i] = (w[0] & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

ORC_API void orc_draw_keys(uint64_t seed, int64_t mp, uint64_t* keys) {
  for (int64_t i = 0; i < mp; ++i) {
    uint32_t w[4];
    draw(seed, (uint64_t)i, 1u, w);
    keys[i] = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
  }
}

typedef struct { uint64_t key; int64_t idx; } keyidx;
static int cmp_keyidx(const void* a, const void* b) {
  const keyidx* x = (const keyidx*)a;
  const keyidx* y = (const keyidx*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}
static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Section 2.1.1: S keeps a random subset of s of the mp rows (without
 * replacement).  Each row gets a 64-bit key; the subset is the s smallest
 * (key, row) pairs in lexicographic order; rows are returned ascending.
 * Returns 0, or -1 when s is out of range. */
ORC_API int orc_draw_rows(uint64_t seed, int64_t mp, int64_t s, int64_t* rows) {
  if (s < 0 || s > mp) return -1;
  keyidx* all = (keyidx*)malloc(sizeof(keyidx) * (size_t)(mp > 0 ? mp : 1));
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(mp > 0 ? mp : 1));
  orc_draw_keys(seed, mp, keys);
  for (int64_t i = 0; i < mp; ++i) { all[i].key = keys[i]; all[i].idx = i; }
  qsort(all, (size_t)mp, sizeof(keyidx), cmp_keyidx);
  for (int64_t k = 0; k < s; ++k) rows[k] = all[k].idx;
  qsort(rows, (size_t)s, sizeof(int64_t), cmp_i64);
  free(all);
  free(keys);
  return 0;
}

/* Section 2.1.1 (Gaussian embedding): s x L matrix G with entries N(0, 1/s),
 * so that E[G^T G] = I.  Entry k = i*L + j uses Philox call k/4 of stream 2;
 * words (w0,w1) give two normals by Box-Muller, (w2,w3) the next two:
 * u1 = (w0+1) 2^-32 in (0,1], u2 = w1 2^-32 in [0,1),
 * r = sqrt(-2 ln u1), z = r cos(2 pi u2), r sin(2 pi u2). */
ORC_API double orc_gauss_entry(uint64_t seed, uint64_t k, double inv_sqrt_s) {
  uint32_t w[4];
  draw(seed, k >> 2, 2u, w);
  int lane = (int)(k & 3u);
  int p = lane >> 1;
  double u1 = ((double)w[2 * p] + 1.0) * 2.3283064365386962890625e-10;
  double u2 = (double)w[2 * p + 1] * 2.3283064365386962890625e-10;
  double r = sqrt(-2.0 * log(u1));
  double t = 6.283185307179586476925286766559 * u2; /* 2 pi */
  double z = (lane & 1) ? r * sin(t) : r * cos(t);
  return z * inv_sqrt_s;
}

ORC_API void orc_draw_gauss(uint64_t seed, int64_t s, int64_t L, double* G) {
  double inv = 1.0 / sqrt((double)s);
  for (int64_t i = 0; i < s; ++i)
    for (int64_t j = 0; j < L; ++j) G[i * L + j] = orc_gauss_entry(seed, (uint64_t)(i * L + j), inv);
}

ORC_API int64_t orc_next_pow2(int64_t m) {
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}

/* ------------------------------------------------------------------------ */
/* Sketches (Section 2.1.1; Algorithm 1 step 2, Algorithm 2 step 2)           */
/* ------------------------------------------------------------------------ */
/* Unnormalized fast Walsh-Hadamard transform, Sylvester order:
 * z <- H z with H_1 = [1], H_{2k} = [[H_k, H_k], [H_k, -H_k]]. */
ORC_API void orc_fwht(double* z, int64_t len) {
  for (int64_t h = 1; h < len; h <<= 1)
    for (int64_t i = 0; i < len; i += 2 * h)
      for (int64_t j = i; j < i + h; ++j) {
        double a = z[j], b = z[j + h];
        z[j] = a + b;
        z[j + h] = a - b;
      }
}

/* SRHT, overdetermined: Y = sqrt(mp/s) S (H/sqrt(mp)) D [A; 0]  (s x n),
 * which simplifies to Y = (1/sqrt(s)) S H D [A; 0].  A is m x n (row stride
 * lda), zero-padded to mp = next power of two rows. */
ORC_API void orc_srht_over(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                           double* Y) {
  int64_t mp = orc_next_pow2(m);
  int8_t* d = (int8_t*)malloc((size_t)mp);
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)mp);
  orc_draw_signs(seed, mp, d);
  orc_draw_rows(seed, mp, s, rows);
  double scale = 1.0 / sqrt((double)s);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < mp; ++i) z[i] = (i < m) ? (double)d[i] * A[i * lda + j] : 0.0;
    orc_fwht(z, mp);
    for (int64_t k = 0; k < s; ++k) Y[k * n + j] = scale * z[rows[k]];
  }
  free(d); free(rows); free(z);
}

/* SRHT, underdetermined (sketch from the right, Algorithm 2): the n x s
 * embedding X = sqrt(np/s) D (H/sqrt(np)) S^T acts on the columns, so
 * Y = A X = (1/sqrt(s)) [A 0] D H S^T  (m x s), np = next power of two >= n. */
ORC_API void orc_srht_under(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                            double* Y) {
  int64_t np = orc_next_pow2(n);
  int8_t* d = (int8_t*)malloc((size_t)np);
  int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)np);
  orc_draw_signs(seed, np, d);
  orc_draw_rows(seed, np, s, cols);
  double scale = 1.0 / sqrt((double)s);
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < np; ++j) z[j] = (j < n) ? (double)d[j] * A[i * lda + j] : 0.0;
    orc_fwht(z, np);
    for (int64_t k = 0; k < s; ++k) Y[i * s + k] = scale * z[cols[k]];
  }
  free(d); free(cols); free(z);
}

/* Gaussian sketch, overdetermined: Y = G A with G (s x m) from orc_draw_gauss. */
ORC_API void orc_gauss_over(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                            double* Y) {
  double inv = 1.0 / sqrt((double)s);
  for (int64_t k = 0; k < s; ++k)
    for (int64_t j = 0; j < n; ++j) Y[k * n + j] = 0.0;
  for (int64_t k = 0; k < s; ++k)
    for (int64_t i = 0; i < m; ++i) {
      double g = orc_gauss_entry(seed, (uint64_t)(k * m + i), inv);
      for (int64_t j = 0; j < n; ++j) Y[k * n + j] += g * A[i * lda + j];
    }
}

/* Gaussian sketch, underdetermined: Y = A G^T (m x s), G (s x n), i.e. the
 * n x s embedding is X = G^T. */
ORC_API void orc_gauss_under(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                             double* Y) {
  double inv = 1.0 / sqrt((double)s);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = 0; k < s; ++k) {
      double acc = 0.0;
      for (int64_t j = 0; j < n; ++j) acc += A[i * lda + j] * orc_gauss_entry(seed, (uint64_t)(k * n + j), inv);
      Y[i * s + k] = acc;
    }
}

/* SRDCT (Section 2.1.1 with F the discrete cosine transform, the embedding of
 * the paper's Fig. 1 and 2): X = sqrt(mp/s) S C D [I; 0], C the orthonormal
 * DCT-II of length mp (the next power of two, as for the SRHT),
 *   C[k][i] = a_k cos(pi (2i + 1) k / (2 mp)),  a_0 = sqrt(1/mp), a_k = sqrt(2/mp),
 * D and S the SRHT's signs (stream 0) and row subset (stream 1).  Only the s
 * sampled rows of C D [A; 0] are formed, each by its defining sum. */
ORC_API void orc_dct2_rows(const double* z, int64_t N, const int64_t* rows, int64_t s, double* out) {
  for (int64_t q = 0; q < s; ++q) {
    const int64_t k = rows[q];
    const double a = k == 0 ? sqrt(1.0 / (double)N) : sqrt(2.0 / (double)N);
    double acc = 0.0;
    /* the angle's integer part reduced modulo 4 mp first (cos has period 2 pi), so the argument stays
     * below 2 pi and carries no error from a large multiple of pi */
    for (int64_t i = 0; i < N; ++i) {
      const int64_t r = ((2 * i + 1) * k) % (4 * N);
      acc += z[i] * cos(3.14159265358979323846 * (double)r / (double)(2 * N));
    }
    out[q] = a * acc;
  }
}

ORC_API void orc_srdct_over(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                            double* Y) {
  const int64_t mp = orc_next_pow2(m);
  int8_t* d = (int8_t*)malloc((size_t)mp);
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)mp);
  double* o = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
  orc_draw_signs(seed, mp, d);
  orc_draw_rows(seed, mp, s, rows);
  const double scale = sqrt((double)mp / (double)s);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < mp; ++i) z[i] = (i < m) ? (double)d[i] * A[i * lda + j] : 0.0;
    orc_dct2_rows(z, mp, rows, s, o);
    for (int64_t k = 0; k < s; ++k) Y[k * n + j] = scale * o[k];
  }
  free(d); free(rows); free(z); free(o);
}

/* SRDCT on the columns (Algorithm 2): Y = A X^T = sqrt(np/s) [A 0] D C^T S^T (m x s). */
ORC_API void orc_srdct_under(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                             double* Y) {
  const int64_t np = orc_next_pow2(n);
  int8_t* d = (int8_t*)malloc((size_t)np);
  int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)np);
  double* o = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
  orc_draw_signs(seed, np, d);
  orc_draw_rows(seed, np, s, cols);
  const double scale = sqrt((double)np / (double)s);
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < np; ++j) z[j] = (j < n) ? (double)d[j] * A[i * lda + j] : 0.0;
    orc_dct2_rows(z, np, cols, s, o);
    for (int64_t k = 0; k < s; ++k) Y[i * s + k] = scale * o[k];
  }
  free(d); free(cols); free(z); free(o);
}

/* Sparse embedding (Section 2.1.1: one nonzero element in each column; the
 * sparse subspace embedding of Theorem 3.5).  Column i of the s x L matrix X
 * holds sign_i in row h_i, both from Philox stream 4 at index i:
 *   h_i = floor(w0 * s / 2^32)  (multiply-shift: uniform over 0..s-1 to within
 *         s / 2^32), sign_i = -1 when the low bit of w1 is set, +1 otherwise.
 * Every column has unit norm, so E[X^T X] = I with no scaling. */
ORC_API void orc_draw_sparse(uint64_t seed, int64_t L, int64_t s, int32_t* h, int8_t* sign) {
  for (int64_t i = 0; i < L; ++i) {
    uint32_t w[4];
    draw(seed, (uint64_t)i, 4u, w);
    h[i] = (int32_t)(((uint64_t)w[0] * (uint64_t)s) >> 32);
    sign[i] = (w[1] & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

/* Sparse sketch, overdetermined: Y = X A (s x n): Y[h_i] += sign_i A[i] for
 * i = 0..m-1 in ascending order (that order fixes every float64 sum). */
ORC_API void orc_sparse_over(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                             double* Y) {
  int32_t* h = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int8_t* d = (int8_t*)malloc((size_t)(m > 0 ? m : 1));
  orc_draw_sparse(seed, m, s, h, d);
  for (int64_t k = 0; k < s * n; ++k) Y[k] = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) Y[(int64_t)h[i] * n + j] += (double)d[i] * A[i * lda + j];
  free(h); free(d);
}

/* Sparse sketch, underdetermined (from the right, Algorithm 2): the n x s
 * embedding X^T acts on the columns, Y = A X^T (m x s):
 * Y[:, h_j] += sign_j A[:, j] for j = 0..n-1 in ascending order. */
ORC_API void orc_sparse_under(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                              double* Y) {
  int32_t* h = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int8_t* d = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  orc_draw_sparse(seed, n, s, h, d);
  for (int64_t k = 0; k < m * s; ++k) Y[k] = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) Y[i * s + h[j]] += (double)d[j] * A[i * lda + j];
  free(h); free(d);
}

/* ------------------------------------------------------------------------ */
/* Gram matrix and Cholesky (Algorithm 1 steps 3-4, Algorithm 2 steps 3-4)   */
/* ------------------------------------------------------------------------ */
/* C = Y^T Y for Y (r x c): C is c x c. */
ORC_API void orc_gram_tn(const double* Y, int64_t r, int64_t c, double* C) {
  for (int64_t a = 0; a < c; ++a)
    for (int64_t b = 0; b < c; ++b) {
      double acc = 0.0;
      for (int64_t k = 0; k < r; ++k) acc += Y[k * c + a] * Y[k * c + b];
      C[a * c + b] = acc;
    }
}

/* C = Y Y^T for Y (r x c): C is r x r. */
ORC_API void orc_gram_nt(const double* Y, int64_t r, int64_t c, double* C) {
  for (int64_t a = 0; a < r; ++a)
    for (int64_t b = 0; b < r; ++b) {
      double acc = 0.0;
      for (int64_t k = 0; k < c; ++k) acc += Y[a * c + k] * Y[b * c + k];
      C[a * r + b] = acc;
    }
}

/* R = chol(C + lambda I): upper triangular R (n x n, row-major, zeros below
 * the diagonal) with R^T R = C + lambda I.  Row-by-row (up-looking) form:
 * R_jj = sqrt(C_jj + lambda - sum_{k<j} R_kj^2),
 * R_ji = (C_ji - sum_{k<j} R_kj R_ki) / R_jj for i > j.
 * Returns 0, or j+1 when the pivot of row j is not positive (breakdown; the
 * paper assumes kappa(C + lambda I) < O(1/u), Section 2.1.1). */
ORC_API int orc_cholesky_shifted(const double* C, int64_t n, double lambda, double* R) {
  for (int64_t i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double d = C[j * n + j] + lambda;
    for (int64_t k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];
    if (!(d > 0.0)) return (int)(j + 1);
    double rjj = sqrt(d);
    R[j * n + j] = rjj;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = C[j * n + i];
      for (int64_t k = 0; k < j; ++k) t -= R[k * n + j] * R[k * n + i];
      R[j * n + i] = t / rjj;
    }
  }
  return 0;
}

/* Back substitution x = R^-1 v, R upper triangular. */
ORC_API void orc_trsv_upper(const double* R, int64_t n, const double* v, double* x) {
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = v[i];
    for (int64_t k = i + 1; k < n; ++k) t -= R[i * n + k] * x[k];
    x[i] = t / R[i * n + i];
  }
}

/* Forward substitution x = R^-T v (R^T is lower triangular). */
ORC_API void orc_trsv_upper_t(const double* R, int64_t n, const double* v, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double t = v[i];
    for (int64_t k = 0; k < i; ++k) t -= R[k * n + i] * x[k];
    x[i] = t / R[i * n + i];
  }
}

/* ------------------------------------------------------------------------ */
/* LSQR (Paige & Saunders 1982), the solver the paper runs on B R^-1 / R^-T D */
/* ------------------------------------------------------------------------ */
typedef void (*orc_apply)(const void* ctx, const double* in, double* out);
typedef struct {
  int64_t rows, cols; /* the operator M is rows x cols */
  orc_apply mv;       /* out = M in   (in: cols, out: rows) */
  orc_apply rmv;      /* out = M^T in (in: rows, out: cols) */
  const void* ctx;
} orc_op;

static double nrm2(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * x[i];
  return sqrt(s);
}

/* Golub-Kahan bidiagonalization with the Givens (QR) update of the lower
 * bidiagonal system:
 *   beta u = b, alpha v = M^T u, w = v, phibar = beta, rhobar = alpha;
 *   each step: beta u = M v - alpha u;  alpha v = M^T u - beta v;
 *   rho = sqrt(rhobar^2 + beta^2), c = rhobar/rho, s = beta/rho,
 *   theta = s alpha, rhobar = -c alpha, phi = c phibar, phibar = s phibar,
 *   x += (phi/rho) w, w = v - (theta/rho) w.
 * Stopping (atol, btol as in Paige & Saunders): with the running Frobenius
 * estimate ||M|| = sqrt(sum alpha^2 + beta^2), ||r|| = phibar and
 * ||M^T r|| = phibar alpha |c|:
 *   test 2: ||M^T r|| / (||M|| ||r||) <= atol          -> istop 2
 *   test 1: ||r|| <= btol ||b|| + atol ||M|| ||x||      -> istop 1
 *   maxiter reached                                      -> istop 7
 * Returns the number of iterations; x (cols) holds the solution. */
ORC_API int orc_lsqr(const orc_op* op, const double* b, double atol, double btol, int maxiter, double* x,
                     int* istop_out) {
  int64_t m = op->rows, n = op->cols;
  double* u = (double*)malloc(sizeof(double) * (size_t)m);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* tm = (double*)malloc(sizeof(double) * (size_t)m);
  double* tn = (double*)malloc(sizeof(double) * (size_t)n);
  int istop = 0, it = 0;
  for (int64_t j = 0; j < n; ++j) x[j] = 0.0;
  for (int64_t i = 0; i < m; ++i) u[i] = b[i];
  double beta = nrm2(u, m), alpha = 0.0;
  double bnorm = beta;
  if (beta > 0.0) {
    for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    op->rmv(op->ctx, u, v);
    alpha = nrm2(v, n);
  } else {
    for (int64_t j = 0; j < n; ++j) v[j] = 0.0;
  }
  if (alpha > 0.0)
    for (int64_t j = 0; j < n; ++j) v[j] /= alpha;
  for (int64_t j = 0; j < n; ++j) w[j] = v[j];
  double phibar = beta, rhobar = alpha, anorm2 = 0.0;
  if (beta == 0.0 || alpha == 0.0) {
    istop = 1; /* x = 0 is exact (b = 0, or b orthogonal to the range of M) */
  }
  while (!istop && it < maxiter) {
    ++it;
    op->mv(op->ctx, v, tm);
    for (int64_t i = 0; i < m; ++i) u[i] = tm[i] - alpha * u[i];
    beta = nrm2(u, m);
    if (beta > 0.0)
      for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    anorm2 += alpha * alpha + beta * beta;
    op->rmv(op->ctx, u, tn);
    for (int64_t j = 0; j < n; ++j) v[j] = tn[j] - beta * v[j];
    alpha = nrm2(v, n);
    if (alpha > 0.0)
      for (int64_t j = 0; j < n; ++j) v[j] /= alpha;
    double rho = sqrt(rhobar * rhobar + beta * beta);
    double c = rhobar / rho, s = beta / rho;
    double theta = s * alpha;
    rhobar = -c * alpha;
    double phi = c * phibar;
    phibar = s * phibar;
    double t1 = phi / rho, t2 = theta / rho;
    for (int64_t j = 0; j < n; ++j) {
      x[j] += t1 * w[j];
      w[j] = v[j] - t2 * w[j];
    }
    double rnorm = phibar;
    double arnorm = phibar * alpha * fabs(c);
    double anorm = sqrt(anorm2);
    double xnorm = nrm2(x, n);
    if (rnorm == 0.0) { istop = 1; break; }
    double test2 = arnorm / (anorm * rnorm);
    double rtol = btol * bnorm + atol * anorm * xnorm;
    if (test2 <= atol) istop = 2;
    else if (rnorm <= rtol) istop = 1;
  }
  if (!istop) istop = 7;
  if (istop_out) *istop_out = istop;
  free(u); free(v); free(w); free(tm); free(tn);
  return it;
}

/* ---- preconditioned operators ------------------------------------------ */
typedef struct {
  const double* A; int64_t m, n, lda;
  double sqrtl;
  const double* R;     /* Cholesky variants: upper triangular, order n (over) or m (under) */
  const double* V;     /* low-rank variants: n x s_i (over) or m x s_i (under) basis, row-major, ld ldv */
  const double* S;     /* low-rank diagonal */
  int64_t si, ldv;
  double inv_sqrtl;
  double* tmp;         /* scratch, length max(m, n) */
  double* tmp2;
  int under_lr;        /* low-rank preconditioner of the underdetermined form */
} precond_ctx;

/* Low-rank inverse of eq. (RinvOver): out = l^{-1/2} (in - V S V^T in); the
 * vectors have length n (overdetermined) or m (underdetermined, Section 3.2:
 * R^-T = l^{-1/2} (I_m - U S U^T), symmetric). */
static void lr_apply(const precond_ctx* c, const double* in, double* out) {
  const int64_t n = c->under_lr ? c->m : c->n;
  for (int64_t j = 0; j < n; ++j) out[j] = in[j];
  for (int64_t k = 0; k < c->si; ++k) {
    double dot = 0.0;
    for (int64_t j = 0; j < n; ++j) dot += c->V[j * c->ldv + k] * in[j];
    dot *= c->S[k];
    for (int64_t j = 0; j < n; ++j) out[j] -= c->V[j * c->ldv + k] * dot;
  }
  for (int64_t j = 0; j < n; ++j) out[j] *= c->inv_sqrtl;
}

/* Overdetermined operator M = B R^-1, B = [A; sqrt(l) I_n]  ((m+n) x n). */
static void over_mv(const void* vc, const double* y, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  double* t = c->tmp;
  if (c->R) orc_trsv_upper(c->R, c->n, y, t);
  else lr_apply(c, y, t);
  for (int64_t i = 0; i < c->m; ++i) {
    double acc = 0.0;
    for (int64_t j = 0; j < c->n; ++j) acc += c->A[i * c->lda + j] * t[j];
    out[i] = acc;
  }
  for (int64_t j = 0; j < c->n; ++j) out[c->m + j] = c->sqrtl * t[j];
}
static void over_rmv(const void* vc, const double* u, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  double* g = c->tmp;
  for (int64_t j = 0; j < c->n; ++j) g[j] = c->sqrtl * u[c->m + j];
  for (int64_t i = 0; i < c->m; ++i)
    for (int64_t j = 0; j < c->n; ++j) g[j] += c->A[i * c->lda + j] * u[i];
  if (c->R) orc_trsv_upper_t(c->R, c->n, g, out);
  else lr_apply(c, g, out); /* the low-rank R^-1 is symmetric */
}

/* Underdetermined operator M = R^-T D, D = [A sqrt(l) I_m]  (m x (n+m)). */
static void under_mv(const void* vc, const double* z, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  double* p = c->tmp;
  for (int64_t i = 0; i < c->m; ++i) {
    double acc = c->sqrtl * z[c->n + i];
    for (int64_t j = 0; j < c->n; ++j) acc += c->A[i * c->lda + j] * z[j];
    p[i] = acc;
  }
  if (c->R) orc_trsv_upper_t(c->R, c->m, p, out);
  else lr_apply(c, p, out);
}
static void under_rmv(const void* vc, const double* u, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  double* t = c->tmp;
  if (c->R) orc_trsv_upper(c->R, c->m, u, t);
  else lr_apply(c, u, t); /* the low-rank R^-1 is symmetric */
  for (int64_t j = 0; j < c->n; ++j) out[j] = 0.0;
  for (int64_t i = 0; i < c->m; ++i)
    for (int64_t j = 0; j < c->n; ++j) out[j] += c->A[i * c->lda + j] * t[i];
  for (int64_t i = 0; i < c->m; ++i) out[c->n + i] = c->sqrtl * t[i];
}

/* Plain operator M = A (unpreconditioned LSQR, used as a behavioural baseline). */
static void plain_mv(const void* vc, const double* x, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  for (int64_t i = 0; i < c->m; ++i) {
    double acc = 0.0;
    for (int64_t j = 0; j < c->n; ++j) acc += c->A[i * c->lda + j] * x[j];
    out[i] = acc;
  }
}
static void plain_rmv(const void* vc, const double* u, double* out) {
  const precond_ctx* c = (const precond_ctx*)vc;
  for (int64_t j = 0; j < c->n; ++j) out[j] = 0.0;
  for (int64_t i = 0; i < c->m; ++i)
    for (int64_t j = 0; j < c->n; ++j) out[j] += c->A[i * c->lda + j] * u[i];
}

/* Unpreconditioned LSQR on min ||A x - b||  (m x n). */
ORC_API int orc_lsqr_plain(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double tol,
                           int maxiter, double* x, int* istop) {
  precond_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.m = m; c.n = n; c.lda = lda;
  orc_op op = {m, n, plain_mv, plain_rmv, &c};
  return orc_lsqr(&op, b, tol, tol, maxiter, x, istop);
}

/* Overdetermined LSQR with the Cholesky factor R (Algorithm 1 steps 5-6):
 * y = argmin ||B R^-1 y - [b; 0]||, x = R^-1 y. */
ORC_API int orc_lsqr_over_chol(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                               double lambda, const double* R, double tol, int maxiter, double* x, int* istop) {
  precond_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.m = m; c.n = n; c.lda = lda; c.sqrtl = sqrt(lambda); c.R = R;
  c.tmp = (double*)malloc(sizeof(double) * (size_t)(m > n ? m : n));
  double* bh = (double*)calloc((size_t)(m + n), sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) bh[i] = b[i];
  orc_op op = {m + n, n, over_mv, over_rmv, &c};
  int it = orc_lsqr(&op, bh, tol, tol, maxiter, y, istop);
  orc_trsv_upper(R, n, y, x);
  free(c.tmp); free(bh); free(y);
  return it;
}

/* Overdetermined LSQR with the low-rank inverse R^-1 = l^{-1/2}(I - V S V^T)
 * (Algorithm 3 steps 8-9). V is n x si with leading dimension ldv. */
ORC_API int orc_lsqr_over_lr(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double lambda,
                             const double* V, int64_t ldv, const double* S, int64_t si, double tol, int maxiter,
                             double* x, int* istop) {
  precond_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.m = m; c.n = n; c.lda = lda; c.sqrtl = sqrt(lambda); c.inv_sqrtl = 1.0 / sqrt(lambda);
  c.V = V; c.ldv = ldv; c.S = S; c.si = si;
  c.tmp = (double*)malloc(sizeof(double) * (size_t)(m > n ? m : n));
  double* bh = (double*)calloc((size_t)(m + n), sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) bh[i] = b[i];
  orc_op op = {m + n, n, over_mv, over_rmv, &c};
  int it = orc_lsqr(&op, bh, tol, tol, maxiter, y, istop);
  lr_apply(&c, y, x);
  free(c.tmp); free(bh); free(y);
  return it;
}

/* Underdetermined LSQR with the Cholesky factor R (m x m), Algorithm 2
 * steps 5-6: the minimum-norm solution [x; y] of R^-T D [x; y] = R^-T b, from
 * LSQR started at zero; x is the top n coordinates. */
ORC_API int orc_lsqr_under_chol(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                double lambda, const double* R, double tol, int maxiter, double* x, int* istop) {
  precond_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.m = m; c.n = n; c.lda = lda; c.sqrtl = sqrt(lambda); c.R = R;
  c.tmp = (double*)malloc(sizeof(double) * (size_t)(m > n ? m : n));
  double* rb = (double*)malloc(sizeof(double) * (size_t)m);
  double* z = (double*)malloc(sizeof(double) * (size_t)(n + m));
  orc_trsv_upper_t(R, m, b, rb);
  orc_op op = {m, n + m, under_mv, under_rmv, &c};
  int it = orc_lsqr(&op, rb, tol, tol, maxiter, z, istop);
  for (int64_t j = 0; j < n; ++j) x[j] = z[j];
  free(c.tmp); free(rb); free(z);
  return it;
}

/* Underdetermined LSQR with the low-rank preconditioner of Section 3.2
 * (Algorithm 4 step 8): R^-T = l^{-1/2} (I_m - U S U^T) with U (m x s_i, ld
 * ldu); min-norm [x; y] of R^-T D [x; y] = R^-T b; x is the top n coordinates. */
ORC_API int orc_lsqr_under_lr(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double lambda,
                              const double* U, int64_t ldu, const double* S, int64_t si, double tol, int maxiter,
                              double* x, int* istop) {
  precond_ctx c;
  memset(&c, 0, sizeof c);
  c.A = A; c.m = m; c.n = n; c.lda = lda; c.sqrtl = sqrt(lambda); c.inv_sqrtl = 1.0 / sqrt(lambda);
  c.V = U; c.ldv = ldu; c.S = S; c.si = si; c.under_lr = 1;
  c.tmp = (double*)malloc(sizeof(double) * (size_t)(m > n ? m : n));
  double* rb = (double*)malloc(sizeof(double) * (size_t)m);
  double* z = (double*)malloc(sizeof(double) * (size_t)(n + m));
  lr_apply(&c, b, rb);
  orc_op op = {m, n + m, under_mv, under_rmv, &c};
  int it = orc_lsqr(&op, rb, tol, tol, maxiter, z, istop);
  for (int64_t j = 0; j < n; ++j) x[j] = z[j];
  free(c.tmp); free(rb); free(z);
  return it;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Algorithm 3 step 4: [~, Sigma, V] = svd(Y, 'econ'))  */
/* ------------------------------------------------------------------------ */
/* Y is s x n with s <= n.  The columns of W = Y^T (n x s) are rotated in
 * pairs until mutually orthogonal (Hestenes); then sigma_p = ||w_p|| and
 * v_p = w_p / sigma_p.  Rotation for a pair with a = ||w_p||^2, b = ||w_q||^2,
 * g = w_p . w_q:  zeta = (b - a) / (2g), t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)),
 * c = 1/sqrt(1+t^2), sn = c t; w_p <- c w_p - sn w_q, w_q <- sn w_p + c w_q.
 * Outputs sigma (s, descending) and V (n x s, row-major).  Returns sweeps. */
ORC_API int orc_jacobi_svd(const double* Y, int64_t s, int64_t n, double tol, int max_sweeps, double* sigma,
                           double* V) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * s)); /* column p stored contiguously: W[p*n + k] */
  for (int64_t p = 0; p < s; ++p)
    for (int64_t k = 0; k < n; ++k) W[p * n + k] = Y[p * n + k];
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int64_t rotations = 0;
    for (int64_t p = 0; p + 1 < s; ++p)
      for (int64_t q = p + 1; q < s; ++q) {
        double* wp = W + p * n;
        double* wq = W + q * n;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int64_t k = 0; k < n; ++k) {
          a += wp[k] * wp[k];
          b += wq[k] * wq[k];
          g += wp[k] * wq[k];
        }
        if (a == 0.0 || b == 0.0 || !(fabs(g) > tol * sqrt(a * b))) continue;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double sn = c * t;
        for (int64_t k = 0; k < n; ++k) {
          double x = wp[k], y = wq[k];
          wp[k] = c * x - sn * y;
          wq[k] = sn * x + c * y;
        }
        ++rotations;
      }
    if (rotations == 0) break;
  }
  /* norms, then order by sigma descending (stable on ties) */
  double* nrm = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  for (int64_t p = 0; p < s; ++p) { nrm[p] = nrm2(W + p * n, n); ord[p] = p; }
  for (int64_t i = 1; i < s; ++i) { /* insertion sort, stable */
    int64_t key = ord[i], j = i - 1;
    while (j >= 0 && nrm[ord[j]] < nrm[key]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = key;
  }
  for (int64_t q = 0; q < s; ++q) {
    int64_t p = ord[q];
    sigma[q] = nrm[p];
    for (int64_t k = 0; k < n; ++k) V[k * s + q] = nrm[p] > 0.0 ? W[p * n + k] / nrm[p] : 0.0;
  }
  free(W); free(nrm); free(ord);
  return sweep + 1;
}

/* Definition 1.1 / Section 3.1.2: statistical-dimension estimate from the
 * singular values of the sketch, sd = sum_j 1 / (1 + lambda / sigma_j^2),
 * summed in ascending j; zero sigma contributes nothing. */
ORC_API double orc_sd_estimate(const double* sigma, int64_t s, double lambda) {
  double acc = 0.0;
  for (int64_t j = 0; j < s; ++j)
    if (sigma[j] > 0.0) acc += 1.0 / (1.0 + lambda / (sigma[j] * sigma[j]));
  return acc;
}

/* Algorithm 3 step 5: s_i = alpha * ceil(sd_i), clamped to the sketch size s. */
ORC_API int64_t orc_truncation(double sd, double alpha, int64_t s) {
  double t = ceil(alpha * ceil(sd));
  if (t > (double)s) return s;
  if (t < 1.0) return 1;
  return (int64_t)t;
}

/* Algorithm 3 step 7: (S_i)_jj = 1 - sqrt(1 / (1 + sigma_j^2 / lambda_i)). */
ORC_API void orc_lr_diag(const double* sigma, int64_t si, double lambda, double* S) {
  for (int64_t j = 0; j < si; ++j) S[j] = 1.0 - sqrt(1.0 / (1.0 + sigma[j] * sigma[j] / lambda));
}

/* ------------------------------------------------------------------------ */
/* Whole algorithms, one lambda at a time, exactly in the paper's order       */
/* ------------------------------------------------------------------------ */
/* sketch kinds: 0 = SRHT, 1 = Gaussian, 2 = sparse (one nonzero per column), 3 = SRDCT */
static void sketch_over(int kind, const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                        double* Y) {
  if (kind == 0) orc_srht_over(A, m, n, lda, seed, s, Y);
  else if (kind == 1) orc_gauss_over(A, m, n, lda, seed, s, Y);
  else if (kind == 2) orc_sparse_over(A, m, n, lda, seed, s, Y);
  else orc_srdct_over(A, m, n, lda, seed, s, Y);
}
static void sketch_under(int kind, const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                         double* Y) {
  if (kind == 0) orc_srht_under(A, m, n, lda, seed, s, Y);
  else if (kind == 1) orc_gauss_under(A, m, n, lda, seed, s, Y);
  else if (kind == 2) orc_sparse_under(A, m, n, lda, seed, s, Y);
  else orc_srdct_under(A, m, n, lda, seed, s, Y);
}

/* Algorithm 1: X drawn once (step 1), Y = XA (2), C = Y^T Y (3); for each
 * lambda_i: R_i = chol(C + lambda_i I) (4), LSQR on B_i R_i^-1 (5),
 * x_i = R_i^-1 y_i (6).  X_out is n x N (column i = x_{lambda_i}).
 * Returns 0 or -(i+1) for a Cholesky breakdown at lambda index i. */
ORC_API int orc_alg1(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* lambdas,
                     int N, int sketch_kind, int64_t s, uint64_t seed, double tol, int maxiter, double* X_out,
                     int* iters, int* istops) {
  double* Y = (double*)malloc(sizeof(double) * (size_t)(s * n));
  double* C = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* R = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  sketch_over(sketch_kind, A, m, n, lda, seed, s, Y);
  orc_gram_tn(Y, s, n, C);
  for (int i = 0; i < N && !rc; ++i) {
    if (orc_cholesky_shifted(C, n, lambdas[i], R)) { rc = -(i + 1); break; }
    iters[i] = orc_lsqr_over_chol(A, m, n, lda, b, lambdas[i], R, tol, maxiter, x, &istops[i]);
    for (int64_t j = 0; j < n; ++j) X_out[j * N + i] = x[j];
  }
  free(Y); free(C); free(R); free(x);
  return rc;
}

/* Algorithm 2: X (n x s) drawn once, Y = AX (m x s), C = Y Y^T; for each
 * lambda_i: R_i = chol(C + lambda_i I_m), min-norm LSQR on R_i^-T D_i. */
ORC_API int orc_alg2(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* lambdas,
                     int N, int sketch_kind, int64_t s, uint64_t seed, double tol, int maxiter, double* X_out,
                     int* iters, int* istops) {
  double* Y = (double*)malloc(sizeof(double) * (size_t)(m * s));
  double* C = (double*)malloc(sizeof(double) * (size_t)(m * m));
  double* R = (double*)malloc(sizeof(double) * (size_t)(m * m));
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  sketch_under(sketch_kind, A, m, n, lda, seed, s, Y);
  orc_gram_nt(Y, m, s, C);
  for (int i = 0; i < N && !rc; ++i) {
    if (orc_cholesky_shifted(C, m, lambdas[i], R)) { rc = -(i + 1); break; }
    iters[i] = orc_lsqr_under_chol(A, m, n, lda, b, lambdas[i], R, tol, maxiter, x, &istops[i]);
    for (int64_t j = 0; j < n; ++j) X_out[j * N + i] = x[j];
  }
  free(Y); free(C); free(R); free(x);
  return rc;
}

/* Algorithm 3 (overdetermined, low rank): sketch of size s (step 1 is the
 * caller's choice of s), Y = XA, SVD of Y (step 4); for each lambda_i the
 * sd estimate of Section 3.1.2 gives s_i (step 5), V_i, Sigma_i are the
 * leading s_i factors (6), S_i from eq. (step 7), LSQR with
 * R_i^-1 = l_i^{-1/2}(I - V_i S_i V_i^T) (8), x_i = R_i^-1 y (9).
 * si_out (N) receives the truncation ranks. */
ORC_API int orc_alg3(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* lambdas,
                     int N, int sketch_kind, int64_t s, double alpha, uint64_t seed, double tol, int maxiter,
                     double* X_out, int* iters, int* istops, int64_t* si_out, double* sigma_out) {
  double* Y = (double*)malloc(sizeof(double) * (size_t)(s * n));
  double* sig = (double*)malloc(sizeof(double) * (size_t)s);
  double* V = (double*)malloc(sizeof(double) * (size_t)(n * s));
  double* S = (double*)malloc(sizeof(double) * (size_t)s);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  sketch_over(sketch_kind, A, m, n, lda, seed, s, Y);
  orc_jacobi_svd(Y, s, n, 1e-15, 80, sig, V);
  if (sigma_out)
    for (int64_t j = 0; j < s; ++j) sigma_out[j] = sig[j];
  for (int i = 0; i < N; ++i) {
    double sd = orc_sd_estimate(sig, s, lambdas[i]);
    int64_t si = orc_truncation(sd, alpha, s);
    si_out[i] = si;
    orc_lr_diag(sig, si, lambdas[i], S);
    iters[i] = orc_lsqr_over_lr(A, m, n, lda, b, lambdas[i], V, s, S, si, tol, maxiter, x, &istops[i]);
    for (int64_t j = 0; j < n; ++j) X_out[j * N + i] = x[j];
  }
  free(Y); free(sig); free(V); free(S); free(x);
  return 0;
}

/* Algorithm 4 (underdetermined, low rank): Y = AX (m x s, step 3), the SVD
 * [U, Sigma, ~] = svd(Y, 'econ') (step 4) taken as the one-sided Jacobi SVD of
 * Y^T (its right singular vectors are U); for each lambda_i the sd estimate
 * gives s_i (step 5), U_i, Sigma_i the leading s_i factors (6), S_i (7), and
 * min-norm LSQR with R_i^-T = l_i^{-1/2}(I - U_i S_i U_i^T) (8) returns x (9). */
ORC_API int orc_alg4(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* lambdas,
                     int N, int sketch_kind, int64_t s, double alpha, uint64_t seed, double tol, int maxiter,
                     double* X_out, int* iters, int* istops, int64_t* si_out, double* sigma_out) {
  double* Y = (double*)malloc(sizeof(double) * (size_t)(m * s));
  double* Yt = (double*)malloc(sizeof(double) * (size_t)(s * m));
  double* sig = (double*)malloc(sizeof(double) * (size_t)s);
  double* U = (double*)malloc(sizeof(double) * (size_t)(m * s));
  double* S = (double*)malloc(sizeof(double) * (size_t)s);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  sketch_under(sketch_kind, A, m, n, lda, seed, s, Y);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < s; ++j) Yt[j * m + i] = Y[i * s + j];
  orc_jacobi_svd(Yt, s, m, 1e-15, 80, sig, U);
  if (sigma_out)
    for (int64_t j = 0; j < s; ++j) sigma_out[j] = sig[j];
  for (int i = 0; i < N; ++i) {
    double sd = orc_sd_estimate(sig, s, lambdas[i]);
    int64_t si = orc_truncation(sd, alpha, s);
    si_out[i] = si;
    orc_lr_diag(sig, si, lambdas[i], S);
    iters[i] = orc_lsqr_under_lr(A, m, n, lda, b, lambdas[i], U, s, S, si, tol, maxiter, x, &istops[i]);
    for (int64_t j = 0; j < n; ++j) X_out[j * N + i] = x[j];
  }
  free(Y); free(Yt); free(sig); free(U); free(S); free(x);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reference solution of the ridge problem (1.2), independent of Alg 1-3     */
/* ------------------------------------------------------------------------ */
/* Error-free transformations (Knuth's TwoSum; TwoProd through fma). */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double bb = x - a;
  *e = (a - (x - bb)) + (b - bb);
  *s = x;
}
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}
/* (hi, lo) += a * b in double-double. */
static void dd_fma_acc(double* hi, double* lo, double a, double b) {
  double p, pe, s, se;
  two_prod(a, b, &p, &pe);
  two_sum(*hi, p, &s, &se);
  double l = *lo + (se + pe);
  double h2, l2;
  two_sum(s, l, &h2, &l2);
  *hi = h2;
  *lo = l2;
}

ORC_API void orc_two_prod(double a, double b, double* p, double* e) { two_prod(a, b, p, e); }
ORC_API void orc_two_sum(double a, double b, double* s, double* e) { two_sum(a, b, s, e); }

/* Normal-equation residual g = A^T (b - A x) - lambda x, with b - A x and the
 * product with A^T accumulated in double-double.  r_out (m, optional) receives
 * the rounded residual b - A x. */
ORC_API void orc_ridge_residual_dd(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                   double lambda, const double* x, double* g, double* r_out) {
  double* rh = (double*)malloc(sizeof(double) * (size_t)m);
  double* rl = (double*)malloc(sizeof(double) * (size_t)m);
  double* gh = (double*)calloc((size_t)n, sizeof(double));
  double* gl = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double hi = b[i], lo = 0.0;
    for (int64_t j = 0; j < n; ++j) dd_fma_acc(&hi, &lo, -A[i * lda + j], x[j]);
    rh[i] = hi;
    rl[i] = lo;
  }
  /* g_j accumulates over i = 0..m-1 in ascending order; the loop nest walks
   * rows (each thread owns a slice of columns) so A is read row by row. */
#pragma omp parallel
  {
    int64_t nt = 1, t = 0;
#ifdef _OPENMP
    nt = omp_get_num_threads();
    t = omp_get_thread_num();
#endif
    int64_t j0 = n * t / nt, j1 = n * (t + 1) / nt;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = j0; j < j1; ++j) {
        dd_fma_acc(&gh[j], &gl[j], A[i * lda + j], rh[i]);
        dd_fma_acc(&gh[j], &gl[j], A[i * lda + j], rl[i]);
      }
    for (int64_t j = j0; j < j1; ++j) dd_fma_acc(&gh[j], &gl[j], -lambda, x[j]);
  }
  for (int64_t j = 0; j < n; ++j) g[j] = gh[j] + gl[j];
  if (r_out)
    for (int64_t i = 0; i < m; ++i) r_out[i] = rh[i] + rl[i];
  free(rh); free(rl); free(gh); free(gl);
}

/* Householder QR of B = [A; sqrt(lambda) I_n] ((m+n) x n), least-squares
 * solve x = R^-1 (Q^T [b; 0])_{1:n}; then `refine` steps of refinement with
 * the double-double normal-equation residual:  x <- x + (R^T R)^-1 g.
 * Returns 0, or -1 if R is singular. */
ORC_API int orc_ref_ridge_qr(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double lambda,
                             int refine, double* x) {
  int64_t M = m + n;
  double* Bm = (double*)calloc((size_t)(M * n), sizeof(double));
  double* c = (double*)calloc((size_t)M, sizeof(double));
  double* vh = (double*)malloc(sizeof(double) * (size_t)M);
  double sl = sqrt(lambda);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) Bm[i * n + j] = A[i * lda + j];
  for (int64_t j = 0; j < n; ++j) Bm[(m + j) * n + j] = sl;
  for (int64_t i = 0; i < m; ++i) c[i] = b[i];
  int rc = 0;
  for (int64_t k = 0; k < n; ++k) {
    /* Householder vector for column k below the diagonal */
    double nrm = 0.0;
    for (int64_t i = k; i < M; ++i) nrm += Bm[i * n + k] * Bm[i * n + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { rc = -1; break; }
    double alpha = Bm[k * n + k] > 0.0 ? -nrm : nrm;
    for (int64_t i = k; i < M; ++i) vh[i] = Bm[i * n + k];
    vh[k] -= alpha;
    double vv = 0.0;
    for (int64_t i = k; i < M; ++i) vv += vh[i] * vh[i];
    if (vv > 0.0) {
      for (int64_t j = k; j < n; ++j) {
        double d = 0.0;
        for (int64_t i = k; i < M; ++i) d += vh[i] * Bm[i * n + j];
        d = 2.0 * d / vv;
        for (int64_t i = k; i < M; ++i) Bm[i * n + j] -= d * vh[i];
      }
      double d = 0.0;
      for (int64_t i = k; i < M; ++i) d += vh[i] * c[i];
      d = 2.0 * d / vv;
      for (int64_t i = k; i < M; ++i) c[i] -= d * vh[i];
    }
  }
  if (!rc) {
    double* R = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) R[i * n + j] = j >= i ? Bm[i * n + j] : 0.0;
    orc_trsv_upper(R, n, c, x);
    for (int it = 0; it < refine; ++it) {
      orc_ridge_residual_dd(A, m, n, lda, b, lambda, x, g, NULL);
      orc_trsv_upper_t(R, n, g, t);
      orc_trsv_upper(R, n, t, g);
      for (int64_t j = 0; j < n; ++j) x[j] += g[j];
    }
    free(R); free(g); free(t);
  }
  free(Bm); free(c); free(vh);
  return rc;
}

/* Refinement of a given x against the stored A, with an approximate inverse of
 * A^T A + lambda I built from a thin SVD factor pair (V: n x k with
 * orthonormal columns, sigma: k) of a matrix close to A:
 *   P^-1 g = g / lambda + V diag(1/(sigma^2 + lambda) - 1/lambda) V^T g.
 * Each step: g = A^T (b - A x) - lambda x in double-double, x <- x + P^-1 g.
 * This is the reference at sizes where a dense QR is out of reach. */
ORC_API void orc_ref_ridge_refine(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                  double lambda, const double* V, int64_t k, const double* sigma, int steps,
                                  double* x) {
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  for (int it = 0; it < steps; ++it) {
    orc_ridge_residual_dd(A, m, n, lda, b, lambda, x, g, NULL);
    for (int64_t q = 0; q < k; ++q) c[q] = 0.0;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t q = 0; q < k; ++q) c[q] += V[j * k + q] * g[j];
    for (int64_t q = 0; q < k; ++q) c[q] *= 1.0 / (sigma[q] * sigma[q] + lambda) - 1.0 / lambda;
    for (int64_t j = 0; j < n; ++j) {
      double acc = g[j] / lambda;
      for (int64_t q = 0; q < k; ++q) acc += V[j * k + q] * c[q];
      x[j] += acc;
    }
  }
  free(g); free(c);
}

/* ------------------------------------------------------------------------ */
/* L-curve (Section 4.3, Fig. 4): for each lambda_i the points                */
/* (||A x_i - b||, ||x_i||) on a log-log plot; the regularization parameter   */
/* of choice sits at the corner.  The paper does not say how the corner is    */
/* found; the reading taken here is Hansen's: the point of maximum curvature  */
/* of the curve P(t) = ln ||A x - b||, Q(t) = ln ||x||, t = ln lambda,        */
/*   kappa = (P' Q'' - P'' Q') / (P'^2 + Q'^2)^(3/2),                          */
/* with the derivatives taken as three-point differences on the (possibly     */
/* non-uniform) grid of sampled t.  The first and last points have no         */
/* curvature (0) and are never the corner.                                    */
/* ------------------------------------------------------------------------ */

/* Norms of the residual and of x for each row of X (N x n): rn[i] =
 * ||b - A x_i||, xn[i] = ||x_i||, plain float64 sums. */
ORC_API void orc_lcurve_norms(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* X,
                              int N, double* rn, double* xn) {
  for (int i = 0; i < N; ++i) {
    const double* x = X + (int64_t)i * n;
    double rr = 0.0, xx = 0.0;
    for (int64_t r = 0; r < m; ++r) {
      double v = b[r];
      for (int64_t j = 0; j < n; ++j) v -= A[r * lda + j] * x[j];
      rr += v * v;
    }
    for (int64_t j = 0; j < n; ++j) xx += x[j] * x[j];
    rn[i] = sqrt(rr);
    xn[i] = sqrt(xx);
  }
}

/* Curvature of the sampled L-curve.  lambdas ascending (N >= 3), rn, xn > 0.
 * kappa[0] = kappa[N-1] = 0.  Returns the index of the largest kappa over
 * 1..N-2 (the first one on ties), or -1 if N < 3. */
ORC_API int orc_lcurve_curvature(const double* lambdas, const double* rn, const double* xn, int N, double* kappa) {
  for (int i = 0; i < N; ++i) kappa[i] = 0.0;
  if (N < 3) return -1;
  int best = 1;
  for (int k = 1; k < N - 1; ++k) {
    const double t0 = log(lambdas[k - 1]), t1 = log(lambdas[k]), t2 = log(lambdas[k + 1]);
    const double h1 = t1 - t0, h2 = t2 - t1;
    const double P0 = log(rn[k - 1]), P1 = log(rn[k]), P2 = log(rn[k + 1]);
    const double Q0 = log(xn[k - 1]), Q1 = log(xn[k]), Q2 = log(xn[k + 1]);
    /* first derivative: weights of the quadratic through the three points */
    const double a0 = -h2 / (h1 * (h1 + h2)), a1 = (h2 - h1) / (h1 * h2), a2 = h1 / (h2 * (h1 + h2));
    /* second derivative */
    const double c0 = 2.0 / (h1 * (h1 + h2)), c1 = -2.0 / (h1 * h2), c2 = 2.0 / (h2 * (h1 + h2));
    const double dP = a0 * P0 + a1 * P1 + a2 * P2, dQ = a0 * Q0 + a1 * Q1 + a2 * Q2;
    const double ddP = c0 * P0 + c1 * P1 + c2 * P2, ddQ = c0 * Q0 + c1 * Q1 + c2 * Q2;
    const double den = pow(dP * dP + dQ * dQ, 1.5);
    kappa[k] = den > 0.0 ? (dP * ddQ - ddP * dQ) / den : 0.0;
    if (kappa[k] > kappa[best]) best = k;
  }
  return best;
}

/* The second sweep around a corner at index k of the ascending grid: nr
 * parameters log-spaced strictly between lambdas[k-1] and lambdas[k+1],
 *   lambda_j = exp(t_{k-1} + (t_{k+1} - t_{k-1}) j / (nr + 1)),  j = 1..nr. */
ORC_API void orc_lcurve_refine_grid(const double* lambdas, int N, int k, int nr, double* out) {
  const int lo = k > 0 ? k - 1 : 0, hi = k < N - 1 ? k + 1 : N - 1;
  const double a = log(lambdas[lo]), b = log(lambdas[hi]);
  for (int j = 1; j <= nr; ++j) out[j - 1] = exp(a + (b - a) * (double)j / (double)(nr + 1));
}

/* ------------------------------------------------------------------------ */
/* BP2 (Section 4.1): the preconditioner of Algorithm 1 obtained by a QR      */
/* decomposition instead of a Cholesky factorization,                         */
/*   Q R_BP2 = [X A; sqrt(lambda) I_n]   ((s + n) x n),                        */
/* equal to chol(Y^T Y + lambda I) up to the signs of its rows in exact       */
/* arithmetic.  Plain Householder QR, columns left to right; the rows of R are */
/* then scaled by the sign of their diagonal so that diag(R) > 0.             */
/* Returns 0, or -1 when a column is exactly zero (cannot happen for          */
/* lambda > 0).                                                                */
/* ------------------------------------------------------------------------ */
ORC_API int orc_bp2_r(const double* Y, int64_t s, int64_t n, double lambda, double* R) {
  const int64_t M = s + n;
  double* Bm = (double*)calloc((size_t)(M * n), sizeof(double));
  double* v = (double*)malloc(sizeof(double) * (size_t)M);
  const double sl = sqrt(lambda);
  for (int64_t i = 0; i < s; ++i)
    for (int64_t j = 0; j < n; ++j) Bm[i * n + j] = Y[i * n + j];
  for (int64_t j = 0; j < n; ++j) Bm[(s + j) * n + j] = sl;
  int rc = 0;
  for (int64_t k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int64_t i = k; i < M; ++i) nrm += Bm[i * n + k] * Bm[i * n + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { rc = -1; break; }
    const double alpha = Bm[k * n + k] > 0.0 ? -nrm : nrm;  /* reflect onto -sign(b_kk) ||b_k|| e_k */
    for (int64_t i = k; i < M; ++i) v[i] = Bm[i * n + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int64_t i = k; i < M; ++i) vv += v[i] * v[i];
    for (int64_t j = k; j < n; ++j) {
      double d = 0.0;
      for (int64_t i = k; i < M; ++i) d += v[i] * Bm[i * n + j];
      d = 2.0 * d / vv;
      for (int64_t i = k; i < M; ++i) Bm[i * n + j] -= d * v[i];
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    const double sg = Bm[i * n + i] < 0.0 ? -1.0 : 1.0;
    for (int64_t j = 0; j < n; ++j) R[i * n + j] = j >= i ? sg * Bm[i * n + j] : 0.0;
  }
  free(Bm); free(v);
  return rc;
}
