/*
 * mm_oracle.c -- plain, slow, obviously correct CPU reference for semiring
 * matrix multiplication.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the library itself never does.  It shares no
 * code, header, table or constant with the CUDA sources.
 *
 * Every product computes the plain definition of matrix multiplication on a
 * semiring (S, (+), (x), 0, 1) (Section 2, "General MM C = A (x) B on a closed
 * semiring"):
 *
 *     C[i][j] = (+)_{t = 0 .. k-1}  A[i][t] (x) B[t][j]
 *
 * with no recursion, blocking, split-K or Strassen.  Loops run i, then t in
 * ascending order, then j, so every C[i][j] is accumulated in ascending t.
 * OpenMP spreads independent rows across host threads; it does not change the
 * arithmetic of any element.
 *
 * Layout: dense row-major.  A is m x k, B is k x n, C is nrows x n where the
 * computed rows are rows[0..nrows) of the full m x n product (rows == NULL
 * means all m rows, in order).
 *
 * The Strassen and Strassen-Winograd recursions and the Floyd-Warshall closure
 * below exist only so the tests can pin the triple loop against independent
 * algorithms (Section 5 Strassen formulas; the bilinear generalisation that
 * names Strassen-Winograd).
 *
 * Closures.  A closed semiring (Section 2) has a closure A* = 1 (+) A (+) A^2
 * (+) ... for square A.  For (min,+) on [0, 2^30] A* is the all-pairs
 * shortest-path matrix (0 on the diagonal); for (or, and) it is reflexive
 * reachability.  The oracle computes both by the textbook vertex-elimination
 * algorithms (Floyd-Warshall, Warshall), which share nothing with the
 * repeated squaring the GPU path uses.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF ((int64_t)1 << 30) /* +infinity of the (min,+) semiring */

static int64_t row_of(const int64_t* rows, int64_t r) { return rows ? rows[r] : r; }

/* (+, x) over the reals, accumulated in double (Section 2 definition). */
int oracle_mm_f64(int64_t m, int64_t n, int64_t k, const double* A, const double* B,
                  double* C, const int64_t* rows, int64_t nrows) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (!rows) nrows = m;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = row_of(rows, r);
    double* c = C + r * n;
    for (int64_t j = 0; j < n; ++j) c[j] = 0.0; /* additive identity */
    if (i < 0 || i >= m) continue;
    for (int64_t t = 0; t < k; ++t) {
      const double a = A[i * k + t];
      const double* b = B + t * n;
      for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
    }
  }
  return 0;
}

/* (+, x) over the integers, exact in int64 (Section 2 definition). */
int oracle_mm_i64(int64_t m, int64_t n, int64_t k, const int64_t* A, const int64_t* B,
                  int64_t* C, const int64_t* rows, int64_t nrows) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (!rows) nrows = m;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = row_of(rows, r);
    int64_t* c = C + r * n;
    for (int64_t j = 0; j < n; ++j) c[j] = 0;
    if (i < 0 || i >= m) continue;
    for (int64_t t = 0; t < k; ++t) {
      const int64_t a = A[i * k + t];
      const int64_t* b = B + t * n;
      for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
    }
  }
  return 0;
}

/*
 * (min, +) tropical semiring on [0, 2^30] with 2^30 standing for +infinity:
 * (+) = min with identity +inf, (x) = + with identity 0 (Section 2 semiring;
 * the saturating reading of the sentinel).  Sums are formed in int64 so that
 * inf + inf cannot wrap; the result is clamped to the sentinel.
 */
int oracle_mm_minplus(int64_t m, int64_t n, int64_t k, const int32_t* A, const int32_t* B,
                      int32_t* C, const int64_t* rows, int64_t nrows) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (!rows) nrows = m;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = row_of(rows, r);
    int32_t* c = C + r * n;
    int64_t* acc = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!acc) { bad = 1; continue; }
    for (int64_t j = 0; j < n; ++j) acc[j] = ORACLE_INF; /* additive identity */
    if (i >= 0 && i < m) {
      for (int64_t t = 0; t < k; ++t) {
        const int64_t a = A[i * k + t];
        const int32_t* b = B + t * n;
        for (int64_t j = 0; j < n; ++j) {
          const int64_t s = a + (int64_t)b[j];
          if (s < acc[j]) acc[j] = s;
        }
      }
    }
    for (int64_t j = 0; j < n; ++j) c[j] = (int32_t)(acc[j] < ORACLE_INF ? acc[j] : ORACLE_INF);
    free(acc);
  }
  return bad ? -2 : 0;
}

/* Boolean semiring ({0,1}, or, and): any nonzero input byte is true. */
int oracle_mm_orand(int64_t m, int64_t n, int64_t k, const uint8_t* A, const uint8_t* B,
                    uint8_t* C, const int64_t* rows, int64_t nrows) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (!rows) nrows = m;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = row_of(rows, r);
    uint8_t* c = C + r * n;
    for (int64_t j = 0; j < n; ++j) c[j] = 0;
    if (i < 0 || i >= m) continue;
    for (int64_t t = 0; t < k; ++t) {
      if (!A[i * k + t]) continue;
      const uint8_t* b = B + t * n;
      for (int64_t j = 0; j < n; ++j) c[j] |= (uint8_t)(b[j] != 0);
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Strassen-like recursions over exact int64 (pins only).
 * ------------------------------------------------------------------------- */

/* Copy / combine quadrant views.  A view is (ptr, leading dimension). */
static void q_add(int64_t r, int64_t c, const int64_t* X, int64_t ldx, const int64_t* Y,
                  int64_t ldy, int64_t sy, int64_t* Z, int64_t ldz) {
  for (int64_t i = 0; i < r; ++i)
    for (int64_t j = 0; j < c; ++j) Z[i * ldz + j] = X[i * ldx + j] + sy * Y[i * ldy + j];
}

static void q_copy(int64_t r, int64_t c, const int64_t* X, int64_t ldx, int64_t* Z, int64_t ldz) {
  for (int64_t i = 0; i < r; ++i)
    for (int64_t j = 0; j < c; ++j) Z[i * ldz + j] = X[i * ldx + j];
}

/* Classic product on strided views, used at the leaves of the recursion. */
static void leaf_i64(int64_t m, int64_t n, int64_t k, const int64_t* A, int64_t lda,
                     const int64_t* B, int64_t ldb, int64_t* C, int64_t ldc) {
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) C[i * ldc + j] = 0;
    for (int64_t t = 0; t < k; ++t) {
      const int64_t a = A[i * lda + t];
      for (int64_t j = 0; j < n; ++j) C[i * ldc + j] += a * B[t * ldb + j];
    }
  }
}

static int64_t* alloc_i64(int64_t count) {
  return (int64_t*)calloc((size_t)(count > 0 ? count : 1), sizeof(int64_t));
}

static int rec_i64(int variant, int levels, int64_t m, int64_t n, int64_t k, const int64_t* A,
                   int64_t lda, const int64_t* B, int64_t ldb, int64_t* C, int64_t ldc);

/*
 * One level of the paper's Strassen formulas (Section 5): the seven
 * products P_r = S_r (x) T_r with
 *   S1 = A00+A11, S2 = A10+A11, S3 = A00,     S4 = A11,
 *   S5 = A00+A01, S6 = A10-A00, S7 = A01-A11,
 *   T1 = B00+B11, T2 = B00,     T3 = B01-B11, T4 = B10-B00,
 *   T5 = B11,     T6 = B00+B01, T7 = B10+B11,
 * and C00 = P1+P4-P5+P7, C01 = P3+P5, C10 = P2+P4, C11 = P1+P3-P2+P6.
 */
static int strassen_level(int levels, int64_t m, int64_t n, int64_t k, const int64_t* A,
                          int64_t lda, const int64_t* B, int64_t ldb, int64_t* C, int64_t ldc) {
  const int64_t hm = m / 2, hn = n / 2, hk = k / 2;
  const int64_t *A00 = A, *A01 = A + hk, *A10 = A + hm * lda, *A11 = A + hm * lda + hk;
  const int64_t *B00 = B, *B01 = B + hn, *B10 = B + hk * ldb, *B11 = B + hk * ldb + hn;
  int64_t *S = alloc_i64(hm * hk), *T = alloc_i64(hk * hn), *P[8] = {0};
  int rc = (S && T) ? 0 : -2;
  for (int r = 1; r <= 7 && rc == 0; ++r) {
    P[r] = alloc_i64(hm * hn);
    if (!P[r]) { rc = -2; break; }
    switch (r) {
      case 1: q_add(hm, hk, A00, lda, A11, lda, 1, S, hk); q_add(hk, hn, B00, ldb, B11, ldb, 1, T, hn); break;
      case 2: q_add(hm, hk, A10, lda, A11, lda, 1, S, hk); q_copy(hk, hn, B00, ldb, T, hn); break;
      case 3: q_copy(hm, hk, A00, lda, S, hk); q_add(hk, hn, B01, ldb, B11, ldb, -1, T, hn); break;
      case 4: q_copy(hm, hk, A11, lda, S, hk); q_add(hk, hn, B10, ldb, B00, ldb, -1, T, hn); break;
      case 5: q_add(hm, hk, A00, lda, A01, lda, 1, S, hk); q_copy(hk, hn, B11, ldb, T, hn); break;
      case 6: q_add(hm, hk, A10, lda, A00, lda, -1, S, hk); q_add(hk, hn, B00, ldb, B01, ldb, 1, T, hn); break;
      case 7: q_add(hm, hk, A01, lda, A11, lda, -1, S, hk); q_add(hk, hn, B10, ldb, B11, ldb, 1, T, hn); break;
    }
    rc = rec_i64(0, levels - 1, hm, hn, hk, S, hk, T, hn, P[r], hn);
  }
  if (rc == 0) {
    int64_t *C00 = C, *C01 = C + hn, *C10 = C + hm * ldc, *C11 = C + hm * ldc + hn;
    for (int64_t i = 0; i < hm; ++i)
      for (int64_t j = 0; j < hn; ++j) {
        const int64_t o = i * hn + j;
        C00[i * ldc + j] = P[1][o] + P[4][o] - P[5][o] + P[7][o];
        C01[i * ldc + j] = P[3][o] + P[5][o];
        C10[i * ldc + j] = P[2][o] + P[4][o];
        C11[i * ldc + j] = P[1][o] + P[3][o] - P[2][o] + P[6][o];
      }
  }
  for (int r = 1; r <= 7; ++r) free(P[r]);
  free(S);
  free(T);
  return rc;
}

/*
 * One level of Strassen-Winograd (seven products, fifteen additions; the
 * variant the bilinear generalisation names), written from its algebra in
 * the paper's quadrant notation:
 *   S1 = A10+A11, S2 = S1-A00, S3 = A00-A10, S4 = A01-S2,
 *   T1 = B01-B00, T2 = B11-T1, T3 = B11-B01, T4 = T2-B10,
 *   P1 = A00 B00, P2 = A01 B10, P3 = S4 B11, P4 = A11 T4,
 *   P5 = S1 T1,   P6 = S2 T2,   P7 = S3 T3,
 *   U2 = P1+P6, U3 = U2+P7, U4 = U2+P5,
 *   C00 = P1+P2, C01 = U4+P3, C10 = U3-P4, C11 = U3+P5.
 */
static int winograd_level(int levels, int64_t m, int64_t n, int64_t k, const int64_t* A,
                          int64_t lda, const int64_t* B, int64_t ldb, int64_t* C, int64_t ldc) {
  const int64_t hm = m / 2, hn = n / 2, hk = k / 2;
  const int64_t *A00 = A, *A01 = A + hk, *A10 = A + hm * lda, *A11 = A + hm * lda + hk;
  const int64_t *B00 = B, *B01 = B + hn, *B10 = B + hk * ldb, *B11 = B + hk * ldb + hn;
  int64_t *S1 = alloc_i64(hm * hk), *S2 = alloc_i64(hm * hk), *S3 = alloc_i64(hm * hk),
          *S4 = alloc_i64(hm * hk);
  int64_t *T1 = alloc_i64(hk * hn), *T2 = alloc_i64(hk * hn), *T3 = alloc_i64(hk * hn),
          *T4 = alloc_i64(hk * hn);
  int64_t* P[8] = {0};
  int rc = (S1 && S2 && S3 && S4 && T1 && T2 && T3 && T4) ? 0 : -2;
  for (int r = 1; r <= 7 && rc == 0; ++r)
    if (!(P[r] = alloc_i64(hm * hn))) rc = -2;
  if (rc == 0) {
    q_add(hm, hk, A10, lda, A11, lda, 1, S1, hk);
    q_add(hm, hk, S1, hk, A00, lda, -1, S2, hk);
    q_add(hm, hk, A00, lda, A10, lda, -1, S3, hk);
    q_add(hm, hk, A01, lda, S2, hk, -1, S4, hk);
    q_add(hk, hn, B01, ldb, B00, ldb, -1, T1, hn);
    q_add(hk, hn, B11, ldb, T1, hn, -1, T2, hn);
    q_add(hk, hn, B11, ldb, B01, ldb, -1, T3, hn);
    q_add(hk, hn, T2, hn, B10, ldb, -1, T4, hn);
    const int64_t* l[8] = {0, A00, A01, S4, A11, S1, S2, S3};
    const int64_t ll[8] = {0, lda, lda, hk, lda, hk, hk, hk};
    const int64_t* rr[8] = {0, B00, B10, B11, T4, T1, T2, T3};
    const int64_t lr[8] = {0, ldb, ldb, ldb, hn, hn, hn, hn};
    for (int r = 1; r <= 7 && rc == 0; ++r)
      rc = rec_i64(1, levels - 1, hm, hn, hk, l[r], ll[r], rr[r], lr[r], P[r], hn);
  }
  if (rc == 0) {
    int64_t *C00 = C, *C01 = C + hn, *C10 = C + hm * ldc, *C11 = C + hm * ldc + hn;
    for (int64_t i = 0; i < hm; ++i)
      for (int64_t j = 0; j < hn; ++j) {
        const int64_t o = i * hn + j;
        const int64_t u2 = P[1][o] + P[6][o], u3 = u2 + P[7][o], u4 = u2 + P[5][o];
        C00[i * ldc + j] = P[1][o] + P[2][o];
        C01[i * ldc + j] = u4 + P[3][o];
        C10[i * ldc + j] = u3 - P[4][o];
        C11[i * ldc + j] = u3 + P[5][o];
      }
  }
  for (int r = 1; r <= 7; ++r) free(P[r]);
  free(S1); free(S2); free(S3); free(S4);
  free(T1); free(T2); free(T3); free(T4);
  return rc;
}

static int rec_i64(int variant, int levels, int64_t m, int64_t n, int64_t k, const int64_t* A,
                   int64_t lda, const int64_t* B, int64_t ldb, int64_t* C, int64_t ldc) {
  if (levels <= 0) {
    leaf_i64(m, n, k, A, lda, B, ldb, C, ldc);
    return 0;
  }
  if ((m | n | k) & 1) return -3;
  return variant == 0 ? strassen_level(levels, m, n, k, A, lda, B, ldb, C, ldc)
                      : winograd_level(levels, m, n, k, A, lda, B, ldb, C, ldc);
}

/* variant 0 = the paper's Strassen formulas, 1 = Strassen-Winograd.
 * m, n, k must be divisible by 2^levels.  Returns 0, or <0 on bad shape. */
int oracle_strassen_i64(int variant, int levels, int64_t m, int64_t n, int64_t k,
                        const int64_t* A, const int64_t* B, int64_t* C) {
  if (levels < 0 || m < 0 || n < 0 || k < 0) return -1;
  const int64_t mask = ((int64_t)1 << levels) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return -3;
  return rec_i64(variant, levels, m, n, k, A, k, B, n, C, n);
}

/* Floyd-Warshall all-pairs shortest paths on an n x n int64 distance matrix,
 * in place, with ORACLE_INF as "no edge" and sums clamped to ORACLE_INF. */
int oracle_floyd_warshall(int64_t n, int64_t* D) {
  if (n < 0) return -1;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t div = D[i * n + v];
      if (div >= ORACLE_INF) continue;
      for (int64_t j = 0; j < n; ++j) {
        int64_t s = div + D[v * n + j];
        if (s > ORACLE_INF) s = ORACLE_INF;
        if (s < D[i * n + j]) D[i * n + j] = s;
      }
    }
  return 0;
}

/* (min,+) closure A* = 1 (+) A (+) A^2 (+) ... of an n x n int64 matrix in
 * place: the semiring's 1 (0 on the diagonal, the sentinel elsewhere) is
 * folded in first, then Floyd-Warshall eliminates every vertex. */
int oracle_closure_minplus(int64_t n, int64_t* D) {
  if (n < 0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (D[i * n + i] > 0) D[i * n + i] = 0;
  return oracle_floyd_warshall(n, D);
}

/* (or, and) closure of an n x n 0/1 matrix in place (nonzero input = true):
 * reflexive diagonal, then Warshall's vertex elimination
 * R[i][j] |= R[i][v] & R[v][j] for v = 0 .. n-1. */
int oracle_closure_orand(int64_t n, uint8_t* R) {
  if (n < 0) return -1;
  for (int64_t e = 0; e < n * n; ++e) R[e] = R[e] ? 1 : 0;
  for (int64_t i = 0; i < n; ++i) R[i * n + i] = 1;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t i = 0; i < n; ++i) {
      if (!R[i * n + v]) continue;
      for (int64_t j = 0; j < n; ++j) R[i * n + j] |= R[v * n + j];
    }
  return 0;
}

/* Rows `rows[0..nrows)` of the (min,+) closure of an n x n matrix with
 * entries in [0, 2^30] (sentinel = no arc): one dense Dijkstra per source
 * (nonnegative arc lengths), O(n^2) each, sums clamped to the sentinel.
 * Writes out[r][j] = shortest distance rows[r] -> j (0 for j = rows[r]). */
int oracle_closure_minplus_rows(int64_t n, const int32_t* D, int64_t nrows, const int64_t* rows,
                                int64_t* out) {
  if (n < 0 || nrows < 0) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t src = rows[r];
    int64_t* dist = out + r * n;
    uint8_t* done = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!done) {
      bad = 1;
      continue;
    }
    for (int64_t j = 0; j < n; ++j) dist[j] = ORACLE_INF;
    dist[src] = 0;
    for (int64_t it = 0; it < n; ++it) {
      int64_t u = -1;
      for (int64_t j = 0; j < n; ++j)
        if (!done[j] && (u < 0 || dist[j] < dist[u])) u = j;
      if (u < 0 || dist[u] >= ORACLE_INF) break;
      done[u] = 1;
      for (int64_t j = 0; j < n; ++j) {
        const int64_t w = D[u * n + j];
        if (w >= ORACLE_INF || done[j]) continue;
        int64_t d = dist[u] + w;
        if (d > ORACLE_INF) d = ORACLE_INF;
        if (d < dist[j]) dist[j] = d;
      }
    }
    free(done);
  }
  return bad ? -2 : 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
