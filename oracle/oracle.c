/*
 * oracle.c -- plain, slow FP64 CPU oracle for TT arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The product path (the
 * CUDA library in paper_2011_06532_gb300/) never calls it, shares no code,
 * header, table or constant with it, and fails loudly when its own native
 * library is missing.
 *
 * Source of every formula: Al Daas, Ballard, Benner, "Parallel Algorithms for
 * Tensor Train Arithmetic" (arXiv 2011.06532).  Citations name the section,
 * algorithm or equation.
 *
 * Conventions
 *   A TT tensor has N cores; core n (0-based) is R[n] x I[n] x R[n+1] with
 *   R[0] = R[N] = 1 (Sec. 2.1).  Entry (a, i, b) of core n is stored at
 *   a + R[n]*(i + I[n]*b): the "vec-oriented" order of Sec. 3.1, in which the
 *   horizontal unfolding H (R[n] x I[n]R[n+1]) and the vertical unfolding
 *   V (R[n]I[n] x R[n+1]) of Sec. 2.2 are both column-major with no copy.
 *   All cores of one tensor are concatenated in one flat double array, core n
 *   starting at offset sum_{m<n} R[m]I[m]R[m+1].
 *   A full tensor is stored with its first index fastest.
 *
 * Parity status: every exported function is pinned by tests/test_oracle_pins.py
 * against closed forms, invariants, brute force on tiny tensors and values the
 * paper fixes.  No function here is "parity unpinned".
 *
 * Return codes: 0 ok, 1 invalid argument, 2 allocation failure, 4 numerical
 * failure (Jacobi not converged).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENUM 4

/* ------------------------------------------------------------------------ */
/* Householder QR (the local QR of Alg. 1 and Alg. 2; LAPACK-style reflectors) */
/* ------------------------------------------------------------------------ */

/*
 * In-place Householder QR of the m x b column-major matrix A (leading
 * dimension lda).  Reflector j is H_j = I - tau[j] v v^T with v[j] = 1 and
 * v[j+1..m-1] stored below the diagonal of column j; R is left on and above
 * the diagonal.  A zero subcolumn gives tau = 0 (H = I).  k = min(m, b)
 * reflectors are produced.
 */
static void house_qr(i64 m, i64 b, double *A, i64 lda, double *tau) {
  i64 k = m < b ? m : b;
  for (i64 j = 0; j < k; ++j) {
    double *col = A + j * lda;
    double alpha = col[j];
    double sig = 0.0;
    for (i64 r = j + 1; r < m; ++r) sig += col[r] * col[r];
    if (sig == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double nrm = sqrt(alpha * alpha + sig);
    double beta = alpha >= 0.0 ? -nrm : nrm;
    tau[j] = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (i64 r = j + 1; r < m; ++r) col[r] *= scal;
    col[j] = beta;
    for (i64 c = j + 1; c < b; ++c) {
      double *cc = A + c * lda;
      double w = cc[j];
      for (i64 r = j + 1; r < m; ++r) w += col[r] * cc[r];
      w *= tau[j];
      cc[j] -= w;
      for (i64 r = j + 1; r < m; ++r) cc[r] -= w * col[r];
    }
  }
}

/* Q = H_0 H_1 ... H_{k-1} [I_k; 0]  (m x k, column-major, ld m). */
static void house_form_q(i64 m, i64 k, const double *A, i64 lda, const double *tau, double *Q) {
  memset(Q, 0, sizeof(double) * (size_t)(m * k));
  for (i64 c = 0; c < k; ++c) Q[c + c * m] = 1.0;
  for (i64 j = k - 1; j >= 0; --j) {
    const double *v = A + j * lda;
    for (i64 c = j; c < k; ++c) {
      double *qc = Q + c * m;
      double w = qc[j];
      for (i64 r = j + 1; r < m; ++r) w += v[r] * qc[r];
      w *= tau[j];
      qc[j] -= w;
      for (i64 r = j + 1; r < m; ++r) qc[r] -= w * v[r];
    }
  }
}

/*
 * Economy QR A = Q R of the m x b column-major matrix A (not modified):
 * Q is m x k and R is k x b (both column-major), k = min(m, b).
 */
int orc_qr(i64 m, i64 b, const double *A, double *Q, double *R) {
  if (m < 1 || b < 1) return ORC_EINVAL;
  i64 k = m < b ? m : b;
  double *W = (double *)malloc(sizeof(double) * (size_t)(m * b));
  double *tau = (double *)malloc(sizeof(double) * (size_t)k);
  if (!W || !tau) {
    free(W);
    free(tau);
    return ORC_ENOMEM;
  }
  memcpy(W, A, sizeof(double) * (size_t)(m * b));
  house_qr(m, b, W, m, tau);
  for (i64 c = 0; c < b; ++c)
    for (i64 r = 0; r < k; ++r) R[r + k * c] = (r <= c) ? W[r + m * c] : 0.0;
  house_form_q(m, k, W, m, tau, Q);
  free(W);
  free(tau);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes): the SVD of Alg. 2, applied to the R of a QR */
/* ------------------------------------------------------------------------ */

/*
 * B (m x n, m >= n, column-major) is overwritten by U*diag(S); V (n x n) holds
 * the accumulated rotations.  Sweeps over all column pairs (p, q) in row-cyclic
 * order until no pair has |b_p^T b_q| > tol * ||b_p|| ||b_q||.
 * Returns the number of sweeps, or -1 if not converged.
 */
static int jacobi_sweeps(i64 m, i64 n, double *B, double *V, int maxsweeps) {
  double tol = 1e-15 * (double)(m > 1 ? m : 1);
  for (i64 c = 0; c < n * n; ++c) V[c] = 0.0;
  for (i64 c = 0; c < n; ++c) V[c + n * c] = 1.0;
  for (int sweep = 1; sweep <= maxsweeps; ++sweep) {
    int rotated = 0;
    for (i64 p = 0; p < n - 1; ++p) {
      for (i64 q = p + 1; q < n; ++q) {
        double *bp = B + p * m, *bq = B + q * m;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (i64 r = 0; r < m; ++r) {
          alpha += bp[r] * bp[r];
          beta += bq[r] * bq[r];
          gamma += bp[r] * bq[r];
        }
        if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (i64 r = 0; r < m; ++r) {
          double x = bp[r], y = bq[r];
          bp[r] = c * x - s * y;
          bq[r] = s * x + c * y;
        }
        double *vp = V + p * n, *vq = V + q * n;
        for (i64 r = 0; r < n; ++r) {
          double x = vp[r], y = vq[r];
          vp[r] = c * x - s * y;
          vq[r] = s * x + c * y;
        }
      }
    }
    if (!rotated) return sweep;
  }
  return -1;
}

static double norm2_pairwise(const double *x, i64 n, i64 stride);

/*
 * Thin SVD B = U diag(S) V^T of the m x n column-major matrix B (not
 * modified), k = min(m, n): U is m x k, S has k entries in non-increasing
 * order, V is n x k.  A wide B is handled through B^T.  Ties keep the original
 * column order.  A column with sigma = 0 gets U(:,j) = e_j (only reached for a
 * zero matrix by the rounding code, where any unit vector is valid).
 */
int orc_svd(i64 m, i64 n, const double *B, double *U, double *S, double *V) {
  if (m < 1 || n < 1) return ORC_EINVAL;
  int wide = m < n;
  i64 mm = wide ? n : m, nn = wide ? m : n; /* work on an mm x nn tall matrix */
  double *W = (double *)malloc(sizeof(double) * (size_t)(mm * nn));
  double *Vw = (double *)malloc(sizeof(double) * (size_t)(nn * nn));
  double *sig = (double *)malloc(sizeof(double) * (size_t)nn);
  i64 *ord = (i64 *)malloc(sizeof(i64) * (size_t)nn);
  if (!W || !Vw || !sig || !ord) {
    free(W); free(Vw); free(sig); free(ord);
    return ORC_ENOMEM;
  }
  if (!wide) {
    memcpy(W, B, sizeof(double) * (size_t)(m * n));
  } else {
    for (i64 c = 0; c < n; ++c)
      for (i64 r = 0; r < m; ++r) W[c + n * r] = B[r + m * c];
  }
  int sw = jacobi_sweeps(mm, nn, W, Vw, 100);
  if (sw < 0) {
    free(W); free(Vw); free(sig); free(ord);
    return ORC_ENUM;
  }
  for (i64 c = 0; c < nn; ++c) {
    sig[c] = norm2_pairwise(W + c * mm, mm, 1);
    ord[c] = c;
  }
  /* stable insertion sort by decreasing sigma */
  for (i64 a = 1; a < nn; ++a) {
    i64 key = ord[a];
    i64 b2 = a - 1;
    while (b2 >= 0 && sig[ord[b2]] < sig[key]) {
      ord[b2 + 1] = ord[b2];
      --b2;
    }
    ord[b2 + 1] = key;
  }
  /* left vectors of the tall matrix: W(:,c)/sigma_c; right vectors: Vw */
  double *Ut = wide ? V : U; /* tall-side left vectors, mm x nn */
  double *Vt = wide ? U : V; /* tall-side right vectors, nn x nn */
  for (i64 j = 0; j < nn; ++j) {
    i64 c = ord[j];
    S[j] = sig[c];
    for (i64 r = 0; r < mm; ++r) Ut[r + mm * j] = sig[c] > 0.0 ? W[r + mm * c] / sig[c] : (r == j ? 1.0 : 0.0);
    for (i64 r = 0; r < nn; ++r) Vt[r + nn * j] = Vw[r + nn * c];
  }
  free(W); free(Vw); free(sig); free(ord);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

/* sqrt(sum x_k^2) with pairwise summation of the squares. */
static double sumsq_pairwise(const double *x, i64 n, i64 stride) {
  if (n <= 16) {
    double s = 0.0;
    for (i64 k = 0; k < n; ++k) s += x[k * stride] * x[k * stride];
    return s;
  }
  i64 h = n / 2;
  return sumsq_pairwise(x, h, stride) + sumsq_pairwise(x + h * stride, n - h, stride);
}
static double norm2_pairwise(const double *x, i64 n, i64 stride) { return sqrt(sumsq_pairwise(x, n, stride)); }

static i64 core_size(const i64 *I, const i64 *R, i64 n) { return R[n] * I[n] * R[n + 1]; }

static int check_tt(i64 N, const i64 *I, const i64 *R) {
  if (N < 1 || !I || !R) return ORC_EINVAL;
  if (R[0] != 1 || R[N] != 1) return ORC_EINVAL;
  for (i64 n = 0; n < N; ++n)
    if (I[n] < 1 || R[n] < 1) return ORC_EINVAL;
  return ORC_OK;
}

/* Working TT: one malloc'd buffer per core, each with the capacity of the input core. */
typedef struct {
  i64 N;
  i64 *I, *r;
  double **c;
} wtt;

static void wtt_free(wtt *w) {
  if (w->c)
    for (i64 n = 0; n < w->N; ++n) free(w->c[n]);
  free(w->c);
  free(w->I);
  free(w->r);
  memset(w, 0, sizeof(*w));
}

static int wtt_load(wtt *w, i64 N, const i64 *I, const i64 *R, const double *cores) {
  memset(w, 0, sizeof(*w));
  w->N = N;
  w->I = (i64 *)malloc(sizeof(i64) * (size_t)N);
  w->r = (i64 *)malloc(sizeof(i64) * (size_t)(N + 1));
  w->c = (double **)calloc((size_t)N, sizeof(double *));
  if (!w->I || !w->r || !w->c) {
    wtt_free(w);
    return ORC_ENOMEM;
  }
  memcpy(w->I, I, sizeof(i64) * (size_t)N);
  memcpy(w->r, R, sizeof(i64) * (size_t)(N + 1));
  i64 off = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 sz = core_size(I, R, n);
    w->c[n] = (double *)malloc(sizeof(double) * (size_t)sz);
    if (!w->c[n]) {
      wtt_free(w);
      return ORC_ENOMEM;
    }
    memcpy(w->c[n], cores + off, sizeof(double) * (size_t)sz);
    off += sz;
  }
  return ORC_OK;
}

static void wtt_store(const wtt *w, i64 *R_out, double *out) {
  memcpy(R_out, w->r, sizeof(i64) * (size_t)(w->N + 1));
  i64 off = 0;
  for (i64 n = 0; n < w->N; ++n) {
    i64 sz = core_size(w->I, w->r, n);
    memcpy(out + off, w->c[n], sizeof(double) * (size_t)sz);
    off += sz;
  }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: TT right-orthonormalization                                       */
/* ------------------------------------------------------------------------ */

/*
 * For n = N-1 down to 1: QR of H(X_n)^T = Q R (economy, k = min(I_n R_{n+1},
 * R_n)); H(X_n) <- Q^T (rank R_n becomes k); V(X_{n-1}) <- V(X_{n-1}) R^T,
 * the pass of the triangular factor to the left neighbour (Alg. 1; Eq.
 * nonunique of Sec. 2.1 shows the tensor is unchanged).
 */
static int right_orth(wtt *w) {
  for (i64 n = w->N - 1; n >= 1; --n) {
    i64 b = w->r[n], In = w->I[n], rr = w->r[n + 1];
    i64 m = In * rr;
    i64 k = m < b ? m : b;
    double *A = (double *)malloc(sizeof(double) * (size_t)(m * b));
    double *Q = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *R = (double *)malloc(sizeof(double) * (size_t)(k * b));
    if (!A || !Q || !R) {
      free(A); free(Q); free(R);
      return ORC_ENOMEM;
    }
    /* A = H(X_n)^T: A[col, a] = H[a, col] */
    const double *X = w->c[n];
    for (i64 a = 0; a < b; ++a)
      for (i64 col = 0; col < m; ++col) A[col + m * a] = X[a + b * col];
    int st = orc_qr(m, b, A, Q, R);
    if (st) {
      free(A); free(Q); free(R);
      return st;
    }
    /* H(X_n) <- Q^T (k x m) */
    double *Xn = w->c[n];
    for (i64 col = 0; col < m; ++col)
      for (i64 a = 0; a < k; ++a) Xn[a + k * col] = Q[col + m * a];
    /* V(X_{n-1}) (M x b) <- V(X_{n-1}) R^T (M x k) */
    i64 M = w->r[n - 1] * w->I[n - 1];
    double *P = w->c[n - 1];
    double *T = (double *)malloc(sizeof(double) * (size_t)(M * k));
    if (!T) {
      free(A); free(Q); free(R);
      return ORC_ENOMEM;
    }
    for (i64 a2 = 0; a2 < k; ++a2)
      for (i64 row = 0; row < M; ++row) {
        double s = 0.0;
        for (i64 a = 0; a < b; ++a) s += P[row + M * a] * R[a2 + k * a];
        T[row + M * a2] = s;
      }
    memcpy(P, T, sizeof(double) * (size_t)(M * k));
    w->r[n] = k;
    free(T); free(A); free(Q); free(R);
  }
  return ORC_OK;
}

int orc_tt_orth_right(i64 N, const i64 *I, const i64 *R, const double *cores, i64 *R_out, double *out) {
  int st = check_tt(N, I, R);
  if (st) return st;
  wtt w;
  if ((st = wtt_load(&w, N, I, R, cores))) return st;
  st = right_orth(&w);
  if (!st) wtt_store(&w, R_out, out);
  wtt_free(&w);
  return st;
}

/* Norm via orthonormalization (Sec. 3.2.4, second approach): ||X|| = ||X_1||_F
 * once X is right-orthonormal (Sec. 2.3). */
int orc_tt_norm(i64 N, const i64 *I, const i64 *R, const double *cores, double *nrm) {
  int st = check_tt(N, I, R);
  if (st) return st;
  wtt w;
  if ((st = wtt_load(&w, N, I, R, cores))) return st;
  st = right_orth(&w);
  if (!st) *nrm = norm2_pairwise(w.c[0], core_size(w.I, w.r, 0), 1);
  wtt_free(&w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Left-orthonormalization: the mirror of Alg. 1 ("the approach for left     */
/* orthonormalization is analogous", Sec. 3.4; left-orthonormal TTs, Sec. 2.3)*/
/* ------------------------------------------------------------------------ */

/*
 * For n = 0 up to N-2: QR of V(X_n) = Q R (economy, k = min(R_n I_n, R_{n+1}));
 * V(X_n) <- Q (rank R_{n+1} becomes k); H(X_{n+1}) <- R H(X_{n+1}), the pass of
 * the triangular factor to the right neighbour (Eq. nonunique of Sec. 2.1: the
 * tensor is unchanged).  Afterwards V(X_n) has orthonormal columns for n < N-1
 * and ||X|| = ||X_N||_F (Sec. 2.3, Sec. 3.2.4).
 */
static int left_orth(wtt *w) {
  for (i64 n = 0; n + 1 < w->N; ++n) {
    i64 m = w->r[n] * w->I[n], b = w->r[n + 1];
    i64 k = m < b ? m : b;
    double *Q = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *R = (double *)malloc(sizeof(double) * (size_t)(k * b));
    i64 cols = w->I[n + 1] * w->r[n + 2];
    double *T = (double *)malloc(sizeof(double) * (size_t)(k * cols));
    if (!Q || !R || !T) {
      free(Q); free(R); free(T);
      return ORC_ENOMEM;
    }
    int st = orc_qr(m, b, w->c[n], Q, R);
    if (st) {
      free(Q); free(R); free(T);
      return st;
    }
    /* V(X_n) <- Q (m x k) */
    memcpy(w->c[n], Q, sizeof(double) * (size_t)(m * k));
    /* H(X_{n+1}) (b x cols) <- R H(X_{n+1}) (k x cols) */
    const double *H = w->c[n + 1];
    for (i64 col = 0; col < cols; ++col)
      for (i64 a2 = 0; a2 < k; ++a2) {
        double s = 0.0;
        for (i64 a = 0; a < b; ++a) s += R[a2 + k * a] * H[a + b * col];
        T[a2 + k * col] = s;
      }
    memcpy(w->c[n + 1], T, sizeof(double) * (size_t)(k * cols));
    w->r[n + 1] = k;
    free(Q); free(R); free(T);
  }
  return ORC_OK;
}

int orc_tt_orth_left(i64 N, const i64 *I, const i64 *R, const double *cores, i64 *R_out, double *out) {
  int st = check_tt(N, I, R);
  if (st) return st;
  wtt w;
  if ((st = wtt_load(&w, N, I, R, cores))) return st;
  st = left_orth(&w);
  if (!st) wtt_store(&w, R_out, out);
  wtt_free(&w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: TT rounding                                                        */
/* ------------------------------------------------------------------------ */

/*
 * Rank rule for the delta-truncated SVD (Alg. 2, Alg. 6): the smallest L >= 1
 * whose discarded tail sum_{j >= L} sigma_j^2 is <= delta^2.  Tails are summed
 * from the smallest sigma upward.  Returns L and stores the tail in *tail.
 */
static i64 pick_rank(i64 k, const double *S, double delta, double *tail) {
  double *t = (double *)malloc(sizeof(double) * (size_t)(k + 1));
  if (!t) return -1;
  t[k] = 0.0;
  for (i64 j = k - 1; j >= 0; --j) t[j] = t[j + 1] + S[j] * S[j];
  double d2 = delta * delta;
  i64 L = k;
  for (i64 l = 1; l <= k; ++l)
    if (t[l] <= d2) {
      L = l;
      break;
    }
  *tail = t[L];
  free(t);
  return L;
}

/*
 * TT rounding, Alg. 2 (right-to-left orthonormalization, then left-to-right
 * truncation).  Input tensor (N, I, R, cores); output ranks in R_out[0..N] and
 * cores (flat, new ranks) in out, which must hold at least as many doubles as
 * the input.  Optional diagnostics (may be NULL): nrm_out = ||X|| from
 * ||X_1||_F after the first sweep, delta_out = eps ||X|| / sqrt(N-1), tails_out
 * [N-1] = discarded sum of squared singular values at each cut.
 * N = 1: nothing to truncate, the tensor is copied.
 */
int orc_tt_round(i64 N, const i64 *I, const i64 *R, const double *cores, double eps, i64 *R_out, double *out,
                 double *nrm_out, double *delta_out, double *tails_out) {
  int st = check_tt(N, I, R);
  if (st) return st;
  if (!(eps >= 0.0)) return ORC_EINVAL;
  wtt w;
  if ((st = wtt_load(&w, N, I, R, cores))) return st;
  if (N == 1) {
    if (nrm_out) *nrm_out = norm2_pairwise(w.c[0], I[0], 1);
    if (delta_out) *delta_out = 0.0;
    wtt_store(&w, R_out, out);
    wtt_free(&w);
    return ORC_OK;
  }
  if ((st = right_orth(&w))) {
    wtt_free(&w);
    return st;
  }
  double nrm = norm2_pairwise(w.c[0], core_size(w.I, w.r, 0), 1);
  double delta = eps * nrm / sqrt((double)(N - 1));
  if (nrm_out) *nrm_out = nrm;
  if (delta_out) *delta_out = delta;
  for (i64 n = 0; n + 1 < N && !st; ++n) {
    i64 m = w.r[n] * w.I[n], b = w.r[n + 1];
    i64 k = m < b ? m : b;
    double *Q = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *Rf = (double *)malloc(sizeof(double) * (size_t)(k * b));
    double *Ur = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *S = (double *)malloc(sizeof(double) * (size_t)k);
    double *Vr = (double *)malloc(sizeof(double) * (size_t)(b * k));
    if (!Q || !Rf || !Ur || !S || !Vr) st = ORC_ENOMEM;
    /* SVD of V(X_n) through its QR: V = Q R, R = Ur S Vr^T */
    if (!st) st = orc_qr(m, b, w.c[n], Q, Rf);
    if (!st) st = orc_svd(k, b, Rf, Ur, S, Vr);
    i64 L = 0;
    double tail = 0.0;
    if (!st) {
      L = pick_rank(k, S, delta, &tail);
      if (L < 1) st = ORC_ENOMEM;
    }
    if (!st) {
      if (tails_out) tails_out[n] = tail;
      /* V(X_n) <- Q Ur(:, :L)  (m x L) */
      double *Xn = w.c[n];
      for (i64 l = 0; l < L; ++l)
        for (i64 row = 0; row < m; ++row) {
          double s = 0.0;
          for (i64 j = 0; j < k; ++j) s += Q[row + m * j] * Ur[j + k * l];
          Xn[row + m * l] = s;
        }
      /* H(X_{n+1}) <- diag(S(:L)) Vr(:, :L)^T H(X_{n+1})  (L x I_{n+1} R_{n+2}) */
      i64 cols = w.I[n + 1] * w.r[n + 2];
      double *H = w.c[n + 1];
      double *T = (double *)malloc(sizeof(double) * (size_t)(L * cols));
      if (!T) {
        st = ORC_ENOMEM;
      } else {
        for (i64 col = 0; col < cols; ++col)
          for (i64 l = 0; l < L; ++l) {
            double s = 0.0;
            for (i64 a = 0; a < b; ++a) s += Vr[a + b * l] * H[a + b * col];
            T[l + L * col] = S[l] * s;
          }
        memcpy(H, T, sizeof(double) * (size_t)(L * cols));
        free(T);
        w.r[n + 1] = L;
      }
    }
    free(Q); free(Rf); free(Ur); free(S); free(Vr);
  }
  if (!st) wtt_store(&w, R_out, out);
  wtt_free(&w);
  return st;
}

/*
 * TT rounding in the other ordering (Sec. 3.4: "the other ordering works
 * analogously"; the LRL variant of Sec. 4.3.2): left-orthonormalization, then
 * truncation from right to left.  ||X|| = ||X_N||_F after the first sweep
 * (Sec. 2.3), delta = eps ||X|| / sqrt(N-1) as in Alg. 2.  For n = N-1 down to
 * 1 the SVD of H(X_n) is taken through the QR of its transpose:
 * H(X_n)^T = Q R, R = Ur S Vr^T, so H(X_n) = Vr S (Q Ur)^T; the rank L follows
 * the same rule as Alg. 2 (pick_rank), H(X_n) <- (Q Ur(:, :L))^T and
 * V(X_{n-1}) <- V(X_{n-1}) Vr(:, :L) diag(S(:L)).  Arguments as orc_tt_round;
 * tails_out[n-1] is the tail discarded at the cut between cores n-1 and n.
 */
int orc_tt_round_lrl(i64 N, const i64 *I, const i64 *R, const double *cores, double eps, i64 *R_out, double *out,
                     double *nrm_out, double *delta_out, double *tails_out) {
  int st = check_tt(N, I, R);
  if (st) return st;
  if (!(eps >= 0.0)) return ORC_EINVAL;
  wtt w;
  if ((st = wtt_load(&w, N, I, R, cores))) return st;
  if (N == 1) {
    if (nrm_out) *nrm_out = norm2_pairwise(w.c[0], I[0], 1);
    if (delta_out) *delta_out = 0.0;
    wtt_store(&w, R_out, out);
    wtt_free(&w);
    return ORC_OK;
  }
  if ((st = left_orth(&w))) {
    wtt_free(&w);
    return st;
  }
  double nrm = norm2_pairwise(w.c[N - 1], core_size(w.I, w.r, N - 1), 1);
  double delta = eps * nrm / sqrt((double)(N - 1));
  if (nrm_out) *nrm_out = nrm;
  if (delta_out) *delta_out = delta;
  for (i64 n = N - 1; n >= 1 && !st; --n) {
    i64 b = w.r[n], m = w.I[n] * w.r[n + 1];
    i64 k = m < b ? m : b;
    double *A = (double *)malloc(sizeof(double) * (size_t)(m * b));
    double *Q = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *Rf = (double *)malloc(sizeof(double) * (size_t)(k * b));
    double *Ur = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *S = (double *)malloc(sizeof(double) * (size_t)k);
    double *Vr = (double *)malloc(sizeof(double) * (size_t)(b * k));
    if (!A || !Q || !Rf || !Ur || !S || !Vr) st = ORC_ENOMEM;
    if (!st) {
      /* A = H(X_n)^T (m x b) */
      const double *X = w.c[n];
      for (i64 a = 0; a < b; ++a)
        for (i64 col = 0; col < m; ++col) A[col + m * a] = X[a + b * col];
      st = orc_qr(m, b, A, Q, Rf);
    }
    if (!st) st = orc_svd(k, b, Rf, Ur, S, Vr);
    i64 L = 0;
    double tail = 0.0;
    if (!st) {
      L = pick_rank(k, S, delta, &tail);
      if (L < 1) st = ORC_ENOMEM;
    }
    if (!st) {
      if (tails_out) tails_out[n - 1] = tail;
      /* H(X_n) <- (Q Ur(:, :L))^T  (L x m) */
      double *Xn = w.c[n];
      for (i64 col = 0; col < m; ++col)
        for (i64 l = 0; l < L; ++l) {
          double s = 0.0;
          for (i64 j = 0; j < k; ++j) s += Q[col + m * j] * Ur[j + k * l];
          Xn[l + L * col] = s;
        }
      /* V(X_{n-1}) (M x b) <- V(X_{n-1}) Vr(:, :L) diag(S(:L))  (M x L) */
      i64 M = w.r[n - 1] * w.I[n - 1];
      double *P = w.c[n - 1];
      double *T = (double *)malloc(sizeof(double) * (size_t)(M * L));
      if (!T) {
        st = ORC_ENOMEM;
      } else {
        for (i64 l = 0; l < L; ++l)
          for (i64 row = 0; row < M; ++row) {
            double s2 = 0.0;
            for (i64 a = 0; a < b; ++a) s2 += P[row + M * a] * Vr[a + b * l];
            T[row + M * l] = S[l] * s2;
          }
        memcpy(P, T, sizeof(double) * (size_t)(M * L));
        free(T);
        w.r[n] = L;
      }
    }
    free(A); free(Q); free(Rf); free(Ur); free(S); free(Vr);
  }
  if (!st) wtt_store(&w, R_out, out);
  wtt_free(&w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Basic operations (Sec. 3.2)                                                */
/* ------------------------------------------------------------------------ */

/*
 * Summation, Sec. 3.2.1: interior slices are block diagonal diag(X_n(i),
 * Y_n(i)); the first core is [X_1 Y_1], the last [X_N; Y_N]; ranks add.
 * For N = 1 the single core is the entrywise sum.  Ro receives the ranks.
 */
int orc_tt_add(i64 N, const i64 *I, const i64 *Ra, const double *a, const i64 *Rb, const double *b, i64 *Ro,
               double *out) {
  if (check_tt(N, I, Ra) || check_tt(N, I, Rb)) return ORC_EINVAL;
  if (N == 1) {
    Ro[0] = Ro[1] = 1;
    for (i64 i = 0; i < I[0]; ++i) out[i] = a[i] + b[i];
    return ORC_OK;
  }
  Ro[0] = 1;
  Ro[N] = 1;
  for (i64 n = 1; n < N; ++n) Ro[n] = Ra[n] + Rb[n];
  i64 oa = 0, ob = 0, oo = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 ra0 = Ra[n], ra1 = Ra[n + 1], rb0 = Rb[n], rb1 = Rb[n + 1], r0 = Ro[n], r1 = Ro[n + 1], In = I[n];
    const double *A = a + oa, *B = b + ob;
    double *Z = out + oo;
    memset(Z, 0, sizeof(double) * (size_t)(r0 * In * r1));
    /* offsets of the Y block: rows shift by ra0 except in the first core,
       columns shift by ra1 except in the last core */
    i64 row_shift = (n == 0) ? 0 : ra0;
    i64 col_shift = (n == N - 1) ? 0 : ra1;
    for (i64 c = 0; c < ra1; ++c)
      for (i64 i = 0; i < In; ++i)
        for (i64 r = 0; r < ra0; ++r) Z[r + r0 * (i + In * c)] = A[r + ra0 * (i + In * c)];
    for (i64 c = 0; c < rb1; ++c)
      for (i64 i = 0; i < In; ++i)
        for (i64 r = 0; r < rb0; ++r) Z[(r + row_shift) + r0 * (i + In * (c + col_shift))] = B[r + rb0 * (i + In * c)];
    oa += ra0 * In * ra1;
    ob += rb0 * In * rb1;
    oo += r0 * In * r1;
  }
  return ORC_OK;
}

/*
 * Hadamard product, Sec. 3.2.2: Z_n(i) = X_n(i) kron Y_n(i), ranks multiply.
 * Kronecker index convention: row (p, q) -> p * rows(Y) + q, likewise columns.
 */
int orc_tt_hadamard(i64 N, const i64 *I, const i64 *Ra, const double *a, const i64 *Rb, const double *b, i64 *Ro,
                    double *out) {
  if (check_tt(N, I, Ra) || check_tt(N, I, Rb)) return ORC_EINVAL;
  for (i64 n = 0; n <= N; ++n) Ro[n] = Ra[n] * Rb[n];
  i64 oa = 0, ob = 0, oo = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 ra0 = Ra[n], ra1 = Ra[n + 1], rb0 = Rb[n], rb1 = Rb[n + 1], r0 = Ro[n], In = I[n];
    const double *A = a + oa, *B = b + ob;
    double *Z = out + oo;
    for (i64 i = 0; i < In; ++i)
      for (i64 p = 0; p < ra0; ++p)
        for (i64 s = 0; s < ra1; ++s)
          for (i64 q = 0; q < rb0; ++q)
            for (i64 t = 0; t < rb1; ++t)
              Z[(p * rb0 + q) + r0 * (i + In * (s * rb1 + t))] = A[p + ra0 * (i + In * s)] * B[q + rb0 * (i + In * t)];
    oa += ra0 * In * ra1;
    ob += rb0 * In * rb1;
    oo += r0 * In * Ro[n + 1];
  }
  return ORC_OK;
}

/*
 * Inner product <X, Y>, Sec. 3.2.3, Eq. innerprodsum: W_0 = [1];
 * W_n = sum_i Y_n(i)^T W_{n-1} X_n(i) (R^Y x R^X); the result is the final 1x1 W.
 */
int orc_tt_dot(i64 N, const i64 *I, const i64 *Rx, const double *x, const i64 *Ry, const double *y, double *out) {
  if (check_tt(N, I, Rx) || check_tt(N, I, Ry)) return ORC_EINVAL;
  i64 maxr = 1;
  for (i64 n = 0; n <= N; ++n) {
    if (Rx[n] > maxr) maxr = Rx[n];
    if (Ry[n] > maxr) maxr = Ry[n];
  }
  double *W = (double *)calloc((size_t)(maxr * maxr), sizeof(double));
  double *Wn = (double *)calloc((size_t)(maxr * maxr), sizeof(double));
  double *T = (double *)calloc((size_t)(maxr * maxr), sizeof(double));
  if (!W || !Wn || !T) {
    free(W); free(Wn); free(T);
    return ORC_ENOMEM;
  }
  W[0] = 1.0; /* W is Ry[n] x Rx[n], column-major */
  i64 ox = 0, oy = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 px = Rx[n], qx = Rx[n + 1], py = Ry[n], qy = Ry[n + 1], In = I[n];
    const double *X = x + ox, *Y = y + oy;
    memset(Wn, 0, sizeof(double) * (size_t)(qy * qx));
    for (i64 i = 0; i < In; ++i) {
      /* T = W X_n(i)   (py x qx) */
      for (i64 s = 0; s < qx; ++s)
        for (i64 p = 0; p < py; ++p) {
          double acc = 0.0;
          for (i64 r = 0; r < px; ++r) acc += W[p + py * r] * X[r + px * (i + In * s)];
          T[p + py * s] = acc;
        }
      /* Wn += Y_n(i)^T T   (qy x qx) */
      for (i64 s = 0; s < qx; ++s)
        for (i64 q = 0; q < qy; ++q) {
          double acc = 0.0;
          for (i64 p = 0; p < py; ++p) acc += Y[p + py * (i + In * q)] * T[p + py * s];
          Wn[q + qy * s] += acc;
        }
    }
    memcpy(W, Wn, sizeof(double) * (size_t)(qy * qx));
    ox += px * In * qx;
    oy += py * In * qy;
  }
  *out = W[0];
  free(W); free(Wn); free(T);
  return ORC_OK;
}

/*
 * The same inner product through the two-multiplication form of Sec. 3.2.3:
 * H(Z_n) = W_{n-1} H(X_n), then W_n = V(Y_n)^T V(Z_n).
 */
int orc_tt_dot_two_step(i64 N, const i64 *I, const i64 *Rx, const double *x, const i64 *Ry, const double *y,
                        double *out) {
  if (check_tt(N, I, Rx) || check_tt(N, I, Ry)) return ORC_EINVAL;
  i64 maxc = 1, maxr = 1;
  for (i64 n = 0; n < N; ++n) {
    i64 c = Ry[n] * I[n] * Rx[n + 1];
    if (c > maxc) maxc = c;
  }
  for (i64 n = 0; n <= N; ++n) {
    if (Rx[n] > maxr) maxr = Rx[n];
    if (Ry[n] > maxr) maxr = Ry[n];
  }
  double *W = (double *)calloc((size_t)(maxr * maxr), sizeof(double));
  double *Z = (double *)calloc((size_t)maxc, sizeof(double));
  if (!W || !Z) {
    free(W); free(Z);
    return ORC_ENOMEM;
  }
  W[0] = 1.0;
  i64 ox = 0, oy = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 px = Rx[n], qx = Rx[n + 1], py = Ry[n], qy = Ry[n + 1], In = I[n];
    const double *X = x + ox, *Y = y + oy;
    i64 cols = In * qx;
    /* H(Z) (py x cols) = W (py x px) * H(X) (px x cols) */
    for (i64 c = 0; c < cols; ++c)
      for (i64 p = 0; p < py; ++p) {
        double acc = 0.0;
        for (i64 r = 0; r < px; ++r) acc += W[p + py * r] * X[r + px * c];
        Z[p + py * c] = acc;
      }
    /* W_n (qy x qx) = V(Y)^T (qy x py In) * V(Z) (py In x qx) */
    i64 rows = py * In;
    for (i64 s = 0; s < qx; ++s)
      for (i64 q = 0; q < qy; ++q) {
        double acc = 0.0;
        for (i64 row = 0; row < rows; ++row) acc += Y[row + rows * q] * Z[row + rows * s];
        W[q + qy * s] = acc;
      }
    ox += px * In * qx;
    oy += py * In * qy;
  }
  *out = W[0];
  free(W); free(Z);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Full-tensor helpers for brute-force checks on tiny tensors                 */
/* ------------------------------------------------------------------------ */

/*
 * Expands a TT to its full tensor (first index fastest) by the chain of slice
 * products of Sec. 2.1: T_(1:n) = T_(1:n-1) H(X_n), reshaped.
 */
int orc_tt_full(i64 N, const i64 *I, const i64 *R, const double *cores, double *full) {
  if (check_tt(N, I, R)) return ORC_EINVAL;
  i64 total = 1;
  for (i64 n = 0; n < N; ++n) total *= I[n];
  /* T holds a (P x r) column-major matrix; its size never exceeds total * maxr */
  i64 maxr = 1;
  for (i64 n = 0; n <= N; ++n)
    if (R[n] > maxr) maxr = R[n];
  double *T = (double *)malloc(sizeof(double) * (size_t)(total * maxr));
  double *T2 = (double *)malloc(sizeof(double) * (size_t)(total * maxr));
  if (!T || !T2) {
    free(T); free(T2);
    return ORC_ENOMEM;
  }
  T[0] = 1.0;
  i64 P = 1, off = 0;
  for (i64 n = 0; n < N; ++n) {
    i64 r0 = R[n], r1 = R[n + 1], In = I[n];
    const double *C = cores + off;
    /* T2 (P x In r1) = T (P x r0) * H(C) (r0 x In r1) */
    for (i64 col = 0; col < In * r1; ++col)
      for (i64 p = 0; p < P; ++p) {
        double acc = 0.0;
        for (i64 a = 0; a < r0; ++a) acc += T[p + P * a] * C[a + r0 * col];
        T2[p + P * col] = acc;
      }
    double *sw = T; T = T2; T2 = sw;
    P *= In;
    off += r0 * In * r1;
  }
  memcpy(full, T, sizeof(double) * (size_t)total);
  free(T); free(T2);
  return ORC_OK;
}

/*
 * TT-SVD of a full tensor (first index fastest) with the same delta rule as
 * rounding: delta = eps ||A|| / sqrt(N-1); for n = 0..N-2 the remainder C,
 * viewed as (r_n I_n) x rest, gets a delta-truncated SVD; core n = U(:, :L),
 * C <- diag(S(:L)) V(:, :L)^T.  The last core is the final remainder.  In
 * exact arithmetic this is the sequence of projections that Alg. 2 applies
 * (Sec. 2.4, Eq. quadprodTT), so it serves as a brute-force check of rounding.
 * R_out gets the ranks; out (flat cores) must hold total * maxrank doubles.
 */
int orc_tt_svd(i64 N, const i64 *I, const double *full, double eps, i64 *R_out, double *out) {
  if (N < 1 || !(eps >= 0.0)) return ORC_EINVAL;
  i64 total = 1;
  for (i64 n = 0; n < N; ++n) {
    if (I[n] < 1) return ORC_EINVAL;
    total *= I[n];
  }
  double *C = (double *)malloc(sizeof(double) * (size_t)total);
  if (!C) return ORC_ENOMEM;
  memcpy(C, full, sizeof(double) * (size_t)total);
  double nrm = norm2_pairwise(C, total, 1);
  double delta = N > 1 ? eps * nrm / sqrt((double)(N - 1)) : 0.0;
  R_out[0] = 1;
  i64 r = 1, rest = total, off = 0;
  int st = ORC_OK;
  for (i64 n = 0; n + 1 < N && !st; ++n) {
    i64 m = r * I[n];
    rest /= I[n];
    i64 k = m < rest ? m : rest;
    double *U = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *S = (double *)malloc(sizeof(double) * (size_t)k);
    double *V = (double *)malloc(sizeof(double) * (size_t)(rest * k));
    if (!U || !S || !V) st = ORC_ENOMEM;
    if (!st) st = orc_svd(m, rest, C, U, S, V);
    if (!st) {
      double tail;
      i64 L = pick_rank(k, S, delta, &tail);
      memcpy(out + off, U, sizeof(double) * (size_t)(m * L));
      off += m * L;
      /* C <- diag(S) V^T  (L x rest) */
      for (i64 col = 0; col < rest; ++col)
        for (i64 l = 0; l < L; ++l) C[l + L * col] = S[l] * V[col + rest * l];
      r = L;
      R_out[n + 1] = L;
    }
    free(U); free(S); free(V);
  }
  if (!st) {
    memcpy(out + off, C, sizeof(double) * (size_t)(r * I[N - 1]));
    R_out[N] = 1;
  }
  free(C);
  return st;
}
