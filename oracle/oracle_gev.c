/*
 * FP64 CPU oracle for the dense generalized Hermitian eigenproblem  H C = S C Lambda  (Eq. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  The GPU solver never calls it and shares no code with it.
 *
 * It computes the plain definition of the method's result by a deliberately slow, different route
 * from the GPU path (section "Current Status of the Implementation", reduction steps 1-3 and the
 * back-transformation C = U^{-1} C~):
 *
 *   1. unblocked Cholesky  S = L L^H  (L = U^H, lower; the paper writes S = U^T U),
 *   2. A = L^{-1} H L^{-H}  by two forward substitutions (no explicit inverse),
 *   3. one-stage Householder tridiagonalisation  A = Q T Q^H  (the "ELPA1" one-stage route),
 *   4. implicit QL with Wilkinson shifts on the real tridiagonal T, accumulating rotations,
 *   5. stable ascending sort, keep the k lowest, back-transform  Y = Q Z,
 *   6. C = L^{-H} Y  by back substitution, then a per-column phase normalisation,
 *   7. residual ||HC - SC Lambda||_1 / (||H||_1 ||C||_1) and orthogonality ||C^H S C - I||_1.
 *
 * The file is compiled twice: once as real (prefix oracle_d_) and once with ORACLE_COMPLEX defined
 * (prefix oracle_z_, scalars are C99 double complex, same memory layout as numpy complex128).
 * All matrices are column-major with a leading dimension; only the lower triangle of H and S is read.
 * Loops marked with OpenMP compute every output element in one thread, in a fixed order, so the
 * results do not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_COMPLEX
typedef double complex scalar;
#define CONJ(x) conj(x)
#define RE(x) creal(x)
#define ABS2(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define SABS(x) cabs(x)
#define FN(name) oracle_z_##name
#else
typedef double scalar;
#define CONJ(x) (x)
#define RE(x) (x)
#define ABS2(x) ((x) * (x))
#define SABS(x) fabs(x)
#define FN(name) oracle_d_##name
#endif

#define AT(M, ld, i, j) (M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)]

/* ---------------------------------------------------------------------------------------------
 * Step 1 (reduction step 1): unblocked Cholesky of the lower triangle, in place.
 * Returns 0, or p+1 when the p-th (0-based) pivot is not positive (S not positive definite,
 * the precondition stated alongside the reduction steps).  The strict upper triangle is zeroed.
 * ------------------------------------------------------------------------------------------- */
int FN(potrf)(int n, scalar* A, int lda) {
  for (int j = 0; j < n; ++j) {
    double djj = RE(AT(A, lda, j, j));
    for (int p = 0; p < j; ++p) djj -= ABS2(AT(A, lda, j, p));
    if (!(djj > 0.0)) return j + 1;
    double ljj = sqrt(djj);
    AT(A, lda, j, j) = ljj;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      scalar s = AT(A, lda, i, j);
      for (int p = 0; p < j; ++p) s -= AT(A, lda, i, p) * CONJ(AT(A, lda, j, p));
      AT(A, lda, i, j) = s / ljj;
    }
  }
  for (int j = 1; j < n; ++j)
    for (int i = 0; i < j; ++i) AT(A, lda, i, j) = 0;
  return 0;
}

/* Solve L X = B in place (L lower, non-unit), B is n x m. Forward substitution per column. */
static void forward_subst(int n, int m, const scalar* L, int ldl, scalar* B, int ldb) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < n; ++i) {
      scalar s = AT(B, ldb, i, c);
      for (int p = 0; p < i; ++p) s -= AT(L, ldl, i, p) * AT(B, ldb, p, c);
      AT(B, ldb, i, c) = s / AT(L, ldl, i, i);
    }
  }
}

/* ---------------------------------------------------------------------------------------------
 * Step 2 (reduction steps 2-3): A = L^{-1} H L^{-H}, with H given by its lower triangle.
 * X = L^{-1} H by forward substitution; then A^H = L^{-1} X^H by a second forward substitution.
 * A is returned full (both triangles) after symmetrisation A <- (A + A^H)/2; the largest
 * |A - A^H| entry before symmetrisation is written to *asym (a rounding diagnostic).
 * ------------------------------------------------------------------------------------------- */
void FN(reduce)(int n, const scalar* H, int ldh, const scalar* L, int ldl, scalar* A, int lda,
                double* asym) {
  scalar* X = (scalar*)malloc(sizeof(scalar) * (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      AT(X, n, i, j) = (i >= j) ? AT(H, ldh, i, j) : CONJ(AT(H, ldh, j, i));
  forward_subst(n, n, L, ldl, X, n); /* X = L^{-1} H */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(A, lda, i, j) = CONJ(AT(X, n, j, i)); /* A <- X^H */
  forward_subst(n, n, L, ldl, A, lda); /* A = L^{-1} X^H = (X L^{-H})^H */
  /* The buffer now holds M = (L^{-1} H L^{-H})^H, so the product's entry (i,j) is conj(M(j,i)).
     Replace the buffer by the Hermitian part of the product. */
  double worst = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int i = j; i < n; ++i) {
      scalar pij = CONJ(AT(A, lda, j, i)); /* product (i,j) */
      scalar pji = CONJ(AT(A, lda, i, j)); /* product (j,i) */
      double d = SABS(pij - CONJ(pji));
      if (d > worst) worst = d;
      scalar m = 0.5 * (pij + CONJ(pji));
      if (i == j) m = RE(m);
      AT(A, lda, i, j) = m;
      AT(A, lda, j, i) = CONJ(m);
    }
  }
  if (asym) *asym = worst;
  free(X);
}

/* ---------------------------------------------------------------------------------------------
 * Step 3 (one-stage tridiagonalisation): A (full Hermitian, both triangles, overwritten) is
 * reduced to a real symmetric tridiagonal T = Q^H A Q with Q = H_0 H_1 ... H_{n-3},
 * H_j = I - tau_j v_j v_j^H acting on rows j+1..n-1, v_j(0) = 1.  Each reflector is chosen so
 * that H_j^H applied to column j below the diagonal gives (beta, 0, ..., 0) with beta real, so T is
 * real also for complex input.  d[0..n-1], e[0..n-2] receive T; v_j(1:) is stored in A below the
 * subdiagonal of column j and tau_j in tau[j].
 * ------------------------------------------------------------------------------------------- */
void FN(sytrd)(int n, scalar* A, int lda, double* d, double* e, scalar* tau) {
  scalar* v = (scalar*)malloc(sizeof(scalar) * (size_t)n);
  scalar* y = (scalar*)malloc(sizeof(scalar) * (size_t)n);
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1; /* length of the column below the diagonal */
    scalar* x = &AT(A, lda, j + 1, j);
    scalar alpha = x[0];
    double xnorm2 = 0.0;
    for (int i = 1; i < m; ++i) xnorm2 += ABS2(x[i]);
    scalar t = 0;
    double beta;
#ifdef ORACLE_COMPLEX
    int trivial = (xnorm2 == 0.0 && cimag(alpha) == 0.0);
#else
    int trivial = (xnorm2 == 0.0);
#endif
    if (trivial) {
      beta = RE(alpha);
      t = 0;
      v[0] = 1;
      for (int i = 1; i < m; ++i) v[i] = 0;
    } else {
      double nrm = sqrt(ABS2(alpha) + xnorm2);
      beta = (RE(alpha) >= 0.0) ? -nrm : nrm;
      t = (beta - alpha) / beta;
      scalar scale = 1.0 / (alpha - beta);
      v[0] = 1;
      for (int i = 1; i < m; ++i) v[i] = x[i] * scale;
    }
    tau[j] = t;
    d[j] = RE(AT(A, lda, j, j));
    e[j] = beta;
    /* store reflector; column j below the diagonal becomes (beta, 0, ...) in T */
    for (int i = 1; i < m; ++i) x[i] = v[i];
    x[0] = beta;
    AT(A, lda, j, j + 1) = beta;
    if (t != 0) {
      /* trailing block B = A[j+1:, j+1:] <- H^H B H with H = I - t v v^H:
         y = B v; w = t y - (|t|^2/2) (v^H y) v; B <- B - w v^H - v w^H  */
      scalar* B = &AT(A, lda, j + 1, j + 1);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < m; ++i) {
        scalar s = 0;
        for (int p = 0; p < m; ++p) s += AT(B, lda, i, p) * v[p];
        y[i] = s;
      }
      scalar vy = 0;
      for (int i = 0; i < m; ++i) vy += CONJ(v[i]) * y[i];
      double half = 0.5 * ABS2(t) * RE(vy);
      for (int i = 0; i < m; ++i) y[i] = t * y[i] - half * v[i]; /* y now holds w */
#pragma omp parallel for schedule(static)
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < m; ++i)
          AT(B, lda, i, c) -= y[i] * CONJ(v[c]) + v[i] * CONJ(y[c]);
      for (int i = 0; i < m; ++i) AT(B, lda, i, i) = RE(AT(B, lda, i, i));
    }
  }
  d[n - 1] = RE(AT(A, lda, n - 1, n - 1));
  if (n >= 1) tau[n - 1] = 0;
  free(v);
  free(y);
}

/* Apply Q = H_0 H_1 ... H_{n-3} (reflectors stored by sytrd in A and tau) to Z (n x k), in place:
   Z <- Q Z, applying H_{n-3} first. */
void FN(ormtr)(int n, int k, const scalar* A, int lda, const scalar* tau, scalar* Z, int ldz) {
  for (int j = n - 2; j >= 0; --j) {
    scalar t = tau[j];
    if (t == 0) continue;
    const int m = n - j - 1;
    const scalar* vt = &AT(A, lda, j + 1, j); /* vt[0] holds beta; the reflector's v[0] is 1 */
#pragma omp parallel for schedule(static)
    for (int c = 0; c < k; ++c) {
      scalar* z = &AT(Z, ldz, j + 1, c);
      scalar s = z[0];
      for (int i = 1; i < m; ++i) s += CONJ(vt[i]) * z[i];
      s *= t;
      z[0] -= s;
      for (int i = 1; i < m; ++i) z[i] -= vt[i] * s;
    }
  }
}

/* ---------------------------------------------------------------------------------------------
 * Step 4: implicit QL with Wilkinson shifts on the real symmetric tridiagonal (d, e), e[i]
 * coupling rows i and i+1.  Rotations are accumulated into the real n x n matrix Z, which the
 * caller initialises (identity for the eigenvectors of T).  Returns 0, or -1 when more than
 * 30*n QL iterations were needed in total.  Eigenvalues are left unsorted in d.
 * ------------------------------------------------------------------------------------------- */
static int steql_impl(int n, double* d, double* e_in, double* Z, int ldz) {
  if (n <= 0) return 0;
  double* e = (double*)calloc((size_t)n, sizeof(double));
  for (int i = 0; i + 1 < n; ++i) e[i] = e_in[i];
  const double eps = 2.220446049250313e-16;
  long total = 0, cap = 30L * n;
  int status = 0;
  for (int l = 0; l < n; ++l) {
    for (;;) {
      int m = l;
      while (m + 1 < n) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
        ++m;
      }
      if (m == l) break;
      if (++total > cap) {
        status = -1;
        goto done;
      }
      /* shift: eigenvalue of the leading 2x2 block at l closest to d[l], in the form g = d[m] - shift */
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      int early = 0;
      for (int i = m - 1; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) { /* the rotation vanished: split and restart at l */
          d[i + 1] -= p;
          e[m] = 0.0;
          early = 1;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        for (int q = 0; q < n; ++q) {
          double zi = AT(Z, ldz, q, i), zi1 = AT(Z, ldz, q, i + 1);
          AT(Z, ldz, q, i + 1) = s * zi + c * zi1;
          AT(Z, ldz, q, i) = c * zi - s * zi1;
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
done:
  free(e);
  return status;
}

/* Stable ascending order of w[0..n-1] (insertion into a merge sort on indices). */
static void stable_argsort(int n, const double* w, int* idx) {
  int* tmp = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int width = 1; width < n; width *= 2) {
    for (int lo = 0; lo < n; lo += 2 * width) {
      int mid = lo + width < n ? lo + width : n, hi = lo + 2 * width < n ? lo + 2 * width : n;
      int a = lo, b = mid, o = lo;
      while (a < mid && b < hi) tmp[o++] = (w[idx[b]] < w[idx[a]]) ? idx[b++] : idx[a++];
      while (a < mid) tmp[o++] = idx[a++];
      while (b < hi) tmp[o++] = idx[b++];
    }
    memcpy(idx, tmp, sizeof(int) * (size_t)n);
  }
  free(tmp);
}

/* Phase normalisation of each column: the entry of largest modulus (first index on exact ties)
   is made real and positive. */
void FN(normalize_phase)(int n, int k, scalar* C, int ldc) {
  for (int c = 0; c < k; ++c) {
    int best = 0;
    double bv = -1.0;
    for (int i = 0; i < n; ++i) {
      double a = ABS2(AT(C, ldc, i, c));
      if (a > bv) { bv = a; best = i; }
    }
    scalar piv = AT(C, ldc, best, c);
    double ap = SABS(piv);
    if (ap == 0.0) continue;
    scalar ph = CONJ(piv) / ap;
    for (int i = 0; i < n; ++i) AT(C, ldc, i, c) *= ph;
    AT(C, ldc, best, c) = ap;
  }
}

static double norm1_herm_lower(int n, const scalar* M, int ld) {
  /* 1-norm of the Hermitian matrix whose lower triangle is stored */
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += SABS(i >= j ? AT(M, ld, i, j) : AT(M, ld, j, i));
    if (s > best) best = s;
  }
  return best;
}

/* Residual ||H C - S C diag(w)||_1 / (||H||_1 ||C||_1) and orthogonality ||C^H S C - I||_1
   (H, S lower triangles; C is n x k). */
void FN(check)(int n, int k, const scalar* H, int ldh, const scalar* S, int lds, const double* w,
               const scalar* C, int ldc, double* resid, double* ortho) {
  scalar* HC = (scalar*)malloc(sizeof(scalar) * (size_t)n * (k > 0 ? k : 1));
  scalar* SC = (scalar*)malloc(sizeof(scalar) * (size_t)n * (k > 0 ? k : 1));
#pragma omp parallel for schedule(static)
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < n; ++i) {
      scalar h = 0, s = 0;
      for (int p = 0; p < n; ++p) {
        scalar hip = i >= p ? AT(H, ldh, i, p) : CONJ(AT(H, ldh, p, i));
        scalar sip = i >= p ? AT(S, lds, i, p) : CONJ(AT(S, lds, p, i));
        h += hip * AT(C, ldc, p, c);
        s += sip * AT(C, ldc, p, c);
      }
      AT(HC, n, i, c) = h;
      AT(SC, n, i, c) = s;
    }
  }
  double rmax = 0.0, cmax = 0.0;
  for (int c = 0; c < k; ++c) {
    double rs = 0.0, cs = 0.0;
    for (int i = 0; i < n; ++i) {
      rs += SABS(AT(HC, n, i, c) - AT(SC, n, i, c) * w[c]);
      cs += SABS(AT(C, ldc, i, c));
    }
    if (rs > rmax) rmax = rs;
    if (cs > cmax) cmax = cs;
  }
  double hn = norm1_herm_lower(n, H, ldh);
  *resid = (hn > 0 && cmax > 0) ? rmax / (hn * cmax) : rmax;
  double omax = 0.0;
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    for (int r = 0; r < k; ++r) {
      scalar g = 0;
      for (int i = 0; i < n; ++i) g += CONJ(AT(C, ldc, i, r)) * AT(SC, n, i, c);
      if (r == c) g -= 1.0;
      s += SABS(g);
    }
    if (s > omax) omax = s;
  }
  *ortho = omax;
  free(HC);
  free(SC);
}

/* ---------------------------------------------------------------------------------------------
 * The whole oracle: k lowest eigenpairs of the pencil (H, S).
 *   inputs : H, S lower triangles (n x n, ld), 1 <= k <= n
 *   outputs: w[k] ascending, C (n x k, ldc), diag[4] = {residual, orthogonality, asymmetry of A,
 *            QL iterations status}
 *   returns 0; p+1 > 0 when S is not positive definite at pivot p; -1 when QL did not converge;
 *            -2 for bad arguments.
 * ------------------------------------------------------------------------------------------- */
int FN(gev)(int n, const scalar* H, int ldh, const scalar* S, int lds, int k, double* w,
            scalar* C, int ldc, double* diag) {
  if (n < 0 || k < 0 || k > n || ldh < (n > 1 ? n : 1) || lds < (n > 1 ? n : 1) ||
      ldc < (n > 1 ? n : 1))
    return -2;
  if (n == 0 || k == 0) return 0;
  const size_t nn = (size_t)n * n;
  scalar* L = (scalar*)malloc(sizeof(scalar) * nn);
  scalar* A = (scalar*)malloc(sizeof(scalar) * nn);
  double* d = (double*)malloc(sizeof(double) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  scalar* tau = (scalar*)malloc(sizeof(scalar) * n);
  double* Zr = (double*)calloc(nn, sizeof(double));
  int* idx = (int*)malloc(sizeof(int) * n);
  scalar* Y = (scalar*)malloc(sizeof(scalar) * (size_t)n * k);
  int status = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(L, n, i, j) = (i >= j) ? AT(S, lds, i, j) : 0;
  int info = FN(potrf)(n, L, n);
  if (info) { status = info; goto out; }
  double asym = 0.0;
  FN(reduce)(n, H, ldh, L, n, A, n, &asym);
  FN(sytrd)(n, A, n, d, e, tau);
  for (int i = 0; i < n; ++i) AT(Zr, n, i, i) = 1.0;
  if (steql_impl(n, d, e, Zr, n)) { status = -1; goto out; }
  stable_argsort(n, d, idx);
  for (int c = 0; c < k; ++c) {
    w[c] = d[idx[c]];
    for (int i = 0; i < n; ++i) AT(Y, n, i, c) = AT(Zr, n, i, idx[c]);
  }
  FN(ormtr)(n, k, A, n, tau, Y, n); /* Y = Q Z */
  /* C = L^{-H} Y: back substitution with the upper-triangular L^H */
#pragma omp parallel for schedule(static)
  for (int c = 0; c < k; ++c) {
    for (int i = n - 1; i >= 0; --i) {
      scalar s = AT(Y, n, i, c);
      for (int p = i + 1; p < n; ++p) s -= CONJ(AT(L, n, p, i)) * AT(C, ldc, p, c);
      AT(C, ldc, i, c) = s / AT(L, n, i, i);
    }
  }
  FN(normalize_phase)(n, k, C, ldc);
  if (diag) {
    double r = 0, o = 0;
    FN(check)(n, k, H, ldh, S, lds, w, C, ldc, &r, &o);
    diag[0] = r;
    diag[1] = o;
    diag[2] = asym;
    diag[3] = 0;
  }
out:
  free(L); free(A); free(d); free(e); free(tau); free(Zr); free(idx); free(Y);
  return status;
}

/* ---------------------------------------------------------------------------------------------
 * Ill-conditioned overlap (section "Current Status of the Implementation", the paragraph on
 * numerically singular S): the pencil is transformed to the basis of the eigenvectors D_i of S,
 * omitting every D_i whose eigenvalue sigma_i is below delta, and the reduced standard problem is
 * solved.  In the paper's order:
 *   1. S = D diag(sigma) D^H  (one-stage tridiagonalisation + QL of the full Hermitian S, ascending),
 *   2. keep the m eigenvectors with sigma_i >= delta: X = D_kept diag(sigma_kept)^{-1/2}  (n x m),
 *   3. H~ = X^H H X  (m x m, plain products, Hermitian part kept),
 *   4. H~ Y = Y Lambda  (one-stage tridiagonalisation + QL), the k lowest,
 *   5. C = X Y, then the per-column phase normalisation.
 * C^H S C = I on the kept space.  *m receives the kept count.  Returns 0; -1 when QL did not
 * converge; -2 for bad arguments; -3 when k > m (fewer kept basis vectors than wanted pairs).
 * ------------------------------------------------------------------------------------------- */
static int herm_eig(int n, scalar* A, double* w, scalar* V) {
  /* all eigenpairs of the full Hermitian A (overwritten): w ascending, V (n x n) */
  double* d = (double*)malloc(sizeof(double) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  scalar* tau = (scalar*)malloc(sizeof(scalar) * n);
  double* Zr = (double*)calloc((size_t)n * n, sizeof(double));
  int* idx = (int*)malloc(sizeof(int) * n);
  int st = 0;
  FN(sytrd)(n, A, n, d, e, tau);
  for (int i = 0; i < n; ++i) AT(Zr, n, i, i) = 1.0;
  if (steql_impl(n, d, e, Zr, n)) { st = -1; goto out; }
  stable_argsort(n, d, idx);
  for (int c = 0; c < n; ++c) {
    w[c] = d[idx[c]];
    for (int i = 0; i < n; ++i) AT(V, n, i, c) = AT(Zr, n, i, idx[c]);
  }
  FN(ormtr)(n, n, A, n, tau, V, n);
out:
  free(d); free(e); free(tau); free(Zr); free(idx);
  return st;
}

int FN(gev_reduced)(int n, const scalar* H, int ldh, const scalar* S, int lds, double delta, int k,
                    double* w, scalar* C, int ldc, int* m_out) {
  if (n < 1 || k < 1 || k > n || ldh < n || lds < n || ldc < n || !(delta >= 0.0)) return -2;
  const size_t nn = (size_t)n * n;
  scalar* A = (scalar*)malloc(sizeof(scalar) * nn);
  scalar* D = (scalar*)malloc(sizeof(scalar) * nn);
  double* sig = (double*)malloc(sizeof(double) * n);
  int status = 0, m = 0;
  scalar *X = NULL, *HX = NULL, *Ht = NULL, *Yt = NULL;
  double* wt = NULL;
  /* 1. eigenvectors of S */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(A, n, i, j) = (i >= j) ? AT(S, lds, i, j) : CONJ(AT(S, lds, j, i));
  if (herm_eig(n, A, sig, D)) { status = -1; goto out; }
  /* 2. the kept basis: sigma ascending, so the kept ones are the last m */
  int first = 0;
  while (first < n && sig[first] < delta) ++first;
  m = n - first;
  if (m_out) *m_out = m;
  if (k > m) { status = -3; goto out; }
  X = (scalar*)malloc(sizeof(scalar) * (size_t)n * m);
  for (int c = 0; c < m; ++c) {
    const double f = 1.0 / sqrt(sig[first + c]);
    for (int i = 0; i < n; ++i) AT(X, n, i, c) = f * AT(D, n, i, first + c);
  }
  /* 3. H~ = X^H H X */
  HX = (scalar*)malloc(sizeof(scalar) * (size_t)n * m);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < n; ++i) {
      scalar acc = 0;
      for (int p = 0; p < n; ++p)
        acc += ((i >= p) ? AT(H, ldh, i, p) : CONJ(AT(H, ldh, p, i))) * AT(X, n, p, c);
      AT(HX, n, i, c) = acc;
    }
  Ht = (scalar*)malloc(sizeof(scalar) * (size_t)m * m);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c)
    for (int r = 0; r < m; ++r) {
      scalar acc = 0;
      for (int i = 0; i < n; ++i) acc += CONJ(AT(X, n, i, r)) * AT(HX, n, i, c);
      AT(Ht, m, r, c) = acc;
    }
  for (int c = 0; c < m; ++c)
    for (int r = c; r < m; ++r) {
      scalar h = 0.5 * (AT(Ht, m, r, c) + CONJ(AT(Ht, m, c, r)));
      if (r == c) h = RE(h);
      AT(Ht, m, r, c) = h;
      AT(Ht, m, c, r) = CONJ(h);
    }
  /* 4. the reduced standard problem */
  Yt = (scalar*)malloc(sizeof(scalar) * (size_t)m * m);
  wt = (double*)malloc(sizeof(double) * m);
  if (herm_eig(m, Ht, wt, Yt)) { status = -1; goto out; }
  /* 5. C = X Y (the k lowest) */
#pragma omp parallel for schedule(static)
  for (int c = 0; c < k; ++c)
    for (int i = 0; i < n; ++i) {
      scalar acc = 0;
      for (int r = 0; r < m; ++r) acc += AT(X, n, i, r) * AT(Yt, m, r, c);
      AT(C, ldc, i, c) = acc;
    }
  for (int c = 0; c < k; ++c) w[c] = wt[c];
  FN(normalize_phase)(n, k, C, ldc);
out:
  free(A); free(D); free(sig); free(X); free(HX); free(Ht); free(Yt); free(wt);
  return status;
}

/* ---------------------------------------------------------------------------------------------
 * Density matrix of the computed orbitals (section "Circumventing the eigenvalue problem"):
 *   P_ij = sum_l  g_l conj(c_li) c_lj,
 * with c_li = C(i, l) the coefficient of basis function i in orbital l (column l of C).  The weights
 * g_l are the occupation numbers f_l for the density matrix, or f_l * lambda_l for its
 * energy-weighted counterpart (section "ELSI").  The plain definition: every entry of the full n x n
 * P is the sum over l, taken in increasing l.
 * ------------------------------------------------------------------------------------------- */
void FN(density)(int n, int k, const scalar* C, int ldc, const double* g, scalar* P, int ldp) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      scalar s = 0;
      for (int l = 0; l < k; ++l) s += g[l] * CONJ(AT(C, ldc, i, l)) * AT(C, ldc, j, l);
      AT(P, ldp, i, j) = s;
    }
  }
}

#ifndef ORACLE_COMPLEX
/* The tridiagonal solver alone (real): eigenvalues ascending into w (length n) and the
   corresponding orthonormal eigenvectors into Z (n x n, ldz).  Returns 0 or -1 (no convergence). */
int oracle_d_steql(int n, const double* d_in, const double* e_in, double* w, double* Z, int ldz) {
  if (n <= 0) return 0;
  double* d = (double*)malloc(sizeof(double) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* Zt = (double*)calloc((size_t)n * n, sizeof(double));
  int* idx = (int*)malloc(sizeof(int) * n);
  memcpy(d, d_in, sizeof(double) * n);
  for (int i = 0; i + 1 < n; ++i) e[i] = e_in[i];
  for (int i = 0; i < n; ++i) AT(Zt, n, i, i) = 1.0;
  int st = steql_impl(n, d, e, Zt, n);
  if (st == 0) {
    stable_argsort(n, d, idx);
    for (int c = 0; c < n; ++c) {
      w[c] = d[idx[c]];
      for (int i = 0; i < n; ++i) AT(Z, ldz, i, c) = AT(Zt, n, i, idx[c]);
    }
  }
  free(d); free(e); free(Zt); free(idx);
  return st;
}
#endif
