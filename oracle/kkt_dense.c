/*
 * Oracle for the batched nonlinear constraint projection -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the package's smoke() and bench.py's cpu_baseline / reference arm may load
 * this file's shared library.  The CUDA library never links, includes or calls it, and it
 * shares no code with the CUDA library.
 *
 * What it computes (the paper's projection, eq. (2) of the Sampling section and the
 * projection restated in "Jacobian Structure"):
 *
 *     u* = argmin_u  1/2 ||u - u_hat||^2   subject to  h(u) = 0,
 *
 * solved by plain Newton iterations on the KKT conditions of Appendix B (the
 * "newtonKKTsystem" equation): with L(u, lam) = f(u) + lam^T h(u), F = [grad_u L ; h] and
 *
 *     [ W  J^T ] [du  ]     [ grad f + J^T lam ]
 *     [ J  0   ] [dlam] = - [ h                ],   W = Hess_uu L,
 *
 * each Newton system is assembled as a DENSE symmetric indefinite matrix and factored with
 * Bunch-Kaufman diagonal pivoting (P K P^T = L D L^T, D with 1x1 and 2x2 blocks).
 *
 * Constraint form.  Every constraint row r of the problems built by problems.py is
 *     h_r(u) = sum_j A_rj u_j + sum_j Q_rj u_j^2 - b_r,
 * a linear part plus a diagonal quadratic part (initial-condition, mass, energy, boundary
 * invariant, discrete divergence and kinetic-energy rows all have this form).  Hence
 *     J_rj = A_rj + 2 Q_rj u_j,     W = I + sum_r lam_r * 2 diag(Q_r).
 *
 * Globalisation (the paper is silent; the reading taken here):
 *   Newton-Raphson on F(u, lam) = 0 exactly as Appendix B derives it, from u = u0 (default
 *   u_hat), lam = 0; stop when ||F||_inf <= tol_kkt; merit phi = 1/2 ||F||_2^2, for which
 *   the Newton step is a descent direction whenever K is nonsingular; Armijo backtracking
 *   (halve t until phi(t) <= (1 - 2 c1 t) phi(0), at most max_backtracks halvings) from
 *   the largest t <= 1 that keeps every diagonal entry of W at >= w_keep times its current
 *   value (W is diagonal and linear in lam for these constraint forms; this keeps W positive
 *   definite, hence K of inertia (n, m, 0) when J has full row rank, and makes a limit
 *   point a strict local minimum).  At a converged point the inertia of K is checked
 *   (second-order sufficient condition); failure gives status NOT_MINIMUM.
 *   Optional (max_corrections > 0): Ipopt-style inertia correction W <- W + delta I.
 *
 * Separability.  The objective is a sum over variables and each constraint touches a
 * subset of them, so the projection splits exactly into independent problems, one per
 * connected component of the variable/active-row graph (the paper's block-diagonal
 * structure across samples, "Jacobian Structure", applied inside a sample as well).
 * With split_components = 1 each component is its own Newton-KKT problem with its own line
 * search and stopping test; with 0 the whole sample is one system (used to check the split).
 * Rows with active = 0 (rows implied by other rows, e.g. the t = 0 mass row that the
 * worked example of Appendix C also omits) take no part in the solve and get lam = 0.
 *
 * Adjoint (implicit-function theorem on F(u, lam; u_hat, theta) = 0): solve
 *     K [a ; b] = [gbar ; 0]
 * with the KKT matrix at the solution (no inertia correction); then dL/du_hat = a and
 * dL/dtheta = -b^T dh/dtheta (the latter is applied in problems.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORA_OK = 0, ORA_MAXITER = 1, ORA_LINESEARCH = 2, ORA_NONFINITE = 3, ORA_SINGULAR = 6,
       ORA_NOT_MINIMUM = 7 };

typedef struct {
  double tol_kkt;
  int max_iter;
  int max_backtracks;
  double c1;
  double delta0;
  int max_corrections;
  int split_components;
  double w_keep;
  int restore;          /* 1: keep grad_u L = 0 along the iteration (start u_hat) */
} ora_opts;

typedef struct {
  int iters;
  int backtracks;
  int status;
  int corrections;
  double kkt_inf;
  double phi;
} ora_stats;

/* ------------------------------------------------------------------------------------- */
/* Bunch-Kaufman LDL^T on a full N x N symmetric matrix (Golub & Van Loan, Matrix         */
/* Computations, diagonal pivoting with the Bunch-Kaufman strategy, alpha=(1+sqrt 17)/8). */
/* ------------------------------------------------------------------------------------- */

typedef struct {
  int N;
  double *L;    /* N x N unit lower triangular (row-major) */
  double *D;    /* N x N block diagonal (only 1x1 / 2x2 blocks are nonzero) */
  int *perm;    /* (P A P^T)[i][j] = A[perm[i]][perm[j]] */
  int *bsize;   /* bsize[k] = 1 or 2 at the first index of each block, 0 at the second */
  int n_pos, n_neg, n_zero;
} ldl_t;

static void ldl_alloc(ldl_t *f, int N) {
  f->N = N;
  f->L = (double *)calloc((size_t)N * N, sizeof(double));
  f->D = (double *)calloc((size_t)N * N, sizeof(double));
  f->perm = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
  f->bsize = (int *)calloc((size_t)(N > 0 ? N : 1), sizeof(int));
}

static void ldl_free(ldl_t *f) {
  free(f->L); free(f->D); free(f->perm); free(f->bsize);
}

/* symmetric interchange of rows/columns p and q of the working matrix M (N x N), of rows p
 * and q of the already computed columns 0..k-1 of L, and of the permutation. */
static void bk_swap(int N, double *M, double *L, int *perm, int k, int p, int q) {
  if (p == q) return;
  for (int j = 0; j < N; ++j) { double t = M[p * N + j]; M[p * N + j] = M[q * N + j]; M[q * N + j] = t; }
  for (int i = 0; i < N; ++i) { double t = M[i * N + p]; M[i * N + p] = M[i * N + q]; M[i * N + q] = t; }
  for (int j = 0; j < k; ++j) { double t = L[p * N + j]; L[p * N + j] = L[q * N + j]; L[q * N + j] = t; }
  int t = perm[p]; perm[p] = perm[q]; perm[q] = t;
}

/* Factor A (N x N, full symmetric, row-major; not modified).  Fills f.  The inertia counts
 * eigenvalue signs of D; a pivot whose magnitude is below ztol counts as zero. */
static void ldl_factor(const double *A, ldl_t *f, double ztol) {
  const int N = f->N;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  double *M = (double *)malloc(sizeof(double) * (size_t)N * N + 8);
  memcpy(M, A, sizeof(double) * (size_t)N * N);
  memset(f->L, 0, sizeof(double) * (size_t)N * N);
  memset(f->D, 0, sizeof(double) * (size_t)N * N);
  for (int i = 0; i < N; ++i) { f->perm[i] = i; f->bsize[i] = 0; }
  f->n_pos = f->n_neg = f->n_zero = 0;
  int k = 0;
  while (k < N) {
    double akk = fabs(M[k * N + k]);
    double colmax = 0.0;
    int r = k;
    for (int i = k + 1; i < N; ++i) {
      double v = fabs(M[i * N + k]);
      if (v > colmax) { colmax = v; r = i; }
    }
    int s = 1;
    if (akk >= alpha * colmax || colmax == 0.0) {
      s = 1;
    } else {
      double rowmax = 0.0;
      for (int j = k; j < N; ++j) {
        if (j == r) continue;
        double v = fabs(M[r * N + j]);
        if (v > rowmax) rowmax = v;
      }
      if (akk * rowmax >= alpha * colmax * colmax) {
        s = 1;
      } else if (fabs(M[r * N + r]) >= alpha * rowmax) {
        s = 1;
        bk_swap(N, M, f->L, f->perm, k, k, r);
      } else {
        s = 2;
        bk_swap(N, M, f->L, f->perm, k, k + 1, r);
      }
    }
    f->L[k * N + k] = 1.0;
    if (s == 1) {
      double d = M[k * N + k];
      f->D[k * N + k] = d;
      f->bsize[k] = 1;
      if (fabs(d) <= ztol) f->n_zero++;
      else if (d > 0) f->n_pos++;
      else f->n_neg++;
      if (d != 0.0) {
        for (int i = k + 1; i < N; ++i) f->L[i * N + k] = M[i * N + k] / d;
        for (int i = k + 1; i < N; ++i)
          for (int j = k + 1; j < N; ++j)
            M[i * N + j] -= f->L[i * N + k] * d * f->L[j * N + k];
      }
      k += 1;
    } else {
      double e11 = M[k * N + k], e21 = M[(k + 1) * N + k], e22 = M[(k + 1) * N + k + 1];
      double det = e11 * e22 - e21 * e21;
      f->D[k * N + k] = e11; f->D[k * N + k + 1] = e21;
      f->D[(k + 1) * N + k] = e21; f->D[(k + 1) * N + k + 1] = e22;
      f->L[(k + 1) * N + k + 1] = 1.0;
      f->bsize[k] = 2; f->bsize[k + 1] = 0;
      /* eigenvalue signs of the symmetric 2x2 block */
      double tr = e11 + e22;
      double scale = fabs(e11) + fabs(e22) + fabs(e21);
      if (fabs(det) <= ztol * scale) {
        f->n_zero++;
        if (tr > 0) f->n_pos++; else f->n_neg++;
      } else if (det < 0) { f->n_pos++; f->n_neg++; }
      else if (tr > 0) f->n_pos += 2;
      else f->n_neg += 2;
      /* E^{-1} = [e22 -e21; -e21 e11] / det */
      for (int i = k + 2; i < N; ++i) {
        double m1 = M[i * N + k], m2 = M[i * N + k + 1];
        f->L[i * N + k] = (m1 * e22 - m2 * e21) / det;
        f->L[i * N + k + 1] = (m2 * e11 - m1 * e21) / det;
      }
      for (int i = k + 2; i < N; ++i)
        for (int j = k + 2; j < N; ++j)
          M[i * N + j] -= f->L[i * N + k] * M[j * N + k] + f->L[i * N + k + 1] * M[j * N + k + 1];
      k += 2;
    }
  }
  free(M);
}

/* Solve A x = rhs with the factorization (x may alias rhs).  Returns 0, or -1 on a zero pivot. */
static int ldl_solve(const ldl_t *f, const double *rhs, double *x) {
  const int N = f->N;
  double *y = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  for (int i = 0; i < N; ++i) y[i] = rhs[f->perm[i]];
  /* L z = y */
  for (int i = 0; i < N; ++i) {
    double s = y[i];
    for (int j = 0; j < i; ++j) s -= f->L[i * N + j] * y[j];
    y[i] = s;
  }
  /* D w = z */
  int bad = 0;
  for (int k = 0; k < N;) {
    if (f->bsize[k] == 1) {
      double d = f->D[k * N + k];
      if (d == 0.0) { bad = 1; y[k] = 0.0; } else y[k] /= d;
      k += 1;
    } else {
      double e11 = f->D[k * N + k], e21 = f->D[(k + 1) * N + k], e22 = f->D[(k + 1) * N + k + 1];
      double det = e11 * e22 - e21 * e21;
      if (det == 0.0) { bad = 1; y[k] = y[k + 1] = 0.0; }
      else {
        double z1 = y[k], z2 = y[k + 1];
        y[k] = (e22 * z1 - e21 * z2) / det;
        y[k + 1] = (e11 * z2 - e21 * z1) / det;
      }
      k += 2;
    }
  }
  /* L^T v = w */
  for (int i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int j = i + 1; j < N; ++j) s -= f->L[j * N + i] * y[j];
    y[i] = s;
  }
  for (int i = 0; i < N; ++i) x[f->perm[i]] = y[i];
  free(y);
  return bad ? -1 : 0;
}

/* Exposed for tests: factor a dense symmetric matrix, report inertia, solve one rhs. */
int ora_ldl_solve_dense(int N, const double *A, const double *rhs, double *x, int *inertia3) {
  ldl_t f;
  ldl_alloc(&f, N);
  double amax = 0.0;
  for (int i = 0; i < N * N; ++i) if (fabs(A[i]) > amax) amax = fabs(A[i]);
  ldl_factor(A, &f, (double)N * 2.220446049250313e-16 * (amax > 0 ? amax : 1.0));
  int rc = ldl_solve(&f, rhs, x);
  if (inertia3) { inertia3[0] = f.n_pos; inertia3[1] = f.n_neg; inertia3[2] = f.n_zero; }
  ldl_free(&f);
  return rc;
}

/* ------------------------------------------------------------------------------------- */
/* Components of the variable / active-row graph (union-find).                             */
/* ------------------------------------------------------------------------------------- */

static int uf_find(int *parent, int x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

/* comp_of_var[n] (and comp_of_row[m], -1 for inactive rows) get component labels
 * 0..ncomp-1, numbered in order of their smallest variable.  Returns ncomp. */
int ora_components(int n, int m, const int *a_ptr, const int *a_col, const int *q_ptr,
                   const int *q_col, const unsigned char *active, int split,
                   int *comp_of_var, int *comp_of_row) {
  int *parent = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) parent[j] = j;
  if (split) {
    for (int r = 0; r < m; ++r) {
      if (!active[r]) continue;
      int first = -1;
      for (int p = a_ptr[r]; p < a_ptr[r + 1]; ++p) {
        int c = a_col[p];
        if (first < 0) first = c; else { int x = uf_find(parent, first), y = uf_find(parent, c); if (x != y) parent[y] = x; }
      }
      for (int p = q_ptr[r]; p < q_ptr[r + 1]; ++p) {
        int c = q_col[p];
        if (first < 0) first = c; else { int x = uf_find(parent, first), y = uf_find(parent, c); if (x != y) parent[y] = x; }
      }
    }
  } else {
    for (int j = 1; j < n; ++j) parent[j] = 0;
  }
  int *label = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) label[j] = -1;
  int nc = 0;
  for (int j = 0; j < n; ++j) {
    int root = uf_find(parent, j);
    if (label[root] < 0) label[root] = nc++;
    comp_of_var[j] = label[root];
  }
  for (int r = 0; r < m; ++r) {
    comp_of_row[r] = -1;
    if (!active[r]) continue;
    int c = -1;
    if (a_ptr[r + 1] > a_ptr[r]) c = a_col[a_ptr[r]];
    else if (q_ptr[r + 1] > q_ptr[r]) c = q_col[q_ptr[r]];
    if (c >= 0) comp_of_row[r] = comp_of_var[c];
  }
  free(label);
  free(parent);
  return nc;
}

/* ------------------------------------------------------------------------------------- */
/* One component: gather its variables and rows with local indexing.                      */
/* ------------------------------------------------------------------------------------- */

typedef struct {
  int nv, mr;
  int *var;         /* global variable index of each local variable */
  int *row;         /* global row index of each local row */
  /* local CSR (columns are local variable indices) */
  int *ap, *ac; double *av;
  int *qp, *qc; double *qv;
} comp_t;

static void comp_build(comp_t *c, int id, int n, int m, const int *cv, const int *cr,
                       const int *a_ptr, const int *a_col, const double *a_val,
                       const int *q_ptr, const int *q_col, const double *q_val, int *g2l) {
  c->nv = 0; c->mr = 0;
  for (int j = 0; j < n; ++j) if (cv[j] == id) c->nv++;
  for (int r = 0; r < m; ++r) if (cr[r] == id) c->mr++;
  c->var = (int *)malloc(sizeof(int) * (size_t)(c->nv + 1));
  c->row = (int *)malloc(sizeof(int) * (size_t)(c->mr + 1));
  int t = 0;
  for (int j = 0; j < n; ++j) if (cv[j] == id) { g2l[j] = t; c->var[t++] = j; }
  t = 0;
  for (int r = 0; r < m; ++r) if (cr[r] == id) c->row[t++] = r;
  int na = 0, nq = 0;
  for (int k = 0; k < c->mr; ++k) {
    int r = c->row[k];
    na += a_ptr[r + 1] - a_ptr[r];
    nq += q_ptr[r + 1] - q_ptr[r];
  }
  c->ap = (int *)malloc(sizeof(int) * (size_t)(c->mr + 1));
  c->qp = (int *)malloc(sizeof(int) * (size_t)(c->mr + 1));
  c->ac = (int *)malloc(sizeof(int) * (size_t)(na + 1));
  c->av = (double *)malloc(sizeof(double) * (size_t)(na + 1));
  c->qc = (int *)malloc(sizeof(int) * (size_t)(nq + 1));
  c->qv = (double *)malloc(sizeof(double) * (size_t)(nq + 1));
  na = nq = 0;
  for (int k = 0; k < c->mr; ++k) {
    int r = c->row[k];
    c->ap[k] = na; c->qp[k] = nq;
    for (int p = a_ptr[r]; p < a_ptr[r + 1]; ++p) { c->ac[na] = g2l[a_col[p]]; c->av[na] = a_val[p]; na++; }
    for (int p = q_ptr[r]; p < q_ptr[r + 1]; ++p) { c->qc[nq] = g2l[q_col[p]]; c->qv[nq] = q_val[p]; nq++; }
  }
  c->ap[c->mr] = na; c->qp[c->mr] = nq;
}

static void comp_free(comp_t *c) {
  free(c->var); free(c->row); free(c->ap); free(c->ac); free(c->av);
  free(c->qp); free(c->qc); free(c->qv);
}

/* F = [grad_u L ; h] at (u, lam) for one component; b is the component's local rhs. */
static void eval_F(const comp_t *c, const double *u, const double *uh, const double *lam,
                   const double *b, double *F) {
  const int nv = c->nv;
  for (int j = 0; j < nv; ++j) F[j] = u[j] - uh[j];       /* grad f */
  for (int k = 0; k < c->mr; ++k) {
    double h = -b[k];
    for (int p = c->ap[k]; p < c->ap[k + 1]; ++p) {
      int j = c->ac[p];
      h += c->av[p] * u[j];
      F[j] += lam[k] * c->av[p];                           /* J^T lam, linear part */
    }
    for (int p = c->qp[k]; p < c->qp[k + 1]; ++p) {
      int j = c->qc[p];
      h += c->qv[p] * u[j] * u[j];
      F[j] += lam[k] * 2.0 * c->qv[p] * u[j];              /* J^T lam, quadratic part */
    }
    F[nv + k] = h;
  }
}

/* K = [W + delta I, J^T ; J, 0] at (u, lam). */
static void build_K(const comp_t *c, const double *u, const double *lam, double delta, double *K) {
  const int nv = c->nv, N = c->nv + c->mr;
  memset(K, 0, sizeof(double) * (size_t)N * N);
  for (int j = 0; j < nv; ++j) K[j * N + j] = 1.0 + delta;   /* Hessian of f = I */
  for (int k = 0; k < c->mr; ++k) {
    int rk = nv + k;
    for (int p = c->ap[k]; p < c->ap[k + 1]; ++p) {
      int j = c->ac[p];
      K[rk * N + j] += c->av[p];
      K[j * N + rk] += c->av[p];
    }
    for (int p = c->qp[k]; p < c->qp[k + 1]; ++p) {
      int j = c->qc[p];
      double Jrj = 2.0 * c->qv[p] * u[j];
      K[rk * N + j] += Jrj;
      K[j * N + rk] += Jrj;
      K[j * N + j] += lam[k] * 2.0 * c->qv[p];             /* lam_r * Hess h_r */
    }
  }
}

static double norm_inf(const double *x, int N) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    double a = fabs(x[i]);
    if (!(a <= s)) s = a;                                  /* NaN propagates */
  }
  return s;
}

static double half_sq(const double *x, int N) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += x[i] * x[i];
  return 0.5 * s;
}

/* The minimiser of L(., lam) for these row forms: grad_u L = u - u_hat + A^T lam
 * + 2 diag(sum_r lam_r Q_r) u = W(lam) u - u_hat + A^T lam = 0, so u = W^-1 (u_hat - A^T lam)
 * with the diagonal W(lam) = I + sum_r lam_r 2 diag(Q_r) (positive along the iteration). */
static void stationary_u(const comp_t *c, const double *uh, const double *lam, double *wd,
                         double *u) {
  const int nv = c->nv;
  for (int j = 0; j < nv; ++j) { wd[j] = 1.0; u[j] = uh[j]; }
  for (int k = 0; k < c->mr; ++k) {
    for (int p = c->ap[k]; p < c->ap[k + 1]; ++p) u[c->ac[p]] -= lam[k] * c->av[p];
    for (int p = c->qp[k]; p < c->qp[k + 1]; ++p) wd[c->qc[p]] += lam[k] * 2.0 * c->qv[p];
  }
  for (int j = 0; j < nv; ++j) u[j] /= wd[j];
}

/* Newton-KKT on one component.  u holds u0 on entry and the result on exit.
 *
 * restore = 0 (primal-dual): the iterate (u, lam) moves along the Newton-KKT
 * step of Appendix B, (u, lam) + t (du, dlam).
 * After the stopping test one polishing step is taken (below).
 *
 * restore = 1 (used when the iteration starts at u0 = u_hat): the same Newton-KKT
 * step and line search, but every trial point is (u(lam_t), lam_t) with lam_t = lam + t dlam
 * and u(lam) = argmin_u L(u, lam) (stationary_u), so grad_u L = 0 along the whole iteration
 * and the Newton-KKT step reduces to S dlam = h with S = J W^-1 J^T.  The start u = u_hat,
 * lam = 0 is such a point. */
static void newton_component(const comp_t *c, const double *uh, const double *b, double *u,
                             double *lam, const ora_opts *o, ora_stats *st) {
  const int nv = c->nv, N = c->nv + c->mr;
  double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1));
  double *Ft = (double *)malloc(sizeof(double) * (size_t)(N + 1));
  double *dz = (double *)malloc(sizeof(double) * (size_t)(N + 1));
  double *ut = (double *)malloc(sizeof(double) * (size_t)(nv + 1));
  double *lt = (double *)malloc(sizeof(double) * (size_t)(c->mr + 1));
  double *K = (double *)malloc(sizeof(double) * (size_t)N * N + 8);
  double *wd = (double *)malloc(sizeof(double) * (size_t)(nv + 1));
  const int restore = o->restore;
  ldl_t f;
  ldl_alloc(&f, N);
  for (int k = 0; k < c->mr; ++k) lam[k] = 0.0;
  if (restore) stationary_u(c, uh, lam, wd, u);
  st->iters = 0; st->backtracks = 0; st->status = ORA_OK; st->corrections = 0;
  eval_F(c, u, uh, lam, b, F);
  double phi = half_sq(F, N);
  double res = norm_inf(F, N);
  for (int it = 0;; ++it) {
    if (!isfinite(res)) { st->status = ORA_NONFINITE; break; }
    if (res <= o->tol_kkt) { st->status = ORA_OK; break; }
    if (it >= o->max_iter) { st->status = ORA_MAXITER; break; }
    /* Newton-KKT system.  max_corrections = 0: plain Newton-Raphson on F = 0 (Appendix B);
     * its step is a descent direction of phi whenever K is nonsingular.  max_corrections > 0:
     * additionally shift W <- W + delta I until the inertia is (n, m, 0). */
    double delta = 0.0;
    int ok = 0;
    for (int corr = 0; corr <= o->max_corrections; ++corr) {
      build_K(c, u, lam, delta, K);
      double kmax = 0.0;
      for (int i = 0; i < N * N; ++i) if (fabs(K[i]) > kmax) kmax = fabs(K[i]);
      ldl_factor(K, &f, (double)N * 2.220446049250313e-16 * (kmax > 0 ? kmax : 1.0));
      if (f.n_zero == 0 && (o->max_corrections == 0 || (f.n_pos == nv && f.n_neg == c->mr))) {
        ok = 1;
        break;
      }
      delta = (delta == 0.0) ? o->delta0 : delta * 10.0;
      st->corrections++;
    }
    if (!ok) { st->status = ORA_SINGULAR; break; }
    for (int i = 0; i < N; ++i) Ft[i] = -F[i];
    if (ldl_solve(&f, Ft, dz) != 0) { st->status = ORA_SINGULAR; break; }
    /* Largest first trial t <= 1 that keeps every diagonal entry of W = I + sum_r lam_r
     * 2 diag(Q_r) (linear in lam) at >= w_keep times its current value, when the current W
     * is positive definite: fraction to the boundary of {lam : W(lam) > 0}. */
    double t = 1.0;
    if (o->w_keep > 0.0) {
      for (int j = 0; j < nv; ++j) {
        double w = 1.0, dw = 0.0;
        for (int k = 0; k < c->mr; ++k)
          for (int p = c->qp[k]; p < c->qp[k + 1]; ++p)
            if (c->qc[p] == j) { w += 2.0 * c->qv[p] * lam[k]; dw += 2.0 * c->qv[p] * dz[nv + k]; }
        if (w > 0.0 && dw < 0.0) {
          double tm = (1.0 - o->w_keep) * w / (-dw);
          if (tm < t) t = tm;
        }
      }
    }
    /* Armijo backtracking on phi = 1/2 ||F||^2 */
    int nb = 0, accepted = 0;
    double phit = phi;
    for (;;) {
      for (int k = 0; k < c->mr; ++k) lt[k] = lam[k] + t * dz[nv + k];
      if (restore)
        stationary_u(c, uh, lt, wd, ut);
      else
        for (int j = 0; j < nv; ++j) ut[j] = u[j] + t * dz[j];
      eval_F(c, ut, uh, lt, b, Ft);
      phit = half_sq(Ft, N);
      if (phit <= (1.0 - 2.0 * o->c1 * t) * phi) { accepted = 1; break; }
      if (nb >= o->max_backtracks) break;
      nb++;
      t *= 0.5;
    }
    st->backtracks += nb;
    if (!accepted) { st->status = ORA_LINESEARCH; break; }
    memcpy(u, ut, sizeof(double) * (size_t)nv);
    memcpy(lam, lt, sizeof(double) * (size_t)c->mr);
    memcpy(F, Ft, sizeof(double) * (size_t)N);
    phi = phit;
    res = norm_inf(F, N);
    st->iters = it + 1;
  }
  /* Polishing step: the stopping test bounds ||F||, and the multipliers only
   * through the conditioning of the KKT matrix, which is large on slices whose boundary circle
   * is nearly degenerate; one more full Newton-KKT step leaves them at the rounding level.  It
   * is kept when ||F||_inf does not increase (and, with restore, W stays positive); it is not
   * counted in the iterations. */
  if (st->status == ORA_OK && c->mr > 0) {
    build_K(c, u, lam, 0.0, K);
    double kmax = 0.0;
    for (int i = 0; i < N * N; ++i) if (fabs(K[i]) > kmax) kmax = fabs(K[i]);
    ldl_factor(K, &f, (double)N * 2.220446049250313e-16 * (kmax > 0 ? kmax : 1.0));
    for (int j = 0; j < N; ++j) Ft[j] = -F[j];
    if (f.n_zero == 0 && ldl_solve(&f, Ft, dz) == 0) {
      for (int k = 0; k < c->mr; ++k) lt[k] = lam[k] + dz[nv + k];
      int wpos = 1;
      if (restore) {
        stationary_u(c, uh, lt, wd, ut);
        for (int j = 0; j < nv; ++j) if (!(wd[j] > 0.0)) wpos = 0;
      } else {
        for (int j = 0; j < nv; ++j) ut[j] = u[j] + dz[j];
      }
      eval_F(c, ut, uh, lt, b, Ft);
      const double rt = norm_inf(Ft, N);
      if (wpos && rt <= res) {
        memcpy(u, ut, sizeof(double) * (size_t)nv);
        memcpy(lam, lt, sizeof(double) * (size_t)c->mr);
        memcpy(F, Ft, sizeof(double) * (size_t)N);
        phi = half_sq(F, N);
        res = rt;
      }
    }
  }
  /* second-order sufficient condition at a converged point: K has inertia (n, m, 0) iff W
   * is positive definite on null(J) (J of full row rank) */
  if (st->status == ORA_OK && c->mr + nv > 0) {
    build_K(c, u, lam, 0.0, K);
    double kmax = 0.0;
    for (int i = 0; i < N * N; ++i) if (fabs(K[i]) > kmax) kmax = fabs(K[i]);
    ldl_factor(K, &f, (double)N * 2.220446049250313e-16 * (kmax > 0 ? kmax : 1.0));
    if (!(f.n_pos == nv && f.n_neg == c->mr && f.n_zero == 0)) st->status = ORA_NOT_MINIMUM;
  }
  st->kkt_inf = res;
  st->phi = phi;
  ldl_free(&f);
  free(F); free(Ft); free(dz); free(ut); free(lt); free(K); free(wd);
}

/* Adjoint on one component: K [a ; bl] = [gbar ; 0] with K at (u, lam), no correction. */
static int adjoint_component(const comp_t *c, const double *u, const double *lam,
                             const double *gbar, double *a, double *bl) {
  const int nv = c->nv, N = c->nv + c->mr;
  double *K = (double *)malloc(sizeof(double) * (size_t)N * N + 8);
  double *rhs = (double *)malloc(sizeof(double) * (size_t)(N + 1));
  ldl_t f;
  ldl_alloc(&f, N);
  build_K(c, u, lam, 0.0, K);
  double kmax = 0.0;
  for (int i = 0; i < N * N; ++i) if (fabs(K[i]) > kmax) kmax = fabs(K[i]);
  ldl_factor(K, &f, (double)N * 2.220446049250313e-16 * (kmax > 0 ? kmax : 1.0));
  for (int j = 0; j < nv; ++j) rhs[j] = gbar[j];
  for (int k = 0; k < c->mr; ++k) rhs[nv + k] = 0.0;
  int rc = ldl_solve(&f, rhs, rhs);
  for (int j = 0; j < nv; ++j) a[j] = rhs[j];
  for (int k = 0; k < c->mr; ++k) bl[k] = rhs[nv + k];
  ldl_free(&f);
  free(K); free(rhs);
  return rc;
}

static int status_rank(int s) {  /* worse status wins when aggregating a sample */
  switch (s) {
    case ORA_OK: return 0;
    case ORA_MAXITER: return 1;
    case ORA_LINESEARCH: return 2;
    case ORA_NOT_MINIMUM: return 3;
    case ORA_SINGULAR: return 4;
    case ORA_NONFINITE: return 5;
    default: return 6;
  }
}

/* ------------------------------------------------------------------------------------- */
/* Batch entry points.  All samples share the row structure (A, Q, active); b, u_hat and  */
/* u0 are per sample.                                                                      */
/* ------------------------------------------------------------------------------------- */

typedef struct {
  int ncomp;
  comp_t *comps;
} plan_t;

static void plan_build(plan_t *P, int n, int m, const int *a_ptr, const int *a_col,
                       const double *a_val, const int *q_ptr, const int *q_col,
                       const double *q_val, const unsigned char *active, int split) {
  int *cv = (int *)malloc(sizeof(int) * (size_t)(n + 1));
  int *cr = (int *)malloc(sizeof(int) * (size_t)(m + 1));
  int *g2l = (int *)malloc(sizeof(int) * (size_t)(n + 1));
  P->ncomp = ora_components(n, m, a_ptr, a_col, q_ptr, q_col, active, split, cv, cr);
  P->comps = (comp_t *)calloc((size_t)P->ncomp, sizeof(comp_t));
  /* one pass per component is O(ncomp * (n+m)); fine for oracle sizes */
  for (int id = 0; id < P->ncomp; ++id)
    comp_build(&P->comps[id], id, n, m, cv, cr, a_ptr, a_col, a_val, q_ptr, q_col, q_val, g2l);
  free(cv); free(cr); free(g2l);
}

static void plan_free(plan_t *P) {
  for (int i = 0; i < P->ncomp; ++i) comp_free(&P->comps[i]);
  free(P->comps);
}

int ora_project_batch(int n, int m, const int *a_ptr, const int *a_col, const double *a_val,
                      const int *q_ptr, const int *q_col, const double *q_val,
                      const unsigned char *active, int B, const double *b, const double *u_hat,
                      const double *u0, const ora_opts *o, int nthreads, double *u,
                      double *lam, ora_stats *stats) {
  plan_t P;
  plan_build(&P, n, m, a_ptr, a_col, a_val, q_ptr, q_col, q_val, active, o->split_components);
  const long total = (long)B * P.ncomp;
  ora_stats *cs = (ora_stats *)calloc((size_t)(total > 0 ? total : 1), sizeof(ora_stats));
  for (long s = 0; s < (long)B * m; ++s) lam[s] = 0.0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long w = 0; w < total; ++w) {
    const int s = (int)(w / P.ncomp);
    const comp_t *c = &P.comps[w % P.ncomp];
    double *lu = (double *)malloc(sizeof(double) * (size_t)(c->nv + 1));
    double *luh = (double *)malloc(sizeof(double) * (size_t)(c->nv + 1));
    double *lb = (double *)malloc(sizeof(double) * (size_t)(c->mr + 1));
    double *ll = (double *)malloc(sizeof(double) * (size_t)(c->mr + 1));
    const double *uh_s = u_hat + (size_t)s * n;
    const double *u0_s = (u0 ? u0 : u_hat) + (size_t)s * n;
    for (int j = 0; j < c->nv; ++j) { luh[j] = uh_s[c->var[j]]; lu[j] = u0_s[c->var[j]]; }
    for (int k = 0; k < c->mr; ++k) lb[k] = b[(size_t)s * m + c->row[k]];
    newton_component(c, luh, lb, lu, ll, o, &cs[w]);
    for (int j = 0; j < c->nv; ++j) u[(size_t)s * n + c->var[j]] = lu[j];
    for (int k = 0; k < c->mr; ++k) lam[(size_t)s * m + c->row[k]] = ll[k];
    free(lu); free(luh); free(lb); free(ll);
  }
  for (int s = 0; s < B; ++s) {
    ora_stats agg = {0, 0, ORA_OK, 0, 0.0, 0.0};
    for (int ci = 0; ci < P.ncomp; ++ci) {
      const ora_stats *q = &cs[(long)s * P.ncomp + ci];
      if (q->iters > agg.iters) agg.iters = q->iters;
      agg.backtracks += q->backtracks;
      agg.corrections += q->corrections;
      if (status_rank(q->status) > status_rank(agg.status)) agg.status = q->status;
      if (!(q->kkt_inf <= agg.kkt_inf)) agg.kkt_inf = q->kkt_inf;
      agg.phi += q->phi;
    }
    stats[s] = agg;
  }
  free(cs);
  plan_free(&P);
  return 0;
}

int ora_adjoint_batch(int n, int m, const int *a_ptr, const int *a_col, const double *a_val,
                      const int *q_ptr, const int *q_col, const double *q_val,
                      const unsigned char *active, int B, const double *u, const double *lam,
                      const double *gbar, int split, int nthreads, double *a, double *bl) {
  plan_t P;
  plan_build(&P, n, m, a_ptr, a_col, a_val, q_ptr, q_col, q_val, active, split);
  const long total = (long)B * P.ncomp;
  int bad = 0;
  for (long s = 0; s < (long)B * m; ++s) bl[s] = 0.0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
  for (long w = 0; w < total; ++w) {
    const int s = (int)(w / P.ncomp);
    const comp_t *c = &P.comps[w % P.ncomp];
    double *lu = (double *)malloc(sizeof(double) * (size_t)(c->nv + 1));
    double *lg = (double *)malloc(sizeof(double) * (size_t)(c->nv + 1));
    double *la = (double *)malloc(sizeof(double) * (size_t)(c->nv + 1));
    double *ll = (double *)malloc(sizeof(double) * (size_t)(c->mr + 1));
    double *lb = (double *)malloc(sizeof(double) * (size_t)(c->mr + 1));
    for (int j = 0; j < c->nv; ++j) {
      lu[j] = u[(size_t)s * n + c->var[j]];
      lg[j] = gbar[(size_t)s * n + c->var[j]];
    }
    for (int k = 0; k < c->mr; ++k) ll[k] = lam[(size_t)s * m + c->row[k]];
    if (adjoint_component(c, lu, ll, lg, la, lb) != 0) bad |= 1;
    for (int j = 0; j < c->nv; ++j) a[(size_t)s * n + c->var[j]] = la[j];
    for (int k = 0; k < c->mr; ++k) bl[(size_t)s * m + c->row[k]] = lb[k];
    free(lu); free(lg); free(la); free(ll); free(lb);
  }
  plan_free(&P);
  return bad ? -1 : 0;
}

/* Threads an OpenMP region of this library would use (for reporting). */
int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
