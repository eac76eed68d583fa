/*
 * oracle.c -- plain FP64 CPU oracle for the ridge-regularized matching LP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the solver library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Problem (Sec. 3.1, Eq. primal):
 *     min_{x in C}  c^T x + (gamma/2) ||x||^2   s.t.  A x <= b,
 * with m capacity families (Sec. 3.3, Eq. dest-capacity; Def. 1):
 *     sum_i a_kij x_ij <= b_kj  for every family k and item j,
 * and per-user simple sets C_i (Sec. 3.3): the simplex {x >= 0, sum x <= z}
 * (kind 0), the simplex with equality (kind 1), the box [0, z] (kind 2), or
 * the box cut by one budget, {0 <= x <= z, sum x <= cut} (kind 3: the paper
 * lists a box-cut projection among its primitives without defining it; this
 * is the reading taken).
 *
 * Dual (Sec. 3.2, Eq. dual):  g(lam) = min_{x in C} c^T x + gamma/2 ||x||^2
 *                                       + lam^T (A x - b),
 * primal recovery (Eq. primal-recovery):  x*(lam) = Proj_C(-(A^T lam + c)/gamma),
 * gradient (Eq. dual-gradient, Danskin):   grad g(lam) = A x*(lam) - b.
 *
 * Optionally a global count constraint sum_ij x_ij <= M (the example of a new
 * coupling constraint in Sec. 5: one more dual coordinate mu, one more term in
 * A^T lam, one more gradient entry).
 *
 * Everything is sequential FP64 in the natural order: users in index order,
 * elements of a user in storage order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t I, J, nnz;
  const int64_t* row_ptr; /* I+1 */
  const int32_t* col;     /* nnz, item of each edge */
  const double* c;        /* nnz */
  const double* a;        /* nnz */
  const double* b;        /* J */
  int32_t kind;           /* 0 simplex <=, 1 simplex ==, 2 box */
  int32_t _pad;
  double z;               /* simplex radius or box upper bound */
  double M;               /* global count bound sum_ij x_ij <= M (Sec. 5); INFINITY: none */
  int32_t m;              /* capacity families (Def. 1): a is [nnz x m] edge-major, b [m x J] */
  int32_t _pad2;
  double cut;             /* kind 3: per-user budget sum_j x_ij <= cut */
} orc_problem;

/* The dual vector is lam[k J + j] for family k and item j (m J entries), then
 * mu when there is a global count constraint: mu >= 0 is the dual of
 * sum_ij x_ij <= M, which adds mu to every edge's cost (one more row of ones
 * in A). */
static int has_count(const orc_problem* p) { return isfinite(p->M); }
static int64_t fams(const orc_problem* p) { return p->m > 0 ? p->m : 1; }
static int64_t mJ(const orc_problem* p) { return fams(p) * p->J; }

/* ------------------------------------------------------------------------ */
/* Projections onto one user's simple set (Sec. 3.3, Sec. 4.3)               */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void* p, const void* q) {
  double a = *(const double*)p, b = *(const double*)q;
  return (a < b) - (a > b);
}

/* Sort-based simplex projection of Duchi et al. (2008), as the fused kernel of
 * Sec. 4.3 describes it: sort descending, prefix sums, cutoff index rho as the
 * last k with mu_k - (S_k - z)/k > 0, threshold theta = (S_rho - z)/rho, then
 * x = max(v - theta, 0).  For the inequality simplex the input is returned
 * clipped at zero when it is already feasible (the early exit of Sec. 4.3,
 * tested exactly: sum max(v,0) <= z). */
static double proj_simplex_sort(const double* v, int64_t n, double z, int eq, double* x) {
  if (n <= 0) return 0.0;
  if (!eq) {
    double s = 0;
    for (int64_t k = 0; k < n; ++k) s += v[k] > 0 ? v[k] : 0;
    if (s <= z) {
      for (int64_t k = 0; k < n; ++k) x[k] = v[k] > 0 ? v[k] : 0;
      return 0.0;
    }
  }
  double* mu = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(mu, v, sizeof(double) * (size_t)n);
  qsort(mu, (size_t)n, sizeof(double), cmp_desc);
  double S = 0, S_rho = 0;
  int64_t rho = 0;
  for (int64_t k = 1; k <= n; ++k) {
    S += mu[k - 1];
    if (mu[k - 1] - (S - z) / (double)k > 0) {
      rho = k;
      S_rho = S;
    }
  }
  free(mu);
  double theta = (S_rho - z) / (double)rho;
  for (int64_t k = 0; k < n; ++k) {
    double t = v[k] - theta;
    x[k] = t > 0 ? t : 0;
  }
  return theta;
}

/* Same projection by bisection on theta for f(theta) = sum max(v - theta, 0) = z
 * (f is continuous and decreasing), run until the bracket stops shrinking. */
static double proj_simplex_bisect(const double* v, int64_t n, double z, int eq, double* x) {
  if (n <= 0) return 0.0;
  double vmax = v[0], vmin = v[0], s = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (v[k] > vmax) vmax = v[k];
    if (v[k] < vmin) vmin = v[k];
    s += v[k] > 0 ? v[k] : 0;
  }
  double theta;
  if (!eq && s <= z) {
    theta = 0.0;
  } else {
    double lo = eq ? vmin - z / (double)n : 0.0; /* f(lo) >= z */
    double hi = vmax;                           /* f(hi) = 0 <= z */
    for (int it = 0; it < 5000; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      double f = 0;
      for (int64_t k = 0; k < n; ++k) f += v[k] > mid ? v[k] - mid : 0;
      if (f > z)
        lo = mid;
      else
        hi = mid;
    }
    theta = 0.5 * (lo + hi);
  }
  for (int64_t k = 0; k < n; ++k) {
    double t = v[k] - theta;
    x[k] = t > 0 ? t : 0;
  }
  return theta;
}

/* Box [0, u]: coordinate-wise clipping. */
static void proj_box(const double* v, int64_t n, double u, double* x) {
  for (int64_t k = 0; k < n; ++k) x[k] = v[k] < 0 ? 0 : (v[k] > u ? u : v[k]);
}

/* Box cut by one budget, {0 <= x <= z, sum x <= cut}: x = clip(v - theta, 0,
 * z) with theta = 0 when the clipped input already meets the budget, else the
 * root of phi(theta) = sum clip(v - theta, 0, z) - cut, which is continuous,
 * nonincreasing and piecewise linear with breakpoints at v_k and v_k - z.
 * Method 0 locates the root between consecutive breakpoints and solves the
 * linear piece there; method 1 bisects on theta. */
static double boxcut_phi(const double* v, int64_t n, double z, double cut, double t) {
  double f = -cut;
  for (int64_t k = 0; k < n; ++k) {
    double y = v[k] - t;
    f += y <= 0 ? 0 : (y >= z ? z : y);
  }
  return f;
}

static int cmp_asc(const void* p, const void* q) {
  double a = *(const double*)p, b = *(const double*)q;
  return (a > b) - (a < b);
}

static double proj_boxcut(const double* v, int64_t n, double z, double cut, int32_t method, double* x) {
  double theta = 0.0;
  if (n > 0 && boxcut_phi(v, n, z, cut, 0.0) > 0) {
    double vmax = v[0];
    for (int64_t k = 1; k < n; ++k)
      if (v[k] > vmax) vmax = v[k];
    if (method == 1) {
      double lo = 0.0, hi = vmax; /* phi(lo) > 0 >= phi(hi) = -cut */
      for (int it = 0; it < 5000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (boxcut_phi(v, n, z, cut, mid) > 0)
          lo = mid;
        else
          hi = mid;
      }
      theta = 0.5 * (lo + hi);
    } else {
      /* breakpoints in (0, vmax], ascending, with 0 in front */
      double* bp = (double*)malloc(sizeof(double) * (size_t)(2 * n + 1));
      int64_t nb = 0;
      bp[nb++] = 0.0;
      for (int64_t k = 0; k < n; ++k) {
        if (v[k] > 0) bp[nb++] = v[k];
        if (v[k] - z > 0) bp[nb++] = v[k] - z;
      }
      qsort(bp + 1, (size_t)(nb - 1), sizeof(double), cmp_asc);
      /* first breakpoint where phi <= 0 (exists: phi(vmax) = -cut) */
      int64_t r = 1;
      while (r < nb && boxcut_phi(v, n, z, cut, bp[r]) > 0) ++r;
      const double ta = bp[r - 1], tb = r < nb ? bp[r] : vmax;
      /* on (ta, tb) the free set F = {v - z < t < v} and the capped set U =
       * {v - z >= t} are fixed: phi(t) = sum_F (v - t) + z |U| - cut */
      const double mid = 0.5 * (ta + tb);
      double sf = 0;
      int64_t nf = 0, nu = 0;
      for (int64_t k = 0; k < n; ++k) {
        if (v[k] - z >= mid)
          ++nu;
        else if (v[k] > mid) {
          sf += v[k];
          ++nf;
        }
      }
      theta = nf > 0 ? (sf + z * (double)nu - cut) / (double)nf : tb;
      if (theta < ta) theta = ta;
      if (theta > tb) theta = tb;
      free(bp);
    }
  }
  for (int64_t k = 0; k < n; ++k) {
    double y = v[k] - theta;
    x[k] = y <= 0 ? 0 : (y >= z ? z : y);
  }
  return theta;
}

/* Exported: project one segment.  method 0 = sort (Duchi) or breakpoints,
 * 1 = bisection.  Returns theta (0 for the box). */
double orc_project(const double* v, int64_t n, int32_t kind, double z, double cut, int32_t method, double* x) {
  if (kind == 2) {
    proj_box(v, n, z, x);
    return 0.0;
  }
  if (kind == 3) return proj_boxcut(v, n, z, cut, method, x);
  if (method == 1) return proj_simplex_bisect(v, n, z, kind == 1, x);
  return proj_simplex_sort(v, n, z, kind == 1, x);
}

/* ------------------------------------------------------------------------ */
/* One dual evaluation (Eqs. dual, primal-recovery, dual-gradient)           */
/* ------------------------------------------------------------------------ */

/* Evaluates, at dual point lam and ridge gamma:
 *   x      = Proj_C(-(A^T lam + c)/gamma)              (per edge, may be NULL)
 *   Ax_kj  = sum_i a_kij x_ij                          (per family and item)
 *   Cx_j   = sum_i c_ij x_ij,  Qx_j = sum_i x_ij^2     (per item, may be NULL)
 *   obj    = sum (c x + gamma/2 x^2)                   (scalar)
 * and returns g(lam) = obj + lam^T (Ax - b) (+ mu (sum x - M)). */
double orc_sweep(const orc_problem* p, const double* lam, double gamma, double* x_out, double* Ax, double* Cx,
                 double* Qx, double* obj_out, double* count_out) {
  const int64_t m = fams(p), J = p->J;
  int64_t maxd = 0;
  for (int64_t i = 0; i < p->I; ++i) {
    int64_t d = p->row_ptr[i + 1] - p->row_ptr[i];
    if (d > maxd) maxd = d;
  }
  const double mu = has_count(p) ? lam[mJ(p)] : 0.0;
  double* v = (double*)malloc(sizeof(double) * (size_t)(maxd > 0 ? maxd : 1));
  double* x = (double*)malloc(sizeof(double) * (size_t)(maxd > 0 ? maxd : 1));
  for (int64_t q = 0; q < m * J; ++q) Ax[q] = 0;
  for (int64_t j = 0; j < J; ++j) {
    if (Cx) Cx[j] = 0;
    if (Qx) Qx[j] = 0;
  }
  double obj = 0, count = 0;
  for (int64_t i = 0; i < p->I; ++i) {
    int64_t e0 = p->row_ptr[i], d = p->row_ptr[i + 1] - e0;
    for (int64_t k = 0; k < d; ++k) {
      int64_t e = e0 + k;
      double t = p->c[e] + mu;
      for (int64_t f = 0; f < m; ++f) t += p->a[e * m + f] * lam[f * J + p->col[e]];
      v[k] = -t / gamma;
    }
    orc_project(v, d, p->kind, p->z, p->cut, 0, x);
    for (int64_t k = 0; k < d; ++k) {
      int64_t e = e0 + k;
      int32_t j = p->col[e];
      for (int64_t f = 0; f < m; ++f) Ax[f * J + j] += p->a[e * m + f] * x[k];
      if (Cx) Cx[j] += p->c[e] * x[k];
      if (Qx) Qx[j] += x[k] * x[k];
      obj += p->c[e] * x[k] + 0.5 * gamma * x[k] * x[k];
      count += x[k];
      if (x_out) x_out[e] = x[k];
    }
  }
  free(v);
  free(x);
  double g = obj;
  for (int64_t q = 0; q < m * J; ++q) g += lam[q] * (Ax[q] - p->b[q]);
  if (has_count(p)) g += mu * (count - p->M);
  if (obj_out) *obj_out = obj;
  if (count_out) *count_out = count;
  return g;
}

/* g(lam) and grad g(lam) = A x*(lam) - b (Eq. dual-gradient), m J entries;
 * with a count constraint one more, sum_ij x_ij - M. */
double orc_dual(const orc_problem* p, const double* lam, double gamma, double* grad, double* x_out) {
  double count = 0;
  double g = orc_sweep(p, lam, gamma, x_out, grad, NULL, NULL, NULL, &count);
  for (int64_t q = 0; q < mJ(p); ++q) grad[q] -= p->b[q];
  if (has_count(p)) grad[mJ(p)] = count - p->M;
  return g;
}

/* s_kj = sum_i a_kij: the coupling between row (k, j) of A and the count row
 * of ones (an entry of A A^T). */
void orc_row_sum(const orc_problem* p, double* s1) {
  const int64_t m = fams(p), J = p->J;
  for (int64_t q = 0; q < m * J; ++q) s1[q] = 0;
  for (int64_t e = 0; e < p->nnz; ++e)
    for (int64_t f = 0; f < m; ++f) s1[f * J + p->col[e]] += p->a[e * m + f];
}

/* n_kj = sum_i a_kij^2, the diagonal of A A^T.  With one capacity family the
 * rows of A have disjoint supports (Def. 1: each D_i is diagonal), so
 * A A^T = diag(n) and ||A||_2^2 = max_j n_j; App. B.2 bounds the gradient's
 * Lipschitz constant by ||A||_2^2 / gamma. */
void orc_row_sq(const orc_problem* p, double* n2) {
  const int64_t m = fams(p), J = p->J;
  for (int64_t q = 0; q < m * J; ++q) n2[q] = 0;
  for (int64_t e = 0; e < p->nnz; ++e)
    for (int64_t f = 0; f < m; ++f) n2[f * J + p->col[e]] += p->a[e * m + f] * p->a[e * m + f];
}

/* Gershgorin row sums of A A^T over the capacity rows: for row (k, j),
 * sum_l |sum_i a_kij a_lij| (the m x m block of item j; the blocks of
 * different items do not couple, Def. 1). */
static void gram_rows(const orc_problem* p, double* r) {
  const int64_t m = fams(p), J = p->J;
  double* G = (double*)calloc((size_t)(m * m * J), sizeof(double));
  for (int64_t e = 0; e < p->nnz; ++e)
    for (int64_t f = 0; f < m; ++f)
      for (int64_t l = 0; l < m; ++l) G[(f * m + l) * J + p->col[e]] += p->a[e * m + f] * p->a[e * m + l];
  for (int64_t f = 0; f < m; ++f)
    for (int64_t j = 0; j < J; ++j) {
      double t = 0;
      for (int64_t l = 0; l < m; ++l) t += fabs(G[(f * m + l) * J + j]);
      r[f * J + j] = t;
    }
  free(G);
}

/* ------------------------------------------------------------------------ */
/* Certified duality gap                                                     */
/* ------------------------------------------------------------------------ */

/* At dual point lam >= 0: evaluates g(lam), then makes x(lam) feasible by
 * scaling each item's column: s_j = min(1, b_j / (Ax)_j), x~_ij = s_j x_ij
 * (stays in every simplex-<= and box set when a, b >= 0), and evaluates the
 * primal objective there, P(x~) = sum_j s_j Cx_j + gamma/2 s_j^2 Qx_j.
 * Weak duality gives P(x~) >= P* >= g(lam).
 * out[0] = g(lam), out[1] = P(x~), out[2] = (P - g)/max(|g|, 1e-30),
 * out[3] = max_j (Ax - b)_j^+, out[4] = -lam^T (Ax - b) / max(|g|, 1e-30)
 * (the gap of the unscaled point x(lam), as the paper's quality table
 * reports it), out[5] = primal objective of the unscaled x(lam). */
void orc_certify(const orc_problem* p, const double* lam, double gamma, double* out) {
  const int64_t J = p->J, m = fams(p);
  double* Ax = (double*)malloc(sizeof(double) * (size_t)(m * J));
  double* Cx = (double*)malloc(sizeof(double) * (size_t)J);
  double* Qx = (double*)malloc(sizeof(double) * (size_t)J);
  double obj = 0, count = 0;
  double g = orc_sweep(p, lam, gamma, NULL, Ax, Cx, Qx, &obj, &count);
  /* item scaling s_j = min(1, min_k b_kj / (A_k x)_j); with a count constraint
   * a common factor t = min(1, M / sum x) on top keeps sum x~ <= t sum x <= M */
  double t = 1.0;
  if (has_count(p) && count > p->M) t = p->M / count;
  double P = 0, viol = 0, lg = 0;
  for (int64_t j = 0; j < J; ++j) {
    double s = 1.0;
    for (int64_t f = 0; f < m; ++f) {
      const int64_t q = f * J + j;
      if (Ax[q] > p->b[q] && p->b[q] / Ax[q] < s) s = p->b[q] / Ax[q];
    }
    s *= t;
    P += s * Cx[j] + 0.5 * gamma * s * s * Qx[j];
  }
  for (int64_t q = 0; q < m * J; ++q) {
    double r = Ax[q] - p->b[q];
    if (r > viol) viol = r;
    lg += lam[q] * r;
  }
  if (has_count(p)) {
    double r = count - p->M;
    if (r > viol) viol = r;
    lg += lam[m * J] * r;
  }
  double den = fabs(g) > 1e-30 ? fabs(g) : 1e-30;
  out[0] = g;
  out[1] = P;
  out[2] = (P - g) / den;
  out[3] = viol;
  out[4] = -lg / den;
  out[5] = obj;
  free(Ax);
  free(Cx);
  free(Qx);
}

static double stage_gamma(double gamma0, double gamma_end, double factor, int64_t s) {
  double g = gamma0;
  for (int64_t k = 0; k < s; ++k) {
    double n = g * factor;
    g = n > gamma_end ? n : gamma_end;
  }
  return g;
}

/* Runs T iterations of
 *     G     = grad g(y) = A x*(y) - b
 *     lam+  = max(0, y + step .* G)
 *     theta+ = (1 + sqrt(1 + 4 theta^2)) / 2
 *     y+    = lam+ + ((theta - 1)/theta+) (lam+ - lam)
 * from lam = y = lam0, theta = 1, where step_j = gamma / max_k n_k (the fixed
 * step 1/L with L = ||A||^2/gamma) or, with row normalization (App. B.2),
 * step_j = gamma / n_j (a diagonal step: the same iteration run on the scaled
 * rows A' = D A, b' = D b with D_jj = n_j^-1/2, mapped back to lam).
 * gamma follows the stage schedule: iteration t is in stage t / iters_per_stage;
 * when the stage's gamma differs from the previous one the new stage starts
 * from the last lam (warm start) with theta = 1 and y = lam (Sec. 6).
 * Outputs: lam_out, y_out (state after T iterations), theta_out, and per
 * iteration t: traj_g[t] = g(y_t), traj_gamma[t] (either may be NULL). */
/* Per-coordinate curvature bounds h_k (step_k = gamma / h_k).  One family:
 * A A^T = diag(n) (Def. 1), so h_j = n_j with row normalization and
 * h = max_j n_j = ||A||^2 otherwise (App. B.2).  With m families A A^T is
 * block diagonal with one m x m block per item, and with the count row it
 * gains the row and column s (s_kj = sum_i a_kij) and the corner nnz;
 * Gershgorin row sums bound it in every case: the diagonal scaling by their
 * inverses is a valid preconditioner, and their maximum bounds ||A||^2. */
static int64_t curvature(const orc_problem* p, int32_t precondition, double* h) {
  const int64_t MJ = mJ(p), D = MJ + (has_count(p) ? 1 : 0);
  gram_rows(p, h);
  if (has_count(p)) {
    double* s1 = (double*)malloc(sizeof(double) * (size_t)MJ);
    orc_row_sum(p, s1);
    double tot = 0;
    for (int64_t q = 0; q < MJ; ++q) {
      h[q] += fabs(s1[q]);
      tot += fabs(s1[q]);
    }
    h[MJ] = (double)p->nnz + tot;
    free(s1);
  }
  if (!precondition) {
    double mx = 0;
    for (int64_t k = 0; k < D; ++k)
      if (h[k] > mx) mx = h[k];
    for (int64_t k = 0; k < D; ++k) h[k] = mx;
  }
  return D;
}

void orc_fista(const orc_problem* p, double gamma0, double gamma_end, double factor, int64_t iters_per_stage,
               int32_t precondition, int32_t restart, int64_t T, const double* lam0, double* lam_out,
               double* y_out, double* theta_out, double* traj_g, double* traj_gamma) {
  int64_t D1 = mJ(p) + 1;
  double* h = (double*)malloc(sizeof(double) * (size_t)D1);
  double* lam = (double*)malloc(sizeof(double) * (size_t)D1);
  double* y = (double*)malloc(sizeof(double) * (size_t)D1);
  double* G = (double*)malloc(sizeof(double) * (size_t)D1);
  double* nl = (double*)malloc(sizeof(double) * (size_t)D1);
  const int64_t D = curvature(p, precondition, h);
  for (int64_t k = 0; k < D; ++k) lam[k] = y[k] = lam0[k];
  double theta = 1.0;
  if (iters_per_stage <= 0) iters_per_stage = T > 0 ? T : 1;
  for (int64_t t = 0; t < T; ++t) {
    int64_t s = t / iters_per_stage;
    double gamma = stage_gamma(gamma0, gamma_end, factor, s);
    double g = orc_dual(p, y, gamma, G, NULL);
    if (traj_g) traj_g[t] = g;
    if (traj_gamma) traj_gamma[t] = gamma;
    for (int64_t k = 0; k < D; ++k) {
      double step = h[k] > 0 ? gamma / h[k] : 0.0;
      double v = y[k] + step * G[k];
      nl[k] = v > 0 ? v : 0;
    }
    int64_t s1 = (t + 1) / iters_per_stage;
    double gamma_next = stage_gamma(gamma0, gamma_end, factor, s1);
    int restart_now = gamma_next != gamma;
    if (restart && !restart_now) {
      /* adaptive restart (O'Donoghue & Candes 2015, gradient-mapping test
         for ascent, in the metric of the per-coordinate steps): restart when
         the step just taken opposes the momentum */
      double dot = 0.0;
      for (int64_t k = 0; k < D; ++k) {
        double step = h[k] > 0 ? gamma / h[k] : 0.0;
        if (step > 0) dot += (nl[k] - y[k]) * (nl[k] - lam[k]) / step;
      }
      restart_now = dot < 0.0;
    }
    if (restart_now) {
      theta = 1.0;
      for (int64_t k = 0; k < D; ++k) {
        lam[k] = nl[k];
        y[k] = nl[k];
      }
    } else {
      double th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      double beta = (theta - 1.0) / th1;
      for (int64_t k = 0; k < D; ++k) {
        y[k] = nl[k] + beta * (nl[k] - lam[k]);
        lam[k] = nl[k];
      }
      theta = th1;
    }
  }
  for (int64_t k = 0; k < D; ++k) {
    lam_out[k] = lam[k];
    if (y_out) y_out[k] = y[k];
  }
  if (theta_out) *theta_out = theta;
  free(h);
  free(lam);
  free(y);
  free(G);
  free(nl);
}

/* Gamma of stage s under the continuation schedule (exported for tests). */
double orc_stage_gamma(double gamma0, double gamma_end, double factor, int64_t s) {
  return stage_gamma(gamma0, gamma_end, factor, s);
}

/* ------------------------------------------------------------------------ */
/* Timing only: the same fixed-gamma iteration with the sweep split over      */
/* threads.  Users are cut into nthreads contiguous ranges of equal edge      */
/* count; each thread projects its users and sums A x into its own J-vector;  */
/* the vectors are added in thread order, then the O(J) step runs serially.   */
/* Deterministic for a fixed thread count.  Parity tests use orc_fista.       */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_problem* p;
  const double* y;
  double gamma;
  int64_t u0, u1;
  double* Ax;
} sweep_job;

static void* sweep_range(void* arg) {
  sweep_job* jb = (sweep_job*)arg;
  const orc_problem* p = jb->p;
  int64_t maxd = 1;
  for (int64_t i = jb->u0; i < jb->u1; ++i) {
    int64_t d = p->row_ptr[i + 1] - p->row_ptr[i];
    if (d > maxd) maxd = d;
  }
  double* v = (double*)malloc(sizeof(double) * (size_t)maxd);
  double* x = (double*)malloc(sizeof(double) * (size_t)maxd);
  for (int64_t j = 0; j < p->J; ++j) jb->Ax[j] = 0;
  for (int64_t i = jb->u0; i < jb->u1; ++i) {
    int64_t e0 = p->row_ptr[i], d = p->row_ptr[i + 1] - e0;
    for (int64_t k = 0; k < d; ++k) v[k] = -(p->c[e0 + k] + p->a[e0 + k] * jb->y[p->col[e0 + k]]) / jb->gamma;
    orc_project(v, d, p->kind, p->z, p->cut, 0, x);
    for (int64_t k = 0; k < d; ++k) jb->Ax[p->col[e0 + k]] += p->a[e0 + k] * x[k];
  }
  free(v);
  free(x);
  return NULL;
}

void orc_fista_threads(const orc_problem* p, double gamma, int32_t precondition, int64_t T, int32_t nthreads,
                       double* lam_out) {
  /* (timing of the one-family capacity problem; the wrapper rejects others) */
  int64_t J = p->J;
  if (nthreads < 1) nthreads = 1;
  double* n2 = (double*)malloc(sizeof(double) * (size_t)J);
  double* lam = (double*)calloc((size_t)J, sizeof(double));
  double* y = (double*)calloc((size_t)J, sizeof(double));
  double* Ax = (double*)malloc(sizeof(double) * (size_t)J * (size_t)nthreads);
  sweep_job* jobs = (sweep_job*)malloc(sizeof(sweep_job) * (size_t)nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  orc_row_sq(p, n2);
  double nmax = 0;
  for (int64_t j = 0; j < J; ++j)
    if (n2[j] > nmax) nmax = n2[j];
  int64_t u = 0;
  for (int32_t t = 0; t < nthreads; ++t) {
    int64_t target = p->nnz * (t + 1) / nthreads;
    int64_t u1 = u;
    while (u1 < p->I && p->row_ptr[u1] < target) ++u1;
    if (t == nthreads - 1) u1 = p->I;
    jobs[t].p = p;
    jobs[t].y = y;
    jobs[t].gamma = gamma;
    jobs[t].u0 = u;
    jobs[t].u1 = u1;
    jobs[t].Ax = Ax + (size_t)J * (size_t)t;
    u = u1;
  }
  double theta = 1.0;
  for (int64_t it = 0; it < T; ++it) {
    for (int32_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, sweep_range, &jobs[t]);
    sweep_range(&jobs[0]);
    for (int32_t t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    double th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
    double beta = (theta - 1.0) / th1;
    for (int64_t j = 0; j < J; ++j) {
      double G = -p->b[j];
      for (int32_t t = 0; t < nthreads; ++t) G += Ax[(size_t)J * (size_t)t + (size_t)j];
      double step = precondition ? (n2[j] > 0 ? gamma / n2[j] : 0.0) : (nmax > 0 ? gamma / nmax : 0.0);
      double v = y[j] + step * G;
      double nl = v > 0 ? v : 0;
      y[j] = nl + beta * (nl - lam[j]);
      lam[j] = nl;
    }
    theta = th1;
  }
  for (int64_t j = 0; j < J; ++j) lam_out[j] = lam[j];
  free(n2);
  free(lam);
  free(y);
  free(Ax);
  free(jobs);
  free(th);
}

/* ------------------------------------------------------------------------ */
/* Solve to a certified gap with the sweep split over threads (the CPU       */
/* baseline of time-to-gap, and reference optima on samples).  The iteration */
/* is orc_fista's -- gamma continuation, step gamma / h, momentum restart at  */
/* a change of gamma and optionally the adaptive restart -- with A x summed   */
/* per thread over contiguous user ranges and the thread vectors added in     */
/* thread order (one thread: orc_fista's arithmetic exactly).  Before         */
/* iteration t, when t is a multiple of gap_every and the gamma of t is       */
/* gamma_end, the certified gap of orc_certify at lam is evaluated (the sums  */
/* split over threads the same way); the solve stops when it is <= target or  */
/* after max_iters iterations.  One capacity family, no count constraint.     */
/* stats[0] = iterations taken, stats[1] = last certified gap (NaN if none),  */
/* stats[2] = g(lam), stats[3] = P(x~) of that check.                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_problem* p;
  const double* y;
  double gamma;
  int64_t u0, u1;
  double *Ax, *Cx, *Qx; /* Cx, Qx NULL: gradient sweep only */
  double obj;
} solve_job;

static void* solve_range(void* arg) {
  solve_job* jb = (solve_job*)arg;
  const orc_problem* p = jb->p;
  int64_t maxd = 1;
  for (int64_t i = jb->u0; i < jb->u1; ++i) {
    int64_t d = p->row_ptr[i + 1] - p->row_ptr[i];
    if (d > maxd) maxd = d;
  }
  double* v = (double*)malloc(sizeof(double) * (size_t)maxd);
  double* x = (double*)malloc(sizeof(double) * (size_t)maxd);
  for (int64_t j = 0; j < p->J; ++j) {
    jb->Ax[j] = 0;
    if (jb->Cx) jb->Cx[j] = jb->Qx[j] = 0;
  }
  double obj = 0;
  for (int64_t i = jb->u0; i < jb->u1; ++i) {
    int64_t e0 = p->row_ptr[i], d = p->row_ptr[i + 1] - e0;
    for (int64_t k = 0; k < d; ++k) {
      double t = p->c[e0 + k] + 0.0;
      t += p->a[e0 + k] * jb->y[p->col[e0 + k]];
      v[k] = -t / jb->gamma;
    }
    orc_project(v, d, p->kind, p->z, p->cut, 0, x);
    for (int64_t k = 0; k < d; ++k) {
      int32_t j = p->col[e0 + k];
      jb->Ax[j] += p->a[e0 + k] * x[k];
      if (jb->Cx) {
        jb->Cx[j] += p->c[e0 + k] * x[k];
        jb->Qx[j] += x[k] * x[k];
        obj += p->c[e0 + k] * x[k] + 0.5 * jb->gamma * x[k] * x[k];
      }
    }
  }
  jb->obj = obj;
  free(v);
  free(x);
  return NULL;
}

static void run_jobs(solve_job* jobs, pthread_t* th, int32_t nthreads) {
  for (int32_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, solve_range, &jobs[t]);
  solve_range(&jobs[0]);
  for (int32_t t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

void orc_solve_threads(const orc_problem* p, double gamma0, double gamma_end, double factor, int64_t iters_per_stage,
                       int32_t precondition, int32_t restart, double target, int64_t gap_every, int64_t max_iters,
                       int32_t nthreads, const double* lam0, double* lam_out, double* stats) {
  const int64_t J = p->J;
  if (nthreads < 1) nthreads = 1;
  if (gap_every < 1) gap_every = 1;
  if (iters_per_stage <= 0) iters_per_stage = max_iters > 0 ? max_iters : 1;
  double* h = (double*)malloc(sizeof(double) * (size_t)(J + 1));
  double* lam = (double*)malloc(sizeof(double) * (size_t)J);
  double* y = (double*)malloc(sizeof(double) * (size_t)J);
  double* G = (double*)malloc(sizeof(double) * (size_t)J);
  double* nl = (double*)malloc(sizeof(double) * (size_t)J);
  double* buf = (double*)malloc(sizeof(double) * (size_t)J * 3 * (size_t)nthreads);
  solve_job* jobs = (solve_job*)malloc(sizeof(solve_job) * (size_t)nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  curvature(p, precondition, h);
  for (int64_t k = 0; k < J; ++k) lam[k] = y[k] = lam0[k];
  int64_t u = 0;
  for (int32_t t = 0; t < nthreads; ++t) {
    int64_t want = p->nnz * (t + 1) / nthreads;
    int64_t u1 = u;
    while (u1 < p->I && p->row_ptr[u1] < want) ++u1;
    if (t == nthreads - 1) u1 = p->I;
    jobs[t].p = p;
    jobs[t].u0 = u;
    jobs[t].u1 = u1;
    jobs[t].Ax = buf + (size_t)J * (size_t)(3 * t);
    jobs[t].Cx = buf + (size_t)J * (size_t)(3 * t + 1);
    jobs[t].Qx = buf + (size_t)J * (size_t)(3 * t + 2);
    u = u1;
  }
  double theta = 1.0, last_gap = NAN, last_g = NAN, last_P = NAN;
  int64_t t = 0;
  for (;; ++t) {
    const double gamma = stage_gamma(gamma0, gamma_end, factor, t / iters_per_stage);
    if (t % gap_every == 0 && gamma == gamma_end) {
      /* certified gap at lam (orc_certify's scaled point) */
      for (int32_t k = 0; k < nthreads; ++k) {
        jobs[k].y = lam;
        jobs[k].gamma = gamma;
      }
      run_jobs(jobs, th, nthreads);
      double obj = jobs[0].obj, P = 0;
      for (int32_t k = 1; k < nthreads; ++k) obj += jobs[k].obj;
      double g = obj;
      for (int64_t j = 0; j < J; ++j) {
        double Ax = jobs[0].Ax[j], Cx = jobs[0].Cx[j], Qx = jobs[0].Qx[j];
        for (int32_t k = 1; k < nthreads; ++k) {
          Ax += jobs[k].Ax[j];
          Cx += jobs[k].Cx[j];
          Qx += jobs[k].Qx[j];
        }
        const double s = (Ax > p->b[j] && p->b[j] / Ax < 1.0) ? p->b[j] / Ax : 1.0;
        P += s * Cx + 0.5 * gamma * s * s * Qx;
        g += lam[j] * (Ax - p->b[j]);
      }
      last_g = g;
      last_P = P;
      last_gap = (P - g) / (fabs(g) > 1e-30 ? fabs(g) : 1e-30);
      if (last_gap <= target) break;
    }
    if (t >= max_iters) break;
    /* one iteration at y (gradient sums only) */
    for (int32_t k = 0; k < nthreads; ++k) {
      jobs[k].y = y;
      jobs[k].gamma = gamma;
      jobs[k].Cx = jobs[k].Qx = NULL;
    }
    run_jobs(jobs, th, nthreads);
    for (int32_t k = 0; k < nthreads; ++k) {
      jobs[k].Cx = buf + (size_t)J * (size_t)(3 * k + 1);
      jobs[k].Qx = buf + (size_t)J * (size_t)(3 * k + 2);
    }
    for (int64_t j = 0; j < J; ++j) {
      double Ax = jobs[0].Ax[j];
      for (int32_t k = 1; k < nthreads; ++k) Ax += jobs[k].Ax[j];
      G[j] = Ax - p->b[j];
    }
    for (int64_t k = 0; k < J; ++k) {
      double step = h[k] > 0 ? gamma / h[k] : 0.0;
      double v = y[k] + step * G[k];
      nl[k] = v > 0 ? v : 0;
    }
    const double gamma_next = stage_gamma(gamma0, gamma_end, factor, (t + 1) / iters_per_stage);
    int restart_now = gamma_next != gamma;
    if (restart && !restart_now) {
      double dot = 0.0;
      for (int64_t k = 0; k < J; ++k) {
        double step = h[k] > 0 ? gamma / h[k] : 0.0;
        if (step > 0) dot += (nl[k] - y[k]) * (nl[k] - lam[k]) / step;
      }
      restart_now = dot < 0.0;
    }
    if (restart_now) {
      theta = 1.0;
      for (int64_t k = 0; k < J; ++k) lam[k] = y[k] = nl[k];
    } else {
      double th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      double beta = (theta - 1.0) / th1;
      for (int64_t k = 0; k < J; ++k) {
        y[k] = nl[k] + beta * (nl[k] - lam[k]);
        lam[k] = nl[k];
      }
      theta = th1;
    }
  }
  for (int64_t k = 0; k < J; ++k) lam_out[k] = lam[k];
  stats[0] = (double)t;
  stats[1] = last_gap;
  stats[2] = last_g;
  stats[3] = last_P;
  free(h);
  free(lam);
  free(y);
  free(G);
  free(nl);
  free(buf);
  free(jobs);
  free(th);
}
