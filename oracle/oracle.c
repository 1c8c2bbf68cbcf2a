/*
 * Oracle (CPU, FP64) for the P1 finite element system (rho*K + M) u = f of the
 * reduced optimality equation -rho*Lap(u) + u = ubar, u = 0 on the boundary
 * (Langer, Steinbach, Yang, arXiv 2102.03515, Sec. 1 eq. (sigular), Sec. 2 eq. (linsys)).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement that the CUDA library is checked against.  It shares no code,
 * header, table or constant with the CUDA library; only tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.
 *
 * Contents (each function cites the passage it follows):
 *   - Kuhn subdivision of the unit cube into 6 n^3 tetrahedra (the paper uses an
 *     admissible simplicial decomposition, Sec. 2; the Kuhn type is our reading).
 *   - P1 element stiffness / mass matrices and the load vector by quadrature
 *     (Sec. 2, the entries of K, M and f below eq. (linsys)).
 *   - Assembly with homogeneous Dirichlet rows/columns removed (V_h = S_h^1 cap H_0^1).
 *   - Jacobi-preconditioned CG in FP64 (Sec. 4 stops PCG on a relative residual).
 *   - Dense Cholesky factorisation and solve (brute force on tiny meshes).
 *   - L2 and H1-seminorm errors by quadrature (Sec. 4.1, Tables 1-2).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so x86 and
 * aarch64 hosts give identical results), with -fopenmp where the compiler has it: the
 * independent rows of assembly and of A x are then shared out among threads (the thread
 * count is set by ora_set_threads, 1 by default) without changing any result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the row loops of assembly and of A x (1 = serial; without OpenMP always 1).
 * Returns the count in effect. */
int ora_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
  omp_set_num_threads(nthreads);
  return nthreads;
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------ mesh */

/* Vertex (i,j,k), 0 <= i,j,k <= n, has index i + (n+1)*(j + (n+1)*k). */
static int64_t vid(int n, int i, int j, int k) {
  return (int64_t)i + (int64_t)(n + 1) * ((int64_t)j + (int64_t)(n + 1) * k);
}

/* Uniform vertex coordinates h*(i,j,k), h = 1/n. */
void ora_uniform_xyz(int n, double *xyz) {
  double h = 1.0 / n;
  for (int k = 0; k <= n; k++)
    for (int j = 0; j <= n; j++)
      for (int i = 0; i <= n; i++) {
        int64_t v = vid(n, i, j, k);
        xyz[3 * v + 0] = i * h;
        xyz[3 * v + 1] = j * h;
        xyz[3 * v + 2] = k * h;
      }
}

/* Kuhn subdivision: cube (i,j,k) is cut into the 6 tetrahedra that follow the
 * monotone lattice paths from its corner (i,j,k) to (i+1,j+1,k+1); the path for
 * the permutation s steps along axis s[0], then s[1], then s[2].  Cubes are
 * visited with i fastest, the permutations in the order below. */
static const int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

void ora_kuhn_tets(int n, int32_t *tets) {
  int64_t t = 0;
  for (int k = 0; k < n; k++)
    for (int j = 0; j < n; j++)
      for (int i = 0; i < n; i++)
        for (int p = 0; p < 6; p++) {
          int c[3] = {i, j, k};
          tets[4 * t + 0] = (int32_t)vid(n, c[0], c[1], c[2]);
          for (int s = 0; s < 3; s++) {
            c[PERMS[p][s]] += 1;
            tets[4 * t + 1 + s] = (int32_t)vid(n, c[0], c[1], c[2]);
          }
          t++;
        }
}

/* ------------------------------------------------------- element algebra */

/* Affine map of tet X (4x3): J = [x1-x0 | x2-x0 | x3-x0].  Returns det J.
 * grad[a][:] is the gradient of the barycentric coordinate lambda_a; the
 * gradients of lambda_1..3 are the rows of J^{-1}, and grad lambda_0 is minus
 * their sum. */
static double tet_geometry(const double X[4][3], double grad[4][3]) {
  double J[3][3];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) J[r][c] = X[c + 1][r] - X[0][r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  /* inverse = adjugate / det */
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int d = 0; d < 3; d++) {
    grad[1][d] = inv[0][d];
    grad[2][d] = inv[1][d];
    grad[3][d] = inv[2][d];
    grad[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
  }
  return det;
}

/* Element matrices of one tet (Sec. 2, entries of K and M):
 *   K_e[a][b] = |tau| grad(lambda_a) . grad(lambda_b)
 *   M_e[a][b] = |tau| (1 + delta_ab) / 20     (exact integral of lambda_a lambda_b)
 * Returns det J (sign = orientation); |tau| = |det J| / 6. */
double ora_element(const double *X12, double *Ke16, double *Me16) {
  double X[4][3], g[4][3];
  for (int a = 0; a < 4; a++)
    for (int d = 0; d < 3; d++) X[a][d] = X12[3 * a + d];
  double det = tet_geometry(X, g);
  double vol = fabs(det) / 6.0;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      Ke16[4 * a + b] = vol * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
      Me16[4 * a + b] = vol * (a == b ? 2.0 : 1.0) / 20.0;
    }
  return det;
}

/* ------------------------------------------------------------ targets */

enum { T_SINE = 0, T_BOX = 1, T_BUMPS = 2, T_SINE_PLUS_ONE = 3, T_SINE_SCALED = 4,
       T_QUADVALS = 5 };

typedef struct {
  int kind;
  int nb;           /* number of Gaussian bumps (T_BUMPS) */
  const double *c;  /* nb x 3 centres */
  const double *w;  /* nb widths */
  const double *a;  /* nb amplitudes */
  double lo, hi;    /* box (lo,hi)^3 for T_BOX */
  double scale;     /* factor for T_SINE_SCALED */
  const double *qv; /* T_QUADVALS: ubar at the 4 points of the degree-2 rule of each tet,
                       [tet][point], point q with barycentric weight A on local vertex q */
} target_t;


static const double PI = 3.14159265358979323846;

/* Targets of Sec. 4: smooth sine (4.1), discontinuous box (4.2), sine plus one
 * (4.3); Gaussian bumps are the synthetic targets of the batched workload. */
static double target_eval(const target_t *T, const double x[3]) {
  switch (T->kind) {
    case T_SINE:
      return sin(PI * x[0]) * sin(PI * x[1]) * sin(PI * x[2]);
    case T_SINE_SCALED:
      return T->scale * sin(PI * x[0]) * sin(PI * x[1]) * sin(PI * x[2]);
    case T_SINE_PLUS_ONE:
      return 1.0 + sin(PI * x[0]) * sin(PI * x[1]) * sin(PI * x[2]);
    case T_BOX:
      return (x[0] > T->lo && x[0] < T->hi && x[1] > T->lo && x[1] < T->hi &&
              x[2] > T->lo && x[2] < T->hi)
                 ? 1.0
                 : 0.0;
    case T_BUMPS: {
      double s = 0.0;
      for (int b = 0; b < T->nb; b++) {
        double dx = x[0] - T->c[3 * b], dy = x[1] - T->c[3 * b + 1], dz = x[2] - T->c[3 * b + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        s += T->a[b] * exp(-r2 / (2.0 * T->w[b] * T->w[b]));
      }
      return s;
    }
  }
  return 0.0;
}

/* ubar at point q of tet t for the load vector: the given values (T_QUADVALS, 4-point rule
 * only) or the target at x. */
static double target_at(const target_t *T, int64_t t, int q, const double x[3]) {
  return T->kind == T_QUADVALS ? T->qv[4 * t + q] : target_eval(T, x);
}

/* Gradient of the smooth sine targets (for the H1-seminorm error, Table 2). */
static void sine_grad(double scale, const double x[3], double g[3]) {
  double s0 = sin(PI * x[0]), s1 = sin(PI * x[1]), s2 = sin(PI * x[2]);
  double c0 = cos(PI * x[0]), c1 = cos(PI * x[1]), c2 = cos(PI * x[2]);
  g[0] = scale * PI * c0 * s1 * s2;
  g[1] = scale * PI * s0 * c1 * s2;
  g[2] = scale * PI * s0 * s1 * c2;
}

/* ------------------------------------------------------------ quadrature */

/* Degree-2, 4-point rule of Hammer and Stroud on a tetrahedron: the points have
 * barycentric coordinates that are the 4 permutations of (A, B, B, B) with
 * A = (5 + 3 sqrt 5)/20 and B = (5 - sqrt 5)/20, each with weight |tau|/4.
 * Level L > 0 applies the rule on each of the 8^L sub-tetrahedra of L rounds
 * of Bey's red refinement.  Everything is expressed in barycentric coordinates
 * of the parent tet. */
typedef struct {
  int np;
  double *bary; /* np x 4 */
  double *wt;   /* np, summing to 1 */
} qrule_t;

static void bey_children(const double P[4][4], double C[8][4][4]) {
  double m[4][4][4]; /* m[a][b] = midpoint of edge ab */
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++)
      for (int d = 0; d < 4; d++) m[a][b][d] = 0.5 * (P[a][d] + P[b][d]);
  /* children of Bey's refinement: 4 corner tets and 4 from the inner octahedron
   * cut along the diagonal x02-x13 */
  const int kids[8][4][2] = {
      {{0, 0}, {0, 1}, {0, 2}, {0, 3}}, {{0, 1}, {1, 1}, {1, 2}, {1, 3}},
      {{0, 2}, {1, 2}, {2, 2}, {2, 3}}, {{0, 3}, {1, 3}, {2, 3}, {3, 3}},
      {{0, 1}, {0, 2}, {0, 3}, {1, 3}}, {{0, 1}, {0, 2}, {1, 2}, {1, 3}},
      {{0, 2}, {0, 3}, {1, 3}, {2, 3}}, {{0, 2}, {1, 2}, {1, 3}, {2, 3}}};
  for (int c = 0; c < 8; c++)
    for (int v = 0; v < 4; v++)
      for (int d = 0; d < 4; d++) C[c][v][d] = m[kids[c][v][0]][kids[c][v][1]][d];
}

static void qrule_fill(const double P[4][4], int level, double wscale, double *bary, double *wt,
                       int *idx) {
  if (level == 0) {
    const double A = (5.0 + 3.0 * sqrt(5.0)) / 20.0, B = (5.0 - sqrt(5.0)) / 20.0;
    for (int q = 0; q < 4; q++) {
      double mu[4] = {B, B, B, B};
      mu[q] = A;
      for (int d = 0; d < 4; d++) {
        double s = 0.0;
        for (int v = 0; v < 4; v++) s += mu[v] * P[v][d];
        bary[4 * (*idx) + d] = s;
      }
      wt[*idx] = wscale * 0.25;
      (*idx)++;
    }
    return;
  }
  double C[8][4][4];
  bey_children(P, C);
  for (int c = 0; c < 8; c++) qrule_fill(C[c], level - 1, wscale / 8.0, bary, wt, idx);
}

static qrule_t qrule_make(int level) {
  qrule_t r;
  r.np = 4;
  for (int l = 0; l < level; l++) r.np *= 8;
  r.bary = (double *)malloc(sizeof(double) * 4 * r.np);
  r.wt = (double *)malloc(sizeof(double) * r.np);
  double P[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  int idx = 0;
  qrule_fill(P, level, 1.0, r.bary, r.wt, &idx);
  return r;
}

static void qrule_free(qrule_t *r) {
  free(r->bary);
  free(r->wt);
}

/* Export the rule (for tests of its exactness on polynomials). */
int ora_qrule(int level, double *bary, double *wt) {
  qrule_t r = qrule_make(level);
  memcpy(bary, r.bary, sizeof(double) * 4 * r.np);
  memcpy(wt, r.wt, sizeof(double) * r.np);
  int np = r.np;
  qrule_free(&r);
  return np;
}

/* ------------------------------------------------------------ assembly */

/* Sparse matrix in CSR with sorted column indices. */
typedef struct {
  int64_t nrows, nnz;
  int64_t *rowptr;
  int32_t *col;
  double *K, *M;
  double *f;
} ora_sys_t;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Assemble K, M (Sec. 2: K_ij = int grad phi_j . grad phi_i, M_ij = int phi_j phi_i)
 * and f_i = int ubar phi_i by the quadrature rule of the given level, on a mesh
 * given by vertex coordinates and tetrahedra.  dof[v] >= 0 numbers the unknowns;
 * dof[v] < 0 marks Dirichlet vertices, whose rows and columns are dropped
 * (homogeneous boundary condition, V_h subset H_0^1).
 *
 * Rows are built vertex by vertex: a vertex's incident tets are visited in
 * increasing tet index, its element contributions added in that order.
 * Returns 0, or -1 on allocation failure / -2 on a degenerate tet. */
int ora_assemble(int64_t nv, const double *xyz, int64_t nt, const int32_t *tets,
                 const int32_t *dof, int64_t ndof, const target_t *T, int qlevel,
                 ora_sys_t *out) {
  memset(out, 0, sizeof(*out));
  if (T->kind == T_QUADVALS && qlevel != 0) return -3;   /* values given for 4 points */
  int64_t *inc_ptr = (int64_t *)calloc(nv + 1, sizeof(int64_t));
  if (!inc_ptr) return -1;
  for (int64_t t = 0; t < nt; t++)
    for (int a = 0; a < 4; a++) inc_ptr[tets[4 * t + a] + 1]++;
  for (int64_t v = 0; v < nv; v++) inc_ptr[v + 1] += inc_ptr[v];
  int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * inc_ptr[nv]);
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nv);
  if (!inc || !fill) return -1;
  memcpy(fill, inc_ptr, sizeof(int64_t) * nv);
  for (int64_t t = 0; t < nt; t++)
    for (int a = 0; a < 4; a++) inc[fill[tets[4 * t + a]]++] = t;
  free(fill);

  /* row patterns: neighbouring dofs through incident tets, sorted, unique */
  int64_t *rowptr = (int64_t *)calloc(ndof + 1, sizeof(int64_t));
  int64_t *row_vertex = (int64_t *)malloc(sizeof(int64_t) * (ndof > 0 ? ndof : 1));
  if (!rowptr || !row_vertex) return -1;
  for (int64_t v = 0; v < nv; v++)
    if (dof[v] >= 0) row_vertex[dof[v]] = v;
  int maxdeg = 0;
  for (int64_t v = 0; v < nv; v++) {
    int64_t d = inc_ptr[v + 1] - inc_ptr[v];
    if (d > maxdeg) maxdeg = (int)d;
  }
  /* rows are independent: with OpenMP they are shared out among threads (each with its
   * own scratch list); every row is computed the same way whatever the thread count */
  int alloc_fail = 0;
#pragma omp parallel reduction(| : alloc_fail)
  {
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (4 * (size_t)maxdeg + 1));
    if (!buf) alloc_fail = 1;
#pragma omp for schedule(static, 1024)
    for (int64_t r = 0; r < ndof; r++) {
      if (!buf) continue;
      int64_t v = row_vertex[r];
      int cnt = 0;
      for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++)
        for (int a = 0; a < 4; a++) {
          int32_t w = dof[tets[4 * inc[e] + a]];
          if (w >= 0) buf[cnt++] = w;
        }
      qsort(buf, cnt, sizeof(int32_t), cmp_i32);
      int u = 0;
      for (int q = 0; q < cnt; q++)
        if (u == 0 || buf[q] != buf[u - 1]) buf[u++] = buf[q];
      rowptr[r + 1] = u;   /* row length; the prefix sum follows */
    }
    free(buf);
  }
  if (alloc_fail) return -1;
  for (int64_t r = 0; r < ndof; r++) rowptr[r + 1] += rowptr[r];
  int64_t nnz = rowptr[ndof];
  int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  double *K = (double *)calloc(nnz > 0 ? nnz : 1, sizeof(double));
  double *M = (double *)calloc(nnz > 0 ? nnz : 1, sizeof(double));
  double *f = (double *)calloc(ndof > 0 ? ndof : 1, sizeof(double));
  if (!col || !K || !M || !f) return -1;

  qrule_t Q = qrule_make(qlevel);
  int bad = 0;
#pragma omp parallel reduction(| : bad, alloc_fail)
  {
  int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (4 * (size_t)maxdeg + 1));
  if (!buf) alloc_fail = 1;
#pragma omp for schedule(static, 1024)
  for (int64_t r = 0; r < ndof; r++) {
    if (!buf) continue;
    int64_t v = row_vertex[r];
    int cnt = 0;
    for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++)
      for (int a = 0; a < 4; a++) {
        int32_t w = dof[tets[4 * inc[e] + a]];
        if (w >= 0) buf[cnt++] = w;
      }
    qsort(buf, cnt, sizeof(int32_t), cmp_i32);
    int u = 0;
    for (int q = 0; q < cnt; q++)
      if (u == 0 || buf[q] != buf[u - 1]) buf[u++] = buf[q];
    int32_t *rc = col + rowptr[r];
    memcpy(rc, buf, sizeof(int32_t) * u);

    for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++) {
      const int32_t *tv = tets + 4 * inc[e];
      double X[12], Ke[16], Me[16];
      int loc = -1;
      for (int a = 0; a < 4; a++) {
        for (int d = 0; d < 3; d++) X[3 * a + d] = xyz[3 * (int64_t)tv[a] + d];
        if (tv[a] == v) loc = a;
      }
      double det = ora_element(X, Ke, Me);
      if (!(det != 0.0)) bad = 1;
      double vol = fabs(det) / 6.0;
      for (int b = 0; b < 4; b++) {
        int32_t w = dof[tv[b]];
        if (w < 0) continue;
        /* binary search for column w in row r */
        int lo = 0, hi = u - 1;
        while (lo < hi) {
          int mid = (lo + hi) / 2;
          if (rc[mid] < w) lo = mid + 1; else hi = mid;
        }
        K[rowptr[r] + lo] += Ke[4 * loc + b];
        M[rowptr[r] + lo] += Me[4 * loc + b];
      }
      /* load: sum_q w_q |tau| ubar(x_q) lambda_loc(x_q) */
      double acc = 0.0;
      for (int q = 0; q < Q.np; q++) {
        double x[3] = {0, 0, 0};
        for (int a = 0; a < 4; a++)
          for (int d = 0; d < 3; d++) x[d] += Q.bary[4 * q + a] * X[3 * a + d];
        acc += Q.wt[q] * target_at(T, inc[e], q, x) * Q.bary[4 * q + loc];
      }
      f[r] += vol * acc;
    }
  }
  free(buf);
  }
  qrule_free(&Q);
  free(inc);
  free(inc_ptr);
  free(row_vertex);
  if (alloc_fail) return -1;
  out->nrows = ndof;
  out->nnz = nnz;
  out->rowptr = rowptr;
  out->col = col;
  out->K = K;
  out->M = M;
  out->f = f;
  return bad ? -2 : 0;
}

void ora_sys_free(ora_sys_t *s) {
  free(s->rowptr);
  free(s->col);
  free(s->K);
  free(s->M);
  free(s->f);
  memset(s, 0, sizeof(*s));
}

/* Signed volumes (det J / 6) of all tets: used to check that jitter keeps the
 * mesh admissible (every det > 0 for the positively oriented Kuhn tets). */
void ora_tet_dets(int64_t nt, const int32_t *tets, const double *xyz, double *det_out) {
  for (int64_t t = 0; t < nt; t++) {
    double X[4][3], g[4][3];
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)tets[4 * t + a] + d];
    det_out[t] = tet_geometry(X, g);
  }
}

/* ------------------------------------------------------------ solvers */

/* y = (rho K + M) x, summing each row in column order (rows shared out among OpenMP
 * threads when built with it; each row's sum is the same whatever the thread count). */
void ora_apply(const ora_sys_t *s, double rho, const double *x, double *y) {
#pragma omp parallel for schedule(static, 4096)
  for (int64_t r = 0; r < s->nrows; r++) {
    double acc = 0.0;
    for (int64_t e = s->rowptr[r]; e < s->rowptr[r + 1]; e++)
      acc += (rho * s->K[e] + s->M[e]) * x[s->col[e]];
    y[r] = acc;
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* Conjugate gradients preconditioned by the diagonal of A = rho K + M
 * (Hestenes-Stiefel form).  x holds the initial guess on entry (zero for the
 * reading x0 = 0) and the iterate on exit.  Stops when ||r||_2 <= tol ||b||_2
 * or after maxit iterations; the returned residual is recomputed as b - A x.
 * Returns the iteration count (negative on breakdown). */
int ora_jacobi_pcg(const ora_sys_t *s, double rho, const double *b, double *x, double tol,
                   int maxit, double *relres_out) {
  int64_t n = s->nrows;
  double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
  double *dinv = (double *)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; i++) {
    double d = 0.0;
    for (int64_t e = s->rowptr[i]; e < s->rowptr[i + 1]; e++)
      if (s->col[e] == i) d = rho * s->K[e] + s->M[e];
    dinv[i] = 1.0 / d;
  }
  ora_apply(s, rho, x, q);
  for (int64_t i = 0; i < n; i++) r[i] = b[i] - q[i];
  double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  for (int64_t i = 0; i < n; i++) z[i] = dinv[i] * r[i];
  memcpy(p, z, sizeof(double) * n);
  double rz = dot(n, r, z);
  int it = 0, status = 0;
  while (it < maxit && sqrt(dot(n, r, r)) > tol * bnorm) {
    ora_apply(s, rho, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) { status = -1; break; }
    double alpha = rz / pq;
    for (int64_t i = 0; i < n; i++) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    for (int64_t i = 0; i < n; i++) z[i] = dinv[i] * r[i];
    double rz_new = dot(n, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    it++;
  }
  ora_apply(s, rho, x, q);
  for (int64_t i = 0; i < n; i++) r[i] = b[i] - q[i];
  if (relres_out) *relres_out = sqrt(dot(n, r, r)) / bnorm;
  free(r); free(z); free(p); free(q); free(dinv);
  return status < 0 ? -(it + 1) : it;
}

/* Dense Cholesky A = L L^T in place (lower triangle, row-major n x n), then
 * forward/back substitution.  Returns 0, or the 1-based index of a non-positive
 * pivot. */
int ora_cholesky(int n, double *A) {
  for (int j = 0; j < n; j++) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; k++) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    A[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; i++) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; k++) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / ljj;
    }
  }
  return 0;
}

void ora_cholesky_solve(int n, const double *L, const double *b, double *x) {
  for (int i = 0; i < n; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= L[(size_t)i * n + k] * x[k];
    x[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = x[i];
    for (int k = i + 1; k < n; k++) s -= L[(size_t)k * n + i] * x[k];
    x[i] = s / L[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------ errors */

/* Squared L2 norm of (uex - u_h) over the mesh, and the squared L2 norm of the
 * gradient difference (H1 seminorm; only for the sine kinds, else returns 0 in
 * *h1sq).  u_h = sum_v U[v] phi_v with U given on all vertices (zeros on the
 * boundary).  Quadrature: the rule of the given level on each tet (Sec. 4.1,
 * Tables 1 and 2 report these norms). */
void ora_errors(int64_t nv, const double *xyz, int64_t nt, const int32_t *tets,
                const double *U, const target_t *T, int qlevel, double *l2sq, double *h1sq) {
  (void)nv;
  qrule_t Q = qrule_make(qlevel);
  double e2 = 0.0, g2 = 0.0;
  int has_grad = (T->kind == T_SINE || T->kind == T_SINE_SCALED || T->kind == T_SINE_PLUS_ONE);
  double gscale = (T->kind == T_SINE_SCALED) ? T->scale : 1.0;
  for (int64_t t = 0; t < nt; t++) {
    double X[4][3], g[4][3], uv[4];
    for (int a = 0; a < 4; a++) {
      int32_t v = tets[4 * t + a];
      uv[a] = U[v];
      for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)v + d];
    }
    double det = tet_geometry(X, g);
    double vol = fabs(det) / 6.0;
    double guh[3] = {0, 0, 0};
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) guh[d] += uv[a] * g[a][d];
    for (int q = 0; q < Q.np; q++) {
      double x[3] = {0, 0, 0}, uh = 0.0;
      for (int a = 0; a < 4; a++) {
        for (int d = 0; d < 3; d++) x[d] += Q.bary[4 * q + a] * X[a][d];
        uh += Q.bary[4 * q + a] * uv[a];
      }
      double diff = target_eval(T, x) - uh;
      e2 += vol * Q.wt[q] * diff * diff;
      if (has_grad) {
        double ge[3];
        sine_grad(gscale, x, ge);
        double dd = 0.0;
        for (int d = 0; d < 3; d++) dd += (ge[d] - guh[d]) * (ge[d] - guh[d]);
        g2 += vol * Q.wt[q] * dd;
      }
    }
  }
  qrule_free(&Q);
  *l2sq = e2;
  *h1sq = g2;
}

/* ------------------------------------------------------------ post-processing */

/* Target values at points (npts x 3 coordinates); used for the control recovery of
 * Sec. 2, z = (ubar - u) / rho, evaluated at the vertices. */
void ora_target_values(const target_t *T, int64_t npts, const double *xyz, double *out) {
  for (int64_t i = 0; i < npts; i++) out[i] = target_eval(T, xyz + 3 * i);
}

/* ------------------------------------------------------------ single rows */

/* Rows of K, M and f for selected interior vertices of the Kuhn mesh with n cells per side,
 * each built from the tets of the 8 cubes around the vertex that contain it (the same
 * element matrices and quadrature as ora_assemble, without building the whole mesh).
 * xyz may be NULL (uniform grid).  vtx: vertex ids i + (n+1)(j + (n+1)k) of interior
 * vertices.  Outputs per row: up to 15 unknown columns (sorted, -1 padded), K, M values and
 * f.  Returns 0, or -1 if a vertex is not interior. */
int ora_kuhn_rows(int n, const double *xyz, const target_t *T, int qlevel, int64_t nsel,
                  const int64_t *vtx, int32_t *cols, double *Kout, double *Mout, double *fout) {
  if (T->kind == T_QUADVALS && qlevel != 0) return -3;   /* values given for 4 points */
  qrule_t Q = qrule_make(qlevel);
  const int m = n - 1;
  const double h = 1.0 / n;
  for (int64_t s = 0; s < nsel; s++) {
    int64_t v = vtx[s];
    int i = (int)(v % (n + 1)), j = (int)((v / (n + 1)) % (n + 1)), k = (int)(v / ((int64_t)(n + 1) * (n + 1)));
    if (i < 1 || j < 1 || k < 1 || i > m || j > m || k > m) {
      qrule_free(&Q);
      return -1;
    }
    int32_t rc[32];
    double rk[32], rm[32];
    int u = 0;
    double fv = 0.0;
    /* cubes with corner c = (i,j,k) - (a,b,d), in increasing cube id */
    for (int dz = 1; dz >= 0; dz--)
      for (int dy = 1; dy >= 0; dy--)
        for (int dx = 1; dx >= 0; dx--) {
          int c[3] = {i - dx, j - dy, k - dz};
          if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= n || c[1] >= n || c[2] >= n) continue;
          for (int p = 0; p < 6; p++) {
            int w[4][3];
            for (int d = 0; d < 3; d++) w[0][d] = c[d];
            for (int st = 0; st < 3; st++) {
              for (int d = 0; d < 3; d++) w[st + 1][d] = w[st][d];
              w[st + 1][PERMS[p][st]] += 1;
            }
            int loc = -1;
            for (int a = 0; a < 4; a++)
              if (w[a][0] == i && w[a][1] == j && w[a][2] == k) loc = a;
            if (loc < 0) continue;
            double X[12], Ke[16], Me[16];
            for (int a = 0; a < 4; a++) {
              int64_t id = vid(n, w[a][0], w[a][1], w[a][2]);
              for (int d = 0; d < 3; d++)
                X[3 * a + d] = xyz ? xyz[3 * id + d] : w[a][d] * h;
            }
            double det = ora_element(X, Ke, Me);
            double vol = fabs(det) / 6.0;
            for (int b = 0; b < 4; b++) {
              int bi = w[b][0], bj = w[b][1], bk = w[b][2];
              if (bi < 1 || bj < 1 || bk < 1 || bi > m || bj > m || bk > m) continue;
              int32_t col = (bi - 1) + m * ((bj - 1) + m * (bk - 1));
              int q = 0;
              while (q < u && rc[q] != col) q++;
              if (q == u) {
                rc[u] = col;
                rk[u] = 0.0;
                rm[u] = 0.0;
                u++;
              }
              rk[q] += Ke[4 * loc + b];
              rm[q] += Me[4 * loc + b];
            }
            double acc = 0.0;
            for (int q = 0; q < Q.np; q++) {
              double x[3] = {0, 0, 0};
              for (int a = 0; a < 4; a++)
                for (int d = 0; d < 3; d++) x[d] += Q.bary[4 * q + a] * X[3 * a + d];
              const int64_t tid = 6 * (c[0] + (int64_t)n * (c[1] + (int64_t)n * c[2])) + p;
              acc += Q.wt[q] * target_at(T, tid, q, x) * Q.bary[4 * q + loc];
            }
            fv += vol * acc;
          }
        }
    /* sort the row by column */
    for (int a = 1; a < u; a++)
      for (int b = a; b > 0 && rc[b - 1] > rc[b]; b--) {
        int32_t tc = rc[b]; rc[b] = rc[b - 1]; rc[b - 1] = tc;
        double tk = rk[b]; rk[b] = rk[b - 1]; rk[b - 1] = tk;
        double tm = rm[b]; rm[b] = rm[b - 1]; rm[b - 1] = tm;
      }
    for (int q = 0; q < 15; q++) {
      cols[15 * s + q] = q < u ? rc[q] : -1;
      Kout[15 * s + q] = q < u ? rk[q] : 0.0;
      Mout[15 * s + q] = q < u ? rm[q] : 0.0;
    }
    fout[s] = fv;
  }
  qrule_free(&Q);
  return 0;
}
