/*
 * FP64 CPU oracle for block nAIR (arXiv 1704.05001).  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg call it; the
 * GPU library never does.  It shares no code with the CUDA path.
 *
 * Plain loops, one step of the method after another, in the order the paper
 * gives them:
 *   - block Jacobi smoothing and coarse-grid correction, Eq. relax / Eq. cgc;
 *   - block form P = [W; I], R = [Z I], K = R A P, Eq. block / Eq. rap;
 *   - classical strength of connection and C/F splitting, Sec. 5.1;
 *   - truncated Neumann approximation of A_ff^{-1}, Eq. neumann (Sec. 4.1),
 *     restricted to strong F-F connections, R = [-A_cf Delta, I];
 *   - one-point interpolation, Sec. 5.1;
 *   - block nAIR and filtering, Sec. 5.2;
 *   - V-cycle with no pre-relaxation, F-relaxation with one more sweep than
 *     the Neumann degree, then a C sweep (Sec. 5, Remark on C-relaxation);
 *     optionally the F-cycle of the scaling study (Sec. 6);
 *   - GMRES acceleration (Sec. 6), as flexible GMRES(m) with CGS2;
 *   - for A^T: the transposed cycle of the same hierarchy (R^T interpolates,
 *     P^T restricts, pre-relaxation; Corollary on ideal interpolation).
 *
 * Canonical arithmetic (so that the GPU path can be compared bit for bit on
 * C/F splittings and sparsity patterns): every value upstream of a threshold
 * is computed with correctly rounded IEEE operations in a fixed order:
 *   block products c_rc = fma(a_rt, b_tc, c_rc), t ascending, summed over the
 *   inner block index in ascending order; squared block norms s = fma(x, x, s)
 *   over the block in row-major order; Gauss-Jordan inverses as below.
 * Build with -ffp-contract=off so that the compiler adds no contraction.
 *
 * The parity build is single-threaded.  A second build with -fopenmp exists
 * only to time the oracle on all host cores: its pragmas split loops whose
 * iterations write disjoint rows (every row's arithmetic is unchanged), and its
 * dot products add fixed contiguous chunks in order, so it is deterministic
 * but rounds dot products differently from the single-threaded build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_SINGULAR_BLOCK 2
#define ORC_ERR_NOT_CONVERGED 3
#define ORC_ERR_BREAKDOWN 4
#define ORC_ERR_OOM 5

#define MAXLEV 64

typedef struct {
  int nrows, ncols;
  int *rp, *ci; /* row pointer (nrows + 1), sorted unique column indices */
  double *v;    /* nnzb * b * b, row-major inside each block */
} Bsr;

typedef struct {
  int E, nC, nF, coarsest;
  Bsr A;
  double *Dinv;          /* E blocks */
  double *snorm;         /* squared Frobenius norm of every block of A */
  unsigned char *strong; /* one flag per block of A */
  int *lam;              /* lambda_i = |{j : i in S_j}| */
  signed char *cf;       /* 1 = C, 0 = F */
  int *cidx, *fidx;      /* fine element -> coarse index / F index (or -1) */
  int *c2f, *f2f;        /* coarse index / F index -> fine element */
  int *ipc;              /* fine element -> coarse column of P (C: itself; F: one-point source or -1) */
  Bsr L, Delta, Rcf, AP; /* Rcf columns are F indices; AP is E x nC */
  int n;                 /* coarsest: dense size */
  double *lu;            /* coarsest: LU factors (row-major n x n) */
  int *piv;
} Level;

typedef struct {
  int b, nlev;
  Level lev[MAXLEV];
  int f_sweeps, c_sweeps;
  int transposed; /* solve with A^T and the transposed cycle (adjoint) */
  int cycle_type; /* 0: V-cycle, 1: F-cycle (forward preconditioner) */
  /* scalar nAIR: the hierarchy (b = 1) is built for D^{-1} A; the Krylov solve
   * keeps the block matrix A (block size bo) and D^{-1} */
  int scalar, bo;
  Bsr Ao;
  double *Do;
} Hier;

static void bsr_free(Bsr *m) {
  free(m->rp);
  free(m->ci);
  free(m->v);
  memset(m, 0, sizeof(*m));
}

static int bsr_nnzb(const Bsr *m) { return m->rp ? m->rp[m->nrows] : 0; }

static double block_norm2(int b, const double *x) {
  double s = 0.0;
  for (int k = 0; k < b * b; ++k) s = fma(x[k], x[k], s);
  return s;
}

/* ---------------------------------------------------------------------------
 * a1: inverse of one b x b block, in-place Gauss-Jordan with partial pivoting.
 * Pivot = first row (from k down) with the largest |entry| in column k.  The
 * pivot row is multiplied by the reciprocal of the pivot (one IEEE division per
 * step), every other row r gets
 * M[r][c] = fma(-l, M[k][c], M[r][c]) with l = M[r][k]; columns are swapped
 * back at the end.  A zero pivot is a singular block.
 * ------------------------------------------------------------------------- */
static int gj_inverse(int b, const double *A, double *M) {
  int piv[64];
  memcpy(M, A, sizeof(double) * b * b);
  for (int k = 0; k < b; ++k) {
    int p = k;
    double best = fabs(M[k * b + k]);
    for (int r = k + 1; r < b; ++r) {
      double a = fabs(M[r * b + k]);
      if (a > best) { best = a; p = r; }
    }
    piv[k] = p;
    if (p != k)
      for (int c = 0; c < b; ++c) {
        double t = M[k * b + c];
        M[k * b + c] = M[p * b + c];
        M[p * b + c] = t;
      }
    double d = M[k * b + k];
    if (d == 0.0 || d != d) return ORC_ERR_SINGULAR_BLOCK;
    double rinv = 1.0 / d;
    M[k * b + k] = 1.0;
    for (int c = 0; c < b; ++c) M[k * b + c] = M[k * b + c] * rinv;
    for (int r = 0; r < b; ++r) {
      if (r == k) continue;
      double l = M[r * b + k];
      M[r * b + k] = 0.0;
      for (int c = 0; c < b; ++c) M[r * b + c] = fma(-l, M[k * b + c], M[r * b + c]);
    }
  }
  for (int k = b - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k)
      for (int r = 0; r < b; ++r) {
        double t = M[r * b + k];
        M[r * b + k] = M[r * b + p];
        M[r * b + p] = t;
      }
  }
  return ORC_OK;
}

/* splitmix64 (Steele, Lea, Flood 2014): the tie-break hash of the C/F keys. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* key_i = (lambda_i, h(i), i), compared lexicographically; returns 1 if i > j */
static int key_greater(const int *lam, uint64_t seed, int i, int j) {
  if (lam[i] != lam[j]) return lam[i] > lam[j];
  uint64_t hi = splitmix64((uint64_t)i ^ seed), hj = splitmix64((uint64_t)j ^ seed);
  if (hi != hj) return hi > hj;
  return i > j;
}

/* ---------------------------------------------------------------------------
 * a2: strength.  j in S_i iff j != i, s_ij > 0 and s_ij >= theta^2 max_{k != i} s_ik,
 * s = squared Frobenius norm of the block (block analogue of the scalar rule
 * |a_ij| >= phi max_j |a_ij|, Fig. neumann caption and Sec. 4.3).
 * ------------------------------------------------------------------------- */
static void strength(Level *L, int b, double theta2) {
  const Bsr *A = &L->A;
  int nnzb = bsr_nnzb(A);
  L->snorm = (double *)malloc(sizeof(double) * (nnzb ? nnzb : 1));
  L->strong = (unsigned char *)calloc(nnzb ? nnzb : 1, 1);
  for (int p = 0; p < nnzb; ++p) L->snorm[p] = block_norm2(b, A->v + (size_t)p * b * b);
  for (int i = 0; i < A->nrows; ++i) {
    double smax = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (A->ci[p] != i && L->snorm[p] > smax) smax = L->snorm[p];
    double thr = theta2 * smax;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      L->strong[p] = (A->ci[p] != i && L->snorm[p] > 0.0 && L->snorm[p] >= thr);
  }
}

/* ---------------------------------------------------------------------------
 * a3: C/F splitting.  Classical strength and measure lambda_i = |S_i^T|
 * (Sec. 5.1), selected by parallel independent-set rounds (PMIS form):
 * lambda_i = 0 -> F; each round, an undecided point whose key beats every
 * undecided neighbour in S u S^T becomes C, then every undecided point that
 * strongly depends on a C point becomes F.
 * ------------------------------------------------------------------------- */
static void cf_split(Level *L, uint64_t seed) {
  const Bsr *A = &L->A;
  int E = A->nrows;
  L->lam = (int *)calloc(E > 0 ? (size_t)E : 1, sizeof(int));
  L->cf = (signed char *)malloc(E > 0 ? (size_t)E : 1);
  for (int i = 0; i < E; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (L->strong[p]) L->lam[A->ci[p]]++;
  /* S^T adjacency */
  int *tp = (int *)calloc(E + 1, sizeof(int));
  for (int i = 0; i < E; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (L->strong[p]) tp[A->ci[p] + 1]++;
  for (int i = 0; i < E; ++i) tp[i + 1] += tp[i];
  int *tc = (int *)malloc(sizeof(int) * (tp[E] ? tp[E] : 1));
  int *fill = (int *)malloc(sizeof(int) * (E ? E : 1));
  for (int i = 0; i < E; ++i) fill[i] = tp[i];
  for (int i = 0; i < E; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (L->strong[p]) tc[fill[A->ci[p]]++] = i;
  enum { U = -1, F = 0, C = 1 };
  signed char *st = L->cf;
  for (int i = 0; i < E; ++i) st[i] = (L->lam[i] == 0) ? F : U;
  signed char *newc = (signed char *)malloc(E ? E : 1);
  for (;;) {
    int undecided = 0;
    for (int i = 0; i < E; ++i) undecided += (st[i] == U);
    if (!undecided) break;
    for (int i = 0; i < E; ++i) {
      newc[i] = 0;
      if (st[i] != U) continue;
      int best = 1;
      for (int p = A->rp[i]; p < A->rp[i + 1] && best; ++p) {
        int j = A->ci[p];
        if (L->strong[p] && st[j] == U && key_greater(L->lam, seed, j, i)) best = 0;
      }
      for (int p = tp[i]; p < tp[i + 1] && best; ++p) {
        int j = tc[p];
        if (st[j] == U && key_greater(L->lam, seed, j, i)) best = 0;
      }
      newc[i] = (signed char)best;
    }
    for (int i = 0; i < E; ++i)
      if (newc[i]) st[i] = C;
    for (int i = 0; i < E; ++i) {
      if (st[i] != U) continue;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (L->strong[p] && st[A->ci[p]] == C) { st[i] = F; break; }
    }
  }
  free(newc);
  free(tp);
  free(tc);
  free(fill);
}

/* sorted insertion of column j into the touched list */
static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------------
 * Block sparse product, row by row with a dense accumulator (Gustavson):
 *   out_i = init_{imap(i)} + sum_{m in row i of Lf, ascending} Lf_im * Rt_{rmap(m)}
 * A block with no init starts from +0.  Every scalar is one fma chain over
 * (m ascending, t ascending).  negate flips the sign of the result.
 * ------------------------------------------------------------------------- */
static void spgemm(int b, int nrows, int ncols, const Bsr *Lf, const int *rmap, const Bsr *Rt,
                   const Bsr *init, const int *imap, int negate, Bsr *out) {
  size_t bb = (size_t)b * b;
  double *acc = (double *)malloc(sizeof(double) * bb * (ncols ? ncols : 1));
  char *flag = (char *)calloc(ncols ? ncols : 1, 1);
  int *touched = (int *)malloc(sizeof(int) * (ncols ? ncols : 1));
  int cap = 1024, nnz = 0;
  out->nrows = nrows;
  out->ncols = ncols;
  out->rp = (int *)malloc(sizeof(int) * (nrows + 1));
  out->ci = (int *)malloc(sizeof(int) * cap);
  out->v = (double *)malloc(sizeof(double) * bb * cap);
  out->rp[0] = 0;
  for (int i = 0; i < nrows; ++i) {
    int nt = 0;
    if (init) {
      int ii = imap ? imap[i] : i;
      for (int p = init->rp[ii]; p < init->rp[ii + 1]; ++p) {
        int j = init->ci[p];
        flag[j] = 1;
        touched[nt++] = j;
        memcpy(acc + (size_t)j * bb, init->v + (size_t)p * bb, sizeof(double) * bb);
      }
    }
    for (int p = Lf->rp[i]; p < Lf->rp[i + 1]; ++p) {
      int m = rmap ? rmap[Lf->ci[p]] : Lf->ci[p];
      const double *a = Lf->v + (size_t)p * bb;
      for (int q = Rt->rp[m]; q < Rt->rp[m + 1]; ++q) {
        int j = Rt->ci[q];
        double *c = acc + (size_t)j * bb;
        if (!flag[j]) {
          flag[j] = 1;
          touched[nt++] = j;
          for (size_t k = 0; k < bb; ++k) c[k] = 0.0;
        }
        const double *bv = Rt->v + (size_t)q * bb;
        for (int r = 0; r < b; ++r)
          for (int cc = 0; cc < b; ++cc) {
            double s = c[r * b + cc];
            for (int t = 0; t < b; ++t) s = fma(a[r * b + t], bv[t * b + cc], s);
            c[r * b + cc] = s;
          }
      }
    }
    qsort(touched, nt, sizeof(int), cmp_int);
    if (nnz + nt > cap) {
      while (nnz + nt > cap) cap *= 2;
      out->ci = (int *)realloc(out->ci, sizeof(int) * cap);
      out->v = (double *)realloc(out->v, sizeof(double) * bb * cap);
    }
    for (int k = 0; k < nt; ++k) {
      int j = touched[k];
      out->ci[nnz] = j;
      double *dst = out->v + (size_t)nnz * bb, *src = acc + (size_t)j * bb;
      for (size_t e = 0; e < bb; ++e) dst[e] = negate ? -src[e] : src[e];
      flag[j] = 0;
      ++nnz;
    }
    out->rp[i + 1] = nnz;
  }
  free(acc);
  free(flag);
  free(touched);
}

/* ---------------------------------------------------------------------------
 * a8: filtering (Sec. 5.2, block form): drop off-diagonal block X_ij when
 * ||X_ij||_F^2 <= tol^2 ||X_ii||_F^2; the diagonal block (column == row) stays.
 * ------------------------------------------------------------------------- */
static void filter_bsr(int b, Bsr *M, double tol2) {
  size_t bb = (size_t)b * b;
  int w = 0;
  int *newrp = (int *)malloc(sizeof(int) * (M->nrows + 1));
  newrp[0] = 0;
  for (int i = 0; i < M->nrows; ++i) {
    double dn = 0.0;
    for (int p = M->rp[i]; p < M->rp[i + 1]; ++p)
      if (M->ci[p] == i) dn = block_norm2(b, M->v + (size_t)p * bb);
    double thr = tol2 * dn;
    for (int p = M->rp[i]; p < M->rp[i + 1]; ++p) {
      int keep = (M->ci[p] == i) || !(block_norm2(b, M->v + (size_t)p * bb) <= thr);
      if (keep) {
        M->ci[w] = M->ci[p];
        if (w != p) memmove(M->v + (size_t)w * bb, M->v + (size_t)p * bb, sizeof(double) * bb);
        ++w;
      }
    }
    newrp[i + 1] = w;
  }
  free(M->rp);
  M->rp = newrp;
}

/* one-point interpolation and the column merge A P (Sec. 5.1: each F point takes
 * the value of its strongest C connection, P has one identity block per row) */
static void interpolation(Level *L) {
  const Bsr *A = &L->A;
  int E = A->nrows;
  L->ipc = (int *)malloc(sizeof(int) * E);
  for (int i = 0; i < E; ++i) {
    if (L->cf[i] == 1) { L->ipc[i] = L->cidx[i]; continue; }
    int best = -1;
    double bs = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int j = A->ci[p];
      if (!L->strong[p] || L->cf[j] != 1) continue;
      if (best < 0 || L->snorm[p] > bs) { best = j; bs = L->snorm[p]; }
    }
    L->ipc[i] = best < 0 ? -1 : L->cidx[best];
  }
}

/* (A P)_{r,J} = sum over j ascending with ipc(j) = J of A_rj (block adds) */
static void form_ap(int b, Level *L) {
  const Bsr *A = &L->A;
  size_t bb = (size_t)b * b;
  int E = A->nrows, nC = L->nC;
  Bsr *o = &L->AP;
  o->nrows = E;
  o->ncols = nC;
  o->rp = (int *)malloc(sizeof(int) * (E + 1));
  int cap = bsr_nnzb(A) ? bsr_nnzb(A) : 1;
  o->ci = (int *)malloc(sizeof(int) * cap);
  o->v = (double *)malloc(sizeof(double) * bb * cap);
  double *acc = (double *)malloc(sizeof(double) * bb * (nC ? nC : 1));
  char *flag = (char *)calloc(nC ? nC : 1, 1);
  int *touched = (int *)malloc(sizeof(int) * (nC ? nC : 1));
  int nnz = 0;
  o->rp[0] = 0;
  for (int r = 0; r < E; ++r) {
    int nt = 0;
    for (int p = A->rp[r]; p < A->rp[r + 1]; ++p) {
      int J = L->ipc[A->ci[p]];
      if (J < 0) continue;
      const double *a = A->v + (size_t)p * bb;
      double *c = acc + (size_t)J * bb;
      if (!flag[J]) {
        flag[J] = 1;
        touched[nt++] = J;
        memcpy(c, a, sizeof(double) * bb);
      } else {
        for (size_t k = 0; k < bb; ++k) c[k] = c[k] + a[k];
      }
    }
    qsort(touched, nt, sizeof(int), cmp_int);
    for (int k = 0; k < nt; ++k) {
      int J = touched[k];
      o->ci[nnz] = J;
      memcpy(o->v + (size_t)nnz * bb, acc + (size_t)J * bb, sizeof(double) * bb);
      flag[J] = 0;
      ++nnz;
    }
    o->rp[r + 1] = nnz;
  }
  free(acc);
  free(flag);
  free(touched);
}

/* dense LU with partial pivoting (first maximal pivot) for the coarsest level */
static int dense_lu(int n, double *a, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[(size_t)k * n + k]);
    for (int r = k + 1; r < n; ++r)
      if (fabs(a[(size_t)r * n + k]) > best) { best = fabs(a[(size_t)r * n + k]); p = r; }
    piv[k] = p;
    if (best == 0.0) return ORC_ERR_SINGULAR_BLOCK;
    if (p != k)
      for (int c = 0; c < n; ++c) {
        double t = a[(size_t)k * n + c];
        a[(size_t)k * n + c] = a[(size_t)p * n + c];
        a[(size_t)p * n + c] = t;
      }
    for (int r = k + 1; r < n; ++r) {
      double l = a[(size_t)r * n + k] / a[(size_t)k * n + k];
      a[(size_t)r * n + k] = l;
      for (int c = k + 1; c < n; ++c) a[(size_t)r * n + c] -= l * a[(size_t)k * n + c];
    }
  }
  return ORC_OK;
}

static void dense_lu_solve(int n, const double *a, const int *piv, double *x) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int r = 0; r < n; ++r) {
    double s = x[r];
    for (int c = 0; c < r; ++c) s -= a[(size_t)r * n + c] * x[c];
    x[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = x[r];
    for (int c = r + 1; c < n; ++c) s -= a[(size_t)r * n + c] * x[c];
    x[r] = s / a[(size_t)r * n + r];
  }
}

static void level_free(Level *L) {
  bsr_free(&L->A);
  bsr_free(&L->L);
  bsr_free(&L->Delta);
  bsr_free(&L->Rcf);
  bsr_free(&L->AP);
  free(L->Dinv); free(L->snorm); free(L->strong); free(L->lam); free(L->cf);
  free(L->cidx); free(L->fidx); free(L->c2f); free(L->f2f); free(L->ipc);
  free(L->lu); free(L->piv);
  memset(L, 0, sizeof(*L));
}

void orc_free(void *h) {
  Hier *H = (Hier *)h;
  if (!H) return;
  for (int l = 0; l < H->nlev; ++l) level_free(&H->lev[l]);
  bsr_free(&H->Ao);
  free(H->Do);
  free(H);
}

/* build level l + 1 from level l: splitting, Delta, R, P and K = R A P */
static int coarsen(Hier *H, int l, double theta2, double tol2, int targets, int k, uint64_t seed,
                   int *stop) {
  int b = H->b;
  size_t bb = (size_t)b * b;
  Level *L = &H->lev[l];
  const Bsr *A = &L->A;
  int E = A->nrows;
  strength(L, b, theta2);
  cf_split(L, seed);
  L->cidx = (int *)malloc(sizeof(int) * E);
  L->fidx = (int *)malloc(sizeof(int) * E);
  int nC = 0, nF = 0;
  for (int i = 0; i < E; ++i) {
    if (L->cf[i] == 1) { L->cidx[i] = nC++; L->fidx[i] = -1; }
    else { L->fidx[i] = nF++; L->cidx[i] = -1; }
  }
  L->nC = nC;
  L->nF = nF;
  if (nC == 0 || (long long)nC * 10 > (long long)E * 9) { *stop = 1; return ORC_OK; }
  L->c2f = (int *)malloc(sizeof(int) * (nC ? nC : 1));
  L->f2f = (int *)malloc(sizeof(int) * (nF ? nF : 1));
  for (int i = 0; i < E; ++i) {
    if (L->cf[i] == 1) L->c2f[L->cidx[i]] = i;
    else L->f2f[L->fidx[i]] = i;
  }
  /* L = -D_ff^{-1} A_ff restricted to strong F-F off-diagonal blocks */
  {
    Bsr *M = &L->L;
    M->nrows = nF; M->ncols = nF;
    M->rp = (int *)malloc(sizeof(int) * (nF + 1));
    int cnt = 0;
    M->rp[0] = 0;
    for (int f = 0; f < nF; ++f) {
      int i = L->f2f[f];
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (L->strong[p] && L->cf[A->ci[p]] == 0) ++cnt;
      M->rp[f + 1] = cnt;
    }
    M->ci = (int *)malloc(sizeof(int) * (cnt ? cnt : 1));
    M->v = (double *)malloc(sizeof(double) * bb * (cnt ? cnt : 1));
    int w = 0;
    for (int f = 0; f < nF; ++f) {
      int i = L->f2f[f];
      const double *d = L->Dinv + (size_t)i * bb;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        int j = A->ci[p];
        if (!(L->strong[p] && L->cf[j] == 0)) continue;
        M->ci[w] = L->fidx[j];
        const double *a = A->v + (size_t)p * bb;
        double *o = M->v + (size_t)w * bb;
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < b; ++c) {
            double s = 0.0;
            for (int t = 0; t < b; ++t) s = fma(d[r * b + t], a[t * b + c], s);
            o[r * b + c] = -s;
          }
        ++w;
      }
    }
  }
  /* Horner: T_0 = D^{-1}, T_{t+1} = D^{-1} + L T_t, Delta = T_k (Eq. neumann) */
  Bsr Dg;
  Dg.nrows = nF; Dg.ncols = nF;
  Dg.rp = (int *)malloc(sizeof(int) * (nF + 1));
  Dg.ci = (int *)malloc(sizeof(int) * (nF ? nF : 1));
  Dg.v = (double *)malloc(sizeof(double) * bb * (nF ? nF : 1));
  for (int f = 0; f < nF; ++f) {
    Dg.rp[f] = f;
    Dg.ci[f] = f;
    memcpy(Dg.v + (size_t)f * bb, L->Dinv + (size_t)L->f2f[f] * bb, sizeof(double) * bb);
  }
  Dg.rp[nF] = nF;
  Bsr T;
  T.nrows = nF; T.ncols = nF;
  T.rp = (int *)malloc(sizeof(int) * (nF + 1));
  T.ci = (int *)malloc(sizeof(int) * (nF ? nF : 1));
  T.v = (double *)malloc(sizeof(double) * bb * (nF ? nF : 1));
  memcpy(T.rp, Dg.rp, sizeof(int) * (nF + 1));
  memcpy(T.ci, Dg.ci, sizeof(int) * (nF ? nF : 1));
  memcpy(T.v, Dg.v, sizeof(double) * bb * (nF ? nF : 1));
  for (int t = 0; t < k; ++t) {
    Bsr Tn;
    spgemm(b, nF, nF, &L->L, NULL, &T, &Dg, NULL, 0, &Tn);
    if (targets & 1) filter_bsr(b, &Tn, tol2);
    bsr_free(&T);
    T = Tn;
  }
  L->Delta = T;
  bsr_free(&Dg);
  /* R_cf = -A_cf Delta over all A_cf blocks */
  {
    Bsr Acf;
    Acf.nrows = nC; Acf.ncols = nF;
    Acf.rp = (int *)malloc(sizeof(int) * (nC + 1));
    int cnt = 0;
    Acf.rp[0] = 0;
    for (int c = 0; c < nC; ++c) {
      int i = L->c2f[c];
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (L->cf[A->ci[p]] == 0) ++cnt;
      Acf.rp[c + 1] = cnt;
    }
    Acf.ci = (int *)malloc(sizeof(int) * (cnt ? cnt : 1));
    Acf.v = (double *)malloc(sizeof(double) * bb * (cnt ? cnt : 1));
    int w = 0;
    for (int c = 0; c < nC; ++c) {
      int i = L->c2f[c];
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        int j = A->ci[p];
        if (L->cf[j] != 0) continue;
        Acf.ci[w] = L->fidx[j];
        memcpy(Acf.v + (size_t)w * bb, A->v + (size_t)p * bb, sizeof(double) * bb);
        ++w;
      }
    }
    spgemm(b, nC, nF, &Acf, NULL, &L->Delta, NULL, NULL, 1, &L->Rcf);
    bsr_free(&Acf);
  }
  interpolation(L);
  form_ap(b, L);
  /* K = (AP)_C + R_cf (AP)_F, then filtering */
  Level *Nx = &H->lev[l + 1];
  memset(Nx, 0, sizeof(*Nx));
  spgemm(b, nC, nC, &L->Rcf, L->f2f, &L->AP, &L->AP, L->c2f, 0, &Nx->A);
  if (targets & 2) filter_bsr(b, &Nx->A, tol2);
  Nx->E = nC;
  *stop = 0;
  return ORC_OK;
}

static int level_dinv(Hier *H, Level *L) {
  int b = H->b;
  size_t bb = (size_t)b * b;
  int E = L->A.nrows;
  L->E = E;
  L->Dinv = (double *)malloc(sizeof(double) * bb * (E ? E : 1));
  for (int i = 0; i < E; ++i) {
    int dp = -1;
    for (int p = L->A.rp[i]; p < L->A.rp[i + 1]; ++p)
      if (L->A.ci[p] == i) dp = p;
    if (dp < 0) return ORC_ERR_INVALID_ARG;
    int st = gj_inverse(b, L->A.v + (size_t)dp * bb, L->Dinv + (size_t)i * bb);
    if (st) return st;
  }
  return ORC_OK;
}

static int make_coarsest(Hier *H, Level *L, int max_dense) {
  int b = H->b;
  size_t bb = (size_t)b * b;
  int n = L->A.nrows * b;
  if (n > max_dense) return ORC_ERR_INVALID_ARG;
  L->coarsest = 1;
  L->n = n;
  L->lu = (double *)calloc(n > 0 ? (size_t)n * (size_t)n : 1, sizeof(double));
  L->piv = (int *)malloc(sizeof(int) * (n ? n : 1));
  for (int i = 0; i < L->A.nrows; ++i)
    for (int p = L->A.rp[i]; p < L->A.rp[i + 1]; ++p) {
      int j = L->A.ci[p];
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c)
          L->lu[(size_t)(i * b + r) * n + j * b + c] = L->A.v[(size_t)p * bb + r * b + c];
    }
  return dense_lu(n, L->lu, L->piv);
}

/* Setup (Sec. 5): repeated coarsening until the level is small enough. */
void *orc_setup(int E, int b, const int *rp, const int *ci, const double *v, double theta,
                double filter_tol, int filter_targets, int neumann_degree, int max_levels,
                int max_coarse, int max_dense, unsigned long long seed, int *status) {
  *status = ORC_OK;
  if (E <= 0 || b <= 0 || b > 32 || neumann_degree < 0 || max_levels < 1) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  Hier *H = (Hier *)calloc(1, sizeof(Hier));
  H->b = b;
  size_t bb = (size_t)b * b;
  Level *L0 = &H->lev[0];
  int nnzb = rp[E];
  L0->A.nrows = E; L0->A.ncols = E;
  L0->A.rp = (int *)malloc(sizeof(int) * (E + 1));
  L0->A.ci = (int *)malloc(sizeof(int) * (nnzb ? nnzb : 1));
  L0->A.v = (double *)malloc(sizeof(double) * bb * (nnzb ? nnzb : 1));
  memcpy(L0->A.rp, rp, sizeof(int) * (E + 1));
  memcpy(L0->A.ci, ci, sizeof(int) * nnzb);
  memcpy(L0->A.v, v, sizeof(double) * bb * nnzb);
  double theta2 = theta * theta, tol2 = filter_tol * filter_tol;
  H->nlev = 1;
  for (int l = 0;; ++l) {
    Level *L = &H->lev[l];
    int st = level_dinv(H, L);
    if (st) { *status = st; orc_free(H); return NULL; }
    int stop = (l == max_levels - 1) || (L->A.nrows <= max_coarse) || (l == MAXLEV - 1);
    if (!stop) {
      st = coarsen(H, l, theta2, tol2, filter_targets, neumann_degree, seed, &stop);
      if (st) { *status = st; orc_free(H); return NULL; }
    }
    if (stop) {
      st = make_coarsest(H, L, max_dense);
      if (st) { *status = st; orc_free(H); return NULL; }
      break;
    }
    H->nlev = l + 2;
  }
  return H;
}

/* ---------------------------------------------------------------------------
 * Scalar nAIR (Sec. 5.2: the default form): scale A by its block-diagonal
 * inverse, so that every diagonal block becomes the identity, and coarsen the
 * scaled matrix degree of freedom by degree of freedom (block size 1, with the
 * same strength, splitting, Neumann, interpolation and filtering rules).  The
 * diagonal blocks are set to I exactly; an off-diagonal block D_ii^{-1} A_ij is
 * a block product in the canonical order; exact zeros are not stored.  The
 * Krylov solve keeps A, preconditioned by the scalar cycle applied to D^{-1} v.
 * ------------------------------------------------------------------------- */
void *orc_setup_scalar(int E, int b, const int *rp, const int *ci, const double *v, double theta,
                       double filter_tol, int filter_targets, int neumann_degree, int max_levels,
                       int max_coarse, int max_dense, unsigned long long seed, int *status) {
  *status = ORC_OK;
  if (E <= 0 || b <= 0 || b > 32) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  size_t bb = (size_t)b * b;
  int nnzb = rp[E];
  double *D = (double *)malloc(sizeof(double) * bb * E);
  for (int i = 0; i < E; ++i) {
    int dp = -1;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) dp = p;
    int st = dp < 0 ? ORC_ERR_INVALID_ARG : gj_inverse(b, v + (size_t)dp * bb, D + (size_t)i * bb);
    if (st) { free(D); *status = st; return NULL; }
  }
  /* scaled scalar rows: (i, r) -> the identity entry and the nonzeros of row r
   * of D_ii^{-1} A_ij, j != i, in ascending column order */
  int n = E * b;
  int *srp = (int *)malloc(sizeof(int) * (n + 1));
  int *sci = (int *)malloc(sizeof(int) * ((size_t)nnzb * bb + n + 1));
  double *sv = (double *)malloc(sizeof(double) * ((size_t)nnzb * bb + n + 1));
  double *blk = (double *)malloc(sizeof(double) * bb);
  int w = 0;
  srp[0] = 0;
  for (int i = 0; i < E; ++i) {
    const double *Di = D + (size_t)i * bb;
    for (int r = 0; r < b; ++r) {
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int j = ci[p];
        if (j == i) {
          sci[w] = i * b + r;
          sv[w++] = 1.0;
          continue;
        }
        const double *a = v + (size_t)p * bb;
        for (int c = 0; c < b; ++c) {
          double acc = 0.0;
          for (int t = 0; t < b; ++t) acc = fma(Di[r * b + t], a[t * b + c], acc);
          blk[c] = acc;
        }
        for (int c = 0; c < b; ++c)
          if (blk[c] != 0.0) {
            sci[w] = j * b + c;
            sv[w++] = blk[c];
          }
      }
      srp[i * b + r + 1] = w;
    }
  }
  free(blk);
  Hier *H = (Hier *)orc_setup(n, 1, srp, sci, sv, theta, filter_tol, filter_targets, neumann_degree,
                              max_levels, max_coarse, max_dense, seed, status);
  free(srp);
  free(sci);
  free(sv);
  if (!H) { free(D); return NULL; }
  H->scalar = 1;
  H->bo = b;
  H->Do = D;
  H->Ao.nrows = H->Ao.ncols = E;
  H->Ao.rp = (int *)malloc(sizeof(int) * (E + 1));
  H->Ao.ci = (int *)malloc(sizeof(int) * (nnzb ? nnzb : 1));
  H->Ao.v = (double *)malloc(sizeof(double) * bb * (nnzb ? nnzb : 1));
  memcpy(H->Ao.rp, rp, sizeof(int) * (E + 1));
  memcpy(H->Ao.ci, ci, sizeof(int) * nnzb);
  memcpy(H->Ao.v, v, sizeof(double) * bb * nnzb);
  return H;
}

/* y_i = D_i^{-1} x_i, or (D_i^{-1})^T x_i when transposed, for E blocks of size b */
static void block_diag_apply(int E, int b, const double *D, const double *x, double *y, int transposed) {
  size_t bb = (size_t)b * b;
  for (int i = 0; i < E; ++i)
    for (int r = 0; r < b; ++r) {
      double s = 0.0;
      for (int c = 0; c < b; ++c)
        s += (transposed ? D[(size_t)i * bb + c * b + r] : D[(size_t)i * bb + r * b + c]) * x[(size_t)i * b + c];
      y[(size_t)i * b + r] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Solve phase
 * ------------------------------------------------------------------------- */
static void spmv(int b, const Bsr *A, const double *x, double *y) {
  size_t bb = (size_t)b * b;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A->nrows; ++i)
    for (int r = 0; r < b; ++r) {
      double s = 0.0;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        const double *a = A->v + (size_t)p * bb + r * b;
        const double *xj = x + (size_t)A->ci[p] * b;
        for (int c = 0; c < b; ++c) s += a[c] * xj[c];
      }
      y[(size_t)i * b + r] = s;
    }
}

/* one block-Jacobi sweep on the rows with cf == which (Eq. relax with M the
 * block diagonal D): x_i <- x_i + D_ii^{-1} (f - A x)_i, every row from the
 * sweep's starting x, in its classical form x_i <- D_ii^{-1} (f_i - sum_{j != i}
 * A_ij x_j) (the same map, since D_ii^{-1} A_ii = I) */
static void jacobi(int b, const Level *L, int which, const double *f, double *x, double *tmp) {
  size_t bb = (size_t)b * b;
  const Bsr *A = &L->A;
  memcpy(tmp, x, sizeof(double) * (size_t)A->nrows * b);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A->nrows; ++i) {
    if (L->cf[i] != which) continue;
    double res[32];
    for (int r = 0; r < b; ++r) {
      double s = f[(size_t)i * b + r];
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        if (A->ci[p] == i) continue;
        const double *a = A->v + (size_t)p * bb + r * b;
        const double *xj = tmp + (size_t)A->ci[p] * b;
        for (int c = 0; c < b; ++c) s -= a[c] * xj[c];
      }
      res[r] = s;
    }
    const double *d = L->Dinv + (size_t)i * bb;
    for (int r = 0; r < b; ++r) {
      double s = 0.0;
      for (int c = 0; c < b; ++c) s += d[r * b + c] * res[c];
      x[(size_t)i * b + r] = s;
    }
  }
}

/* One cycle on level l for A_l x = f, with no pre-relaxation (Sec. 5):
 * restrict the residual with R = [R_cf I] (the right-hand side itself when x
 * enters as zero), solve the coarse problem approximately, add P x_c, then
 * f_sweeps F-Jacobi sweeps and c_sweeps C-Jacobi sweeps.  The coarse problem
 * gets one V-cycle from zero (type 0, V-cycle), or one F-cycle from zero
 * followed by one V-cycle from its result (type 1, F-cycle; Sec. 6 scaling
 * study).  The coarsest level is solved exactly. */
static void cycle(const Hier *H, int l, int type, const double *f, double *x, int zero) {
  int b = H->b;
  size_t bb = (size_t)b * b;
  const Level *L = &H->lev[l];
  size_t n = (size_t)L->A.nrows * b;
  if (L->coarsest) {
    memcpy(x, f, sizeof(double) * n);
    dense_lu_solve(L->n, L->lu, L->piv, x);
    return;
  }
  int nC = L->nC;
  double *fc = (double *)malloc(sizeof(double) * (size_t)nC * b + 8);
  double *xc = (double *)calloc((size_t)nC * b + 8, sizeof(double));
  double *tmp = (double *)malloc(sizeof(double) * n + 8);
  double *r = (double *)malloc(sizeof(double) * n + 8);
  if (zero) {
    memcpy(r, f, sizeof(double) * n);
  } else {
    spmv(b, &L->A, x, r);
    for (size_t k = 0; k < n; ++k) r[k] = f[k] - r[k];
  }
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nC; ++c) {
    int i = L->c2f[c];
    for (int rr = 0; rr < b; ++rr) {
      double s = r[(size_t)i * b + rr];
      for (int p = L->Rcf.rp[c]; p < L->Rcf.rp[c + 1]; ++p) {
        const double *rv = L->Rcf.v + (size_t)p * bb + rr * b;
        const double *ff = r + (size_t)L->f2f[L->Rcf.ci[p]] * b;
        for (int t = 0; t < b; ++t) s += rv[t] * ff[t];
      }
      fc[(size_t)c * b + rr] = s;
    }
  }
  cycle(H, l + 1, type, fc, xc, 1);
  if (type == 1) cycle(H, l + 1, 0, fc, xc, 0);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < L->A.nrows; ++i)
    for (int rr = 0; rr < b; ++rr) {
      double v = L->ipc[i] >= 0 ? xc[(size_t)L->ipc[i] * b + rr] : 0.0;
      x[(size_t)i * b + rr] = zero ? v : x[(size_t)i * b + rr] + v;
    }
  for (int s = 0; s < H->f_sweeps; ++s) jacobi(b, L, 0, f, x, tmp);
  for (int s = 0; s < H->c_sweeps; ++s) jacobi(b, L, 1, f, x, tmp);
  free(fc);
  free(xc);
  free(tmp);
  free(r);
}

static void precond_apply(const Hier *H, const double *v, double *z);

int orc_vcycle(void *h, const double *f, double *x, int f_sweeps, int c_sweeps) {
  Hier *H = (Hier *)h;
  H->f_sweeps = f_sweeps;
  H->c_sweeps = c_sweeps;
  H->transposed = 0;
  precond_apply(H, f, x);
  return ORC_OK;
}

/* cycle of the preconditioner: 0 = V-cycle, 1 = F-cycle */
int orc_set_cycle(void *h, int type) {
  if (type != 0 && type != 1) return ORC_ERR_INVALID_ARG;
  ((Hier *)h)->cycle_type = type;
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Adjoint preconditioner from the forward hierarchy.  For A^T the transfer
 * operators swap roles (Sec. 2, Corollary on ideal interpolation; Remark on
 * pre-F-relaxation): R^T = [Z^T; I] interpolates, where Z^T = R_cf^T
 * approximates the ideal interpolation -(A^T)_ff^{-1} (A^T)_fc of A^T, and
 * P^T = [W^T I] restricts, with coarse operators K^T.  Relaxation comes
 * before the coarse-grid correction: the C sweeps, then the F sweeps, each a
 * block-Jacobi sweep on A^T whose blocks (D_ii^{-1})^T are the inverses of the
 * diagonal blocks of A^T.  As a linear map this cycle is the transpose of the
 * forward V-cycle (the two error propagators are adjoint to each other).
 * ------------------------------------------------------------------------- */

/* y = A^T x: y_j = sum over blocks (i, j) of A_ij^T x_i */
static void spmv_t(int b, const Bsr *A, const double *x, double *y) {
  size_t bb = (size_t)b * b;
  memset(y, 0, sizeof(double) * (size_t)A->ncols * b);
  for (int i = 0; i < A->nrows; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      const double *a = A->v + (size_t)p * bb;
      double *yj = y + (size_t)A->ci[p] * b;
      const double *xi = x + (size_t)i * b;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) yj[c] += a[r * b + c] * xi[r];
    }
}

/* y = (A - D)^T x: A^T without its diagonal blocks */
static void spmv_t_off(int b, const Bsr *A, const double *x, double *y) {
  size_t bb = (size_t)b * b;
  memset(y, 0, sizeof(double) * (size_t)A->ncols * b);
  for (int i = 0; i < A->nrows; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      if (A->ci[p] == i) continue;
      const double *a = A->v + (size_t)p * bb;
      double *yj = y + (size_t)A->ci[p] * b;
      const double *xi = x + (size_t)i * b;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) yj[c] += a[r * b + c] * xi[r];
    }
}

/* one block-Jacobi sweep on A^T over the rows with cf == which, in the same
 * classical form: x_i <- (D_ii^{-1})^T (f - (A - D)^T x)_i, every row from the
 * sweep's starting x */
static void jacobi_t(int b, const Level *L, int which, const double *f, double *x, double *tmp) {
  size_t bb = (size_t)b * b;
  spmv_t_off(b, &L->A, x, tmp);
  for (int i = 0; i < L->A.nrows; ++i) {
    if (L->cf[i] != which) continue;
    double res[32];
    for (int r = 0; r < b; ++r) res[r] = f[(size_t)i * b + r] - tmp[(size_t)i * b + r];
    const double *d = L->Dinv + (size_t)i * bb;
    double *xi = x + (size_t)i * b;
    for (int r = 0; r < b; ++r) {
      double s = 0.0;
      for (int c = 0; c < b; ++c) s += d[c * b + r] * res[c];
      xi[r] = s;
    }
  }
}

/* x = K^{-T} f from the factors P K = L U of dense_lu: K^T = U^T L^T P, so
 * solve U^T y = f, then L^T z = y, then undo the row interchanges */
static void dense_lu_solve_t(int n, const double *a, const int *piv, double *x) {
  for (int r = 0; r < n; ++r) {
    double s = x[r];
    for (int c = 0; c < r; ++c) s -= a[(size_t)c * n + r] * x[c];
    x[r] = s / a[(size_t)r * n + r];
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = x[r];
    for (int c = r + 1; c < n; ++c) s -= a[(size_t)c * n + r] * x[c];
    x[r] = s;
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
}

/* transposed cycle with zero initial guess: c_sweeps C sweeps and f_sweeps F
 * sweeps on A^T, residual, restriction with P^T (each C point takes its own
 * residual plus those of the F points interpolating from it), recursion on
 * K^T, interpolation with R^T (x_C += x_c, x_F += R_cf^T x_c) */
static void vcycle_t(const Hier *H, int l, const double *f, double *x) {
  int b = H->b;
  size_t bb = (size_t)b * b;
  const Level *L = &H->lev[l];
  size_t n = (size_t)L->A.nrows * b;
  if (L->coarsest) {
    memcpy(x, f, sizeof(double) * n);
    dense_lu_solve_t(L->n, L->lu, L->piv, x);
    return;
  }
  int nC = L->nC;
  double *rc = (double *)calloc((size_t)nC * b + 8, sizeof(double));
  double *xc = (double *)malloc(sizeof(double) * (size_t)nC * b + 8);
  double *tmp = (double *)malloc(sizeof(double) * n + 8);
  memset(x, 0, sizeof(double) * n);
  for (int s = 0; s < H->c_sweeps; ++s) jacobi_t(b, L, 1, f, x, tmp);
  for (int s = 0; s < H->f_sweeps; ++s) jacobi_t(b, L, 0, f, x, tmp);
  spmv_t(b, &L->A, x, tmp);
  for (size_t k = 0; k < n; ++k) tmp[k] = f[k] - tmp[k];
  for (int i = 0; i < L->A.nrows; ++i) {
    int J = L->ipc[i];
    if (J < 0) continue;
    for (int r = 0; r < b; ++r) rc[(size_t)J * b + r] += tmp[(size_t)i * b + r];
  }
  vcycle_t(H, l + 1, rc, xc);
  for (int c = 0; c < nC; ++c) {
    const double *xcc = xc + (size_t)c * b;
    double *xi = x + (size_t)L->c2f[c] * b;
    for (int r = 0; r < b; ++r) xi[r] += xcc[r];
    for (int p = L->Rcf.rp[c]; p < L->Rcf.rp[c + 1]; ++p) {
      const double *rv = L->Rcf.v + (size_t)p * bb;
      double *xf = x + (size_t)L->f2f[L->Rcf.ci[p]] * b;
      for (int r = 0; r < b; ++r)
        for (int t = 0; t < b; ++t) xf[r] += rv[t * b + r] * xcc[t];
    }
  }
  free(rc);
  free(xc);
  free(tmp);
}

int orc_vcycle_t(void *h, const double *f, double *x, int f_sweeps, int c_sweeps) {
  Hier *H = (Hier *)h;
  H->f_sweeps = f_sweeps;
  H->c_sweeps = c_sweeps;
  H->transposed = 1;
  precond_apply(H, f, x);
  H->transposed = 0;
  return ORC_OK;
}

/* the operator and preconditioner of the Krylov solve: A and the V-cycle, or
 * A^T and the transposed cycle */
static void op_apply(const Hier *H, const double *x, double *y) {
  const Bsr *A = H->scalar ? &H->Ao : &H->lev[0].A;
  int b = H->scalar ? H->bo : H->b;
  if (H->transposed) spmv_t(b, A, x, y);
  else spmv(b, A, x, y);
}

/* the preconditioner: the cycle, or its transpose; for scalar nAIR the cycle of
 * D^{-1} A applied to D^{-1} v (transposed: D^{-T} applied after the cycle) */
static void precond_apply(const Hier *H, const double *v, double *z) {
  if (!H->scalar) {
    if (H->transposed) vcycle_t(H, 0, v, z);
    else cycle(H, 0, H->cycle_type, v, z, 1);
    return;
  }
  size_t n = (size_t)H->lev[0].A.nrows;
  double *t = (double *)malloc(sizeof(double) * n + 8);
  int E = (int)(n / H->bo);
  if (H->transposed) {
    vcycle_t(H, 0, v, t);
    block_diag_apply(E, H->bo, H->Do, t, z, 1);
  } else {
    block_diag_apply(E, H->bo, H->Do, v, t, 0);
    cycle(H, 0, H->cycle_type, t, z, 1);
  }
  free(t);
}

static double dot(size_t n, const double *a, const double *b) {
#ifdef _OPENMP
  /* multi-threaded timing build: 64 contiguous chunks, then their sums in order */
  double part[64];
#pragma omp parallel for schedule(static)
  for (int c = 0; c < 64; ++c) {
    size_t lo = n * (size_t)c / 64, hi = n * (size_t)(c + 1) / 64;
    double t = 0.0;
    for (size_t i = lo; i < hi; ++i) t += a[i] * b[i];
    part[c] = t;
  }
  double s = 0.0;
  for (int c = 0; c < 64; ++c) s += part[c];
  return s;
#else
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
#endif
}

/* Flexible GMRES(m), right preconditioned by one V-cycle, classical Gram-Schmidt
 * applied twice, Givens rotations.  hist[j] = Arnoldi residual estimate / ||b||
 * (hist[0] = initial residual).  Stops at hist <= tol; relres is the true
 * residual ||b - A x|| / ||b|| at exit. */
int orc_solve(void *h, const double *bvec, double *x, int f_sweeps, int c_sweeps, int restart,
              int maxiter, double tol, double *hist, int hist_cap, int *hist_len, int *iters,
              double *relres) {
  Hier *H = (Hier *)h;
  H->f_sweeps = f_sweeps;
  H->c_sweeps = c_sweeps;
  int b = H->b;
  size_t n = (size_t)H->lev[0].A.nrows * b;
  int m = restart;
  double *V = (double *)malloc(sizeof(double) * n * (m + 1));
  double *Z = (double *)malloc(sizeof(double) * n * m);
  double *w = (double *)malloc(sizeof(double) * n);
  double *Hm = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)malloc(sizeof(double) * m), *sn = (double *)malloc(sizeof(double) * m);
  double *g = (double *)malloc(sizeof(double) * (m + 1)), *y = (double *)malloc(sizeof(double) * m);
  double *hc = (double *)malloc(sizeof(double) * (m + 1));
  double bnorm = sqrt(dot(n, bvec, bvec));
  int it = 0, nh = 0, status = ORC_ERR_NOT_CONVERGED;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * n);
    *iters = 0; *hist_len = 0; *relres = 0.0;
    status = ORC_OK;
    goto done;
  }
  for (;;) {
    op_apply(H, x, w);
    for (size_t i = 0; i < n; ++i) w[i] = bvec[i] - w[i];
    double beta = sqrt(dot(n, w, w));
    if (nh == 0 && nh < hist_cap) hist[nh++] = beta / bnorm;
    if (beta / bnorm <= tol) { status = ORC_OK; break; }
    if (it >= maxiter) break;
    for (size_t i = 0; i < n; ++i) V[i] = w[i] / beta;
    memset(g, 0, sizeof(double) * (m + 1));
    g[0] = beta;
    int j, conv = 0, brk = 0;
    for (j = 0; j < m && it < maxiter; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      precond_apply(H, vj, zj);
      ++it;
      op_apply(H, zj, w);
      for (int k = 0; k <= j; ++k) hc[k] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int k = 0; k <= j; ++k) {
          double hk = dot(n, V + (size_t)k * n, w);
          Hm[(size_t)k * m + j] += hk;
          hc[k] = hk;
        }
        for (int k = 0; k <= j; ++k) {
          const double *vk = V + (size_t)k * n;
#pragma omp parallel for schedule(static)
          for (size_t i = 0; i < n; ++i) w[i] -= hc[k] * vk[i];
        }
      }
      double hn = sqrt(dot(n, w, w));
      Hm[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0) {
        double *vn = V + (size_t)(j + 1) * n;
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) vn[i] = w[i] / hn;
      }
      for (int k = 0; k < j; ++k) {
        double a = Hm[(size_t)k * m + j], c = Hm[(size_t)(k + 1) * m + j];
        Hm[(size_t)k * m + j] = cs[k] * a + sn[k] * c;
        Hm[(size_t)(k + 1) * m + j] = -sn[k] * a + cs[k] * c;
      }
      double a = Hm[(size_t)j * m + j], c = Hm[(size_t)(j + 1) * m + j];
      double r = hypot(a, c);
      cs[j] = a / r;
      sn[j] = c / r;
      Hm[(size_t)j * m + j] = r;
      Hm[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      double est = fabs(g[j + 1]) / bnorm;
      if (nh < hist_cap) hist[nh++] = est;
      if (est <= tol) { conv = 1; ++j; break; }
      if (hn == 0.0) { brk = 1; ++j; break; }
    }
    /* y = H^{-1} g on the j x j upper triangle; x += Z y */
    for (int r = j - 1; r >= 0; --r) {
      double s = g[r];
      for (int c = r + 1; c < j; ++c) s -= Hm[(size_t)r * m + c] * y[c];
      y[r] = s / Hm[(size_t)r * m + r];
    }
    for (int k = 0; k < j; ++k) {
      const double *zk = Z + (size_t)k * n;
#pragma omp parallel for schedule(static)
      for (size_t i = 0; i < n; ++i) x[i] += y[k] * zk[i];
    }
    memset(Hm, 0, sizeof(double) * (size_t)(m + 1) * m);
    if (conv || brk) { status = ORC_OK; break; }
    if (it >= maxiter) break;
  }
  op_apply(H, x, w);
  for (size_t i = 0; i < n; ++i) w[i] = bvec[i] - w[i];
  *relres = sqrt(dot(n, w, w)) / bnorm;
  *iters = it;
  *hist_len = nh;
  if (status == ORC_OK && *relres > 10.0 * tol && tol > 0) status = ORC_ERR_NOT_CONVERGED;
done:
  free(V); free(Z); free(w); free(Hm); free(cs); free(sn); free(g); free(y); free(hc);
  return status;
}

/* Solve A^T lambda = w with the same flexible GMRES, preconditioned by the
 * transposed cycle of the forward hierarchy (no second setup). */
int orc_solve_t(void *h, const double *w, double *lam, int f_sweeps, int c_sweeps, int restart,
                int maxiter, double tol, double *hist, int hist_cap, int *hist_len, int *iters,
                double *relres) {
  Hier *H = (Hier *)h;
  H->transposed = 1;
  int st = orc_solve(h, w, lam, f_sweeps, c_sweeps, restart, maxiter, tol, hist, hist_cap, hist_len,
                     iters, relres);
  H->transposed = 0;
  return st;
}

/* ---------------------------------------------------------------------------
 * Hierarchy export for the comparisons
 * ------------------------------------------------------------------------- */
int orc_num_levels(void *h) { return ((Hier *)h)->nlev; }

/* sizes: E, nnzb(A), nC, nF, nnzb(L), nnzb(Delta), nnzb(Rcf), nnzb(AP), coarsest */
void orc_level_sizes(void *h, int l, long long *out) {
  Level *L = &((Hier *)h)->lev[l];
  out[0] = L->A.nrows;
  out[1] = bsr_nnzb(&L->A);
  out[2] = L->nC;
  out[3] = L->nF;
  out[4] = bsr_nnzb(&L->L);
  out[5] = bsr_nnzb(&L->Delta);
  out[6] = bsr_nnzb(&L->Rcf);
  out[7] = bsr_nnzb(&L->AP);
  out[8] = L->coarsest;
}

static void *copy_or_null(void *dst, const void *src, size_t bytes) {
  if (src && bytes) memcpy(dst, src, bytes);
  return dst;
}

/* which: 0 A.rp 1 A.ci 2 A.v 3 Dinv 4 cf 5 ipc 6 Delta.rp 7 Delta.ci 8 Delta.v
 *        9 Rcf.rp 10 Rcf.ci 11 Rcf.v 12 strong 13 lam 14 L.rp 15 L.ci 16 L.v */
int orc_level_get(void *h, int l, int which, void *out) {
  Hier *H = (Hier *)h;
  Level *L = &H->lev[l];
  size_t bb = (size_t)H->b * H->b;
  int E = L->A.nrows;
  switch (which) {
    case 0: copy_or_null(out, L->A.rp, sizeof(int) * (E + 1)); break;
    case 1: copy_or_null(out, L->A.ci, sizeof(int) * bsr_nnzb(&L->A)); break;
    case 2: copy_or_null(out, L->A.v, sizeof(double) * bb * bsr_nnzb(&L->A)); break;
    case 3: copy_or_null(out, L->Dinv, sizeof(double) * bb * E); break;
    case 4: copy_or_null(out, L->cf, (size_t)E); break;
    case 5: copy_or_null(out, L->ipc, sizeof(int) * E); break;
    case 6: copy_or_null(out, L->Delta.rp, sizeof(int) * (L->nF + 1)); break;
    case 7: copy_or_null(out, L->Delta.ci, sizeof(int) * bsr_nnzb(&L->Delta)); break;
    case 8: copy_or_null(out, L->Delta.v, sizeof(double) * bb * bsr_nnzb(&L->Delta)); break;
    case 9: copy_or_null(out, L->Rcf.rp, sizeof(int) * (L->nC + 1)); break;
    case 10: copy_or_null(out, L->Rcf.ci, sizeof(int) * bsr_nnzb(&L->Rcf)); break;
    case 11: copy_or_null(out, L->Rcf.v, sizeof(double) * bb * bsr_nnzb(&L->Rcf)); break;
    case 12: copy_or_null(out, L->strong, (size_t)bsr_nnzb(&L->A)); break;
    case 13: copy_or_null(out, L->lam, sizeof(int) * E); break;
    case 14: copy_or_null(out, L->L.rp, sizeof(int) * (L->nF + 1)); break;
    case 15: copy_or_null(out, L->L.ci, sizeof(int) * bsr_nnzb(&L->L)); break;
    case 16: copy_or_null(out, L->L.v, sizeof(double) * bb * bsr_nnzb(&L->L)); break;
    default: return ORC_ERR_INVALID_ARG;
  }
  return ORC_OK;
}

/* block inverse exported for the pins */
int orc_block_inverse(int b, const double *A, double *X) { return gj_inverse(b, A, X); }

/* a8 alone, exported for the pins: the filter of Sec. 5.2 (block form) applied
 * in place to a square block-CSR matrix (nrows block rows, b x b blocks) with
 * tolerance tol.  rp, ci and v are overwritten with the kept blocks, in their
 * original order; returns the new number of blocks. */
int orc_filter(int nrows, int b, int *rp, int *ci, double *v, double tol) {
  size_t bb = (size_t)b * b;
  int nnzb = rp[nrows];
  Bsr M;
  M.nrows = nrows;
  M.ncols = nrows;
  M.rp = (int *)malloc(sizeof(int) * (nrows + 1));
  M.ci = (int *)malloc(sizeof(int) * (nnzb ? nnzb : 1));
  M.v = (double *)malloc(sizeof(double) * bb * (nnzb ? nnzb : 1));
  memcpy(M.rp, rp, sizeof(int) * (nrows + 1));
  memcpy(M.ci, ci, sizeof(int) * nnzb);
  memcpy(M.v, v, sizeof(double) * bb * nnzb);
  filter_bsr(b, &M, tol * tol);
  int kept = M.rp[nrows];
  memcpy(rp, M.rp, sizeof(int) * (nrows + 1));
  memcpy(ci, M.ci, sizeof(int) * kept);
  memcpy(v, M.v, sizeof(double) * bb * kept);
  bsr_free(&M);
  return kept;
}

/* ---------------------------------------------------------------------------
 * Adjoint helpers: block transpose of A, and the gradients of J = w . x with
 * respect to the element absorption and the nodal source when A(sigma) has
 * diagonal blocks A0_ee + sigma_e M_e and the right-hand side is M q:
 *   dJ/dsigma_e = -lambda_e^T M_e x_e,  dJ/dq_e = M_e^T lambda_e,  A^T lambda = w.
 * ------------------------------------------------------------------------- */
void orc_transpose(int E, int b, const int *rp, const int *ci, const double *v, int *trp, int *tci,
                   double *tv) {
  size_t bb = (size_t)b * b;
  int nnzb = rp[E];
  for (int i = 0; i <= E; ++i) trp[i] = 0;
  for (int p = 0; p < nnzb; ++p) trp[ci[p] + 1]++;
  for (int i = 0; i < E; ++i) trp[i + 1] += trp[i];
  int *fill = (int *)malloc(sizeof(int) * (E ? E : 1));
  for (int i = 0; i < E; ++i) fill[i] = trp[i];
  for (int i = 0; i < E; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      int w = fill[j]++;
      tci[w] = i;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) tv[(size_t)w * bb + c * b + r] = v[(size_t)p * bb + r * b + c];
    }
  free(fill);
}

void orc_gradients(int E, int b, const double *M, const double *lam, const double *x, double *gsig,
                   double *gq) {
  size_t bb = (size_t)b * b;
  for (int e = 0; e < E; ++e) {
    const double *Me = M + (size_t)e * bb;
    const double *le = lam + (size_t)e * b, *xe = x + (size_t)e * b;
    double s = 0.0;
    for (int r = 0; r < b; ++r) {
      double mx = 0.0;
      for (int c = 0; c < b; ++c) mx += Me[r * b + c] * xe[c];
      s += le[r] * mx;
    }
    gsig[e] = -s;
    for (int c = 0; c < b; ++c) {
      double t = 0.0;
      for (int r = 0; r < b; ++r) t += Me[r * b + c] * le[r];
      gq[(size_t)e * b + c] = t;
    }
  }
}
