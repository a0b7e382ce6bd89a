// Hierarchy data of the nAIR GPU library and the host-side entry points of
// the setup and solve phases.
#pragma once

#include "common.cuh"

namespace nair {

// block-CSR matrix in device memory; values of type T, b x b row-major blocks
template <typename T>
struct DBsr {
  int nrows = 0, ncols = 0, nnzb = 0;
  int *rp = nullptr, *ci = nullptr;
  T *v = nullptr;
};

// most F sweeps per cycle with their own row lists
static constexpr int kMaxFLists = 8;

// scalar-row form of a level's off-diagonal blocks for its sweeps:
// scalar row (i, r) lists, in ascending block order, the off-diagonal blocks
// p of row i whose row r has a nonzero (offsets srp[i b + r], block indices
// sp).  The entries are also packed for the sweeps: sj[e] is entry e's block
// column and sv[e b .. e b + b) row r of its block (values of the level's
// type), so a sweep streams its values and loads one index per entry.
// perm_f[k] (for F sweep k's rows, fsweep when k = 0) and perm_c (csweep)
// order the scalar rows of each thread block of *_tpc rows by entry count
struct SweepRows {
  int *srp = nullptr, *sp = nullptr, *sj = nullptr;
  int ne = 0;  // packed entries
  void *sv = nullptr;
  int *srs = nullptr;  // per scalar row of an F row: where its F-column entries start (C columns first)
  // with the F sweeps in the scaled variable y_F = D_FF x_F: the entries with an
  // F column scaled from the right, row r of A_ij D_jj^{-1}; the others as in sv
  void *sv2 = nullptr;
  unsigned char *perm_f[kMaxFLists] = {}, *perm_c = nullptr;
  int perm_f_tpc[kMaxFLists] = {}, perm_c_tpc = 0;
};

// One level of the hierarchy (Sec. 5).  Index spaces: elements 0..E-1 of the
// level; F elements numbered 0..nF-1 and C elements 0..nC-1 in ascending
// element order (the C numbering is the next level's element numbering).
template <typename T>
struct Level {
  int E = 0, nC = 0, nF = 0, coarsest = 0, cf_rounds = 0;
  DBsr<T> A;               // level operator
  int *diag = nullptr;     // position of the diagonal block of each row
  T *dinv = nullptr;       // E inverse diagonal blocks (computed in FP64)
  signed char *cf = nullptr;  // 1 = C, 0 = F
  int *c2f = nullptr;      // coarse index -> element (the C rows, ascending)
  int *f2f = nullptr;      // F index -> element (the F rows, ascending)
  int *fsweep = nullptr, *csweep = nullptr;  // F / C rows ordered by row length (sweep work lists)
  // F sweeps after the first in a cycle from a zero iterate.  The C values do
  // not change during the F sweeps, so an F row whose off-diagonal F couplings
  // all lead to rows that kept their value in sweep k - 1 would recompute its
  // previous value from the same inputs: sweep k updates only the rows of
  // fl[k] (F rows with an F coupling to a row of fl[k - 1]; fl[0] = fsweep),
  // in the order of fsweep.  fq[k] (k >= 1) holds the rows of fl[k - 1] that
  // are not in fl[k].  Built for nfl = f_sweeps sweeps (0: not built).
  int nfl = 0;
  int *fl[kMaxFLists] = {}, *fq[kMaxFLists] = {};
  int fl_n[kMaxFLists] = {}, fq_n[kMaxFLists] = {};
  SweepRows sr;  // levels >= 1, FP64
  int *ipc = nullptr;      // element -> coarse column of P (C: itself, F: one-point source) or -1
  DBsr<T> R;               // R_cf, nC rows, columns = element indices (solve form)
  SweepRows rr;            // scalar-row form of R_cf for the restriction (FP64; perm_c: all rows)
  int *R_ci_f = nullptr;   // R_cf columns as F indices (export form)
  // kept only with keep_setup_data
  unsigned char *strong = nullptr;
  int *lam = nullptr;
  DBsr<T> L, Delta;
  // coarsest level: dense inverse
  int n = 0;
  T *ainv = nullptr;
  // cycle vectors: right-hand side, iterate, second sweep buffer, residual;
  // level 0 with scaled couplings also g = D^{-1} f; levels >= 1 in the
  // scalar-row form also h = f_F - A_FC x_C for the F sweeps of a cycle
  T *f = nullptr, *x = nullptr, *x2 = nullptr, *r = nullptr, *g = nullptr, *h = nullptr;
  // F sweeps in y_F = D_FF x_F (sr.sv2 built): the F sweeps of a cycle apply no
  // D^{-1}; the C sweep reads y_F through sr.sv2 and converts x_F = D^{-1} y_F
  int ymode = 0;
};

// Level-0 off-diagonal blocks restricted to their nonzero columns.  An upwind
// DG coupling block is nonzero only in the columns of the p + 1 face nodes of
// the neighbour, so each off-diagonal block keeps W <= b columns (the largest
// count over all blocks, padded with zero columns): off block q of row i is
// q = p - i - (p > diag(i)) for its BSR position p.
template <typename T>
struct L0Comp {
  int W = 0;                         // 0: not built (kernels use the BSR blocks)
  int *oci = nullptr;                // block column of each off-diagonal block
  unsigned long long *ocols = nullptr;  // W local column indices, 8 bits each
  T *ov = nullptr;                   // (nnzb - E) x b x W values
  T *sv = nullptr;                   // the same blocks scaled, D_ii^{-1} A_ij (forward sweeps)
};

template <typename T>
void build_l0comp(const DBsr<T> &A, const int *diag, int b, cudaStream_t s, Mem &mem, L0Comp<T> &C);

// C.sv = D_ii^{-1} A_ij for every compressed off-diagonal block (dinv: E blocks)
template <typename T>
void build_l0scaled(const DBsr<T> &A, const T *dinv, int b, cudaStream_t s, Mem &mem, L0Comp<T> &C);

// The V-cycle replayed as one CUDA graph: it reads its input from and writes its
// output to the two device pointers in dptr (set before each launch), so one
// instantiated graph serves every Krylov vector.
struct VGraph {
  cudaGraphExec_t exec = nullptr;
  void **dptr = nullptr;  // device: [0] input (double*), [1] output (double*)
  long long nodes = 0;    // kernels per replay
};

// device-clock stamps of the block-Jacobi sweeps: slot s holds the earliest
// start and the latest end of the sweep with site index s = level * S + k
struct SweepClock {
  unsigned long long *dev = nullptr;      // [2 * nsites]: starts, then ends
  unsigned long long *slot[2] = {};       // pinned copies of two consecutive cycles
  int nsites = 0, S = 0;
  std::vector<long long> count;        // per (level, class)
  std::vector<double> ms;
  std::vector<long long> site_count;   // per (level, sweep of the cycle)
  std::vector<double> site_ms;
};

// One level of the transposed hierarchy, which preconditions A^T with the
// transpose of the V-cycle: R^T = [R_cf^T; I] interpolates, P^T = [W^T I]
// restricts, and the block-Jacobi sweeps on A_l^T (C sweeps, then F sweeps)
// come before the coarse-grid correction.  Built from a finished level.
template <typename T>
struct TLevel {
  DBsr<T> At;                  // A_l^T (rows sorted by column)
  int *diag = nullptr;         // position of the diagonal block of each row of At
  T *dinvT = nullptr;          // (D_ii^{-1})^T, the inverse diagonal blocks of A_l^T
  int *fsweep = nullptr, *csweep = nullptr;  // F / C rows ordered by At row length
  // F sweeps after the first (they follow the C sweeps, which fix x_C): as
  // Level::fl / fq, for the couplings of A^T; fq[1] lists the F rows the second
  // F sweep copies into its buffer
  int nfl = 0;
  int *fl[kMaxFLists] = {}, *fq[kMaxFLists] = {};
  int fl_n[kMaxFLists] = {}, fq_n[kMaxFLists] = {};
  SweepRows sr;  // levels >= 1, for the rows of A^T
  DBsr<T> Rt;                  // R_cf^T: E rows (blocks on F rows only), nC columns
  int *cself = nullptr;        // element -> its coarse index (C) or -1 (F)
  int *pt_rp = nullptr, *pt_ci = nullptr;  // P^T: coarse J -> F elements with ip = J, ascending
  T *r = nullptr;              // residual after the pre-relaxation
  T *h = nullptr;              // f - (A^T)_FC x_C for the F sweeps (scalar-row levels)
  T *ainvT = nullptr;          // coarsest level: (A_c^{-1})^T
  // F sweeps in y_F = D_FF^T x_F (sr.sv2 built), as Level::ymode; x_F =
  // D_FF^{-T} y_F is formed after the last F sweep
  int ymode = 0;
};

template <typename T>
struct Hier {
  int b = 0, nlev = 0;
  std::vector<Level<T>> lev;
  mutable VGraph graph;
  mutable SweepClock clock;
  L0Comp<T> l0c;
  double setup_ms = 0.0;
  double op_complexity = 0.0, cycle_complexity = 0.0;
  // transposed form (empty until build_transposed)
  std::vector<TLevel<T>> tlev;
  L0Comp<T> tl0c;
  mutable VGraph tgraph;
  // scalar nAIR: the hierarchy is built for D^{-1} A; the preconditioner applies
  // the pre_E blocks of D^{-1} (size pre_b) before the cycle (after the
  // transposed cycle, transposed)
  const T *pre_dinv = nullptr;
  int pre_b = 0, pre_E = 0;
};

struct Params {
  double theta, filter_tol;
  int filter_targets, k, f_sweeps, c_sweeps, max_levels, max_coarse, max_dense;
  uint64_t seed;
  int precision, restart, maxiter;
  double tol;
  int keep, use_graphs, sweep_timing;
  int cycle;   // 0: V-cycle, 1: F-cycle
  int scalar;  // 1: scalar nAIR (hierarchy of D^{-1} A by degree of freedom)
};

Params resolve_params(const nair_params *p, int b);

// setup of the hierarchy for level-0 matrix A0 (device BSR, values T)
template <typename T>
void build_hierarchy(const DBsr<T> &A0, const Params &P, cudaStream_t s, Mem &mem, Hier<T> &H);

// one cycle (P.cycle) with zero initial guess on level 0: x = M^{-1} f (device vectors of T)
template <typename T>
void vcycle(const Hier<T> &H, const Params &P, const T *f, T *x, cudaStream_t s);

// release the V-cycle graph of a hierarchy
void release_graph(VGraph &g);
void release_clock(SweepClock &c);

// transposed cycle with zero initial guess on level 0: x = M^{-T} f
template <typename T>
void vcycle_t(const Hier<T> &H, const Params &P, const T *f, T *x, cudaStream_t s);

// the transposed form of a built hierarchy (adjoint solves without a second setup)
template <typename T>
void build_transposed(Hier<T> &H, int f_sweeps, cudaStream_t s, Mem &mem);

// block transpose of a block-CSR matrix (each block transposed, rows sorted)
template <typename T>
void bsr_transpose(const DBsr<T> &A, int b, DBsr<T> &out, cudaStream_t s, Mem &mem);

// scalar form of a block matrix: D^{-1} A (Dinv: the inverse diagonal blocks,
// diag: their positions) by degree of freedom, identity diagonal, no zeros stored
void scalar_matrix(const DBsr<double> &A, int b, const double *Dinv, const int *diag, DBsr<double> &out,
                   cudaStream_t s, Mem &mem);

// rows of one class ordered by decreasing row length (sweep work list)
int *sweep_list(int n, const int *list, const int *rp, cudaStream_t s, Mem &mem, Mem &tmp);
// thread groups per row the row kernels use for nrows rows of avg blocks
int rowop_groups(long long nrows, int b, double avg);
// row lists of F sweeps 1 .. nf - 1 that update only the F rows whose inputs
// changed (matrix rp / ci, F rows fsweep): rows of sweep k, then for each k the
// rows of sweep k - 1 not in sweep k, 2 (nf - 1) lists of nF slots in the
// returned buffer, their lengths written to cnt on the device; null when the
// level keeps full sweeps.  fsweep_assign sets fl / fq from the read-back lengths.
int *fsweep_lists(int E, int nF, const int *rp, const int *ci, const signed char *cf, const int *fsweep, int nf,
                  int *cnt, cudaStream_t s, Mem &mem, Mem &tmp);
void fsweep_assign(int nF, int nf, int *buf, const int *hcnt, int *fsweep, int **fl, int *fl_n, int **fq,
                   int *fq_n);
// the scalar-row form of R_cf (nC rows, element columns) for the restriction
// (FP64 and the DG block sizes; otherwise rr stays empty)
template <typename T>
void build_restrict_rows(int nC, int b, const DBsr<T> &R, SweepRows &rr, cudaStream_t s, Mem &mem);
// sr.sv2: the packed entries with an F column j (cf[j] == 0) scaled from the
// right by dinv_j (row r of the block times dinv_j), the others copied
template <typename T>
void scale_srow_entries(SweepRows &sr, int b, const T *dinv, const signed char *cf, cudaStream_t s, Mem &mem);
// the scalar-row form of one level's matrix A for its sweep lists (the DG
// block sizes; otherwise sr stays empty and the sweeps use k_rowop)
template <typename T>
void build_sweep_rows_level(int E, int nF, int nC, int b, const DBsr<T> &A, const signed char *cf, int *fsweep,
                            int nfl, int *const *fl, const int *fl_n, int *csweep, SweepRows &sr, cudaStream_t s,
                            Mem &mem);

// position of the diagonal block of every row
void diag_positions(int E, const int *rp, const int *ci, int *out, cudaStream_t s);

// diagonal-block inverses in FP64 of the blocks at positions pos[] (or 0..nblk-1)
template <typename TI>
void block_inverses(int nblk, int b, const TI *A, const int *pos, double *out, int *err_flag,
                    cudaStream_t s);

}  // namespace nair
