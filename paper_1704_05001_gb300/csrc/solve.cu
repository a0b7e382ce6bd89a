// nAIR solve phase on the GPU: the V-cycle (Sec. 5: restriction of the
// right-hand side with R = [R_cf I], recursion, one-point interpolation, then
// block-Jacobi F- and C-relaxation, Eq. relax / Eq. cgc) and flexible GMRES(m)
// with classical Gram-Schmidt applied twice (Sec. 6: GMRES acceleration).
// The Krylov vectors, Arnoldi products and outer residuals are FP64; the
// V-cycle runs in the hierarchy's precision T.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "rowops.cuh"
#include "solve.cuh"

namespace nair {

static constexpr int kThreads = 256;
static inline int grid(long long n) { return std::max(1, cdiv(n, kThreads)); }

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------

// a12: x = P x_c (C: own coarse value, F: one-point source, or 0); used only
// when no relaxation sweep follows (otherwise the first sweep reads P x_c)
template <typename T>
__global__ void k_prolong(int E, int b, const int *__restrict__ ipc, const T *__restrict__ xc,
                          T *__restrict__ x) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)E * b) return;
  const int i = (int)(g / b), r = (int)(g - (long long)i * b);
  const int J = ipc[i];
  x[g] = J >= 0 ? xc[(size_t)J * b + r] : (T)0;
}

// a9: coarsest level, x = A_c^{-1} f (dense), one warp per row
template <typename T>
__global__ void k_dense_mv(int n, const T *__restrict__ M, const T *__restrict__ f, T *__restrict__ x) {
  pdl_launch_dependents();
  pdl_wait();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const T *row = M + (size_t)warp * n;
  T acc = 0;
  for (int c = lane; c < n; c += 32) acc += row[c] * f[c];
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[warp] = acc;
}

// x_i = D_ii^{-1} f_i (trans: (D_ii^{-1})^T f_i) for E blocks: a block-diagonal
// coarsest level, or the scaling of scalar nAIR
template <typename T>
__global__ void k_bdiag_apply(int E, int b, const T *__restrict__ dinv, const T *__restrict__ f,
                              T *__restrict__ x, int trans) {
  pdl_launch_dependents();
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)E * b) return;
  const int i = (int)(g / b), r = (int)(g - (long long)i * b);
  const T *d = dinv + (size_t)i * b * b + (trans ? r : r * b);
  const int step = trans ? b : 1;
  const T *fi = f + (size_t)i * b;
  T acc = 0;
  for (int c = 0; c < b; ++c) acc = fma(d[(size_t)c * step], fi[c], acc);
  x[g] = acc;
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    NAIR_CK(cudaGetDevice(&dev));
    NAIR_CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

// threads per row of the row kernels: enough block groups that each thread
// handles about two blocks of a long (coarse-level) row, keeping the serial
// chain short; on small levels more, until the rows fill about one wave of the
// GPU (those sweeps are bound by each thread's chain of dependent loads, not by
// throughput), up to about one group per block of an average row
int rowop_groups(long long nrows, int b, double avg) {
  int G = 1;
  if (avg > 4.0)
    while (G * 2 <= avg / 2 && G * 2 * b <= 256 && G < 32) G *= 2;
  const long long wave = (long long)sm_count() * 1536;
  while (G < 32 && G * 2 * b <= 256 && G * 2 <= 2 * avg && nrows * b * G * 2 <= wave) G *= 2;
  return G;
}

template <typename T, int OP>
void launch_rowop(RowArgs<T> a, double avg, cudaStream_t s) {
  const int b = a.b;
  const int G = rowop_groups(a.nrows, b, avg);
  a.G = G;
  const int tsz = G * b;
  a.tpc = std::max(1, 256 / tsz);
  const int threads = a.tpc * tsz;
  const size_t smem = ((size_t)a.tpc * tsz + (size_t)a.tpc * b) * sizeof(T);
  a.comp_ctas = cdiv(a.nrows, a.tpc);
  int blocks = a.comp_ctas;
  if (OP == OP_JACOBI && a.ncopy > 0) blocks += cdiv((long long)a.ncopy * b, threads);
  if (blocks == 0) return;
  const dim3 gr(blocks), bl(threads);
  switch (b) {
    case 1: launch_pdl(k_rowop<T, 1, OP>, gr, bl, smem, s, a); break;
    case 3: launch_pdl(k_rowop<T, 3, OP>, gr, bl, smem, s, a); break;
    case 6: launch_pdl(k_rowop<T, 6, OP>, gr, bl, smem, s, a); break;
    case 10: launch_pdl(k_rowop<T, 10, OP>, gr, bl, smem, s, a); break;
    case 15: launch_pdl(k_rowop<T, 15, OP>, gr, bl, smem, s, a); break;
    case 21: launch_pdl(k_rowop<T, 21, OP>, gr, bl, smem, s, a); break;
    case 28: launch_pdl(k_rowop<T, 28, OP>, gr, bl, smem, s, a); break;
    default: launch_pdl(k_rowop<T, 0, OP>, gr, bl, smem, s, a); break;
  }
  NAIR_LAUNCH_CHECK();
}
// the scalar-row kernel for block size b and F-sweep mode FM
template <typename T, int OP, int FM>
static void launch_scalar_rows_b(const RowArgs<T> &a, int b, dim3 gr, dim3 bl, cudaStream_t s) {
  switch (b) {
    case 3: launch_pdl(k_scalar_rows<T, 3, OP, FM>, gr, bl, 0, s, a); break;
    case 6: launch_pdl(k_scalar_rows<T, 6, OP, FM>, gr, bl, 0, s, a); break;
    case 10: launch_pdl(k_scalar_rows<T, 10, OP, FM>, gr, bl, 0, s, a); break;
    case 15: launch_pdl(k_scalar_rows<T, 15, OP, FM>, gr, bl, 0, s, a); break;
    case 21: launch_pdl(k_scalar_rows<T, 21, OP, FM>, gr, bl, 0, s, a); break;
    default: launch_pdl(k_scalar_rows<T, 28, OP, FM>, gr, bl, 0, s, a); break;
  }
}

template <typename T, int OP>
bool launch_scalar_rows(RowArgs<T> a, int G, cudaStream_t s) {
  const int b = a.b;
  a.G = G;
  a.tpc = sweep_rows_tpc(b, G);
  const int threads = a.tpc * b * G;
  a.comp_ctas = cdiv(a.nrows, a.tpc);
  int blocks = a.comp_ctas;
  if (OP == OP_JACOBI && a.ncopy > 0) blocks += cdiv((long long)a.ncopy * b, threads);
  const dim3 gr(blocks), bl(threads);
  if (b != 3 && b != 6 && b != 10 && b != 15 && b != 21 && b != 28) return false;
  if (blocks) {
    if (OP == OP_JACOBI && a.fmode == 1) launch_scalar_rows_b<T, OP_JACOBI, 1>(a, b, gr, bl, s);
    else if (OP == OP_JACOBI && a.fmode == 2) launch_scalar_rows_b<T, OP_JACOBI, 2>(a, b, gr, bl, s);
    else if (OP == OP_JACOBI && a.fmode == 3) launch_scalar_rows_b<T, OP_JACOBI, 3>(a, b, gr, bl, s);
    else if (OP == OP_JACOBI && a.fmode == 4) launch_scalar_rows_b<T, OP_JACOBI, 4>(a, b, gr, bl, s);
    else if (OP == OP_JACOBI && a.fmode == 5) launch_scalar_rows_b<T, OP_JACOBI, 5>(a, b, gr, bl, s);
    else launch_scalar_rows_b<T, OP, 0>(a, b, gr, bl, s);
    NAIR_LAUNCH_CHECK();
  }
  return true;
}
template bool launch_scalar_rows<double, OP_JACOBI>(RowArgs<double>, int, cudaStream_t);
template bool launch_scalar_rows<float, OP_JACOBI>(RowArgs<float>, int, cudaStream_t);
template bool launch_scalar_rows<double, OP_RESTRICT>(RowArgs<double>, int, cudaStream_t);
template bool launch_scalar_rows<float, OP_RESTRICT>(RowArgs<float>, int, cudaStream_t);

template <typename T, int OP>
void launch_rowop_l0(RowArgs<T> a, int W, cudaStream_t s) {
  const int b = a.b;
  a.G = 1;
  a.tpc = std::max(1, 256 / b);
  const int threads = a.tpc * b;
  a.comp_ctas = cdiv(a.nrows, a.tpc);
  int blocks = a.comp_ctas;
  if ((OP == OP_JACOBI || OP == OP_JACOBI_S) && a.ncopy > 0) blocks += cdiv((long long)a.ncopy * b, threads);
  if (blocks == 0) return;
  const dim3 gr(blocks), bl(threads);
  if (b == 3 && W == 2) launch_pdl(k_rowop_l0<T, 3, 2, OP>, gr, bl, 0, s, a);
  else if (b == 6 && W == 3) launch_pdl(k_rowop_l0<T, 6, 3, OP>, gr, bl, 0, s, a);
  else if (b == 10 && W == 4) launch_pdl(k_rowop_l0<T, 10, 4, OP>, gr, bl, 0, s, a);
  else if (b == 15 && W == 5) launch_pdl(k_rowop_l0<T, 15, 5, OP>, gr, bl, 0, s, a);
  else if (b == 21 && W == 6) launch_pdl(k_rowop_l0<T, 21, 6, OP>, gr, bl, 0, s, a);
  else if (b == 28 && W == 7) launch_pdl(k_rowop_l0<T, 28, 7, OP>, gr, bl, 0, s, a);
  else fail(NAIR_ERR_UNSUPPORTED, "no level-0 kernel for this block size and width");
  NAIR_LAUNCH_CHECK();
}

template void launch_rowop<double, OP_SPMV>(RowArgs<double>, double, cudaStream_t);
template void launch_rowop<double, OP_RESID>(RowArgs<double>, double, cudaStream_t);

template <typename T>
static RowArgs<T> row_args(const DBsr<T> &A, int b) {
  RowArgs<T> a{};
  a.nrows = A.nrows;
  a.b = b;
  a.rp = A.rp;
  a.ci = A.ci;
  a.v = A.v;
  return a;
}

// a12 from a nonzero iterate: dst = x + P x_c (dst may be x itself)
template <typename T>
__global__ void k_prolong_add(int E, int b, const int *__restrict__ ipc, const T *__restrict__ xc, const T *x,
                              T *dst) {
  pdl_launch_dependents();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = g < (long long)E * b;
  const int i = in ? (int)(g / b) : 0, r = in ? (int)(g - (long long)i * b) : 0;
  const int J = in ? ipc[i] : -1;
  pdl_wait();
  if (!in) return;
  dst[g] = x[g] + (J >= 0 ? xc[(size_t)J * b + r] : (T)0);
}

// One cycle on level l for A_l x = f (Sec. 5: no pre-relaxation).  zero: x
// enters as zero, so the right-hand side itself is restricted and the first
// sweep reads x = P x_c through the interpolation map; otherwise the residual
// is restricted and x + P x_c is formed first.  The coarse problem gets a
// V-cycle (type 0), or an F-cycle and then a V-cycle from its result (type 1).
template <typename T>
static void vcyc(const Hier<T> &H, const Params &P, int l, int type, const T *f, T *out, bool zero,
                 cudaStream_t s) {
  const Level<T> &L = H.lev[l];
  const int b = H.b;
  const bool comp = l == 0 && H.l0c.W > 0;
  const double avg = (double)L.A.nnzb / L.E;  // blocks per row (F and C rows have similar lengths)
  if (L.coarsest) {  // exact: the initial guess does not matter
    ProfScope ps("coarse_solve", s, l);
    if (L.ainv) {
      launch_pdl(k_dense_mv<T>, dim3(cdiv((long long)L.n * 32, kThreads)), dim3(kThreads), 0, s, L.n,
                 (const T *)L.ainv, f, out);
    } else {  // block-diagonal coarsest matrix: x_i = D_ii^{-1} f_i
      launch_pdl(k_bdiag_apply<T>, dim3(grid((long long)L.E * b)), dim3(kThreads), 0, s, L.E, b,
                 (const T *)L.dinv, f, out, 0);
    }
    NAIR_LAUNCH_CHECK();
    return;
  }
  const Level<T> &N = H.lev[l + 1];
  const T *rhs = f;
  if (!zero) {  // residual of the incoming iterate
    ProfScope ps("resid", s, l);
    RowArgs<T> a = row_args(L.A, b);
    a.x = out;
    a.f = f;
    a.out = L.r;
    if (comp) {
      a.diag = L.diag;
      a.oci = H.l0c.oci;
      a.ocols = H.l0c.ocols;
      a.ov = H.l0c.ov;
      launch_rowop_l0<T, OP_RESID>(a, H.l0c.W, s);
    } else {
      launch_rowop<T, OP_RESID>(a, avg, s);
    }
    rhs = L.r;
  }
  {  // a11: f_c = r_C + R_cf r_F
    ProfScope ps("restrict", s, l);
    RowArgs<T> a = row_args(L.R, b);
    a.nrows = L.nC;
    a.x = rhs;
    a.f = rhs;
    a.c2f = L.c2f;
    a.out = N.f;
    const double avgR = L.nC ? (double)L.R.nnzb / L.nC : 0.0;
    // scalar-row form of R_cf where built (its permutation was sorted for the
    // same thread groups per row)
    const int G = rowop_groups(a.nrows, b, avgR);
    bool done = false;
    if (L.rr.srp && L.rr.perm_c && sweep_rows_tpc(b, G) == L.rr.perm_c_tpc) {
      a.srp = L.rr.srp;
      a.sj = L.rr.sj;
      a.sv = static_cast<const T *>(L.rr.sv);
      a.perm = L.rr.perm_c;
      done = launch_scalar_rows<T, OP_RESTRICT>(a, G, s);
    }
    if (!done) launch_rowop<T, OP_RESTRICT>(a, avgR, s);
  }
  vcyc<T>(H, P, l + 1, type, N.f, N.x, true, s);
  if (type == 1) vcyc<T>(H, P, l + 1, 0, N.f, N.x, false, s);
  const int S = P.f_sweeps + P.c_sweeps;
  // a12-a14: x = P x_c (or x + P x_c), then F sweeps and C sweeps.  Each sweep
  // updates one class (F or C) from a compact row list, so no warp mixes
  // updated and idle rows; rows of the other class are copied into the output
  // buffer only when that buffer holds an older version of them.  The sweeps
  // alternate between two buffers and end in out.
  T *buf[2];
  int buf_ver[2][2] = {{-1, -1}, {-1, -1}};
  const T *in;
  const int *ipc0;
  if (zero) {
    if (S == 0) {
      k_prolong<T><<<grid((long long)L.E * b), kThreads, 0, s>>>(L.E, b, L.ipc, N.x, out);
      NAIR_LAUNCH_CHECK();
      return;
    }
    buf[0] = (S % 2 == 1) ? out : L.x2;
    buf[1] = (S % 2 == 1) ? L.x2 : out;
    in = N.x;  // read through ipc by the first sweep
    ipc0 = L.ipc;
  } else {
    T *start = (S % 2 == 1) ? L.x2 : out;
    {
      ProfScope ps("prolong_add", s, l);
      launch_pdl(k_prolong_add<T>, dim3(grid((long long)L.E * b)), dim3(kThreads), 0, s, L.E, b,
                 (const int *)L.ipc, (const T *)N.x, (const T *)out, start);
      NAIR_LAUNCH_CHECK();
    }
    if (S == 0) return;
    buf[0] = (start == out) ? L.x2 : out;
    buf[1] = start;
    buf_ver[1][0] = buf_ver[1][1] = 0;
    in = start;
    ipc0 = nullptr;
  }
  const int nrow[2] = {L.nF, L.nC};
  const int *rows[2] = {L.fsweep, L.csweep};
  int cur_ver[2] = {0, 0};  // version of each class (0 = the sweeps' starting iterate)
  // level 0 with scaled couplings: g = D^{-1} f once, then x_i = g_i - sum_j S_ij x_j
  const bool scaled = comp && H.l0c.sv && L.g;
  if (scaled) {
    ProfScope ps("dinv_f", s, l);
    launch_pdl(k_bdiag_apply<T>, dim3(grid((long long)L.E * b)), dim3(kThreads), 0, s, L.E, b,
               (const T *)L.dinv, f, L.g, 0);
    NAIR_LAUNCH_CHECK();
  }
  // device-clock stamps only in V-cycles, where every sweep site runs once per cycle
  const bool stamp = H.clock.dev && P.cycle == 0;
  // the F sweeps after the first update only the rows whose inputs changed
  // (fl[k]; x_C is fixed while they run).  A buffer lacks only the rows updated
  // since it was last written, and those are copied: fq[k] for sweep k >= 2,
  // fl[f_sweeps - 1] for the first C sweep.  From a zero iterate the first
  // sweep reads x_c and writes its F rows into both buffers; from a nonzero one
  // it reads one of them, so sweep 1 copies the F rows outside its list (fq[1])
  const int SF = P.f_sweeps;
  const bool short_f = SF >= 2 && L.nfl == SF;
  // the first F sweep (scalar-row form) keeps f - A_FC x_C in L.h for the
  // later F sweeps, which then sum only the F-column part (x_C is fixed while
  // the F sweeps run)
  bool have_h = false;
  // F sweeps in y_F = D_FF x_F (set up where every sweep takes the scalar-row
  // form): y^1 = h - A_FF x_F^0 with h = f_F - A_FC x_C, y^{k+1} = h - sum_j
  // (A_ij D_jj^{-1}) y^k_j, the same block-Jacobi iterates as x = D^{-1} y, with
  // no D^{-1} applied per sweep; the C sweep reads y_F through the scaled
  // blocks and its copy part writes x_F = D_FF^{-1} y_F for every F row
  const bool ymode = L.ymode && short_f && S == SF + 1 && L.sr.sv2;
  for (int k = 0; k < S; ++k) {
    const int cls = k < SF ? 0 : 1, oth = 1 - cls, ob = k % 2;
    RowArgs<T> a = row_args(L.A, b);
    a.x = in;
    a.ipc = (k == 0) ? ipc0 : nullptr;
    a.f = f;
    a.dinv = L.dinv;
    a.diag = L.diag;
    a.nrows = nrow[cls];
    a.list = rows[cls];
    a.out = buf[ob];
    if (short_f && k >= 1 && k < SF) {
      // the C rows of both buffers are current since the first sweep
      a.nrows = L.fl_n[k];
      a.list = L.fl[k];
      if (k >= 2 || !zero) {
        a.ncopy = L.fq_n[k];
        a.copy_list = L.fq[k];
      }
    } else if (short_f && k == SF) {
      a.ncopy = ymode ? L.nF : L.fl_n[SF - 1];
      a.copy_list = ymode ? L.fsweep : L.fl[SF - 1];
    } else if (buf_ver[ob][oth] != cur_ver[oth]) {
      a.ncopy = nrow[oth];
      a.copy_list = rows[oth];
      if (k == 0 && zero) a.out2 = buf[1 - ob];  // both buffers then hold P x_c on that class
    }
    if (short_f && zero && k == 0) a.out2c = buf[1];
    if (stamp) {
      a.stamp = H.clock.dev + (size_t)l * S + k;
      a.ns = H.clock.nsites;
    }
    ProfScope ps(cls == 0 ? "jacobi_F" : "jacobi_C", s, l);
    if (scaled) {
      a.f = L.g;
      a.diag = L.diag;
      a.oci = H.l0c.oci;
      a.ocols = H.l0c.ocols;
      a.ov = H.l0c.sv;
      launch_rowop_l0<T, OP_JACOBI_S>(a, H.l0c.W, s);
    } else if (comp) {
      a.diag = L.diag;
      a.oci = H.l0c.oci;
      a.ocols = H.l0c.ocols;
      a.ov = H.l0c.ov;
      launch_rowop_l0<T, OP_JACOBI>(a, H.l0c.W, s);
    } else {
      // scalar-row form where built: the permutation belongs to the row list in
      // use and was sorted for the same thread groups per row
      const int pk = (short_f && k < SF) ? k : 0;
      const unsigned char *perm = cls == 1 ? L.sr.perm_c : L.sr.perm_f[pk];
      const int ptpc = cls == 1 ? L.sr.perm_c_tpc : L.sr.perm_f_tpc[pk];
      // F sweep lists: groups sized for half a row, as at setup
      const int G = rowop_groups(a.nrows, b, (cls == 0 && b <= 10) ? 0.5 * avg : avg);
      bool done = false;
      if (L.sr.srp && perm && sweep_rows_tpc(b, G) == ptpc) {
        a.srp = L.sr.srp;
        a.sj = L.sr.sj;
        a.sv = static_cast<const T *>(L.sr.sv);
        a.perm = perm;
        if (ymode) {
          a.srs = L.sr.srs;
          a.h = L.h;
          a.fmode = cls == 1 ? 5 : (k == 0 ? 3 : 4);
          if (a.fmode != 3) a.sv = static_cast<const T *>(L.sr.sv2);
        } else if (cls == 0 && L.h && L.sr.srs && (k == 0 || have_h)) {
          a.srs = L.sr.srs;
          a.h = L.h;
          a.fmode = k == 0 ? 1 : 2;
        }
        done = launch_scalar_rows<T, OP_JACOBI>(a, G, s);
        if (done && k == 0 && a.fmode == 1) have_h = true;
      }
      if (!done && ymode) fail(NAIR_ERR_UNSUPPORTED, "scaled F sweeps without the scalar-row form");
      if (!done) launch_rowop<T, OP_JACOBI>(a, avg, s);
    }
    cur_ver[cls] = k + 1;
    buf_ver[ob][cls] = k + 1;
    if (short_f && k < SF) {
      // both buffers hold the C rows of the first sweep; the F rows of buf[ob]
      // are current, those of the other buffer differ by fl[k]
      buf_ver[1 - ob][oth] = buf_ver[ob][oth] = cur_ver[oth];
    } else if (short_f && k == SF) {
      buf_ver[ob][oth] = cur_ver[oth];
    } else if (a.ncopy) {
      buf_ver[ob][oth] = cur_ver[oth];
      if (a.out2) buf_ver[1 - ob][oth] = cur_ver[oth];
    }
    in = buf[ob];
  }
}

template <typename T>
void vcycle(const Hier<T> &H, const Params &P, const T *f, T *x, cudaStream_t s) {
  vcyc<T>(H, P, 0, P.cycle, f, x, true, s);
}
template void vcycle<double>(const Hier<double> &, const Params &, const double *, double *, cudaStream_t);
template void vcycle<float>(const Hier<float> &, const Params &, const float *, float *, cudaStream_t);

// ---------------------------------------------------------------------------
// transposed cycle (preconditioner of A^T): from a zero iterate, C sweeps then
// F sweeps of block Jacobi on A_l^T, the residual, restriction with P^T,
// recursion on K^T, interpolation with R^T = [R_cf^T; I]
// ---------------------------------------------------------------------------

// first sweep from a zero iterate: rows of `list` get (D_ii^{-1})^T f_i, rows
// of `zlist` are zeroed in out and out2
template <typename T>
__global__ void k_first_sweep_t(int nrows, int b, const int *__restrict__ list, const T *__restrict__ dinvT,
                                const T *__restrict__ f, int nzero, const int *__restrict__ zlist,
                                T *__restrict__ out, T *__restrict__ out2) {
  pdl_launch_dependents();
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long na = (long long)nrows * b;
  if (g < na) {
    const int k = (int)(g / b), r = (int)(g - (long long)k * b);
    const int i = list[k];
    const T *d = dinvT + (size_t)i * b * b + r * b;
    const T *fi = f + (size_t)i * b;
    T acc = 0;
    for (int c = 0; c < b; ++c) acc = fma(d[c], fi[c], acc);
    out[(size_t)i * b + r] = acc;
    return;
  }
  g -= na;
  if (g < (long long)nzero * b) {
    const int k = (int)(g / b), r = (int)(g - (long long)k * b);
    const size_t o = (size_t)zlist[k] * b + r;
    out[o] = (T)0;
    if (out2) out2[o] = (T)0;
  }
}

// P^T restriction: f_c[J] = r[c2f[J]] + the sum of r over the F elements with ip = J
template <typename T>
__global__ void k_restrict_pt(int nC, int b, const int *__restrict__ c2f, const int *__restrict__ prp,
                              const int *__restrict__ pci, const T *__restrict__ r, T *__restrict__ fc) {
  pdl_launch_dependents();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = g < (long long)nC * b;
  const int J = in ? (int)(g / b) : 0, c = in ? (int)(g - (long long)J * b) : 0;
  const int self = in ? c2f[J] : 0, q0 = in ? prp[J] : 0, q1 = in ? prp[J + 1] : 0;
  pdl_wait();
  if (!in) return;
  T acc = r[(size_t)self * b + c];
  for (int q = q0; q < q1; ++q) acc += r[(size_t)pci[q] * b + c];
  fc[g] = acc;
}

template <typename T>
static void l0_args(RowArgs<T> &a, const TLevel<T> &TL, const L0Comp<T> &C) {
  a.diag = TL.diag;
  a.oci = C.oci;
  a.ocols = C.ocols;
  a.ov = C.ov;
}

// the end of the y-form F sweeps of the transposed cycle: out_F = D_ii^{-T} y_i
// for the F rows (flist), out_C = y_C copied for the C rows (clist)
template <typename T>
__global__ void k_convert_t(int nF, int b, const int *__restrict__ flist, const T *__restrict__ dinvT,
                            const T *__restrict__ y, int nC, const int *__restrict__ clist, T *__restrict__ out) {
  pdl_launch_dependents();
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long na = (long long)nF * b;
  if (g < na) {
    const int k = (int)(g / b), r = (int)(g - (long long)k * b);
    const int i = flist[k];
    const T *d = dinvT + (size_t)i * b * b + r * b;
    const T *yi = y + (size_t)i * b;
    T acc = 0;
    for (int c = 0; c < b; ++c) acc = fma(d[c], yi[c], acc);
    out[(size_t)i * b + r] = acc;
    return;
  }
  g -= na;
  if (g < (long long)nC * b) {
    const int k = (int)(g / b), r = (int)(g - (long long)k * b);
    const size_t o = (size_t)clist[k] * b + r;
    out[o] = y[o];
  }
}

template <typename T>
static void vcyc_t(const Hier<T> &H, const Params &P, int l, const T *f, T *out, cudaStream_t s) {
  const Level<T> &L = H.lev[l];
  const TLevel<T> &TL = H.tlev[l];
  const int b = H.b;
  if (L.coarsest) {
    ProfScope ps("coarse_solve_t", s, l);
    if (TL.ainvT) {
      launch_pdl(k_dense_mv<T>, dim3(cdiv((long long)L.n * 32, kThreads)), dim3(kThreads), 0, s, L.n,
                 (const T *)TL.ainvT, f, out);
    } else {
      launch_pdl(k_bdiag_apply<T>, dim3(grid((long long)L.E * b)), dim3(kThreads), 0, s, L.E, b,
                 (const T *)TL.dinvT, f, out, 0);
    }
    NAIR_LAUNCH_CHECK();
    return;
  }
  const Level<T> &N = H.lev[l + 1];
  const int S = P.c_sweeps + P.f_sweeps;
  const bool comp = l == 0 && H.tl0c.W > 0;
  const double avg = (double)TL.At.nnzb / L.E;
  const T *r = f;  // residual after the pre-relaxation (f itself without one)
  if (S == 0) {
    NAIR_CK(cudaMemsetAsync(out, 0, sizeof(T) * (size_t)L.E * b, s));
  } else {
    // F sweeps in y_F = D_FF^T x_F (as in the forward cycle): the first stores
    // h and y = h (x_F = 0 after the C sweeps), the later ones y = h - sum_j
    // ((A^T)_ij D_jj^{-T}) y_j with no D^{-T}, and a last pass writes x_F =
    // D_FF^{-T} y_F into out before the residual
    const bool ymode = TL.ymode && P.f_sweeps >= 2 && TL.nfl == P.f_sweeps && P.c_sweeps >= 1 && TL.sr.sv2;
    const int Sp = S + (ymode ? 1 : 0);
    // the sweeps (and the conversion) alternate between two buffers and end in out
    T *buf[2] = {(Sp % 2 == 1) ? out : L.x2, (Sp % 2 == 1) ? L.x2 : out};
    const int nrow[2] = {L.nF, L.nC};
    const int *rows[2] = {TL.fsweep, TL.csweep};
    int cur_ver[2] = {0, 0};  // version of each class (0 = the zero start)
    int buf_ver[2][2] = {{-1, -1}, {-1, -1}};
    // F sweep m >= 1 updates only the rows of fl[m] (their F couplings reach a
    // row updated in sweep m - 1; x_C is fixed) and copies fq[m] into its
    // buffer, which holds every other F row current: the values of sweep m - 2,
    // or for m = 1 none, fq[1] then being all F rows outside fl[1]
    const bool tshort = P.f_sweeps >= 2 && TL.nfl == P.f_sweeps;
    bool have_h = false;  // h = f - (A^T)_FC x_C formed by this cycle's first F sweep
    for (int k = 0; k < S; ++k) {
      const int cls = k < P.c_sweeps ? 1 : 0, oth = 1 - cls, ob = k % 2, m = k - P.c_sweeps;
      ProfScope ps(cls == 0 ? "jacobi_tF" : "jacobi_tC", s, l);
      if (k == 0) {
        const long long tot = (long long)(nrow[cls] + nrow[oth]) * b;
        launch_pdl(k_first_sweep_t<T>, dim3(grid(tot)), dim3(kThreads), 0, s, nrow[cls], b, rows[cls],
                   (const T *)TL.dinvT, f, nrow[oth], rows[oth], buf[0], buf[1]);
        NAIR_LAUNCH_CHECK();
        cur_ver[cls] = 1;
        buf_ver[0][cls] = 1;
        buf_ver[0][oth] = buf_ver[1][oth] = 0;
        continue;
      }
      RowArgs<T> a = row_args(TL.At, b);
      a.x = buf[1 - ob];
      a.f = f;
      a.dinv = TL.dinvT;
      a.diag = TL.diag;
      a.nrows = nrow[cls];
      a.list = rows[cls];
      a.out = buf[ob];
      const bool short_f = tshort && cls == 0 && m >= 1 && buf_ver[ob][1] == cur_ver[1];
      if (short_f) {
        a.nrows = TL.fl_n[m];
        a.list = TL.fl[m];
        a.ncopy = TL.fq_n[m];
        a.copy_list = TL.fq[m];
      } else if (buf_ver[ob][oth] != cur_ver[oth]) {
        a.ncopy = nrow[oth];
        a.copy_list = rows[oth];
      }
      if (comp) {
        l0_args(a, TL, H.tl0c);
        launch_rowop_l0<T, OP_JACOBI>(a, H.tl0c.W, s);
      } else {
        // scalar-row form of A^T where built, as in the forward cycle
        const unsigned char *perm = cls == 1 ? TL.sr.perm_c : TL.sr.perm_f[short_f ? m : 0];
        const int ptpc = cls == 1 ? TL.sr.perm_c_tpc : TL.sr.perm_f_tpc[short_f ? m : 0];
        const int G = rowop_groups(a.nrows, b, (cls == 0 && b <= 10) ? 0.5 * avg : avg);
        bool done = false;
        if (TL.sr.srp && perm && sweep_rows_tpc(b, G) == ptpc) {
          a.srp = TL.sr.srp;
          a.sj = TL.sr.sj;
          a.sv = static_cast<const T *>(TL.sr.sv);
          a.perm = perm;
          // the first F sweep over all F rows forms h; later ones sum the F part
          const bool full = a.nrows == L.nF;
          if (cls == 0 && TL.h && TL.sr.srs && (have_h || full)) {
            a.srs = TL.sr.srs;
            a.h = TL.h;
            a.fmode = ymode ? (have_h ? 4 : 3) : (have_h ? 2 : 1);
            if (a.fmode == 4) a.sv = static_cast<const T *>(TL.sr.sv2);
          }
          done = launch_scalar_rows<T, OP_JACOBI>(a, G, s);
          if (done && (a.fmode == 1 || a.fmode == 3)) have_h = true;
        }
        if (!done && ymode && cls == 0) fail(NAIR_ERR_UNSUPPORTED, "scaled F sweeps without the scalar-row form");
        if (!done) launch_rowop<T, OP_JACOBI>(a, avg, s);
      }
      cur_ver[cls] = k + 1;
      buf_ver[ob][cls] = k + 1;
      if (!short_f && a.ncopy) buf_ver[ob][oth] = cur_ver[oth];
    }
    if (ymode) {
      ProfScope ps("convert_t", s, l);
      const long long tot = (long long)(L.nF + L.nC) * b;
      launch_pdl(k_convert_t<T>, dim3(grid(tot)), dim3(kThreads), 0, s, L.nF, b, (const int *)TL.fsweep,
                 (const T *)TL.dinvT, (const T *)buf[(S - 1) % 2], L.nC, (const int *)TL.csweep, out);
      NAIR_LAUNCH_CHECK();
    }
    ProfScope ps("resid_t", s, l);
    RowArgs<T> a = row_args(TL.At, b);
    a.x = out;
    a.f = f;
    a.out = TL.r;
    if (comp) {
      l0_args(a, TL, H.tl0c);
      launch_rowop_l0<T, OP_RESID>(a, H.tl0c.W, s);
    } else {
      launch_rowop<T, OP_RESID>(a, avg, s);
    }
    r = TL.r;
  }
  {
    ProfScope ps("restrict_t", s, l);
    launch_pdl(k_restrict_pt<T>, dim3(grid((long long)L.nC * b)), dim3(kThreads), 0, s, L.nC, b,
               (const int *)L.c2f, (const int *)TL.pt_rp, (const int *)TL.pt_ci, r, N.f);
    NAIR_LAUNCH_CHECK();
  }
  vcyc_t<T>(H, P, l + 1, N.f, N.x, s);
  {  // x += R^T x_c: F rows through R_cf^T, C rows take their own coarse value
    ProfScope ps("interp_t", s, l);
    RowArgs<T> a = row_args(TL.Rt, b);
    a.x = N.x;
    a.f = out;
    a.c2f = TL.cself;
    a.out = out;
    launch_rowop<T, OP_INTERP_T>(a, (double)TL.Rt.nnzb / L.E, s);
  }
}

template <typename T>
void vcycle_t(const Hier<T> &H, const Params &P, const T *f, T *x, cudaStream_t s) {
  if ((int)H.tlev.size() != H.nlev) fail(NAIR_ERR_INVALID_ARG, "transposed hierarchy not built");
  vcyc_t<T>(H, P, 0, f, x, s);
}
template void vcycle_t<double>(const Hier<double> &, const Params &, const double *, double *, cudaStream_t);
template void vcycle_t<float>(const Hier<float> &, const Params &, const float *, float *, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 Krylov kernels
// ---------------------------------------------------------------------------

static constexpr int kDotGroup = 8;
// Thread blocks of the dot products over the Krylov basis: four per SM on
// long vectors (C5, 5.2 M unknowns: FP64 solve 135.2 -> 134.5 ms against two;
// six: 137.1 ms), two on shorter ones, where four leave each thread only a few
// elements (C2, 0.79 M unknowns: 31.3 -> 32.3 ms with four)
static constexpr int kDotCtas = 608;
static int dot_ctas(long long n) { return n >= (1LL << 22) ? kDotCtas : kDotCtas / 2; }

// partial[k * G + cta] = sum over this CTA's elements of V_k . w, k < nv.
// Vectors are taken NQ at a time with NQ a compile-time count, so no FP64
// instruction is issued for a vector that does not exist (on GB300 every
// warp-wide FP64 instruction is scarce).
template <int NQ>
__device__ __forceinline__ void dot_group(long long lo, long long hi, int k0, const double *__restrict__ V,
                                          long long ldv, const double *__restrict__ w,
                                          double *__restrict__ partial, double (*red)[kThreads / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, G = gridDim.x;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = fma(V[(k0 + q) * ldv + i], wi, acc[q]);
  }
  if constexpr (NQ == 8) {
    // butterfly reduce-scatter: after it, lanes 4k hold the warp's sum of
    // accumulator k (9 additions per lane instead of 8 full reductions)
    double u[4], t[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool hi = lane & 16;
      const double snd = hi ? acc[q] : acc[q + 4];
      const double rcv = __shfl_xor_sync(0xffffffffu, snd, 16);
      u[q] = (hi ? acc[q + 4] : acc[q]) + rcv;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const bool hi = lane & 8;
      const double snd = hi ? u[q] : u[q + 2];
      const double rcv = __shfl_xor_sync(0xffffffffu, snd, 8);
      t[q] = (hi ? u[q + 2] : u[q]) + rcv;
    }
    const bool hi4 = lane & 4;
    double z = (hi4 ? t[1] : t[0]) + __shfl_xor_sync(0xffffffffu, hi4 ? t[0] : t[1], 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    if ((lane & 3) == 0) {
      const int k = ((lane >> 2) & 1) | (((lane >> 3) & 1) << 1) | (((lane >> 4) & 1) << 2);
      red[k][wid] = z;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double a = acc[q];
      for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (lane == 0) red[q][wid] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double a = 0.0;
    for (int w2 = 0; w2 < kThreads / 32; ++w2) a += red[threadIdx.x][w2];
    partial[(size_t)(k0 + threadIdx.x) * G + blockIdx.x] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_multidot(long long n, int nv, const double *__restrict__ V,
                                                       long long ldv, const double *__restrict__ w,
                                                       double *__restrict__ partial) {
  __shared__ double red[kDotGroup][kThreads / 32];
  const int G = gridDim.x;
  const long long chunk = (n + G - 1) / G;
  const long long lo = chunk * blockIdx.x, hi = min(n, lo + chunk);
  int k0 = 0;
  for (; k0 + kDotGroup <= nv; k0 += kDotGroup) dot_group<kDotGroup>(lo, hi, k0, V, ldv, w, partial, red);
  switch (nv - k0) {
    case 1: dot_group<1>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 2: dot_group<2>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 3: dot_group<3>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 4: dot_group<4>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 5: dot_group<5>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 6: dot_group<6>(lo, hi, k0, V, ldv, w, partial, red); break;
    case 7: dot_group<7>(lo, hi, k0, V, ldv, w, partial, red); break;
    default: break;
  }
}

__global__ void k_reduce_partials(int nv, int G, const double *__restrict__ partial,
                                  double *__restrict__ out) {
  const int k = blockIdx.x, lane = threadIdx.x;
  if (k >= nv) return;
  double a = 0.0;
  for (int c = lane; c < G; c += 32) a += partial[(size_t)k * G + c];
  for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if (lane == 0) out[k] = a;
}

// w -= sum_k h_k V_k
__global__ void k_axpy_multi(long long n, int nv, const double *__restrict__ V, long long ldv,
                             const double *__restrict__ h, double *__restrict__ w) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = w[i];
  int k = 0;
  // eight vectors' loads issued together; the updates keep the order of k
  // (C5 FP64 solve 134.5 -> 134.2 ms)
  for (; k + 8 <= nv; k += 8) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = V[(k + q) * ldv + i];
#pragma unroll
    for (int q = 0; q < 8; ++q) a -= h[k + q] * v[q];
  }
  for (; k < nv; ++k) a -= h[k] * V[k * ldv + i];
  w[i] = a;
}

// x += sum_k y_k Z_k
__global__ void k_update(long long n, int nv, const double *__restrict__ Z, long long ldz,
                         const double *__restrict__ y, double *__restrict__ x) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = x[i];
  for (int k = 0; k < nv; ++k) a += y[k] * Z[k * ldz + i];
  x[i] = a;
}

// out = w / d as w times the correctly rounded 1 / d: an FP64 division per
// element costs a dozen FP64-pipe instructions, which made the normalisation
// FP64-bound (81 us per C5 basis vector; within 1.5 ulp of the quotient)
__global__ void k_div(long long n, const double *__restrict__ w, double d, double *__restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 1.0 / d;
  if (i < n) out[i] = w[i] * inv;
}

// out = w / ||w|| from the squared norm on the device (IEEE sqrt, then the
// scaling by its reciprocal as in k_div); zero when the norm is zero
// (breakdown: the host ends the cycle at this column and never uses out)
__global__ void k_div_norm(long long n, const double *__restrict__ w, const double *__restrict__ nrm2,
                           double *__restrict__ out) {
  const double d = sqrt(*nrm2);  // once per thread: a grid-stride loop over the vector
  const double inv = d != 0.0 ? 1.0 / d : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = w[i] * inv;
}

template <typename A, typename B>
__global__ void k_cast(long long n, const A *__restrict__ in, B *__restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (B)in[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void Krylov::ensure(long long n_, int m_, cudaStream_t s) {
  if (n == n_ && m == m_ && V) return;
  mem.release_all();
  mem.s = s;
  n = n_;
  m = m_;
  V = mem.alloc<double>((size_t)n * (m + 1));
  Z = mem.alloc<double>((size_t)n * m);
  w = mem.alloc<double>(n);
  partial = mem.alloc<double>((size_t)kDotCtas * (m + 2));
  hdev = mem.alloc<double>(2 * (m + 2) + 2);
  ydev = mem.alloc<double>(m + 1);
  if (hhost) cudaFreeHost(hhost);
  NAIR_CK(cudaMallocHost(&hhost, sizeof(double) * (2 * (m + 2) + 2 + m + 1)));
  for (int q = 0; q < 2; ++q) {
    if (slot[q]) cudaFreeHost(slot[q]);
    NAIR_CK(cudaMallocHost(&slot[q], sizeof(double) * (2 * (m + 1) + 1)));
    if (!ev[q]) NAIR_CK(cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming));
  }
}

Krylov::~Krylov() {
  if (hhost) cudaFreeHost(hhost);
  for (int q = 0; q < 2; ++q) {
    if (slot[q]) cudaFreeHost(slot[q]);
    if (ev[q]) cudaEventDestroy(ev[q]);
  }
}

static void multidot(Krylov &K, long long n, int nv, const double *V, const double *w, double *out,
                     cudaStream_t s) {
  ProfScope ps("multidot", s);
  const int G = dot_ctas(n);
  k_multidot<<<G, kThreads, 0, s>>>(n, nv, V, n, w, K.partial);
  NAIR_LAUNCH_CHECK();
  k_reduce_partials<<<nv, 32, 0, s>>>(nv, G, K.partial, out);
  NAIR_LAUNCH_CHECK();
}

__global__ void k_set_ptrs(void **dptr, const double *v, double *z) {
  dptr[0] = const_cast<double *>(v);
  dptr[1] = z;
}

template <typename T>
__global__ void k_copy_in(long long n, void *const *__restrict__ ptrs, T *__restrict__ dst) {
  pdl_launch_dependents();
  pdl_wait();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)(static_cast<const double *>(ptrs[0])[i]);
}

template <typename T>
__global__ void k_copy_out(long long n, const T *__restrict__ src, void *const *__restrict__ ptrs) {
  pdl_launch_dependents();
  pdl_wait();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) static_cast<double *>(ptrs[1])[i] = (double)src[i];
}

void release_clock(SweepClock &c) {
  if (c.dev) cudaFree(c.dev);
  for (auto sl : c.slot)
    if (sl) cudaFreeHost(sl);
  c = SweepClock();
}

// reset all sweep stamps (starts to the maximum, ends to zero) on the stream
static void clock_reset(const SweepClock &c, cudaStream_t s) {
  NAIR_CK(cudaMemsetAsync(c.dev, 0xff, sizeof(unsigned long long) * c.nsites, s));
  NAIR_CK(cudaMemsetAsync(c.dev + c.nsites, 0, sizeof(unsigned long long) * c.nsites, s));
}

template <typename T>
static void clock_init(const Hier<T> &H, const Params &P) {
  SweepClock &c = H.clock;
  if (!P.sweep_timing || c.dev) return;
  c.S = P.f_sweeps + P.c_sweeps;
  c.nsites = std::max(1, H.nlev * c.S);
  NAIR_CK(cudaMalloc(&c.dev, sizeof(unsigned long long) * 2 * c.nsites));
  for (auto &sl : c.slot) NAIR_CK(cudaMallocHost(&sl, sizeof(unsigned long long) * 2 * c.nsites));
  c.count.assign(2 * H.nlev, 0);
  c.ms.assign(2 * H.nlev, 0.0);
  c.site_count.assign(c.nsites, 0);
  c.site_ms.assign(c.nsites, 0.0);
}

// queue a copy of the stamps of the cycle just enqueued into pinned slot q
template <typename T>
static void clock_stage(const Hier<T> &H, int q, cudaStream_t s) {
  const SweepClock &c = H.clock;
  if (!c.dev) return;
  NAIR_CK(cudaMemcpyAsync(c.slot[q], c.dev, sizeof(unsigned long long) * 2 * c.nsites, cudaMemcpyDeviceToHost, s));
}

// once slot q's copy has completed: add the stamped sweep durations
template <typename T>
static void clock_collect(const Hier<T> &H, const Params &P, int q) {
  SweepClock &c = H.clock;
  if (!c.dev) return;
  const unsigned long long *h = c.slot[q];
  for (int l = 0; l < H.nlev; ++l)
    for (int k = 0; k < c.S; ++k) {
      const int site = l * c.S + k;
      const unsigned long long t0 = h[site], t1 = h[c.nsites + site];
      if (t1 == 0 || t0 == ~0ULL || t1 < t0) continue;
      const int cls = k < P.f_sweeps ? 0 : 1;
      const double ms = (double)(t1 - t0) * 1e-6;
      c.count[2 * l + cls] += 1;
      c.ms[2 * l + cls] += ms;
      c.site_count[site] += 1;
      c.site_ms[site] += ms;
    }
}

void release_graph(VGraph &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.dptr) cudaFree(g.dptr);
  g = VGraph();
}

// the preconditioner on level-0 vectors: the cycle (or the transposed cycle);
// for scalar nAIR with the block scaling D^{-1} before it (D^{-T} after the
// transposed cycle), through level 0's residual vector, which a cycle from a
// zero guess does not use on level 0
template <typename T>
static void cycle_apply(const Hier<T> &H, const Params &P, const T *f, T *x, bool transposed, cudaStream_t s) {
  if (!H.pre_dinv) {
    if (transposed) vcycle_t<T>(H, P, f, x, s);
    else vcycle<T>(H, P, f, x, s);
    return;
  }
  T *tmp = H.lev[0].r;
  const dim3 g(grid((long long)H.pre_E * H.pre_b));
  if (transposed) {
    vcycle_t<T>(H, P, f, tmp, s);
    ProfScope ps("scaling", s);
    launch_pdl(k_bdiag_apply<T>, g, dim3(kThreads), 0, s, H.pre_E, H.pre_b, H.pre_dinv, (const T *)tmp, x, 1);
    NAIR_LAUNCH_CHECK();
  } else {
    {
      ProfScope ps("scaling", s);
      launch_pdl(k_bdiag_apply<T>, g, dim3(kThreads), 0, s, H.pre_E, H.pre_b, H.pre_dinv, f, tmp, 0);
      NAIR_LAUNCH_CHECK();
    }
    vcycle<T>(H, P, (const T *)tmp, x, s);
  }
}

// capture: copy the input into level 0's right-hand side, V-cycle on fixed
// buffers, copy level 0's solution out (FP64 <-> T casts in mixed precision)
template <typename T>
static void capture_graph(const Hier<T> &H, const Params &P, long long n, bool transposed) {
  VGraph &g = transposed ? H.tgraph : H.graph;
  NAIR_CK(cudaMalloc(&g.dptr, 2 * sizeof(void *)));
  const long long before = thread_launch_count();
  cudaGraph_t graph;
  // capture on a private stream (the caller's may be the legacy default stream,
  // which cannot be captured); the graph is launched on the caller's stream
  cudaStream_t s;
  NAIR_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  NAIR_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    T *f0 = H.lev[0].f, *x0 = H.lev[0].x;
    if (H.clock.dev && !transposed) clock_reset(H.clock, s);
    k_copy_in<T><<<grid(n), kThreads, 0, s>>>(n, g.dptr, f0);
    NAIR_LAUNCH_CHECK();
    cycle_apply<T>(H, P, f0, x0, transposed, s);
    launch_pdl(k_copy_out<T>, dim3(grid(n)), dim3(kThreads), 0, s, n, (const T *)x0, (void *const *)g.dptr);
    NAIR_LAUNCH_CHECK();
  } catch (...) {
    cudaStreamEndCapture(s, &graph);
    throw;
  }
  NAIR_CK(cudaStreamEndCapture(s, &graph));
  g.nodes = thread_launch_count() - before;
  add_launches(-g.nodes);  // captured, not launched
  cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  NAIR_CK(e);
}

template <typename T>
void precond(const Hier<T> &H, const Params &P, const double *v, double *z, cudaStream_t s,
             long long n, bool transposed) {
  if (!transposed) clock_init(H, P);
  if (P.use_graphs && !prof_on()) {
    VGraph &g = transposed ? H.tgraph : H.graph;
    if (!g.exec) capture_graph<T>(H, P, n, transposed);
    // the pointers travel as kernel arguments (copied at launch), so the host
    // may queue the next replay before this one has started
    k_set_ptrs<<<1, 1, 0, s>>>(g.dptr, v, z);
    NAIR_LAUNCH_CHECK();
    NAIR_CK(cudaGraphLaunch(g.exec, s));
    add_launches(g.nodes);
    return;
  }
  if (H.clock.dev && !transposed) clock_reset(H.clock, s);
  if constexpr (std::is_same<T, double>::value) {
    cycle_apply<double>(H, P, v, z, transposed, s);
  } else {
    T *f0 = H.lev[0].f, *x0 = H.lev[0].x;
    k_cast<double, T><<<grid(n), kThreads, 0, s>>>(n, v, f0);
    NAIR_LAUNCH_CHECK();
    cycle_apply<T>(H, P, f0, x0, transposed, s);
    k_cast<T, double><<<grid(n), kThreads, 0, s>>>(n, x0, z);
    NAIR_LAUNCH_CHECK();
  }
}
template void precond<double>(const Hier<double> &, const Params &, const double *, double *, cudaStream_t, long long,
                              bool);
template void precond<float>(const Hier<float> &, const Params &, const double *, double *, cudaStream_t, long long,
                             bool);

// a10: y = A x, or y = b - A x when b is given (FP64, level 0)
void spmv64(const DBsr<double> &A, int b, const double *x, const double *bvec, double *y, cudaStream_t s,
            const L0Comp<double> *C, const int *diag) {
  RowArgs<double> a = row_args(A, b);
  a.x = x;
  a.f = bvec;
  a.out = y;
  const double avg = (double)A.nnzb / A.nrows;
  ProfScope ps(bvec ? "resid64" : "spmv64", s);
  if (C && C->W > 0 && diag) {
    a.diag = diag;
    a.oci = C->oci;
    a.ocols = C->ocols;
    a.ov = C->ov;
    if (bvec) launch_rowop_l0<double, OP_RESID>(a, C->W, s);
    else launch_rowop_l0<double, OP_SPMV>(a, C->W, s);
    return;
  }
  if (bvec) launch_rowop<double, OP_RESID>(a, avg, s);
  else launch_rowop<double, OP_SPMV>(a, avg, s);
}

template <typename T>
nair_status fgmres(const Outer &op, const Hier<T> &H, const Params &P, Krylov &K, const double *bvec,
                   double *x, std::vector<double> &hist, int *iters, double *relres, cudaStream_t s,
                   bool transposed) {
  // transposed: op is A^T and the preconditioner the transposed cycle
  const DBsr<double> &A = op.A;
  const L0Comp<double> *C = &op.C;
  const int *diag0 = op.diag;
  const int b = op.b, m = P.restart;
  const long long n = (long long)A.nrows * b;
  K.ensure(n, m, s);
  double *hh = K.hhost;  // [0, m+1): h1, [m+1, 2m+2): h2, [2m+2]: ||w||^2
  std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  hist.clear();
  // ||b||
  multidot(K, n, 1, bvec, bvec, K.hdev, s);
  NAIR_CK(cudaMemcpyAsync(hh, K.hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(hh[0]);
  int it = 0;
  nair_status status = NAIR_ERR_NOT_CONVERGED;
  if (bnorm == 0.0) {
    NAIR_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *iters = 0;
    *relres = 0.0;
    return NAIR_OK;
  }
  double *V = K.V, *Z = K.Z, *w = K.w;
  // one Arnoldi step for column j: z_j = M^{-1} v_j, w = A z_j, classical
  // Gram-Schmidt twice, ||w||^2; the Hessenberg column is copied to pinned slot
  // j mod 2 (event ev[j mod 2]) and v_{j+1} = w / ||w|| is formed on the device
  auto arnoldi_step = [&](int j) {
    const int q = j & 1;
    double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
    {
      ProfScope ps("vcycle", s);
      precond<T>(H, P, vj, zj, s, n, transposed);
    }
    if (!transposed) clock_stage(H, q, s);
    spmv64(A, b, zj, nullptr, w, s, C, diag0);
    multidot(K, n, j + 1, V, w, K.hdev, s);
    {
      ProfScope ps("axpy_multi", s);
      k_axpy_multi<<<grid(n), kThreads, 0, s>>>(n, j + 1, V, n, K.hdev, w);
      NAIR_LAUNCH_CHECK();
    }
    multidot(K, n, j + 1, V, w, K.hdev + (m + 1), s);
    {
      ProfScope ps("axpy_multi", s);
      k_axpy_multi<<<grid(n), kThreads, 0, s>>>(n, j + 1, V, n, K.hdev + (m + 1), w);
      NAIR_LAUNCH_CHECK();
    }
    multidot(K, n, 1, w, w, K.hdev + 2 * (m + 1), s);
    {
      ProfScope ps("arnoldi_readback", s);
      NAIR_CK(cudaMemcpyAsync(K.slot[q], K.hdev, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
      NAIR_CK(cudaEventRecord(K.ev[q], s));
    }
    k_div_norm<<<std::min(grid(n), 4 * kDotCtas), kThreads, 0, s>>>(n, w, K.hdev + 2 * (m + 1),
                                                                    V + (size_t)(j + 1) * n);
    NAIR_LAUNCH_CHECK();
  };
  for (;;) {
    spmv64(A, b, x, bvec, w, s, C, diag0);
    multidot(K, n, 1, w, w, K.hdev, s);
    NAIR_CK(cudaMemcpyAsync(hh, K.hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
    const double beta = std::sqrt(hh[0]);
    if (!std::isfinite(beta)) return NAIR_ERR_BREAKDOWN;
    if (hist.empty()) hist.push_back(beta / bnorm);
    if (beta / bnorm <= P.tol) { status = NAIR_OK; break; }
    if (it >= P.maxiter) break;
    k_div<<<grid(n), kThreads, 0, s>>>(n, w, beta, V);
    NAIR_LAUNCH_CHECK();
    std::fill(g.begin(), g.end(), 0.0);
    std::fill(Hm.begin(), Hm.end(), 0.0);
    g[0] = beta;
    int j;
    bool conv = false, brk = false, queued = false;
    for (j = 0; j < m && it < P.maxiter; ++j) {
      // column j (if not already in flight), then column j + 1 before column j's
      // Hessenberg entries are read: the host's read-back and Givens work
      // overlap the next iteration on the GPU.  A column enqueued past
      // convergence or breakdown is never used.
      if (!queued) arnoldi_step(j);
      ++it;
      queued = j + 1 < m && it < P.maxiter;
      if (queued) arnoldi_step(j + 1);
      NAIR_CK(cudaEventSynchronize(K.ev[j & 1]));
      const double *hq = K.slot[j & 1];
      if (!transposed) clock_collect(H, P, j & 1);
      for (int k = 0; k <= j; ++k) Hm[(size_t)k * m + j] = hq[k] + hq[m + 1 + k];
      const double hn = std::sqrt(hq[2 * (m + 1)]);
      if (!std::isfinite(hn)) return NAIR_ERR_BREAKDOWN;
      Hm[(size_t)(j + 1) * m + j] = hn;
      for (int k = 0; k < j; ++k) {
        double a = Hm[(size_t)k * m + j], c = Hm[(size_t)(k + 1) * m + j];
        Hm[(size_t)k * m + j] = cs[k] * a + sn[k] * c;
        Hm[(size_t)(k + 1) * m + j] = -sn[k] * a + cs[k] * c;
      }
      double a = Hm[(size_t)j * m + j], c = Hm[(size_t)(j + 1) * m + j];
      double r = std::hypot(a, c);
      cs[j] = a / r;
      sn[j] = c / r;
      Hm[(size_t)j * m + j] = r;
      Hm[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      double est = std::fabs(g[j + 1]) / bnorm;
      hist.push_back(est);
      if (est <= P.tol) { conv = true; ++j; break; }
      if (hn == 0.0) { brk = true; ++j; break; }
    }
    for (int r = j - 1; r >= 0; --r) {
      double sum = g[r];
      for (int c = r + 1; c < j; ++c) sum -= Hm[(size_t)r * m + c] * y[c];
      y[r] = sum / Hm[(size_t)r * m + r];
    }
    double *yh = hh + 2 * (m + 2) + 2;
    for (int k = 0; k < j; ++k) yh[k] = y[k];
    NAIR_CK(cudaMemcpyAsync(K.ydev, yh, sizeof(double) * j, cudaMemcpyHostToDevice, s));
    k_update<<<grid(n), kThreads, 0, s>>>(n, j, Z, n, K.ydev, x);
    NAIR_LAUNCH_CHECK();
    if (conv || brk) { status = NAIR_OK; break; }
    if (it >= P.maxiter) break;
  }
  spmv64(A, b, x, bvec, w, s, C, diag0);
  multidot(K, n, 1, w, w, K.hdev, s);
  NAIR_CK(cudaMemcpyAsync(hh, K.hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
  *relres = std::sqrt(hh[0]) / bnorm;
  *iters = it;
  if (!std::isfinite(*relres)) return NAIR_ERR_BREAKDOWN;
  if (status == NAIR_OK && *relres > 10.0 * P.tol && P.tol > 0) status = NAIR_ERR_NOT_CONVERGED;
  return status;
}

template nair_status fgmres<double>(const Outer &, const Hier<double> &, const Params &, Krylov &, const double *,
                                    double *, std::vector<double> &, int *, double *, cudaStream_t, bool);
template nair_status fgmres<float>(const Outer &, const Hier<float> &, const Params &, Krylov &, const double *,
                                   double *, std::vector<double> &, int *, double *, cudaStream_t, bool);

}  // namespace nair
