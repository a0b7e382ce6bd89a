// Adjoint operators on the GPU: block transposes of block-CSR matrices and the
// transposed form of a finished hierarchy.  For A^T the transfer operators of
// the forward hierarchy swap roles (Sec. 2, Corollary on ideal interpolation):
// R^T = [R_cf^T; I] interpolates -- R_cf^T approximates the ideal
// interpolation -(A^T)_ff^{-1} (A^T)_fc of A^T -- and P^T = [W^T I] restricts,
// with coarse operators K^T.  An F solve must then come before the coarse-grid
// correction (Remark on pre-F-relaxation), so the block-Jacobi sweeps move in
// front of it.  The result, the transpose of the V-cycle, preconditions A^T
// without a second setup.
#include <algorithm>

#include "hier.cuh"

namespace nair {

static constexpr int kThreads = 256;
static inline int grid(long long n) { return std::max(1, cdiv(n, kThreads)); }

// ---------------------------------------------------------------------------
// block-CSR transpose: counts per column, scan, scatter, per-row sort
// ---------------------------------------------------------------------------
__global__ void k_t_count(int nnzb, const int *__restrict__ ci, int *__restrict__ cnt) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnzb) atomicAdd(&cnt[ci[p]], 1);
}

__global__ void k_t_fill(int nr, const int *__restrict__ rp, const int *__restrict__ ci,
                         const int *__restrict__ trp, int *__restrict__ fill, int *__restrict__ tci,
                         int *__restrict__ tsrc) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    const int q = trp[j] + atomicAdd(&fill[j], 1);
    tci[q] = i;
    tsrc[q] = p;
  }
}

// sort each row by column, carrying a companion index when given (insertion
// sort: the rows of a transposed DG operator are short)
__global__ void k_sort_rows(int n, const int *__restrict__ rp, int *__restrict__ ci, int *__restrict__ comp) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = rp[i] + 1; a < rp[i + 1]; ++a) {
    const int c = ci[a], s = comp ? comp[a] : 0;
    int q = a - 1;
    while (q >= rp[i] && ci[q] > c) {
      ci[q + 1] = ci[q];
      if (comp) comp[q + 1] = comp[q];
      --q;
    }
    ci[q + 1] = c;
    if (comp) comp[q + 1] = s;
  }
}

// out block q = (in block tsrc[q])^T
template <typename T>
__global__ void k_t_vals(long long total, int b, const int *__restrict__ tsrc, const T *__restrict__ v,
                         T *__restrict__ tv) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long q = g / bb;
  const int rc = (int)(g - q * bb), r = rc / b, c = rc - r * b;
  tv[g] = v[(size_t)tsrc[q] * bb + c * b + r];
}

// every b x b block transposed in place of position
template <typename T>
__global__ void k_block_transpose(long long total, int b, const T *__restrict__ in, T *__restrict__ out) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long q = g / bb;
  const int rc = (int)(g - q * bb), r = rc / b, c = rc - r * b;
  out[g] = in[(size_t)q * bb + c * b + r];
}

// C elements: own coarse index; F elements: -1
__global__ void k_cself(int E, const signed char *__restrict__ cf, const int *__restrict__ ipc,
                        int *__restrict__ cself) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) cself[i] = cf[i] ? ipc[i] : -1;
}

// P^T lists: F elements that interpolate from coarse point J
__global__ void k_pt_count(int E, const signed char *__restrict__ cf, const int *__restrict__ ipc,
                           int *__restrict__ cnt) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E && !cf[i] && ipc[i] >= 0) atomicAdd(&cnt[ipc[i]], 1);
}

__global__ void k_pt_fill(int E, const signed char *__restrict__ cf, const int *__restrict__ ipc,
                          const int *__restrict__ prp, int *__restrict__ fill, int *__restrict__ pci) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E || cf[i] || ipc[i] < 0) return;
  const int J = ipc[i];
  pci[prp[J] + atomicAdd(&fill[J], 1)] = i;
}

template <typename T>
void bsr_transpose(const DBsr<T> &A, int b, DBsr<T> &out, cudaStream_t s, Mem &mem) {
  const int nr = A.nrows, nc = A.ncols, nnzb = A.nnzb;
  out.nrows = nc;
  out.ncols = nr;
  out.nnzb = nnzb;
  out.rp = mem.alloc<int>(nc + 1);
  out.ci = mem.alloc<int>(nnzb);
  out.v = mem.alloc<T>((size_t)nnzb * b * b);
  Mem tmp;
  tmp.s = s;
  int *cnt = tmp.alloc<int>(nc + 1), *fill = tmp.alloc<int>(nc + 1), *tsrc = tmp.alloc<int>(nnzb);
  NAIR_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (nc + 1), s));
  NAIR_CK(cudaMemsetAsync(fill, 0, sizeof(int) * (nc + 1), s));
  if (nnzb) {
    launch_pdl(k_t_count, dim3(grid(nnzb)), dim3(kThreads), 0, s, nnzb, A.ci, cnt);
    NAIR_LAUNCH_CHECK();
  }
  exclusive_scan(cnt, out.rp, nc, s, tmp, false);
  if (nnzb) {
    launch_pdl(k_t_fill, dim3(grid(nr)), dim3(kThreads), 0, s, nr, A.rp, A.ci, out.rp, fill, out.ci, tsrc);
    NAIR_LAUNCH_CHECK();
    launch_pdl(k_sort_rows, dim3(grid(nc)), dim3(kThreads), 0, s, nc, out.rp, out.ci, tsrc);
    NAIR_LAUNCH_CHECK();
    const long long tot = (long long)nnzb * b * b;
    launch_pdl(k_t_vals<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, tsrc, A.v, out.v);
    NAIR_LAUNCH_CHECK();
  }
}
template void bsr_transpose<double>(const DBsr<double> &, int, DBsr<double> &, cudaStream_t, Mem &);
template void bsr_transpose<float>(const DBsr<float> &, int, DBsr<float> &, cudaStream_t, Mem &);

template <typename T>
void build_transposed(Hier<T> &H, int f_sweeps, cudaStream_t s, Mem &mem) {
  ProfScope ps("transpose_hierarchy", s);
  const int b = H.b;
  H.tlev.assign(H.nlev, TLevel<T>());
  Mem tmp;
  tmp.s = s;
  const int nf = (f_sweeps >= 2 && f_sweeps <= kMaxFLists) ? f_sweeps : 0, m = nf ? 2 * (nf - 1) : 0;
  int *lcnt = m ? tmp.alloc<int>((size_t)H.nlev * m) : nullptr;
  std::vector<int *> lbufs(H.nlev, nullptr);
  for (int l = 0; l < H.nlev; ++l) {
    const Level<T> &L = H.lev[l];
    TLevel<T> &TL = H.tlev[l];
    const int E = L.E;
    const long long tb = (long long)E * b * b;
    TL.dinvT = mem.alloc<T>((size_t)tb);
    launch_pdl(k_block_transpose<T>, dim3(grid(tb)), dim3(kThreads), 0, s, tb, b, L.dinv, TL.dinvT);
    NAIR_LAUNCH_CHECK();
    if (l == 0 || !L.coarsest) {
      // A_l^T: level 0's is also the operator of the outer Krylov solve
      bsr_transpose<T>(L.A, b, TL.At, s, mem);
      TL.diag = mem.alloc<int>(E);
      diag_positions(E, TL.At.rp, TL.At.ci, TL.diag, s);
    }
    if (L.coarsest) {
      if (L.ainv) {
        const long long nn = (long long)L.n * L.n;
        TL.ainvT = mem.alloc<T>((size_t)nn);
        launch_pdl(k_block_transpose<T>, dim3(grid(nn)), dim3(kThreads), 0, s, nn, L.n, L.ainv, TL.ainvT);
        NAIR_LAUNCH_CHECK();
      }
      continue;
    }
    const int nC = L.nC, nF = L.nF;
    TL.fsweep = sweep_list(nF, L.f2f, TL.At.rp, s, mem, tmp);
    TL.csweep = sweep_list(nC, L.c2f, TL.At.rp, s, mem, tmp);
    if (nf)
      lbufs[l] = fsweep_lists(E, nF, TL.At.rp, TL.At.ci, L.cf, TL.fsweep, nf, lcnt + (size_t)l * m, s, mem, tmp);
    // R_cf (nC rows, element columns) -> R_cf^T (element rows, nC columns)
    DBsr<T> R = L.R;
    R.nrows = nC;
    R.ncols = E;
    bsr_transpose<T>(R, b, TL.Rt, s, mem);
    TL.cself = mem.alloc<int>(E);
    launch_pdl(k_cself, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, L.ipc, TL.cself);
    NAIR_LAUNCH_CHECK();
    // P^T: for each coarse point the F elements interpolating from it
    int *cnt = tmp.alloc<int>(nC + 1), *fill = tmp.alloc<int>(nC + 1);
    NAIR_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (nC + 1), s));
    NAIR_CK(cudaMemsetAsync(fill, 0, sizeof(int) * (nC + 1), s));
    launch_pdl(k_pt_count, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, L.ipc, cnt);
    NAIR_LAUNCH_CHECK();
    TL.pt_rp = mem.alloc<int>(nC + 1);
    exclusive_scan(cnt, TL.pt_rp, nC, s, tmp, false);
    TL.pt_ci = mem.alloc<int>(nF);  // at most one entry per F element
    launch_pdl(k_pt_fill, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, L.ipc, TL.pt_rp, fill, TL.pt_ci);
    NAIR_LAUNCH_CHECK();
    launch_pdl(k_sort_rows, dim3(grid(nC)), dim3(kThreads), 0, s, nC, TL.pt_rp, TL.pt_ci, nullptr);
    NAIR_LAUNCH_CHECK();
    TL.r = mem.alloc<T>((size_t)E * b);
  }
  if (!H.lev[0].coarsest) build_l0comp<T>(H.tlev[0].At, H.tlev[0].diag, b, s, mem, H.tl0c);
  std::vector<int> h((size_t)H.nlev * m, 0);
  if (m) NAIR_CK(cudaMemcpyAsync(h.data(), lcnt, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
  for (int l = 0; l < H.nlev; ++l) {
    TLevel<T> &TL = H.tlev[l];
    if (!lbufs[l]) continue;
    TL.nfl = nf;
    fsweep_assign(H.lev[l].nF, nf, lbufs[l], h.data() + (size_t)l * m, TL.fsweep, TL.fl, TL.fl_n, TL.fq, TL.fq_n);
  }
  for (int l = 1; l < H.nlev; ++l) {
    const Level<T> &L = H.lev[l];
    TLevel<T> &TL = H.tlev[l];
    if (L.coarsest) continue;
    build_sweep_rows_level<T>(L.E, L.nF, L.nC, b, TL.At, L.cf, TL.fsweep, TL.nfl, TL.fl, TL.fl_n, TL.csweep, TL.sr,
                              s, mem);
    // the F sweeps follow the C sweeps, so x_C is fixed while they run: the
    // first keeps f - (A^T)_FC x_C for the others, as in the forward cycle
    if (TL.sr.srs && TL.nfl >= 2) TL.h = mem.alloc<T>((size_t)L.E * b);
    // F sweeps in y_F = D_FF^T x_F where each of them takes the scalar-row
    // form (the C sweeps come first and see x_F = 0)
    bool all_rows = TL.h && TL.nfl == nf && nf >= 2;
    for (int k = 0; all_rows && k < TL.nfl; ++k) all_rows = TL.sr.perm_f[k] != nullptr;
    if (all_rows) {
      scale_srow_entries<T>(TL.sr, b, (const T *)TL.dinvT, L.cf, s, mem);
      TL.ymode = 1;
    }
  }
  NAIR_CK(cudaStreamSynchronize(s));
}
template void build_transposed<double>(Hier<double> &, int, cudaStream_t, Mem &);
template void build_transposed<float>(Hier<float> &, int, cudaStream_t, Mem &);

}  // namespace nair
