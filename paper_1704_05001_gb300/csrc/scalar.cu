// Scalar nAIR (Sec. 5.2; the paper's default form): A is scaled by its
// block-diagonal inverse, every diagonal block becoming the identity, and the
// scaled matrix is stored and coarsened degree of freedom by degree of
// freedom (block size 1).  The off-diagonal blocks D_ii^{-1} A_ij are block
// products in the canonical order (acc = fma(d_rt, a_tc, acc), t ascending,
// from zero), the diagonal blocks are set to I exactly, and exact zeros are
// not stored, so the scaled matrix is the same bit for bit whatever the
// launch shape.
#include <algorithm>

#include "hier.cuh"

namespace nair {

static constexpr int kThreads = 256;
static inline int grid(long long n) { return std::max(1, cdiv(n, kThreads)); }

__global__ void k_row_of_block(int E, const int *__restrict__ rp, int *__restrict__ brow) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) brow[p] = i;
}

// S_p = D_i^{-1} A_p for an off-diagonal block p of row i, I for the diagonal block
__global__ void k_scale_blocks(long long total, int b, const int *__restrict__ brow, const int *__restrict__ diag,
                               const double *__restrict__ Dinv, const double *__restrict__ A,
                               double *__restrict__ S) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long p = g / bb;
  const int rc = (int)(g - p * bb), r = rc / b, c = rc - r * b;
  const int i = brow[p];
  if (diag[i] == p) {
    S[g] = (r == c) ? 1.0 : 0.0;
    return;
  }
  const double *d = Dinv + (size_t)i * bb + r * b;
  const double *a = A + (size_t)p * bb + c;
  double acc = 0.0;
  for (int t = 0; t < b; ++t) acc = __fma_rn(d[t], a[(size_t)t * b], acc);
  S[g] = acc;
}

// scalar row (i, r): its nonzeros over the blocks of row i in ascending column
// order; FILL = false counts them, FILL = true writes them at srp[i b + r]
template <bool FILL>
__global__ void k_expand_scalar(int E, int b, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ S, const int *__restrict__ srp, int *__restrict__ cnt,
                              int *__restrict__ sci, double *__restrict__ sv) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)E * b) return;
  const int i = (int)(g / b), r = (int)(g - (long long)i * b);
  const int bb = b * b;
  int w = FILL ? srp[g] : 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const double *row = S + (size_t)p * bb + r * b;
    const int j = ci[p];
    for (int c = 0; c < b; ++c) {
      const double v = row[c];
      if (v != 0.0) {
        if (FILL) {
          sci[w] = j * b + c;
          sv[w] = v;
        }
        ++w;
      }
    }
  }
  if (!FILL) cnt[g] = w;
}

void scalar_matrix(const DBsr<double> &A, int b, const double *Dinv, const int *diag, DBsr<double> &out,
                   cudaStream_t s, Mem &mem) {
  ProfScope ps("scalar_scaling", s);
  const int E = A.nrows, nnzb = A.nnzb;
  const long long n = (long long)E * b;
  if (n > INT32_MAX) fail(NAIR_ERR_UNSUPPORTED, "scalar form: more than 2^31 - 1 unknowns");
  Mem tmp;
  tmp.s = s;
  int *brow = tmp.alloc<int>(nnzb);
  launch_pdl(k_row_of_block, dim3(grid(E)), dim3(kThreads), 0, s, E, A.rp, brow);
  NAIR_LAUNCH_CHECK();
  const long long tot = (long long)nnzb * b * b;
  double *S = tmp.alloc<double>((size_t)tot);
  launch_pdl(k_scale_blocks, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, brow, diag, Dinv, A.v, S);
  NAIR_LAUNCH_CHECK();
  int *cnt = tmp.alloc<int>(n + 1);
  launch_pdl(k_expand_scalar<false>, dim3(grid(n)), dim3(kThreads), 0, s, E, b, A.rp, A.ci, S, nullptr, cnt, nullptr, nullptr);
  NAIR_LAUNCH_CHECK();
  out.nrows = out.ncols = (int)n;
  out.rp = mem.alloc<int>(n + 1);
  const int nnz = exclusive_scan(cnt, out.rp, (int)n, s, tmp, true);
  out.nnzb = nnz;
  out.ci = mem.alloc<int>(nnz);
  out.v = mem.alloc<double>(nnz);
  launch_pdl(k_expand_scalar<true>, dim3(grid(n)), dim3(kThreads), 0, s, E, b, A.rp, A.ci, S, out.rp, nullptr, out.ci, out.v);
  NAIR_LAUNCH_CHECK();
}

}  // namespace nair
