// nAIR setup phase on the GPU (Sec. 4.1, 5.1, 5.2): diagonal-block inverses,
// strength of connection, C/F splitting, truncated Neumann Delta, restriction
// R = [-A_cf Delta  I], one-point interpolation and the coarse operator
// K = R A P with filtering, level after level.
//
// Every value upstream of a threshold (block norms, Delta, R, K) is computed
// with correctly rounded IEEE operations in one fixed order, whatever the
// launch shape: block products c_rc = fma(a_rt, b_tc, c_rc) with t ascending,
// summed over the inner block index in ascending order; squared norms
// s = fma(x, x, s) in row-major order.  Threads parallelise over output
// blocks and their scalars only, never over a summed index, so C/F splittings
// and sparsity patterns are reproducible bit for bit.
#include <algorithm>
#include <type_traits>
#include <climits>
#include <cstdio>

#include "hier.cuh"

namespace nair {

static constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// a1: diagonal-block inverses (in-place Gauss-Jordan, partial pivoting, FP64)
// One thread per block row; bpc blocks per CTA staged in shared memory.
// ---------------------------------------------------------------------------
template <typename TI>
__global__ void k_block_inverse(int nblk, int b, int bpc, const TI *__restrict__ A,
                                const int *__restrict__ pos, double *__restrict__ out,
                                int *__restrict__ err) {
  pdl_wait();
  extern __shared__ double sm[];
  const int ld = b | 1;  // odd row stride: rows of one block fall in distinct banks
  int *piv = reinterpret_cast<int *>(sm + (size_t)bpc * b * ld);
  __shared__ double rinv_s[256];
  const int lb = threadIdx.x / b, t = threadIdx.x % b;
  const long long blk = (long long)blockIdx.x * bpc + lb;
  const bool active = lb < bpc && blk < nblk;
  double *M = sm + (size_t)lb * b * ld;
  if (active) {
    const TI *src = A + (size_t)(pos ? pos[blk] : blk) * b * b;
    for (int c = 0; c < b; ++c) M[t * ld + c] = (double)src[t * b + c];
  }
  __syncthreads();
  bool sing = false;
  for (int k = 0; k < b; ++k) {
    // pivot search by one thread per block (FP64 compares are FP64-pipe work)
    if (active && t == 0) {
      int p = k;
      double best = fabs(M[k * ld + k]);
      for (int r = k + 1; r < b; ++r) {
        double a = fabs(M[r * ld + k]);
        if (a > best) { best = a; p = r; }
      }
      piv[lb * 32 + k] = p;
    }
    __syncthreads();
    const int p = active ? piv[lb * 32 + k] : k;
    if (active && p != k) {  // thread t swaps column t of rows k and p
      double tmp = M[k * ld + t];
      M[k * ld + t] = M[p * ld + t];
      M[p * ld + t] = tmp;
    }
    __syncthreads();
    const double d = active ? M[k * ld + k] : 1.0;
    if (active && (d == 0.0 || d != d)) sing = true;
    if (active && t == 0) rinv_s[lb] = __ddiv_rn(1.0, d);  // one division per step
    __syncthreads();
    if (active) {
      double v = (t == k) ? 1.0 : M[k * ld + t];
      M[k * ld + t] = __dmul_rn(v, rinv_s[lb]);
    }
    __syncthreads();
    if (active && t != k) {
      double l = M[t * ld + k];
      M[t * ld + k] = 0.0;
      for (int c = 0; c < b; ++c) M[t * ld + c] = __fma_rn(-l, M[k * ld + c], M[t * ld + c]);
    }
    __syncthreads();
  }
  if (active) {
    for (int k = b - 1; k >= 0; --k) {
      int p = piv[lb * 32 + k];
      if (p != k) {
        double tmp = M[t * ld + k];
        M[t * ld + k] = M[t * ld + p];
        M[t * ld + p] = tmp;
      }
    }
    double *dst = out + (size_t)blk * b * b;
    for (int c = 0; c < b; ++c) dst[t * b + c] = M[t * ld + c];
    if (sing) atomicOr(err, 1);
  }
}

// The same Gauss-Jordan inverse with one block per segment of SEG lanes (SEG the
// power of two >= B) and row r of the block in the registers of lane r, for
// the DG block sizes.  Every FP64 instruction occupies the scarce FP64 pipe
// whatever the number of active lanes, so everything that is not arithmetic
// on values runs on the integer pipe or through shuffles:
//   - the pivot search compares |x| as integers: for IEEE doubles with the sign
//     cleared, the bit patterns order like the values; a NaN below the
//     diagonal ranks lowest (a comparison with it is false), a NaN on the
//     diagonal highest (nothing compares greater than it);
//   - rows are exchanged logically: each lane tracks the index of the row it
//     holds, so a swap moves two integers, not two rows;
//   - the pivot row is scaled once, one element per lane, through shared memory.
// The values computed (reciprocal, products, fma chains, column order) are
// those of k_block_inverse, so both give identical bits.
template <int B>
struct SegShape {
  static constexpr int SEG = B <= 4 ? 4 : B <= 8 ? 8 : B <= 16 ? 16 : 32;
  static constexpr int NSEG = kThreads / SEG;  // blocks per CTA
  static constexpr int LD = B | 1;
  // shared memory per segment: staging (B x LD doubles), scaled pivot row (B
  // doubles), pivot rows (B ints) and the column order (2 B ints), rounded up
  // to 16 bytes so that every segment's doubles stay aligned
  static constexpr size_t BYTES = (sizeof(double) * (B * LD + B) + sizeof(int) * 3 * B + 15) / 16 * 16;
};

__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

template <int B, typename TI>
__global__ void __launch_bounds__(kThreads) k_block_inverse_seg(int nblk, const TI *__restrict__ A,
                                                                const int *__restrict__ pos,
                                                                double *__restrict__ out, int *__restrict__ err) {
  pdl_wait();
  using S = SegShape<B>;
  constexpr int SEG = S::SEG, LD = S::LD;
  extern __shared__ double smb[];
  const int seg = threadIdx.x / SEG, r = threadIdx.x % SEG;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned segmask = (SEG == 32) ? 0xffffffffu : (((1u << SEG) - 1u) << (lane & ~(unsigned)(SEG - 1)));
  unsigned char *base = reinterpret_cast<unsigned char *>(smb) + (size_t)seg * S::BYTES;
  double *stage = reinterpret_cast<double *>(base);
  double *prow = stage + B * LD;
  int *pk = reinterpret_cast<int *>(prow + B);
  int *content = pk + B, *inv = content + B;
  const long long blk = (long long)blockIdx.x * S::NSEG + seg;
  const bool have = blk < nblk;
  const bool active = have && r < B;
  // coalesced load of the block into the staging area, then row r to registers
  if (have) {
    const TI *src = A + (size_t)(pos ? pos[blk] : blk) * B * B;
    for (int e = r; e < B * B; e += SEG) stage[(e / B) * LD + e % B] = (double)src[e];
  }
  __syncwarp();
  double M[B];
#pragma unroll
  for (int c = 0; c < B; ++c) M[c] = active ? stage[r * LD + c] : 0.0;
  int li = r;  // index of the row this lane holds
  bool sing = false;
#pragma unroll
  for (int k = 0; k < B; ++k) {
    // pivot: first row (in the current order) of largest |M[.][k]| among rows >= k
    const unsigned long long a = abs_key(M[k]);
    const bool nan = a > 0x7FF0000000000000ull;
    unsigned long long key = (!active || li < k) ? 0ull : nan ? (li == k ? ~0ull : 1ull) : a + 1ull;
    int bli = li;
#pragma unroll
    for (int o = SEG / 2; o; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o, SEG);
      const int l2 = __shfl_xor_sync(0xffffffffu, bli, o, SEG);
      if (k2 > key || (k2 == key && l2 < bli)) { key = k2; bli = l2; }
    }
    const int p = bli;
    if (r == 0) pk[k] = p;
    if (li == p) li = k;
    else if (li == k) li = p;
    const bool piv = active && li == k;
    const unsigned pmask = __ballot_sync(0xffffffffu, piv) & segmask;
    const int plane = pmask ? __ffs(pmask) - 1 : (int)(lane & ~(unsigned)(SEG - 1));
    const double d = __shfl_sync(0xffffffffu, M[k], plane);
    const unsigned long long dk = abs_key(d);
    if (active && (dk == 0ull || dk > 0x7FF0000000000000ull)) sing = true;
    const double rinv = __drcp_rn(d);
    if (piv) {
#pragma unroll
      for (int c = 0; c < B; ++c) prow[c] = M[c];
    }
    __syncwarp();
    if (r < B && have) prow[r] = __dmul_rn(r == k ? 1.0 : prow[r], rinv);
    __syncwarp();
    const double l = M[k];
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const double pc = prow[c];
      const double nv = __fma_rn(-l, pc, c == k ? 0.0 : M[c]);
      M[c] = piv ? pc : nv;
    }
    __syncwarp();
  }
  // column order after undoing the row exchanges in reverse (Gauss-Jordan unscramble)
  if (r == 0 && have) {
    for (int c = 0; c < B; ++c) content[c] = c;
    for (int k = B - 1; k >= 0; --k) {
      const int p = pk[k];
      const int t = content[k];
      content[k] = content[p];
      content[p] = t;
    }
    for (int c = 0; c < B; ++c) inv[content[c]] = c;
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int c = 0; c < B; ++c) stage[li * LD + inv[c]] = M[c];
  }
  __syncwarp();
  if (have) {
    double *dst = out + (size_t)blk * B * B;
    for (int e = r; e < B * B; e += SEG) dst[e] = stage[(e / B) * LD + e % B];
  }
  const bool any = __any_sync(0xffffffffu, sing);
  if (any && r == 0 && have) atomicOr(err, 1);
}

template <int B, typename TI>
static void launch_inverse_seg(int nblk, const TI *A, const int *pos, double *out, int *err, cudaStream_t s) {
  using S = SegShape<B>;
  const size_t smem = (size_t)S::NSEG * S::BYTES;
  if (smem > 48 * 1024)
    NAIR_CK(cudaFuncSetAttribute(k_block_inverse_seg<B, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  launch_pdl(k_block_inverse_seg<B, TI>, dim3(cdiv(nblk, S::NSEG)), dim3(kThreads), smem, s, nblk, A, pos, out, err);
  NAIR_LAUNCH_CHECK();
}

template <typename TI>
void block_inverses(int nblk, int b, const TI *A, const int *pos, double *out, int *err,
                    cudaStream_t s) {
  if (nblk <= 0) return;
  switch (b) {
    case 3: launch_inverse_seg<3, TI>(nblk, A, pos, out, err, s); return;
    case 6: launch_inverse_seg<6, TI>(nblk, A, pos, out, err, s); return;
    case 10: launch_inverse_seg<10, TI>(nblk, A, pos, out, err, s); return;
    case 15: launch_inverse_seg<15, TI>(nblk, A, pos, out, err, s); return;
    case 21: launch_inverse_seg<21, TI>(nblk, A, pos, out, err, s); return;
    case 28: launch_inverse_seg<28, TI>(nblk, A, pos, out, err, s); return;
    default: break;
  }
  int bpc = std::max(1, kThreads / b);
  size_t smem = (size_t)bpc * b * (b | 1) * sizeof(double) + (size_t)bpc * 32 * sizeof(int);
  if (smem > 48 * 1024) {
    NAIR_CK(cudaFuncSetAttribute(k_block_inverse<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  }
  launch_pdl(k_block_inverse<TI>, dim3(cdiv(nblk, bpc)), dim3(bpc * b), smem, s, nblk, b, bpc, A, pos, out, err);
  NAIR_LAUNCH_CHECK();
}
template void block_inverses<double>(int, int, const double *, const int *, double *, int *, cudaStream_t);
template void block_inverses<float>(int, int, const float *, const int *, double *, int *, cudaStream_t);

// ---------------------------------------------------------------------------
// structure helpers
// ---------------------------------------------------------------------------
__global__ void k_validate(int E, int ncols, const int *__restrict__ rp, const int *__restrict__ ci,
                           int nnzb, int *__restrict__ err) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  int a = rp[i], e = rp[i + 1];
  if (a > e || a < 0 || e > nnzb) { atomicOr(err, 2); return; }
  int prev = -1;
  bool diag = false;
  for (int p = a; p < e; ++p) {
    int j = ci[p];
    if (j <= prev || j >= ncols) { atomicOr(err, 2); return; }
    prev = j;
    diag |= (j == i);
  }
  if (!diag) atomicOr(err, 4);
}

__global__ void k_diag_pos(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                           int *__restrict__ dpos) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) dpos[i] = find_sorted(ci, rp[i], rp[i + 1], i);
}

__global__ void k_block_rows(int E, const int *__restrict__ rp, int *__restrict__ brow) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) brow[p] = i;
}

template <typename TO>
__global__ void k_convert(long long n, const double *__restrict__ in, TO *__restrict__ out) {
  pdl_wait();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}

// ---------------------------------------------------------------------------
// a2: squared block norms and strength
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_norm2(const T *__restrict__ x, int bb) {
  T s = 0;
#pragma unroll 8
  for (int k = 0; k < bb; ++k) s = fma_rn(x[k], x[k], s);
  return s;
}

template <typename T>
__global__ void k_block_norm2(int nnzb, int b, const T *__restrict__ v, T *__restrict__ s) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnzb) s[p] = block_norm2(v + (size_t)p * b * b, b * b);
}

template <typename T>
__global__ void k_strength(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                           const T *__restrict__ s, T th2, unsigned char *__restrict__ strong) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  T smax = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] != i && s[p] > smax) smax = s[p];
  const T thr = mul_rn(th2, smax);
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    strong[p] = (ci[p] != i && s[p] > (T)0 && s[p] >= thr) ? 1 : 0;
}

__global__ void k_lambda(int nnzb, const int *__restrict__ ci, const unsigned char *__restrict__ strong,
                         int *__restrict__ lam) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnzb && strong[p]) atomicAdd(&lam[ci[p]], 1);
}

// ---------------------------------------------------------------------------
// a3: C/F splitting by independent-set rounds (PMIS form of classical RS)
// states: -1 undecided, 0 F, 1 C
// ---------------------------------------------------------------------------
__global__ void k_pmis_init(int E, const int *__restrict__ lam, signed char *__restrict__ st,
                            uint64_t *__restrict__ h, uint64_t seed, int *__restrict__ mark) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  st[i] = lam[i] == 0 ? 0 : -1;
  h[i] = splitmix64((uint64_t)i ^ seed);
  mark[i] = -1;
}

__device__ __forceinline__ bool key_greater(int i, int j, const int *__restrict__ lam,
                                            const uint64_t *__restrict__ h) {
  if (lam[i] != lam[j]) return lam[i] > lam[j];
  if (h[i] != h[j]) return h[i] > h[j];
  return i > j;
}

__global__ void k_pmis_mark(int nnzb, const int *__restrict__ brow, const int *__restrict__ ci,
                            const unsigned char *__restrict__ strong,
                            const signed char *__restrict__ st, const int *__restrict__ lam,
                            const uint64_t *__restrict__ h, int *__restrict__ mark, int round) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnzb || !strong[p]) return;
  int i = brow[p], j = ci[p];
  if (st[i] != -1 || st[j] != -1) return;
  if (key_greater(j, i, lam, h)) mark[i] = round;
  else mark[j] = round;
}

__global__ void k_pmis_select(int E, signed char *__restrict__ st, const int *__restrict__ mark,
                              int round) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E && st[i] == -1 && mark[i] != round) st[i] = 1;
}

__global__ void k_pmis_fmark(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                             const unsigned char *__restrict__ strong, signed char *__restrict__ st,
                             int *__restrict__ remaining) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E || st[i] != -1) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (strong[p] && st[ci[p]] == 1) {
      st[i] = 0;
      return;
    }
  atomicAdd(remaining, 1);
}

__global__ void k_cf_flags(int E, const signed char *__restrict__ cf, int *__restrict__ isc) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) isc[i] = cf[i] == 1;
}

__global__ void k_cf_index(int E, const signed char *__restrict__ cf, const int *__restrict__ pre,
                           int *__restrict__ cidx, int *__restrict__ fidx, int *__restrict__ c2f,
                           int *__restrict__ f2f) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  int c = pre[i];
  if (cf[i] == 1) {
    cidx[i] = c;
    fidx[i] = -1;
    c2f[c] = i;
  } else {
    cidx[i] = -1;
    fidx[i] = i - c;
    f2f[i - c] = i;
  }
}

// ---------------------------------------------------------------------------
// sweep work lists: the rows of one class ordered by decreasing row length, so
// that rows sharing a warp have similar trip counts (any order gives the same
// sweep result: every row is computed independently)
// ---------------------------------------------------------------------------
static constexpr int kLenBuckets = 64;

__global__ void k_len_count(int n, const int *__restrict__ list, const int *__restrict__ rp,
                            int *__restrict__ counts) {
  pdl_wait();
  __shared__ int h[kLenBuckets];
  for (int k = threadIdx.x; k < kLenBuckets; k += blockDim.x) h[k] = 0;
  __syncthreads();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const int i = list[t];
    atomicAdd(&h[min(rp[i + 1] - rp[i], kLenBuckets - 1)], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kLenBuckets; k += blockDim.x)
    if (h[k]) atomicAdd(&counts[k], h[k]);
}

// offsets of the buckets, longest rows first
__global__ void k_len_offsets(int *__restrict__ counts) {
  pdl_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int run = 0;
  for (int k = kLenBuckets - 1; k >= 0; --k) {
    const int c = counts[k];
    counts[k] = run;
    run += c;
  }
}

__global__ void k_len_scatter(int n, const int *__restrict__ list, const int *__restrict__ rp,
                              int *__restrict__ offs, int *__restrict__ out) {
  pdl_wait();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = list[t];
  out[atomicAdd(&offs[min(rp[i + 1] - rp[i], kLenBuckets - 1)], 1)] = i;
}

// ---------------------------------------------------------------------------
// a6: one-point interpolation: strongest strong C neighbour, first on ties
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_one_point(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                            const unsigned char *__restrict__ strong, const T *__restrict__ s,
                            const signed char *__restrict__ cf, const int *__restrict__ cidx,
                            int *__restrict__ ipc) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  if (cf[i] == 1) { ipc[i] = cidx[i]; return; }
  int best = -1;
  T bs = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (!strong[p] || cf[j] != 1) continue;
    if (best < 0 || s[p] > bs) { best = j; bs = s[p]; }
  }
  ipc[i] = best < 0 ? -1 : cidx[best];
}

// ---------------------------------------------------------------------------
// submatrix extraction: rows sel (rowmap), blocks whose column passes a test
// mode 0: strong F-F blocks of F rows (for L); mode 1: F columns of C rows (A_cf)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool take_block(int mode, int p, int j, const unsigned char *strong,
                                           const signed char *cf) {
  return mode == 0 ? (strong[p] && cf[j] == 0) : (cf[j] == 0);
}

__global__ void k_sub_count(int nrows, int mode, const int *__restrict__ rowmap,
                            const int *__restrict__ rp, const int *__restrict__ ci,
                            const unsigned char *__restrict__ strong,
                            const signed char *__restrict__ cf, int *__restrict__ cnt) {
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int i = rowmap[r], c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) c += take_block(mode, p, ci[p], strong, cf);
  cnt[r] = c;
}

__global__ void k_sub_fill(int nrows, int mode, const int *__restrict__ rowmap,
                           const int *__restrict__ rp, const int *__restrict__ ci,
                           const unsigned char *__restrict__ strong,
                           const signed char *__restrict__ cf, const int *__restrict__ fidx,
                           const int *__restrict__ orp, int *__restrict__ oci,
                           int *__restrict__ osrc, int *__restrict__ orow) {
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int i = rowmap[r], w = orp[r];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (!take_block(mode, p, j, strong, cf)) continue;
    oci[w] = fidx[j];
    osrc[w] = p;
    orow[w] = r;
    ++w;
  }
}

// L_ij = -(D_ii^{-1} A_ij): one block product from +0, then negated
template <typename T>
__global__ void k_L_values(long long total, int b, const int *__restrict__ orow,
                           const int *__restrict__ osrc, const int *__restrict__ rowmap,
                           const T *__restrict__ dinv, const T *__restrict__ Av, T *__restrict__ out,
                           const int *__restrict__ nblk) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long blk = g / bb;
  if (nblk && blk >= *nblk) return;  // grid sized by an upper bound
  const int rc = (int)(g - blk * bb), r = rc / b, c = rc - r * b;
  const T *d = dinv + (size_t)rowmap[orow[blk]] * bb + r * b;
  const T *a = Av + (size_t)osrc[blk] * bb + c;
  T acc = 0;
  for (int t = 0; t < b; ++t) acc = fma_rn(d[t], a[t * b], acc);
  out[g] = -acc;
}

template <typename T>
__global__ void k_copy_blocks(long long total, int b, const int *__restrict__ src,
                              const T *__restrict__ in, T *__restrict__ out,
                              const int *__restrict__ nblk = nullptr) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long blk = g / bb;
  if (nblk && blk >= *nblk) return;  // grid sized by an upper bound
  const int rc = (int)(g - blk * bb);
  out[g] = in[(size_t)src[blk] * bb + rc];
}

__global__ void k_iota(int n, int *__restrict__ a) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) a[i] = i;
}

__global__ void k_map(int n, const int *__restrict__ in, const int *__restrict__ m,
                      int *__restrict__ out) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = m[in[i]];
}

// ---------------------------------------------------------------------------
// Block sparse product  out_i = init_{imap(i)} + sum_{m in Left row i} Left_im * Right_{rmap(m)}
// symbolic: the sorted union of the right rows (and init row), by repeated
// extraction of the smallest head over per-entry cursors (thread per row).
// ---------------------------------------------------------------------------
struct SpgemmIdx {
  int nrows;
  const int *lrp, *lci, *rmap;
  const int *rrp, *rci;
  const int *irp, *ici, *imap;
  const int *rsrc;  // right entry q -> its block in the right value array (null: q)
};

template <bool FILL>
__global__ void k_spgemm_symbolic(SpgemmIdx X, int *__restrict__ cursor, int *__restrict__ cnt,
                                  const int *__restrict__ orp, int *__restrict__ oci,
                                  int *__restrict__ orow) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= X.nrows) return;
  const int l0 = X.lrp[i], l1 = X.lrp[i + 1];
  for (int p = l0; p < l1; ++p) {
    int m = X.rmap ? X.rmap[X.lci[p]] : X.lci[p];
    cursor[p] = X.rrp[m];
  }
  int icur = 0, iend = 0;
  if (X.irp) {
    int ii = X.imap ? X.imap[i] : i;
    icur = X.irp[ii];
    iend = X.irp[ii + 1];
  }
  int count = 0;
  int w = FILL ? orp[i] : 0;
  for (;;) {
    int jmin = INT_MAX;
    if (icur < iend) jmin = X.ici[icur];
    for (int p = l0; p < l1; ++p) {
      int m = X.rmap ? X.rmap[X.lci[p]] : X.lci[p];
      int cpos = cursor[p];
      if (cpos < X.rrp[m + 1]) jmin = min(jmin, X.rci[cpos]);
    }
    if (jmin == INT_MAX) break;
    if (FILL) {
      oci[w] = jmin;
      orow[w] = i;
      ++w;
    }
    ++count;
    if (icur < iend && X.ici[icur] == jmin) ++icur;
    for (int p = l0; p < l1; ++p) {
      int m = X.rmap ? X.rmap[X.lci[p]] : X.lci[p];
      int cpos = cursor[p];
      if (cpos < X.rrp[m + 1] && X.rci[cpos] == jmin) cursor[p] = cpos + 1;
    }
  }
  if (!FILL) cnt[i] = count;
}

// numeric phase: one thread per output scalar (block, r, c); one fma chain over
// (left entry m ascending, t ascending); the init block (if any) is the start value
template <typename T>
__global__ void k_spgemm_numeric(long long total, int b, SpgemmIdx X, const T *__restrict__ lv,
                                 const T *__restrict__ rv, const T *__restrict__ iv,
                                 const int *__restrict__ orow, const int *__restrict__ oci,
                                 int negate, T *__restrict__ ov) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long blk = g / bb;
  const int rc = (int)(g - blk * bb), r = rc / b, c = rc - r * b;
  const int i = orow[blk], j = oci[blk];
  T acc = 0;
  if (X.irp) {
    int ii = X.imap ? X.imap[i] : i;
    int q = find_sorted(X.ici, X.irp[ii], X.irp[ii + 1], j);
    if (q >= 0) acc = iv[(size_t)q * bb + rc];
  }
  for (int p = X.lrp[i]; p < X.lrp[i + 1]; ++p) {
    int m = X.rmap ? X.rmap[X.lci[p]] : X.lci[p];
    int q = find_sorted(X.rci, X.rrp[m], X.rrp[m + 1], j);
    if (q < 0) continue;
    const T *a = lv + (size_t)p * bb + r * b;
    const T *bv = rv + (size_t)(X.rsrc ? X.rsrc[q] : q) * bb + c;
    for (int t = 0; t < b; ++t) acc = fma_rn(a[t], bv[t * b], acc);
  }
  ov[g] = negate ? -acc : acc;
}

// Warp-per-row form of the same product.  The lanes own the row's left entries
// (32 per chunk, at most kMergeChunks chunks) and keep one cursor each into the
// sorted right row it selects; every step the warp takes the smallest head
// column (the next output column), records which entries meet it -- in
// ascending left-entry order, the order of the canonical sum -- and advances
// them.  COUNT gives the output and product counts of each row; FILL writes the
// output columns, each output's slice of (left entry, right entry) pairs, and
// the position of its start value in the init row (or -1).  A row with more
// left entries than the warp holds raises `overflow` (the caller then uses the
// thread-per-row kernels above).
static constexpr int kMergeChunks = 8;

template <bool FILL>
__global__ void k_spgemm_warp(SpgemmIdx X, int *__restrict__ cnt, int *__restrict__ pcnt,
                              const int *__restrict__ orp, const int *__restrict__ prp,
                              int *__restrict__ oci, int *__restrict__ orow, int *__restrict__ pbeg,
                              int2 *__restrict__ pairs, int *__restrict__ iq, int *__restrict__ overflow) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= X.nrows) return;  // uniform across the warp
  const int l0 = X.lrp[i], l1 = X.lrp[i + 1];
  if (l1 - l0 > 32 * kMergeChunks) {
    if (lane == 0) {
      atomicOr(overflow, 1);
      if (!FILL) { cnt[i] = 0; pcnt[i] = 0; }
    }
    return;
  }
  int cur[kMergeChunks], end[kMergeChunks];
#pragma unroll
  for (int c = 0; c < kMergeChunks; ++c) {
    const int p = l0 + c * 32 + lane;
    cur[c] = end[c] = 0;
    if (p < l1) {
      const int m = X.rmap ? X.rmap[X.lci[p]] : X.lci[p];
      cur[c] = X.rrp[m];
      end[c] = X.rrp[m + 1];
    }
  }
  int icur = 0, iend = 0;
  if (X.irp && lane == 0) {
    const int ii = X.imap ? X.imap[i] : i;
    icur = X.irp[ii];
    iend = X.irp[ii + 1];
  }
  int nout = 0, pw = FILL ? prp[i] : 0, w = FILL ? orp[i] : 0;
  for (;;) {
    int h = INT_MAX;
#pragma unroll
    for (int c = 0; c < kMergeChunks; ++c)
      if (cur[c] < end[c]) h = min(h, X.rci[cur[c]]);
    if (icur < iend) h = min(h, X.ici[icur]);
    const int jmin = __reduce_min_sync(0xffffffffu, h);
    if (jmin == INT_MAX) break;
    const int im = (icur < iend && X.ici[icur] == jmin) ? icur : -1;
    if (FILL && lane == 0) {
      oci[w] = jmin;
      orow[w] = i;
      pbeg[w] = pw;
      iq[w] = im;
    }
#pragma unroll
    for (int c = 0; c < kMergeChunks; ++c) {
      const bool mt = cur[c] < end[c] && X.rci[cur[c]] == jmin;
      const unsigned ball = __ballot_sync(0xffffffffu, mt);
      if (FILL && mt)
        pairs[pw + __popc(ball & ((1u << lane) - 1u))] = make_int2(l0 + c * 32 + lane, X.rsrc ? X.rsrc[cur[c]] : cur[c]);
      pw += __popc(ball);
      if (mt) ++cur[c];
    }
    if (im >= 0) ++icur;
    ++w;
    ++nout;
  }
  if (!FILL && lane == 0) {
    cnt[i] = nout;
    pcnt[i] = pw;
  }
}

// numeric phase over the recorded pairs: the start value, then one fma chain over
// the pairs in order (left entry ascending) and t ascending.  B = 0 takes the
// block size b at run time, with eight thread blocks per SM (register cap 32):
// the chains wait on loads, and the extra resident warps gained more than the
// spilled registers cost (C5 FP64 setup with Neumann degree 6: 96.3 -> 92.9
// ms).  For B > 0 the index arithmetic divides by constants and each pair's 2B
// loads are issued before its fma chain, the next pair's indices one pair
// ahead; six thread blocks per SM keep it free of spills (C5 FP64 setup 93.8
// -> 93.1 ms, two boxes; 60 registers and four blocks per SM: 96.1 ms).  With
// masks, a pair takes only the inner indices t where column t of its left
// block and row t of its right block hold a nonzero: the skipped terms are
// exact zeros (finite operands), so each sum is unchanged but for the sign of
// a zero.  The coupling blocks of the DG operator are nonzero only on the
// shared face, and that structure persists down the hierarchy (C5, 32x32x2
// mesh: 40 % of L's and A_cf's level-0 terms kept, 48-72 % of the Galerkin
// product's on every level); C5 FP64 setup 93.0 -> 85.0 ms
template <typename T, int B>
__global__ void __launch_bounds__(256, B ? 6 : 8) k_spgemm_pairs(long long total, int b_rt,
                               const int *__restrict__ pbeg, const int2 *__restrict__ pairs,
                               const int *__restrict__ iq, const T *__restrict__ lv,
                               const T *__restrict__ rv, const T *__restrict__ iv, int negate,
                               T *__restrict__ ov, const unsigned *__restrict__ lmask,
                               const unsigned *__restrict__ rmask) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int b = B ? B : b_rt;
  const int bb = b * b;
  const long long blk = g / bb;
  const int rc = (int)(g - blk * bb), r = rc / b, c = rc - r * b;
  const int q0 = iq[blk];
  T acc = q0 >= 0 ? iv[(size_t)q0 * bb + rc] : (T)0;
  int k = pbeg[blk];
  const int k1 = pbeg[blk + 1];
  if constexpr (B > 0) {
    constexpr unsigned kFull = (1u << B) - 1u;
    int2 pq = k < k1 ? pairs[k] : make_int2(0, 0);
    for (; k < k1; ++k) {
      const T *a = lv + (size_t)pq.x * bb + r * B;
      const T *bv = rv + (size_t)pq.y * bb + c;
      // inner indices t with a nonzero in column t of the left block and in
      // row t of the right one; the others add exact zeros
      const unsigned m = (lmask ? lmask[pq.x] : kFull) & (rmask ? rmask[pq.y] >> 16 : kFull) & kFull;
      if (m == kFull) {
        T av[B], bw[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
          av[t] = a[t];
          bw[t] = bv[t * B];
        }
        if (k + 1 < k1) pq = pairs[k + 1];
#pragma unroll
        for (int t = 0; t < B; ++t) acc = fma_rn(av[t], bw[t], acc);
      } else if (m) {
        if (k + 1 < k1) pq = pairs[k + 1];
        // the next term's operands are loaded while the current one is added
        unsigned mm = m;
        int t = __ffs(mm) - 1;
        T an = a[t], bn = bv[t * B];
        for (mm &= mm - 1u; mm; mm &= mm - 1u) {
          const T ac = an, bc = bn;
          t = __ffs(mm) - 1;
          an = a[t];
          bn = bv[t * B];
          acc = fma_rn(ac, bc, acc);
        }
        acc = fma_rn(an, bn, acc);
      } else if (k + 1 < k1) {
        pq = pairs[k + 1];
      }
    }
  } else {
    for (; k < k1; ++k) {
      const int2 pq = pairs[k];
      const T *a = lv + (size_t)pq.x * bb + r * b;
      const T *bv = rv + (size_t)pq.y * bb + c;
      for (int t = 0; t < b; ++t) acc = fma_rn(a[t], bv[t * b], acc);
    }
  }
  ov[g] = negate ? -acc : acc;
}

// position of the (n + 1)-th set bit of m (n < popcount(m))
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  for (int i = 0; i < n; ++i) m &= m - 1u;
  return __ffs(m) - 1;
}

// Warp per output block, for products whose left blocks have zero rows (R_cf,
// A_cf): the block's b x b sums stay in shared memory, and for each pair the
// lanes take the outputs (r, c) with r a nonzero row of the left block and c
// a nonzero column of the right block, ceil(nr nc / 32) at a time, each an
// fma chain over the inner indices of the pair's mask.  Each output sees the
// same nonzero terms in the same order as in k_spgemm_pairs (pairs in order,
// t ascending); the terms left out are exact zeros.  lmask is required.  The
// blocks of R_cf and A_cf keep about 60 % of their rows zero (the rows of
// element DOFs off the shared faces), which the thread-per-output form can
// skip only where a whole warp's rows are zero (about 12 % of the 4-row
// windows); here a pair costs ceil(nr nc / 32) fma chains instead of about
// three.  C5 FP64 setup 84.9 -> 77.0 ms (the Neumann products, whose L
// blocks have full rows, stay with k_spgemm_pairs).
template <typename T, int B>
__global__ void __launch_bounds__(256) k_spgemm_wblk(int nblk, const int *__restrict__ pbeg,
                                                     const int2 *__restrict__ pairs, const int *__restrict__ iq,
                                                     const T *__restrict__ lv, const T *__restrict__ rv,
                                                     const T *__restrict__ iv, int negate, T *__restrict__ ov,
                                                     const unsigned *__restrict__ lmask,
                                                     const unsigned *__restrict__ rmask) {
  pdl_wait();
  constexpr int bb = B * B;
  constexpr unsigned kFull = (1u << B) - 1u;
  __shared__ T sacc[8][bb];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int blk = blockIdx.x * 8 + wid;
  if (blk >= nblk) return;  // the whole warp; no block-wide barrier follows
  T *acc = sacc[wid];
  const int q0 = iq[blk];
  for (int rc = lane; rc < bb; rc += 32) acc[rc] = q0 >= 0 ? iv[(size_t)q0 * bb + rc] : (T)0;
  __syncwarp();
  const int k1 = pbeg[blk + 1];
  for (int k = pbeg[blk]; k < k1; ++k) {
    const int2 pq = pairs[k];
    const unsigned ml = lmask[pq.x], mr = rmask ? rmask[pq.y] : (kFull | (kFull << 16));
    const unsigned tm = ml & (mr >> 16) & kFull;
    const unsigned rows = (ml >> 16) & kFull, cols = mr & kFull;
    const int nc = __popc(cols), nw = __popc(rows) * nc;
    if (tm) {
      const T *a0 = lv + (size_t)pq.x * bb, *b0 = rv + (size_t)pq.y * bb;
      for (int idx = lane; idx < nw; idx += 32) {
        const int ri = idx / nc, ci = idx - ri * nc;
        const int r = nth_set_bit(rows, ri), c = nth_set_bit(cols, ci);
        T sum = acc[r * B + c];
        for (unsigned mm = tm; mm; mm &= mm - 1u) {
          const int t = __ffs(mm) - 1;
          sum = fma_rn(a0[r * B + t], b0[t * B + c], sum);
        }
        acc[r * B + c] = sum;
      }
    }
    __syncwarp();
  }
  for (int rc = lane; rc < bb; rc += 32) ov[(size_t)blk * bb + rc] = negate ? -acc[rc] : acc[rc];
}

// nonzero pattern of each b x b block (b <= 16): bit c for a nonzero in
// column c, bit 16 + r for one in row r.  Thread per block row; blocks from
// *nblk on (when given) are skipped.  mask must be zero on entry.
template <typename T>
__global__ void k_block_masks(long long rows, int b, const T *__restrict__ v, const int *__restrict__ nblk,
                              unsigned *__restrict__ mask) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= rows) return;
  const long long blk = g / b;
  if (nblk && blk >= *nblk) return;
  const int r = (int)(g - blk * b);
  const T *row = v + (size_t)g * b;
  unsigned cols = 0;
  for (int c = 0; c < b; ++c)
    if (row[c] != (T)0) cols |= 1u << c;
  if (cols) atomicOr(&mask[blk], cols | (1u << (16 + r)));
}

// the masks of k_block_masks for up to cap blocks (null where the pair kernel
// takes no masks: FP32, or b not 3, 6 or 10)
template <typename T>
static unsigned *block_masks(int b, int cap, const T *v, const int *nblk, cudaStream_t s, Mem &tmp) {
  if (sizeof(T) != 8 || !(b == 3 || b == 6 || b == 10) || cap <= 0) return nullptr;
  unsigned *m = tmp.alloc<unsigned>(cap);
  NAIR_CK(cudaMemsetAsync(m, 0, sizeof(unsigned) * cap, s));
  launch_pdl(k_block_masks<T>, dim3(std::max(1, cdiv((long long)cap * b, kThreads))), dim3(kThreads), 0, s, (long long)cap * b, b, v, nblk, m);
  NAIR_LAUNCH_CHECK();
  return m;
}

// The same products with one thread per output block row (DG blocks up to
// 10): thread (blk, r) keeps the B scalars (r, c) of its row as B independent
// fma chains, loads row r of each pair's left block once and streams the right
// block row by row, so every FP64 instruction has B-fold independence and each
// value loaded feeds B or 1 products.  Each scalar's chain is the one above
// (the pairs in order, t ascending), so the results are bitwise equal.
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) k_spgemm_rows(long long total, const int *__restrict__ pbeg,
                                                          const int2 *__restrict__ pairs, const int *__restrict__ iq,
                                                          const T *__restrict__ lv, const T *__restrict__ rv,
                                                          const T *__restrict__ iv, int negate, T *__restrict__ ov) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (output block, row)
  if (g >= total) return;
  constexpr int bb = B * B;
  const long long blk = g / B;
  const int r = (int)(g - blk * B);
  const int q0 = iq[blk];
  T acc[B];
  if (q0 >= 0) {
    const T *s0 = iv + (size_t)q0 * bb + r * B;
#pragma unroll
    for (int c = 0; c < B; ++c) acc[c] = s0[c];
  } else {
#pragma unroll
    for (int c = 0; c < B; ++c) acc[c] = (T)0;
  }
  const int k1 = pbeg[blk + 1];
  for (int k = pbeg[blk]; k < k1; ++k) {
    const int2 pq = pairs[k];
    const T *a = lv + (size_t)pq.x * bb + r * B;
    const T *bm = rv + (size_t)pq.y * bb;
    T av[B];
#pragma unroll
    for (int t = 0; t < B; ++t) av[t] = a[t];
#pragma unroll
    for (int t = 0; t < B; ++t) {
      T br[B];
#pragma unroll
      for (int c = 0; c < B; ++c) br[c] = bm[t * B + c];
#pragma unroll
      for (int c = 0; c < B; ++c) acc[c] = fma_rn(av[t], br[c], acc[c]);
    }
  }
  T *o = ov + (size_t)blk * bb + r * B;
#pragma unroll
  for (int c = 0; c < B; ++c) o[c] = negate ? -acc[c] : acc[c];
}

// ---------------------------------------------------------------------------
// a8: filtering.  Drop X_ij (j != i) when ||X_ij||^2 <= tol^2 ||X_ii||^2
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_filter_flags(int nrows, const int *__restrict__ rp, const int *__restrict__ ci,
                               const T *__restrict__ nrm, T tol2, int *__restrict__ newpos,
                               int *__restrict__ cnt) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  T dn = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) dn = nrm[p];
  const T thr = mul_rn(tol2, dn);
  int k = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    bool keep = ci[p] == i || !(nrm[p] <= thr);
    newpos[p] = keep ? k++ : -1;
  }
  cnt[i] = k;
}

__global__ void k_filter_compact(int nrows, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const int *__restrict__ newpos, const int *__restrict__ nrp,
                                 int *__restrict__ nci, int *__restrict__ src) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = newpos[p];
    if (k < 0) continue;
    nci[nrp[i] + k] = ci[p];
    src[nrp[i] + k] = p;
  }
}

// ---------------------------------------------------------------------------
// a7: A P by column merge: (AP)_{r,J} = sum over j ascending with ipc(j) = J of A_rj
// ---------------------------------------------------------------------------
__global__ void k_ap_count(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                           const int *__restrict__ ipc, int *__restrict__ cnt) {
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= E) return;
  int c = 0;
  for (int p = rp[r]; p < rp[r + 1]; ++p) {
    int J = ipc[ci[p]];
    if (J < 0) continue;
    bool dup = false;
    for (int q = rp[r]; q < p && !dup; ++q) dup = ipc[ci[q]] == J;
    c += !dup;
  }
  cnt[r] = c;
}

// The blocks of row r of AP in ascending column J; for each, first[w] is the
// first block p of A's row r with ipc[ci[p]] = J, and next[p] links the
// following ones in ascending p (-1 ends a list), the order of the sum
__global__ void k_ap_fill(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                          const int *__restrict__ ipc, const int *__restrict__ orp,
                          int *__restrict__ oci, int *__restrict__ first, int *__restrict__ next) {
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= E) return;
  int w = orp[r], last = -1;
  for (;;) {
    int jmin = INT_MAX;
    for (int p = rp[r]; p < rp[r + 1]; ++p) {
      int J = ipc[ci[p]];
      if (J > last && J < jmin) jmin = J;
    }
    if (jmin == INT_MAX) break;
    oci[w] = jmin;
    int prev = -1;
    for (int p = rp[r]; p < rp[r + 1]; ++p) {
      if (ipc[ci[p]] != jmin) continue;
      if (prev < 0) first[w] = p;
      else next[prev] = p;
      prev = p;
    }
    next[prev] = -1;
    ++w;
    last = jmin;
  }
}

// AP values: each output scalar adds its A blocks along the list of k_ap_fill
// (ascending p, the sum's order), with no search of the row (C5 FP64 setup
// 74.2 -> 71.9 ms against scanning the row for each output scalar)
template <typename T>
__global__ void k_ap_values(long long total, int b, const int *__restrict__ first, const int *__restrict__ next,
                            const T *__restrict__ Av, T *__restrict__ out, const int *__restrict__ nblk) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long blk = g / bb;
  if (blk >= *nblk) return;  // grid sized by an upper bound
  const int rc = (int)(g - blk * bb);
  int p = first[blk];
  T acc = Av[(size_t)p * bb + rc];
  for (p = next[p]; p >= 0; p = next[p]) acc = add_rn(acc, Av[(size_t)p * bb + rc]);
  out[g] = acc;
}

// ---------------------------------------------------------------------------
// a9: coarsest level: dense matrix and its inverse (single CTA Gauss-Jordan)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_dense_fill(long long total, int b, int n, const int *__restrict__ brow,
                             const int *__restrict__ ci, const T *__restrict__ v,
                             double *__restrict__ M) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bb = b * b;
  const long long blk = g / bb;
  const int rc = (int)(g - blk * bb), r = rc / b, c = rc - r * b;
  M[(size_t)(brow[blk] * b + r) * n + ci[blk] * b + c] = (double)v[g];
}

static constexpr int kGjThreads = 1024;

// in-place Gauss-Jordan with partial pivoting on an n x n matrix held by one
// thread block (in shared or global memory); same arithmetic as the block inverse
// pivot-search key of |x| in row r of pivot column k: IEEE bit patterns of
// non-negative doubles order like the values, so the search runs on the
// integer pipe; a NaN ranks lowest below the diagonal (a comparison with it is
// false) and highest on it (nothing compares greater); 0 marks no candidate
__device__ __forceinline__ unsigned long long pivot_key(double x, bool diag) {
  const unsigned long long a = abs_key(x);
  return a > 0x7FF0000000000000ull ? (diag ? ~0ull : 1ull) : a + 1ull;
}

// (key, row) pair with the larger key, the smaller row on ties
__device__ __forceinline__ void pivot_max(unsigned long long &key, int &row, unsigned long long k2, int r2) {
  if (k2 > key || (k2 == key && r2 < row)) {
    key = k2;
    row = r2;
  }
}

__device__ void dense_gj_cta(int n, double *__restrict__ M, int *__restrict__ piv,
                             double *__restrict__ lcol, int *__restrict__ err) {
  __shared__ unsigned long long rv[kGjThreads / 32];
  __shared__ int ri[kGjThreads / 32];
  __shared__ int pk;
  __shared__ double dk;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    // pivot: first row of largest |M[r][k]|, r >= k (integer keys, two shuffle levels)
    unsigned long long key = 0;
    int bi = n;
    for (int r = k + tid; r < n; r += blockDim.x) pivot_max(key, bi, pivot_key(M[(size_t)r * n + k], r == k), r);
    for (int o = 16; o; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
      const int r2 = __shfl_xor_sync(0xffffffffu, bi, o);
      pivot_max(key, bi, k2, r2);
    }
    if (lane == 0) {
      rv[wid] = key;
      ri[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
      key = lane < nw ? rv[lane] : 0ull;
      bi = lane < nw ? ri[lane] : n;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, bi, o);
        pivot_max(key, bi, k2, r2);
      }
      if (lane == 0) {
        pk = bi;
        piv[k] = bi;
      }
    }
    __syncthreads();
    const int p = pk;
    if (p != k)
      for (int c = tid; c < n; c += blockDim.x) {
        double t = M[(size_t)k * n + c];
        M[(size_t)k * n + c] = M[(size_t)p * n + c];
        M[(size_t)p * n + c] = t;
      }
    __syncthreads();
    if (tid == 0) {
      dk = M[(size_t)k * n + k];
      if (dk == 0.0 || dk != dk) *err = 1;
      dk = __ddiv_rn(1.0, dk);  // reciprocal of the pivot
    }
    __syncthreads();
    const double rinv = dk;
    for (int c = tid; c < n; c += blockDim.x) {
      double v = (c == k) ? 1.0 : M[(size_t)k * n + c];
      M[(size_t)k * n + c] = __dmul_rn(v, rinv);
    }
    for (int r = tid; r < n; r += blockDim.x) {
      lcol[r] = (r == k) ? 0.0 : M[(size_t)r * n + k];
      if (r != k) M[(size_t)r * n + k] = 0.0;
    }
    __syncthreads();
    {
      const int lane32 = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      for (int r = warp; r < n; r += nw) {
        if (r == k) continue;
        const double l = lcol[r];
        double *row = M + (size_t)r * n;
        const double *prw = M + (size_t)k * n;
        for (int c = lane32; c < n; c += 32) row[c] = __fma_rn(-l, prw[c], row[c]);
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k)
      for (int r = tid; r < n; r += blockDim.x) {
        double t = M[(size_t)r * n + k];
        M[(size_t)r * n + k] = M[(size_t)r * n + p];
        M[(size_t)r * n + p] = t;
      }
    __syncthreads();
  }
}

// the same, with the matrix staged in shared memory (small coarsest levels)
__global__ void __launch_bounds__(kGjThreads) k_dense_gj_smem(int n, double *__restrict__ Mg, int *__restrict__ err) {
  pdl_wait();
  extern __shared__ double sm[];
  double *M = sm, *lcol = sm + (size_t)n * n;
  int *piv = reinterpret_cast<int *>(lcol + n);
  for (long long g = threadIdx.x; g < (long long)n * n; g += blockDim.x) M[g] = Mg[g];
  __syncthreads();
  dense_gj_cta(n, M, piv, lcol, err);
  for (long long g = threadIdx.x; g < (long long)n * n; g += blockDim.x) Mg[g] = M[g];
}

// Larger coarsest matrices: one launch per Gauss-Jordan step k, Min -> Mout,
// the same arithmetic as the in-place single-CTA form.  Every thread block
// finds the pivot of column k itself (first row with the largest |entry|),
// reads the pivot row through the row swap k <-> p, scales it once per column
// into shared memory and updates its tile.
static constexpr int kGjTileRows = 16, kGjTileCols = 256;

__global__ void __launch_bounds__(256) k_gj_step(int n, int k, const double *__restrict__ Min,
                                                 double *__restrict__ Mout, int *__restrict__ piv,
                                                 int *__restrict__ err) {
  __shared__ unsigned long long rv[8];
  __shared__ int ri[8];
  __shared__ int sp;
  __shared__ double prow[kGjTileCols];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  pdl_wait();  // Min is the previous step's output, Mout its input
  unsigned long long key = 0;
  int bi = n;
  for (int r = k + tid; r < n; r += blockDim.x) pivot_max(key, bi, pivot_key(Min[(size_t)r * n + k], r == k), r);
  for (int o = 16; o; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, bi, o);
    pivot_max(key, bi, k2, r2);
  }
  if (lane == 0) { rv[wid] = key; ri[wid] = bi; }
  __syncthreads();
  if (tid == 0) {
    unsigned long long k0 = rv[0];
    int i0 = ri[0];
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) pivot_max(k0, i0, rv[w], ri[w]);
    sp = i0;
  }
  __syncthreads();
  const int p = sp;
  const double d = Min[(size_t)p * n + k];
  if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
    piv[k] = p;
    if (d == 0.0 || d != d) *err = 1;
  }
  const int r0 = blockIdx.y * kGjTileRows, c0 = blockIdx.x * kGjTileCols;
  const double rinv = __ddiv_rn(1.0, d);
  for (int c = tid; c < kGjTileCols; c += blockDim.x) {
    const int cc = c0 + c;
    if (cc < n) prow[c] = __dmul_rn(cc == k ? 1.0 : Min[(size_t)p * n + cc], rinv);
  }
  __syncthreads();
  for (int idx = tid; idx < kGjTileRows * kGjTileCols; idx += blockDim.x) {
    const int r = r0 + idx / kGjTileCols, c = c0 + idx % kGjTileCols;
    if (r >= n || c >= n) continue;
    if (r == k) {
      Mout[(size_t)k * n + c] = prow[c - c0];
      continue;
    }
    const int src = (r == p) ? k : r;
    const double l = Min[(size_t)src * n + k];
    const double a = (c == k) ? 0.0 : Min[(size_t)src * n + c];
    Mout[(size_t)r * n + c] = __fma_rn(-l, prow[c - c0], a);
  }
}

// undo the row interchanges as column swaps, last step first
__global__ void __launch_bounds__(1024) k_gj_unscramble(int n, double *__restrict__ M, const int *__restrict__ piv) {
  pdl_wait();
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double t = M[(size_t)r * n + k];
        M[(size_t)r * n + k] = M[(size_t)r * n + p];
        M[(size_t)r * n + p] = t;
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// level-0 column compression of the off-diagonal blocks
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_colmask(int nnzb, int b, const int *__restrict__ brow, const int *__restrict__ diag,
                          const T *__restrict__ v, unsigned *__restrict__ mask, int *__restrict__ wmax) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnzb) return;
  if (diag[brow[p]] == p) { mask[p] = 0; return; }
  const T *x = v + (size_t)p * b * b;
  unsigned m = 0;
  for (int r = 0; r < b; ++r)
    for (int c = 0; c < b; ++c)
      if (x[r * b + c] != (T)0) m |= 1u << c;
  mask[p] = m;
  atomicMax(wmax, __popc(m));
}

template <typename T>
__global__ void k_comp_fill(int nnzb, int b, int W, const int *__restrict__ brow, const int *__restrict__ diag,
                            const int *__restrict__ ci, const T *__restrict__ v, const unsigned *__restrict__ mask,
                            int *__restrict__ oci, unsigned long long *__restrict__ ocols, T *__restrict__ ov) {
  pdl_wait();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnzb) return;
  const int i = brow[p], d = diag[i];
  if (p == d) return;
  const int q = p - i - (p > d ? 1 : 0);
  unsigned m = mask[p];
  int cols[32];
  int w = 0;
  for (int c = 0; c < b && w < W; ++c)
    if (m & (1u << c)) cols[w++] = c;
  for (int c = 0; c < b && w < W; ++c)  // pad with columns that are zero in this block
    if (!(m & (1u << c))) cols[w++] = c;
  unsigned long long packed = 0;
  for (int k = 0; k < W; ++k) packed |= (unsigned long long)cols[k] << (8 * k);
  oci[q] = ci[p];
  ocols[q] = packed;
  const T *x = v + (size_t)p * b * b;
  T *o = ov + (size_t)q * b * W;
  for (int r = 0; r < b; ++r)
    for (int k = 0; k < W; ++k) o[r * W + k] = x[r * b + cols[k]];
}

static inline int grid1d(long long n) { return std::max(1, cdiv(n, kThreads)); }

static bool l0_supported(int b, int W) {
  return (b == 3 && W == 2) || (b == 6 && W == 3) || (b == 10 && W == 4) || (b == 15 && W == 5) ||
         (b == 21 && W == 6) || (b == 28 && W == 7);
}

template <typename T>
void build_l0comp(const DBsr<T> &A, const int *diag, int b, cudaStream_t s, Mem &mem, L0Comp<T> &C) {
  C = L0Comp<T>();
  const int E = A.nrows, nnzb = A.nnzb, noff = nnzb - E;
  if (noff <= 0) return;
  Mem tmp;
  tmp.s = s;
  int *brow = tmp.alloc<int>(nnzb), *wmax = tmp.alloc<int>(1);
  unsigned *mask = tmp.alloc<unsigned>(nnzb);
  NAIR_CK(cudaMemsetAsync(wmax, 0, sizeof(int), s));
  launch_pdl(k_block_rows, dim3(grid1d(E)), dim3(kThreads), 0, s, E, A.rp, brow);
  NAIR_LAUNCH_CHECK();
  launch_pdl(k_colmask<T>, dim3(grid1d(nnzb)), dim3(kThreads), 0, s, nnzb, b, brow, diag, A.v, mask, wmax);
  NAIR_LAUNCH_CHECK();
  int W = read_int(wmax, s);
  if (W == 0) W = 1;
  for (int w = W; w < b; ++w)
    if (l0_supported(b, w)) { W = w; break; }
  if (!l0_supported(b, W)) return;
  C.W = W;
  C.oci = mem.alloc<int>(noff);
  C.ocols = mem.alloc<unsigned long long>(noff);
  C.ov = mem.alloc<T>((size_t)noff * b * W);
  launch_pdl(k_comp_fill<T>, dim3(grid1d(nnzb)), dim3(kThreads), 0, s, nnzb, b, W, brow, diag, A.ci, A.v, mask, C.oci, C.ocols, C.ov);
  NAIR_LAUNCH_CHECK();
}
template void build_l0comp<double>(const DBsr<double> &, const int *, int, cudaStream_t, Mem &, L0Comp<double> &);
template void build_l0comp<float>(const DBsr<float> &, const int *, int, cudaStream_t, Mem &, L0Comp<float> &);

// row of every compressed off-diagonal block: row i owns q in [rp[i] - i, rp[i + 1] - i - 1)
__global__ void k_l0_qrow(int E, const int *__restrict__ rp, int *__restrict__ qrow) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  for (int q = rp[i] - i; q < rp[i + 1] - i - 1; ++q) qrow[q] = i;
}

// sv[q][r][w] = sum_t dinv[i][r][t] ov[q][t][w], accumulated in FP64
template <typename T>
__global__ void k_l0_scale(long long total, int b, int W, const int *__restrict__ qrow, const T *__restrict__ dinv,
                           const T *__restrict__ ov, T *__restrict__ sv) {
  pdl_wait();
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int bw = b * W;
  const long long q = g / bw;
  const int rw = (int)(g - q * bw), r = rw / W, w = rw - r * W;
  const T *d = dinv + (size_t)qrow[q] * b * b + (size_t)r * b;
  const T *o = ov + (size_t)q * bw + w;
  double acc = 0.0;
  for (int t = 0; t < b; ++t) acc = fma((double)d[t], (double)o[(size_t)t * W], acc);
  sv[g] = (T)acc;
}

template <typename T>
void build_l0scaled(const DBsr<T> &A, const T *dinv, int b, cudaStream_t s, Mem &mem, L0Comp<T> &C) {
  if (C.W <= 0) return;
  const int E = A.nrows, noff = A.nnzb - E;
  Mem tmp;
  tmp.s = s;
  int *qrow = tmp.alloc<int>(noff);
  launch_pdl(k_l0_qrow, dim3(grid1d(E)), dim3(kThreads), 0, s, E, A.rp, qrow);
  NAIR_LAUNCH_CHECK();
  const long long tot = (long long)noff * b * C.W;
  C.sv = mem.alloc<T>((size_t)tot);
  launch_pdl(k_l0_scale<T>, dim3(grid1d(tot)), dim3(kThreads), 0, s, tot, b, C.W, qrow, dinv, C.ov, C.sv);
  NAIR_LAUNCH_CHECK();
}
template void build_l0scaled<double>(const DBsr<double> &, const double *, int, cudaStream_t, Mem &, L0Comp<double> &);
template void build_l0scaled<float>(const DBsr<float> &, const float *, int, cudaStream_t, Mem &, L0Comp<float> &);

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static inline int grid(long long n) { return std::max(1, cdiv(n, kThreads)); }

template <typename T>
static void spgemm_rowwise(int b, const SpgemmIdx &X, int left_nnz, const T *lv, const T *rv,
                           const T *iv, int negate, int ncols, cudaStream_t s, Mem &mem, Mem &tmp,
                           DBsr<T> &out) {
  const int nrows = X.nrows;
  int *cursor = tmp.alloc<int>(left_nnz + 1);
  int *cnt = tmp.alloc<int>(nrows + 1);
  out.nrows = nrows;
  out.ncols = ncols;
  out.rp = mem.alloc<int>(nrows + 1);
  launch_pdl(k_spgemm_symbolic<false>, dim3(grid(nrows)), dim3(kThreads), 0, s, X, cursor, cnt, nullptr, nullptr, nullptr);
  NAIR_LAUNCH_CHECK();
  out.nnzb = exclusive_scan(cnt, out.rp, nrows, s, tmp);
  out.ci = mem.alloc<int>(out.nnzb);
  int *orow = tmp.alloc<int>(out.nnzb);
  launch_pdl(k_spgemm_symbolic<true>, dim3(grid(nrows)), dim3(kThreads), 0, s, X, cursor, nullptr, out.rp, out.ci, orow);
  NAIR_LAUNCH_CHECK();
  out.v = mem.alloc<T>((size_t)out.nnzb * b * b);
  long long total = (long long)out.nnzb * b * b;
  if (total) {
    launch_pdl(k_spgemm_numeric<T>, dim3(grid(total)), dim3(kThreads), 0, s, total, b, X, lv, rv, iv, orow, out.ci,
                                                        negate, out.v);
    NAIR_LAUNCH_CHECK();
  }
  tmp.release(orow);
  tmp.release(cnt);
  tmp.release(cursor);
}

template <typename T>
static void spgemm(int b, const SpgemmIdx &X, int left_nnz, const T *lv, const T *rv, const T *iv,
                   int negate, int ncols, cudaStream_t s, Mem &mem, Mem &tmp, DBsr<T> &out,
                   const unsigned *lmask = nullptr, const unsigned *rmask = nullptr, bool by_block = false) {
  ProfScope ps("spgemm", s);
  const int nrows = X.nrows;
  int *cnt = tmp.alloc<int>(nrows + 1), *pcnt = tmp.alloc<int>(nrows + 1);
  int *prp = tmp.alloc<int>(nrows + 1), *flags = tmp.alloc<int>(4);
  NAIR_CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
  const int wblocks = std::max(1, cdiv((long long)nrows * 32, kThreads));
  launch_pdl(k_spgemm_warp<false>, dim3(wblocks), dim3(kThreads), 0, s, X, cnt, pcnt, nullptr, nullptr, nullptr, nullptr,
                                                    nullptr, nullptr, nullptr, flags);
  NAIR_LAUNCH_CHECK();
  out.nrows = nrows;
  out.ncols = ncols;
  out.rp = mem.alloc<int>(nrows + 1);
  exclusive_scan(cnt, out.rp, nrows, s, tmp, false);
  exclusive_scan(pcnt, prp, nrows, s, tmp, false);
  // one read-back: output blocks, products, overflow flag
  NAIR_CK(cudaMemcpyAsync(flags + 1, out.rp + nrows, sizeof(int), cudaMemcpyDeviceToDevice, s));
  NAIR_CK(cudaMemcpyAsync(flags + 2, prp + nrows, sizeof(int), cudaMemcpyDeviceToDevice, s));
  int h[3];
  {
    static thread_local int *stage = nullptr;
    if (!stage) NAIR_CK(cudaMallocHost(&stage, 4 * sizeof(int)));
    NAIR_CK(cudaMemcpyAsync(stage, flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
    h[0] = stage[0];
    h[1] = stage[1];
    h[2] = stage[2];
  }
  if (h[0]) {  // a row longer than the warp merge holds: thread-per-row kernels
    mem.release(out.rp);
    tmp.release(flags);
    tmp.release(prp);
    tmp.release(pcnt);
    tmp.release(cnt);
    spgemm_rowwise<T>(b, X, left_nnz, lv, rv, iv, negate, ncols, s, mem, tmp, out);
    return;
  }
  out.nnzb = h[1];
  const int nprod = h[2];
  out.ci = mem.alloc<int>(out.nnzb);
  int *orow = tmp.alloc<int>(out.nnzb), *pbeg = tmp.alloc<int>(out.nnzb + 1), *iq = tmp.alloc<int>(out.nnzb);
  int2 *pairs = tmp.alloc<int2>(nprod);
  launch_pdl(k_spgemm_warp<true>, dim3(wblocks), dim3(kThreads), 0, s, X, nullptr, nullptr, out.rp, prp, out.ci, orow, pbeg,
                                                   pairs, iq, flags);
  NAIR_LAUNCH_CHECK();
  NAIR_CK(cudaMemcpyAsync(pbeg + out.nnzb, prp + nrows, sizeof(int), cudaMemcpyDeviceToDevice, s));
  out.v = mem.alloc<T>((size_t)out.nnzb * b * b);
  const long long total = (long long)out.nnzb * b * b;
  if (total) {
    // FP32 (mixed precision) takes the row form; in FP64 one thread per output
    // scalar measured faster (C5 FP64 setup with Neumann degree 6: 95.5 ms
    // against 109.6 ms; FP32: 57.1 -> 52.3 ms with the row form)
    const long long rows = (long long)out.nnzb * b;
    const dim3 gr(grid(rows)), bl(kThreads);
    const bool row_form = sizeof(T) == 4 && (b == 3 || b == 6 || b == 10);
    if (row_form && b == 3) launch_pdl(k_spgemm_rows<T, 3>, gr, bl, 0, s, rows, pbeg, pairs, iq, lv, rv, iv, negate, out.v);
    else if (row_form && b == 6) launch_pdl(k_spgemm_rows<T, 6>, gr, bl, 0, s, rows, pbeg, pairs, iq, lv, rv, iv, negate, out.v);
    else if (row_form) launch_pdl(k_spgemm_rows<T, 10>, gr, bl, 0, s, rows, pbeg, pairs, iq, lv, rv, iv, negate, out.v);
    else if (by_block && lmask && (b == 3 || b == 6 || b == 10)) {
      const dim3 gw(cdiv(out.nnzb, 8));
      if (b == 10) launch_pdl(k_spgemm_wblk<T, 10>, gw, bl, 0, s, out.nnzb, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
      else if (b == 6) launch_pdl(k_spgemm_wblk<T, 6>, gw, bl, 0, s, out.nnzb, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
      else launch_pdl(k_spgemm_wblk<T, 3>, gw, bl, 0, s, out.nnzb, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
    } else if (b == 10) launch_pdl(k_spgemm_pairs<T, 10>, dim3(grid(total)), bl, 0, s, total, b, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
    else if (b == 6) launch_pdl(k_spgemm_pairs<T, 6>, dim3(grid(total)), bl, 0, s, total, b, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
    else if (b == 3) launch_pdl(k_spgemm_pairs<T, 3>, dim3(grid(total)), bl, 0, s, total, b, pbeg, pairs, iq, lv, rv, iv, negate, out.v, lmask, rmask);
    else launch_pdl(k_spgemm_pairs<T, 0>, dim3(grid(total)), bl, 0, s, total, b, pbeg, pairs, iq, lv, rv, iv, negate, out.v,
                                (const unsigned *)nullptr, (const unsigned *)nullptr);
    NAIR_LAUNCH_CHECK();
  }
  tmp.release(pairs);
  tmp.release(iq);
  tmp.release(pbeg);
  tmp.release(orow);
  tmp.release(flags);
  tmp.release(prp);
  tmp.release(pcnt);
  tmp.release(cnt);
  (void)left_nnz;
}

// With defer, the kept count stays on the device (M.nnzb = -1, the buffers sized
// by the unfiltered count): no host round trip.
// With keep_src, the kept blocks are not copied: M keeps its value array, and
// *keep_src (allocated in mem, released by the caller) maps each kept entry to
// its block there.
template <typename T>
static void filter(int b, T tol2, cudaStream_t s, Mem &mem, Mem &tmp, DBsr<T> &M, bool defer = false,
                   int **keep_src = nullptr) {
  const int nrows = M.nrows;
  ProfScope ps("filter", s);
  const int ub = M.nnzb;
  int *newpos = tmp.alloc<int>(ub);
  int *cnt = tmp.alloc<int>(nrows + 1);
  T *nrm = tmp.alloc<T>(ub);
  if (ub) {
    launch_pdl(k_block_norm2<T>, dim3(grid(ub)), dim3(kThreads), 0, s, ub, b, M.v, nrm);
    NAIR_LAUNCH_CHECK();
  }
  launch_pdl(k_filter_flags<T>, dim3(grid(nrows)), dim3(kThreads), 0, s, nrows, M.rp, M.ci, nrm, tol2, newpos, cnt);
  NAIR_LAUNCH_CHECK();
  int *nrp = mem.alloc<int>(nrows + 1);
  const int nn = exclusive_scan(cnt, nrp, nrows, s, tmp, !defer);
  const int cap = defer ? ub : nn;
  int *nci = mem.alloc<int>(cap);
  int *src = keep_src ? mem.alloc<int>(cap) : tmp.alloc<int>(cap);
  launch_pdl(k_filter_compact, dim3(grid(nrows)), dim3(kThreads), 0, s, nrows, M.rp, M.ci, newpos, nrp, nci, src);
  NAIR_LAUNCH_CHECK();
  if (keep_src) {
    mem.release(M.rp);
    mem.release(M.ci);
    tmp.release(nrm);
    tmp.release(cnt);
    tmp.release(newpos);
    M.rp = nrp;
    M.ci = nci;
    M.nnzb = defer ? -1 : nn;
    *keep_src = src;
    return;
  }
  T *nv = mem.alloc<T>((size_t)cap * b * b);
  long long total = (long long)cap * b * b;
  if (total) {
    launch_pdl(k_copy_blocks<T>, dim3(grid(total)), dim3(kThreads), 0, s, total, b, src, M.v, nv, defer ? (const int *)(nrp + nrows) : (const int *)nullptr);
    NAIR_LAUNCH_CHECK();
  }
  mem.release(M.rp);
  mem.release(M.ci);
  mem.release(M.v);
  tmp.release(src);
  tmp.release(nrm);
  tmp.release(cnt);
  tmp.release(newpos);
  M.rp = nrp;
  M.ci = nci;
  M.v = nv;
  M.nnzb = defer ? -1 : nn;
}

template <typename T>
static void release_bsr(Mem &mem, DBsr<T> &M) {
  if (M.rp) mem.release(M.rp);
  if (M.ci) mem.release(M.ci);
  if (M.v) mem.release(M.v);
  M = DBsr<T>();
}

static void check_flag(int *flag, cudaStream_t s, nair_status st, const char *msg) {
  int v = read_int(flag, s);
  if (v) fail(st, msg);
}

int *sweep_list(int n, const int *list, const int *rp, cudaStream_t s, Mem &mem, Mem &tmp) {
  int *out = mem.alloc<int>(n);
  int *counts = tmp.alloc<int>(kLenBuckets);
  NAIR_CK(cudaMemsetAsync(counts, 0, sizeof(int) * kLenBuckets, s));
  if (n) {
    launch_pdl(k_len_count, dim3(grid(n)), dim3(kThreads), 0, s, n, list, rp, counts);
    NAIR_LAUNCH_CHECK();
  }
  launch_pdl(k_len_offsets, dim3(1), dim3(32), 0, s, counts);
  NAIR_LAUNCH_CHECK();
  if (n) {
    launch_pdl(k_len_scatter, dim3(grid(n)), dim3(kThreads), 0, s, n, list, rp, counts, out);
    NAIR_LAUNCH_CHECK();
  }
  tmp.release(counts);
  return out;
}

// ---------------------------------------------------------------------------
// work lists of the F sweeps after the first (cycle from a zero iterate)
// ---------------------------------------------------------------------------
// cur[i] = 1 for the F rows with an off-diagonal F coupling to a row changed
// in the previous sweep (prev = null: the first sweep, which changes every F row)
__global__ void k_fsweep_dep(int E, const int *__restrict__ rp, const int *__restrict__ ci,
                             const signed char *__restrict__ cf, const unsigned char *__restrict__ prev,
                             unsigned char *__restrict__ cur) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  unsigned char c = 0;
  if (!cf[i]) {
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      if (j != i && !cf[j] && (!prev || prev[j])) {
        c = 1;
        break;
      }
    }
  }
  cur[i] = c;
}

// membership flags over the positions q of fsweep for m = 2 (nf - 1) lists:
// t < nf - 1: the rows of sweep k = t + 1; t >= nf - 1: the rows of sweep
// k - 1 that are not in sweep k, k = t - nf + 2 (ch: nf rows of E flags, row k
// for sweep k >= 1; sweep 0 holds every F row)
__global__ void k_fsweep_flags(int nF, int nf, int E, const int *__restrict__ fsweep,
                               const unsigned char *__restrict__ ch, int *__restrict__ flag) {
  pdl_wait();
  const int m = 2 * (nf - 1);
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)m * nF) return;
  const int t = (int)(g / nF), q = (int)(g - (long long)t * nF), i = fsweep[q];
  int v;
  if (t < nf - 1) {
    v = ch[(size_t)(t + 1) * E + i];
  } else {
    const int k = t - nf + 2;
    v = (k == 1 || ch[(size_t)(k - 1) * E + i]) && !ch[(size_t)k * E + i];
  }
  flag[g] = v;
}

// stable compaction of each list (list t at out + t nF) and its length
__global__ void k_fsweep_scatter(int nF, int m, const int *__restrict__ fsweep, const int *__restrict__ flag,
                                 const int *__restrict__ pre, int *__restrict__ out, int *__restrict__ cnt) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < m && cnt) cnt[g] = pre[(size_t)(g + 1) * nF] - pre[(size_t)g * nF];
  if (g >= (long long)m * nF || !flag[g]) return;
  const int t = (int)(g / nF), q = (int)(g - (long long)t * nF);
  out[(size_t)t * nF + pre[g] - pre[(size_t)t * nF]] = fsweep[q];
}

// the row lists of F sweeps 1 .. nf - 1 of one level (matrix rp / ci, its F
// rows fsweep) into a new buffer of 2 (nf - 1) nF entries, list lengths to
// cnt on the device; null when the level keeps full sweeps
int *fsweep_lists(int E, int nF, const int *rp, const int *ci, const signed char *cf, const int *fsweep, int nf,
                  int *cnt, cudaStream_t s, Mem &mem, Mem &tmp) {
  const int m = 2 * (nf - 1);
  const long long tot = (long long)m * nF;
  if (nf < 2 || nF == 0 || tot >= INT_MAX) return nullptr;
  unsigned char *ch = tmp.alloc<unsigned char>((size_t)nf * E);
  for (int k = 1; k < nf; ++k) {
    launch_pdl(k_fsweep_dep, dim3(grid(E)), dim3(kThreads), 0, s, E, rp, ci, cf,
               k == 1 ? (const unsigned char *)nullptr : (const unsigned char *)(ch + (size_t)(k - 1) * E),
               ch + (size_t)k * E);
    NAIR_LAUNCH_CHECK();
  }
  int *flag = tmp.alloc<int>(tot), *pre = tmp.alloc<int>(tot + 1);
  launch_pdl(k_fsweep_flags, dim3(grid(tot)), dim3(kThreads), 0, s, nF, nf, E, fsweep, (const unsigned char *)ch,
             flag);
  NAIR_LAUNCH_CHECK();
  exclusive_scan(flag, pre, (int)tot, s, tmp, false);
  int *buf = mem.alloc<int>(tot);
  launch_pdl(k_fsweep_scatter, dim3(grid(tot)), dim3(kThreads), 0, s, nF, m, fsweep, (const int *)flag,
             (const int *)pre, buf, cnt);
  NAIR_LAUNCH_CHECK();
  return buf;
}

// pointers and lengths of the lists in buf (hcnt: the 2 (nf - 1) lengths)
void fsweep_assign(int nF, int nf, int *buf, const int *hcnt, int *fsweep, int **fl, int *fl_n, int **fq,
                   int *fq_n) {
  fl[0] = fsweep;
  fl_n[0] = nF;
  for (int k = 1; k < nf; ++k) {
    fl[k] = buf + (size_t)(k - 1) * nF;
    fl_n[k] = hcnt[k - 1];
    fq[k] = buf + (size_t)(nf - 1 + k - 1) * nF;
    fq_n[k] = hcnt[nf - 1 + k - 1];
  }
}

// the lists of every non-coarsest level, with one read-back of their lengths
template <typename T>
static void build_fsweep_lists(Hier<T> &H, const Params &P, cudaStream_t s, Mem &mem) {
  const int nf = P.f_sweeps;
  if (nf < 2 || nf > kMaxFLists) return;
  const int m = 2 * (nf - 1);
  Mem tmp;
  tmp.s = s;
  int *cnt = tmp.alloc<int>((size_t)H.nlev * m);
  std::vector<int *> bufs(H.nlev, nullptr);
  for (int l = 0; l < H.nlev; ++l) {
    Level<T> &L = H.lev[l];
    if (L.coarsest) continue;
    bufs[l] = fsweep_lists(L.E, L.nF, L.A.rp, L.A.ci, L.cf, L.fsweep, nf, cnt + (size_t)l * m, s, mem, tmp);
  }
  std::vector<int> h((size_t)H.nlev * m, 0);
  NAIR_CK(cudaMemcpyAsync(h.data(), cnt, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
  for (int l = 0; l < H.nlev; ++l) {
    Level<T> &L = H.lev[l];
    if (!bufs[l]) continue;
    L.nfl = nf;
    fsweep_assign(L.nF, nf, bufs[l], h.data() + (size_t)l * m, L.fsweep, L.fl, L.fl_n, L.fq, L.fq_n);
  }
}

// ---------------------------------------------------------------------------
// scalar-row form of the off-diagonal blocks (sweeps of levels >= 1)
// ---------------------------------------------------------------------------
// FILL = false: number of blocks of row i (the off-diagonal ones when
// skip_diag is set) whose row r has a nonzero; FILL = true: their block
// indices, ascending.  With cf, an F row lists its blocks in C columns first
// and then those in F columns (each part ascending), and srs receives the
// position where the F part starts (the row's start for C rows)
template <typename T, bool FILL>
__global__ void k_srow_entries(int E, int b, const int *__restrict__ rp, const int *__restrict__ ci,
                               const T *__restrict__ v, const int *__restrict__ srp, int *__restrict__ cnt,
                               int *__restrict__ sp, int skip_diag, const signed char *__restrict__ cf,
                               int *__restrict__ srs, unsigned char *__restrict__ nzb) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)E * b) return;
  const int i = (int)(g / b), r = (int)(g - (long long)i * b);
  const bool split = cf && cf[i] == 0;
  int w = FILL ? srp[g] : 0;
  if (FILL && srs) srs[g] = w;
  for (int pass = 0; pass < (split ? 2 : 1); ++pass) {
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (skip_diag && ci[p] == i) continue;
      if (split && (cf[ci[p]] == 1) != (pass == 0)) continue;  // pass 0: C columns, pass 1: F columns
      // the counting pass reads the values and keeps one flag per block row
      // (p, r) for the filling pass, which then reads no values (C5 FP64
      // setup 75.3 -> 73.8 ms)
      bool nz = false;
      if (FILL) {
        nz = nzb[(size_t)p * b + r] != 0;
      } else {
        const T *row = v + ((size_t)p * b + r) * b;
        for (int c = 0; c < b; ++c) nz |= row[c] != (T)0;
        nzb[(size_t)p * b + r] = nz;
      }
      if (nz) {
        if (FILL) sp[w] = p;
        ++w;
      }
    }
    if (FILL && srs && split && pass == 0) srs[g] = w;
  }
  if (!FILL) cnt[g] = w;
}

// packed entries: for scalar row g = (i, r), each entry e's block column sj[e]
// and row r of its block, sv[e b .. e b + b)
template <typename T>
__global__ void k_srow_pack(long long n, int b, const int *__restrict__ srp, const int *__restrict__ sp,
                            const int *__restrict__ ci, const T *__restrict__ v, int *__restrict__ sj,
                            T *__restrict__ sv) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int r = (int)(g % b);
  for (int e = srp[g]; e < srp[g + 1]; ++e) {
    const int p = sp[e];
    sj[e] = ci[p];
    const T *row = v + ((size_t)p * b + r) * b;
    for (int c = 0; c < b; ++c) sv[(size_t)e * b + c] = row[c];
  }
}

// per thread block of a row list (tpc rows, tpc b scalar rows; rows base ..
// when list is null): the scalar rows sorted by entry count (counted from srs
// when given: the F part a later F sweep sums), ties in natural order;
// perm[c tpc b + rank] = the natural slot team b + r
__global__ void k_srow_perm(int n, int b, int tpc, const int *__restrict__ list, const int *__restrict__ srp,
                            const int *__restrict__ srs, unsigned char *__restrict__ perm) {
  pdl_wait();
  __shared__ int key[256];
  const int base = blockIdx.x * tpc, nact = min(tpc, n - base), t = threadIdx.x, m = nact * b;
  int k = 0;
  if (t < m) {
    const int team = t / b, r = t - team * b;
    const size_t q = (size_t)(list ? list[base + team] : base + team) * b + r;
    k = srp[q + 1] - (srs ? srs[q] : srp[q]);
    key[t] = k;
  }
  __syncthreads();
  if (t >= m) return;
  int rank = 0;
  for (int u = 0; u < m; ++u) rank += (key[u] < k) || (key[u] == k && u < t);
  perm[(size_t)base * b + rank] = (unsigned char)t;
}

static bool srow_supported(int b) {
  return b == 3 || b == 6 || b == 10 || b == 15 || b == 21 || b == 28;
}

// largest thread-group count per row that takes the scalar-row form: with 16
// or more groups a thread already handles about one block of a row
static constexpr int kSweepRowsMaxG = 8;

template <typename T>
static unsigned char *srow_perm(int n, int b, double avg, const int *list, const int *srp, cudaStream_t s,
                                Mem &mem, int *tpc_out, const int *srs = nullptr) {
  const int G = rowop_groups(n, b, avg);
  if (G > kSweepRowsMaxG) return nullptr;
  const int tpc = sweep_rows_tpc(b, G);
  *tpc_out = tpc;
  unsigned char *perm = mem.alloc<unsigned char>((size_t)std::max(n, 1) * b);
  if (n > 0) {
    launch_pdl(k_srow_perm, dim3(cdiv(n, tpc)), dim3(tpc * b), 0, s, n, b, tpc, list, srp, srs, perm);
    NAIR_LAUNCH_CHECK();
  }
  return perm;
}

// entry lists and packed entries of the scalar-row form of the E x b scalar
// rows of M (its off-diagonal blocks when skip_diag is set)
template <typename T>
static void srow_pack(int E, int b, const DBsr<T> &M, bool skip_diag, const signed char *cf, SweepRows &sr,
                      cudaStream_t s, Mem &mem) {
  const long long n = (long long)E * b;
  Mem tmp;
  tmp.s = s;
  int *cnt = tmp.alloc<int>(n + 1);
  unsigned char *nzb = tmp.alloc<unsigned char>((size_t)std::max(M.nnzb, 1) * b);
  launch_pdl(k_srow_entries<T, false>, dim3(grid(n)), dim3(kThreads), 0, s, E, b, (const int *)M.rp,
             (const int *)M.ci, (const T *)M.v, (const int *)nullptr, cnt, (int *)nullptr, (int)skip_diag, cf,
             (int *)nullptr, nzb);
  NAIR_LAUNCH_CHECK();
  sr.srp = mem.alloc<int>(n + 1);
  const int ne = exclusive_scan(cnt, sr.srp, (int)n, s, tmp, true);
  sr.ne = ne;
  sr.sp = mem.alloc<int>(std::max(ne, 1));
  if (cf) sr.srs = mem.alloc<int>(n);
  launch_pdl(k_srow_entries<T, true>, dim3(grid(n)), dim3(kThreads), 0, s, E, b, (const int *)M.rp,
             (const int *)M.ci, (const T *)M.v, (const int *)sr.srp, (int *)nullptr, sr.sp, (int)skip_diag, cf,
             sr.srs, nzb);
  NAIR_LAUNCH_CHECK();
  sr.sj = mem.alloc<int>(std::max(ne, 1));
  T *sv = mem.alloc<T>((size_t)std::max(ne, 1) * b);
  sr.sv = sv;
  launch_pdl(k_srow_pack<T>, dim3(grid(n)), dim3(kThreads), 0, s, n, b, (const int *)sr.srp, (const int *)sr.sp,
             (const int *)M.ci, (const T *)M.v, sr.sj, sv);
  NAIR_LAUNCH_CHECK();
}

template <typename T>
void build_restrict_rows(int nC, int b, const DBsr<T> &R, SweepRows &rr, cudaStream_t s, Mem &mem) {
  // FP64 only (the FP32 restriction keeps the block-row kernel)
  if (!std::is_same<T, double>::value || !srow_supported(b) || nC == 0) return;
  const long long n = (long long)nC * b, ub = (long long)R.nnzb * b;
  if (n + 1 >= INT_MAX || ub >= INT_MAX) return;
  const double avg = (double)R.nnzb / nC;
  if (rowop_groups(nC, b, avg) > kSweepRowsMaxG) return;
  srow_pack<T>(nC, b, R, false, nullptr, rr, s, mem);
  rr.perm_c = srow_perm<T>(nC, b, avg, nullptr, rr.srp, s, mem, &rr.perm_c_tpc);
}
template void build_restrict_rows<double>(int, int, const DBsr<double> &, SweepRows &, cudaStream_t, Mem &);
template void build_restrict_rows<float>(int, int, const DBsr<float> &, SweepRows &, cudaStream_t, Mem &);

template <typename T>
void build_sweep_rows_level(int E, int nF, int nC, int b, const DBsr<T> &A, const signed char *cf, int *fsweep,
                            int nfl, int *const *fl, const int *fl_n, int *csweep, SweepRows &sr, cudaStream_t s,
                            Mem &mem) {
  // FP64 and FP32: it saves FP64 issue slots at the price of a shuffled
  // access pattern and a longer setup.  In FP32 alone it did not gain (mixed
  // precision, C5 at Neumann degree 2: 427.6 -> 434.7 ms); with the F sweeps
  // in y = D x it does (degree 6: setup + solve 141.7 -> 132.9 ms)
  if (!srow_supported(b) || E == 0) return;
  const long long n = (long long)E * b, ub = (long long)A.nnzb * b;
  if (n + 1 >= INT_MAX || ub >= INT_MAX) return;
  const double avg = (double)A.nnzb / E;
  if (rowop_groups(nF, b, avg) > kSweepRowsMaxG && rowop_groups(nC, b, avg) > kSweepRowsMaxG) return;
  srow_pack<T>(E, b, A, true, cf, sr, s, mem);
  // F sweeps: thread groups per scalar row sized for half a row (the first
  // F sweep's rows too: C5 FP64 solve 112.5 -> 110.8 ms; for a quarter of a
  // row the later sweeps were slower, 113.1 ms).  Blocks larger than 10 keep
  // the full-row sizing: their scalar rows are long already (C3, b = 28:
  // solve 30.0 -> 28.1 ms with it)
  const double favg = b <= 10 ? 0.5 * avg : avg;
  sr.perm_f[0] = srow_perm<T>(nF, b, favg, fsweep, sr.srp, s, mem, &sr.perm_f_tpc[0]);
  // the later F sweeps sum only the F part of their rows: sorted by its length,
  // their thread groups per row sized for half a row (C5 FP64 solve 119.4 ->
  // 112.4 ms, mixed 80.2 -> 75.5 ms, adjoint 211.8 -> 204.8 ms)
  for (int k = 1; k < nfl; ++k)
    sr.perm_f[k] = srow_perm<T>(fl_n[k], b, favg, fl[k], sr.srp, s, mem, &sr.perm_f_tpc[k], sr.srs);
  sr.perm_c = srow_perm<T>(nC, b, avg, csweep, sr.srp, s, mem, &sr.perm_c_tpc);
}
template void build_sweep_rows_level<double>(int, int, int, int, const DBsr<double> &, const signed char *, int *,
                                             int, int *const *, const int *, int *, SweepRows &, cudaStream_t, Mem &);
template void build_sweep_rows_level<float>(int, int, int, int, const DBsr<float> &, const signed char *, int *,
                                            int, int *const *, const int *, int *, SweepRows &, cudaStream_t, Mem &);

// sv2[e b + c] = sum_t sv[e b + t] dinv[j][t][c] (fma, t ascending) for an
// entry e whose column j = sj[e] is an F element; sv[e b + c] otherwise
template <typename T>
__global__ void k_srow_scale(long long tot, int b, const int *__restrict__ sj, const T *__restrict__ sv,
                             const T *__restrict__ dinv, const signed char *__restrict__ cf, T *__restrict__ sv2) {
  pdl_wait();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= tot) return;
  const long long e = g / b;
  const int c = (int)(g - e * b);
  const int j = sj[e];
  if (cf[j] != 0) {
    sv2[g] = sv[g];
    return;
  }
  const T *row = sv + (size_t)e * b;
  const T *dc = dinv + (size_t)j * b * b + c;
  T acc = 0;
  for (int t = 0; t < b; ++t) acc = fma_rn(row[t], dc[(size_t)t * b], acc);
  sv2[g] = acc;
}

template <typename T>
void scale_srow_entries(SweepRows &sr, int b, const T *dinv, const signed char *cf, cudaStream_t s, Mem &mem) {
  const long long ne = sr.ne;
  T *sv2 = mem.alloc<T>((size_t)std::max(ne, 1LL) * b);
  const long long tot = ne * b;
  if (tot) {
    launch_pdl(k_srow_scale<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, (const int *)sr.sj,
               (const T *)sr.sv, dinv, cf, sv2);
    NAIR_LAUNCH_CHECK();
  }
  sr.sv2 = sv2;
}
template void scale_srow_entries<double>(SweepRows &, int, const double *, const signed char *, cudaStream_t, Mem &);
template void scale_srow_entries<float>(SweepRows &, int, const float *, const signed char *, cudaStream_t, Mem &);

// the scalar-row lists and permutations of every level >= 1 that sweeps
template <typename T>
static void build_sweep_rows(Hier<T> &H, const Params &P, cudaStream_t s, Mem &mem) {
  for (int l = 0; l < H.nlev; ++l) {
    Level<T> &L = H.lev[l];
    if (L.coarsest) continue;
    build_restrict_rows<T>(L.nC, H.b, L.R, L.rr, s, mem);
    if (l == 0) continue;
    build_sweep_rows_level<T>(L.E, L.nF, L.nC, H.b, L.A, L.cf, L.fsweep, L.nfl, L.fl, L.fl_n, L.csweep, L.sr, s,
                              mem);
    // the C part of the F rows, summed once per cycle by the first F sweep
    if (L.sr.srs && L.nfl >= 2) L.h = mem.alloc<T>((size_t)L.E * H.b);
    // F sweeps in y_F = D_FF x_F where every sweep of the cycle takes the
    // scalar-row form (one F sweep list per sweep, one C sweep): the first F
    // sweep stores y = f_F - A_FC x_C - A_FF x_F, each later one y = h -
    // sum_j (A_ij D_jj^{-1}) y_j, so no F sweep applies D^{-1}; the C sweep
    // reads y_F through the same scaled blocks and writes x_F = D_FF^{-1} y_F
    bool all_rows = L.h && L.nfl == P.f_sweeps && P.f_sweeps >= 2 && P.c_sweeps == 1 && L.sr.perm_c;
    for (int k = 0; all_rows && k < L.nfl; ++k) all_rows = L.sr.perm_f[k] != nullptr;
    if (all_rows) {
      scale_srow_entries<T>(L.sr, H.b, L.dinv, L.cf, s, mem);
      L.ymode = 1;
    }
  }
}

// extract rows `rowmap` (nrows of them) of A with the chosen column test
// The output count stays on the device (out.nnzb = -1, buffers sized by the
// upper bound A.nnzb, returned in *ub): no host round trip.
template <typename T>
static void extract(int b, int nrows, int mode, const int *rowmap, const Level<T> &L,
                    const unsigned char *strong, const int *fidx, cudaStream_t s, Mem &mem,
                    Mem &tmp, DBsr<T> &out, int **src_out, int **row_out, int *ub) {
  int *cnt = tmp.alloc<int>(nrows + 1);
  launch_pdl(k_sub_count, dim3(grid(nrows)), dim3(kThreads), 0, s, nrows, mode, rowmap, L.A.rp, L.A.ci, strong, L.cf, cnt);
  NAIR_LAUNCH_CHECK();
  out.nrows = nrows;
  out.rp = mem.alloc<int>(nrows + 1);
  exclusive_scan(cnt, out.rp, nrows, s, tmp, false);
  *ub = L.A.nnzb;
  out.nnzb = -1;
  out.ci = mem.alloc<int>(*ub);
  int *src = tmp.alloc<int>(*ub);
  int *row = tmp.alloc<int>(*ub);
  launch_pdl(k_sub_fill, dim3(grid(nrows)), dim3(kThreads), 0, s, nrows, mode, rowmap, L.A.rp, L.A.ci, strong, L.cf, fidx,
                                               out.rp, out.ci, src, row);
  NAIR_LAUNCH_CHECK();
  out.v = mem.alloc<T>((size_t)*ub * b * b);
  tmp.release(cnt);
  *src_out = src;
  *row_out = row;
}

// Build level l + 1 from level l.  Returns false when level l must be the coarsest.
template <typename T>
static bool coarsen(Hier<T> &H, int l, const Params &P, cudaStream_t s, Mem &mem, Mem &tmp) {
  const int b = H.b, bb = b * b;
  Level<T> &L = H.lev[l];
  const int E = L.E, nnzb = L.A.nnzb;
  // a2: strength
  ProfScope ps_all("setup_level", s, l);
  ProfScope ps_str("strength", s, l);
  T *snorm = tmp.alloc<T>(nnzb);
  unsigned char *strong = (P.keep ? mem.alloc<unsigned char>(nnzb) : tmp.alloc<unsigned char>(nnzb));
  launch_pdl(k_block_norm2<T>, dim3(grid(nnzb)), dim3(kThreads), 0, s, nnzb, b, L.A.v, snorm);
  NAIR_LAUNCH_CHECK();
  const T th2 = (T)(P.theta * P.theta);
  launch_pdl(k_strength<T>, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, snorm, th2, strong);
  NAIR_LAUNCH_CHECK();
  int *lam = P.keep ? mem.alloc<int>(E) : tmp.alloc<int>(E);
  NAIR_CK(cudaMemsetAsync(lam, 0, sizeof(int) * E, s));
  launch_pdl(k_lambda, dim3(grid(nnzb)), dim3(kThreads), 0, s, nnzb, L.A.ci, strong, lam);
  NAIR_LAUNCH_CHECK();
  ps_str.end();
  // a3: C/F splitting
  L.cf = mem.alloc<signed char>(E);
  uint64_t *hash = tmp.alloc<uint64_t>(E);
  int *mark = tmp.alloc<int>(E);
  int *brow = tmp.alloc<int>(nnzb);
  int *remaining = tmp.alloc<int>(1);
  launch_pdl(k_block_rows, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, brow);
  NAIR_LAUNCH_CHECK();
  launch_pdl(k_pmis_init, dim3(grid(E)), dim3(kThreads), 0, s, E, lam, L.cf, hash, P.seed, mark);
  NAIR_LAUNCH_CHECK();
  int rounds = 0;
  ProfScope ps_cf("cf_split", s, l);
  // rounds are issued in batches (four, then two at a time) between read-backs
  // of the undecided count; a round with no undecided point changes nothing
  for (int batch = 4;; batch = 2) {
    for (int rep = 0; rep < batch; ++rep) {
      NAIR_CK(cudaMemsetAsync(remaining, 0, sizeof(int), s));
      launch_pdl(k_pmis_mark, dim3(grid(nnzb)), dim3(kThreads), 0, s, nnzb, brow, L.A.ci, strong, L.cf, lam, hash, mark, rounds);
      NAIR_LAUNCH_CHECK();
      launch_pdl(k_pmis_select, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, mark, rounds);
      NAIR_LAUNCH_CHECK();
      launch_pdl(k_pmis_fmark, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, strong, L.cf, remaining);
      NAIR_LAUNCH_CHECK();
      ++rounds;
    }
    if (read_int(remaining, s) == 0) break;
    if (rounds > E + 2) fail(NAIR_ERR_CUDA, "C/F splitting did not terminate");
  }
  L.cf_rounds = rounds;
  ps_cf.end();
  int *isc = tmp.alloc<int>(E);
  int *pre = tmp.alloc<int>(E + 1);
  launch_pdl(k_cf_flags, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, isc);
  NAIR_LAUNCH_CHECK();
  const int nC = exclusive_scan(isc, pre, E, s, tmp);
  const int nF = E - nC;
  L.nC = nC;
  L.nF = nF;
  if (P.keep) {
    L.strong = strong;
    L.lam = lam;
  }
  if (nC == 0 || (long long)nC * 10 > (long long)E * 9) {
    tmp.release_all();
    return false;
  }
  int *cidx = tmp.alloc<int>(E), *fidx = tmp.alloc<int>(E);
  L.c2f = mem.alloc<int>(nC);
  L.f2f = mem.alloc<int>(nF);
  int *f2f = L.f2f;
  launch_pdl(k_cf_index, dim3(grid(E)), dim3(kThreads), 0, s, E, L.cf, pre, cidx, fidx, L.c2f, f2f);
  NAIR_LAUNCH_CHECK();
  L.fsweep = sweep_list(nF, f2f, L.A.rp, s, mem, tmp);
  L.csweep = sweep_list(nC, L.c2f, L.A.rp, s, mem, tmp);

  // a4: L = -D_ff^{-1} A^S_ff, then Horner T_{t+1} = D^{-1} + L T_t (Eq. neumann)
  ProfScope ps_neu("neumann", s, l);
  DBsr<T> Lm;
  int *src, *row;
  int lub = 0;
  extract<T>(b, nF, 0, f2f, L, strong, fidx, s, mem, tmp, Lm, &src, &row, &lub);
  Lm.ncols = nF;
  long long tot = (long long)lub * bb;
  if (tot) {
    launch_pdl(k_L_values<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, row, src, f2f, L.dinv, L.A.v, Lm.v, Lm.rp + nF);
    NAIR_LAUNCH_CHECK();
  }
  tmp.release(src);
  tmp.release(row);
  DBsr<T> Dg;  // diagonal D_ff^{-1} as a block-CSR matrix
  Dg.nrows = Dg.ncols = Dg.nnzb = nF;
  Dg.rp = tmp.alloc<int>(nF + 1);
  Dg.ci = Dg.rp;  // column i of row i: the same iota array
  Dg.v = tmp.alloc<T>((size_t)nF * bb);
  launch_pdl(k_iota, dim3(grid(nF + 1)), dim3(kThreads), 0, s, nF, Dg.rp);
  NAIR_LAUNCH_CHECK();
  tot = (long long)nF * bb;
  if (tot) {
    launch_pdl(k_copy_blocks<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, f2f, L.dinv, Dg.v, (const int *)nullptr);
    NAIR_LAUNCH_CHECK();
  }
  DBsr<T> Tk;  // T_0 = D^{-1}
  {
    Tk.nrows = Tk.ncols = Tk.nnzb = nF;
    Tk.rp = mem.alloc<int>(nF + 1);
    Tk.ci = mem.alloc<int>(nF);
    Tk.v = mem.alloc<T>((size_t)nF * bb);
    NAIR_CK(cudaMemcpyAsync(Tk.rp, Dg.rp, sizeof(int) * (nF + 1), cudaMemcpyDeviceToDevice, s));
    NAIR_CK(cudaMemcpyAsync(Tk.ci, Dg.rp, sizeof(int) * nF, cudaMemcpyDeviceToDevice, s));
    NAIR_CK(cudaMemcpyAsync(Tk.v, Dg.v, sizeof(T) * nF * bb, cudaMemcpyDeviceToDevice, s));
  }
  const T tol2 = (T)(P.filter_tol * P.filter_tol);
  // zero columns of the L blocks (the face columns of A's couplings): the
  // products skip them
  unsigned *lm_mask = block_masks<T>(b, lub, Lm.v, Lm.rp + nF, s, tmp);
  // the filtered iterates keep the product's value array: tk_src maps their
  // entries into it, so no kept block is copied (the next product reads the
  // blocks through the map; C5 FP64 setup 77.0 -> 73.8 ms)
  int *tk_src = nullptr;
  for (int t = 0; t < P.k; ++t) {
    SpgemmIdx X{nF, Lm.rp, Lm.ci, nullptr, Tk.rp, Tk.ci, Dg.rp, Dg.rp, nullptr, tk_src};
    DBsr<T> Tn;
    int *tn_src = nullptr;
    spgemm<T>(b, X, lub, Lm.v, Tk.v, Dg.v, 0, nF, s, mem, tmp, Tn, lm_mask);
    // (for b = 1 the copy is cheaper than the extra index load in the merge:
    // scalar nAIR setup 973 -> 997 ms with the map)
    if (P.filter_targets & 1) filter<T>(b, tol2, s, mem, tmp, Tn, true, b >= 3 ? &tn_src : nullptr);
    release_bsr(mem, Tk);
    if (tk_src) mem.release(tk_src);
    Tk = Tn;
    tk_src = tn_src;
  }
  if (lm_mask) tmp.release(lm_mask);
  tmp.release(Dg.v);
  tmp.release(Dg.rp);
  ps_neu.end();

  // a5: R_cf = -A_cf Delta over all A_cf blocks
  ProfScope ps_r("restriction", s, l);
  DBsr<T> Acf;
  int aub = 0;
  extract<T>(b, nC, 1, L.c2f, L, strong, fidx, s, tmp, tmp, Acf, &src, &row, &aub);
  tot = (long long)aub * bb;
  if (tot) {
    launch_pdl(k_copy_blocks<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, src, L.A.v, Acf.v, Acf.rp + nC);
    NAIR_LAUNCH_CHECK();
  }
  {
    SpgemmIdx X{nC, Acf.rp, Acf.ci, nullptr, Tk.rp, Tk.ci, nullptr, nullptr, nullptr, tk_src};
    unsigned *acf_mask = block_masks<T>(b, aub, Acf.v, Acf.rp + nC, s, tmp);
    spgemm<T>(b, X, aub, Acf.v, Tk.v, (const T *)nullptr, 1, nF, s, mem, tmp, L.R, acf_mask, nullptr, true);
    if (acf_mask) tmp.release(acf_mask);
  }
  L.R_ci_f = L.R.ci;
  L.R.ci = mem.alloc<int>(L.R.nnzb);
  if (L.R.nnzb) {
    launch_pdl(k_map, dim3(grid(L.R.nnzb)), dim3(kThreads), 0, s, L.R.nnzb, L.R_ci_f, f2f, L.R.ci);
    NAIR_LAUNCH_CHECK();
  }
  L.R.ncols = E;
  ps_r.end();

  // a6: one-point interpolation
  L.ipc = mem.alloc<int>(E);
  launch_pdl(k_one_point<T>, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, strong, snorm, L.cf, cidx, L.ipc);
  NAIR_LAUNCH_CHECK();

  // a7: A P (column merge), then K = (AP)_C + R_cf (AP)_F
  ProfScope ps_k("galerkin", s, l);
  DBsr<T> AP;
  {
    int *cnt = tmp.alloc<int>(E + 1);
    launch_pdl(k_ap_count, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, L.ipc, cnt);
    NAIR_LAUNCH_CHECK();
    AP.nrows = E;
    AP.ncols = nC;
    AP.rp = tmp.alloc<int>(E + 1);
    exclusive_scan(cnt, AP.rp, E, s, tmp, false);
    AP.nnzb = -1;               // at most one block per block of A: sized by nnzb(A)
    AP.ci = tmp.alloc<int>(nnzb);
    int *apfirst = tmp.alloc<int>(nnzb), *apnext = tmp.alloc<int>(nnzb);
    launch_pdl(k_ap_fill, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, L.ipc, AP.rp, AP.ci, apfirst,
               apnext);
    NAIR_LAUNCH_CHECK();
    AP.v = tmp.alloc<T>((size_t)nnzb * bb);
    tot = (long long)nnzb * bb;
    if (tot) {
      launch_pdl(k_ap_values<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, (const int *)apfirst,
                 (const int *)apnext, (const T *)L.A.v, AP.v, (const int *)(AP.rp + E));
      NAIR_LAUNCH_CHECK();
    }
  }
  Level<T> nx;
  {
    SpgemmIdx X{nC, L.R.rp, L.R.ci, nullptr, AP.rp, AP.ci, AP.rp, AP.ci, L.c2f};
    unsigned *r_mask = block_masks<T>(b, L.R.nnzb, L.R.v, (const int *)nullptr, s, tmp);
    unsigned *ap_mask = block_masks<T>(b, nnzb, AP.v, AP.rp + E, s, tmp);
    spgemm<T>(b, X, L.R.nnzb, L.R.v, AP.v, AP.v, 0, nC, s, mem, tmp, nx.A, r_mask, ap_mask, true);
    if (ap_mask) tmp.release(ap_mask);
    if (r_mask) tmp.release(r_mask);
    if (P.filter_targets & 2) filter<T>(b, tol2, s, mem, tmp, nx.A);
  }
  nx.E = nC;
  if (P.keep) {
    Lm.nnzb = read_int(Lm.rp + nF, s);
    if (Tk.nnzb < 0) Tk.nnzb = read_int(Tk.rp + nF, s);
    if (tk_src) {  // Delta's kept blocks, contiguous for the export
      T *dv = mem.alloc<T>((size_t)std::max(Tk.nnzb, 1) * bb);
      const long long tk_tot = (long long)Tk.nnzb * bb;
      if (tk_tot) {
        launch_pdl(k_copy_blocks<T>, dim3(grid(tk_tot)), dim3(kThreads), 0, s, tk_tot, b, (const int *)tk_src,
                   (const T *)Tk.v, dv, (const int *)nullptr);
        NAIR_LAUNCH_CHECK();
      }
      mem.release(Tk.v);
      mem.release(tk_src);
      tk_src = nullptr;
      Tk.v = dv;
    }
    L.L = Lm;
    L.Delta = Tk;
  } else {
    release_bsr(mem, Lm);
    release_bsr(mem, Tk);
    if (tk_src) mem.release(tk_src);
  }
  tmp.release_all();
  H.lev.push_back(nx);
  return true;
}

void diag_positions(int E, const int *rp, const int *ci, int *out, cudaStream_t s) {
  launch_pdl(k_diag_pos, dim3(grid(E)), dim3(kThreads), 0, s, E, rp, ci, out);
  NAIR_LAUNCH_CHECK();
}

template <typename T>
static void level_dinv(Hier<T> &H, Level<T> &L, cudaStream_t s, Mem &mem, Mem &tmp, int *err) {
  const int b = H.b, E = L.E;
  ProfScope ps("dinv", s);
  L.diag = mem.alloc<int>(E);
  launch_pdl(k_diag_pos, dim3(grid(E)), dim3(kThreads), 0, s, E, L.A.rp, L.A.ci, L.diag);
  NAIR_LAUNCH_CHECK();
  double *d64;
  if constexpr (std::is_same<T, double>::value) {
    L.dinv = mem.alloc<T>((size_t)E * b * b);
    d64 = L.dinv;
  } else {
    d64 = tmp.alloc<double>((size_t)E * b * b);
  }
  block_inverses<T>(E, b, L.A.v, L.diag, d64, err, s);
  if constexpr (!std::is_same<T, double>::value) {
    L.dinv = mem.alloc<T>((size_t)E * b * b);
    long long n = (long long)E * b * b;
    launch_pdl(k_convert<T>, dim3(grid(n)), dim3(kThreads), 0, s, n, d64, L.dinv);
    NAIR_LAUNCH_CHECK();
    tmp.release(d64);
  }
  // the singular-block flag is read once, at the end of the hierarchy build
}

template <typename T>
static void make_coarsest(Hier<T> &H, Level<T> &L, const Params &P, cudaStream_t s, Mem &mem,
                          Mem &tmp, int *err) {
  const int b = H.b;
  const int n = L.E * b;
  if (L.A.nnzb == L.E) {
    // block-diagonal coarsest matrix (coarsening stopped on isolated elements):
    // its exact inverse is the diagonal-block inverse already computed
    L.coarsest = 1;
    L.n = n;
    L.ainv = nullptr;
    return;
  }
  if (n > P.max_dense) {
    // a singular diagonal block upstream explains a stalled coarsening first
    check_flag(err, s, NAIR_ERR_SINGULAR_BLOCK, "singular diagonal block");
    char buf[200];
    snprintf(buf, sizeof(buf),
             "coarsest level has %d unknowns, above max_dense = %d (coarsening stalled)", n,
             P.max_dense);
    fail(NAIR_ERR_UNSUPPORTED, buf);
  }
  L.coarsest = 1;
  L.n = n;
  ProfScope ps("coarse_inverse", s);
  double *M = tmp.alloc<double>((size_t)n * n);
  NAIR_CK(cudaMemsetAsync(M, 0, sizeof(double) * n * n, s));
  int *brow = tmp.alloc<int>(L.A.nnzb);
  launch_pdl(k_block_rows, dim3(grid(L.E)), dim3(kThreads), 0, s, L.E, L.A.rp, brow);
  NAIR_LAUNCH_CHECK();
  long long tot = (long long)L.A.nnzb * b * b;
  if (tot) {
    launch_pdl(k_dense_fill<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, b, n, brow, L.A.ci, L.A.v, M);
    NAIR_LAUNCH_CHECK();
  }
  int *piv = tmp.alloc<int>(n);
  // one thread block in shared memory for small matrices; beyond that the
  // elimination (n^3 FMAs on one SM's FP64 pipe) is spread over thread blocks,
  // one launch per step, consecutive steps overlapping their launch latency
  const size_t gj_smem = (size_t)n * n * sizeof(double) + (size_t)n * (sizeof(double) + sizeof(int));
  if (n <= 48) {
    NAIR_CK(cudaFuncSetAttribute(k_dense_gj_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gj_smem));
    launch_pdl(k_dense_gj_smem, dim3(1), dim3(kGjThreads), gj_smem, s, n, M, err);
    NAIR_LAUNCH_CHECK();
  } else {
    double *M2 = tmp.alloc<double>((size_t)n * n);
    dim3 g(cdiv(n, kGjTileCols), cdiv(n, kGjTileRows));
    for (int k = 0; k < n; ++k) {
      launch_pdl(k_gj_step, g, dim3(256), 0, s, n, k, (const double *)M, M2, piv, err);
      NAIR_LAUNCH_CHECK();
      std::swap(M, M2);
    }
    launch_pdl(k_gj_unscramble, dim3(1), dim3(1024), 0, s, n, M, piv);
    NAIR_LAUNCH_CHECK();
  }
  L.ainv = mem.alloc<T>((size_t)n * n);
  tot = (long long)n * n;
  launch_pdl(k_convert<T>, dim3(grid(tot)), dim3(kThreads), 0, s, tot, M, L.ainv);
  NAIR_LAUNCH_CHECK();
  // the flag is read at the end of the hierarchy build
  tmp.release_all();
}

template <typename T>
void build_hierarchy(const DBsr<T> &A0, const Params &P, cudaStream_t s, Mem &mem, Hier<T> &H) {
  Mem tmp;
  tmp.s = s;
  int *err = tmp.alloc<int>(1);
  NAIR_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  H.lev.clear();
  H.lev.reserve(P.max_levels + 1);
  Level<T> l0;
  l0.A = A0;
  l0.E = A0.nrows;
  H.lev.push_back(l0);
  for (int l = 0;; ++l) {
    Level<T> &L = H.lev[l];
    level_dinv<T>(H, L, s, mem, tmp, err);
    bool stop = (l == P.max_levels - 1) || (L.E <= P.max_coarse);
    if (!stop) {
      Mem ltmp;
      ltmp.s = s;
      stop = !coarsen<T>(H, l, P, s, mem, ltmp);
    }
    if (stop) {
      Mem ctmp;
      ctmp.s = s;
      make_coarsest<T>(H, H.lev[l], P, s, mem, ctmp, err);
      break;
    }
  }
  H.nlev = (int)H.lev.size();
  check_flag(err, s, NAIR_ERR_SINGULAR_BLOCK, "singular diagonal block or coarsest-level matrix");
  if (!H.lev[0].coarsest) {
    build_l0comp<T>(H.lev[0].A, H.lev[0].diag, H.b, s, mem, H.l0c);
    // level-0 sweeps with the couplings scaled in advance (they then skip the
    // b^2 FMAs per row of the D^{-1} apply)
    build_l0scaled<T>(H.lev[0].A, H.lev[0].dinv, H.b, s, mem, H.l0c);
  }
  build_fsweep_lists<T>(H, P, s, mem);
  build_sweep_rows<T>(H, P, s, mem);
  // V-cycle vectors and complexities (Sec. 6: OC and CC in work units)
  const int b = H.b;
  double nnz0 = (double)H.lev[0].A.nnzb, oc = 0.0, cc = 0.0;
  for (int l = 0; l < H.nlev; ++l) {
    Level<T> &L = H.lev[l];
    size_t n = (size_t)L.E * b;
    L.f = mem.alloc<T>(n);
    L.x = mem.alloc<T>(n);
    L.x2 = mem.alloc<T>(n);
    L.r = mem.alloc<T>(n);
    if (l == 0 && H.l0c.sv) L.g = mem.alloc<T>(n);
    double a = (double)L.A.nnzb / nnz0;
    oc += a;
    // visits of level l per cycle: 1 in a V-cycle; 1 + l in an F-cycle (one
    // F-type visit, and l V-type visits from a nonzero guess, each adding a residual)
    const double visits = P.cycle == 1 ? 1.0 + l : 1.0, resid = P.cycle == 1 ? (double)l : 0.0;
    if (L.coarsest) {
      cc += visits * (L.ainv ? (double)L.n * L.n / (nnz0 * b * b) : a);
    } else {
      // restriction + (f + c) sweeps over the selected rows, counted as full SpMVs
      cc += visits * (a * (P.f_sweeps + P.c_sweeps) + (double)L.R.nnzb / nnz0) + resid * a;
    }
  }
  H.op_complexity = oc;
  H.cycle_complexity = cc;
  NAIR_CK(cudaStreamSynchronize(s));
}

template void build_hierarchy<double>(const DBsr<double> &, const Params &, cudaStream_t, Mem &, Hier<double> &);
template void build_hierarchy<float>(const DBsr<float> &, const Params &, cudaStream_t, Mem &, Hier<float> &);

// validation kernel wrapper used by the API
void validate_bsr(int E, int ncols, const int *rp, const int *ci, int nnzb, cudaStream_t s, Mem &tmp) {
  int *err = tmp.alloc<int>(1);
  NAIR_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  launch_pdl(k_validate, dim3(grid(E)), dim3(kThreads), 0, s, E, ncols, rp, ci, nnzb, err);
  NAIR_LAUNCH_CHECK();
  int v = read_int(err, s);
  tmp.release(err);
  if (v & 2) fail(NAIR_ERR_INVALID_ARG, "block CSR structure invalid (row pointers or unsorted/out-of-range columns)");
  if (v & 4) fail(NAIR_ERR_INVALID_ARG, "a block row has no diagonal block");
}

}  // namespace nair
