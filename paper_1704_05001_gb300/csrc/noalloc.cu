// Batched block inverses for callers that cannot allocate device memory.
//
// nair_block_inverse allocates a small device status word for every call.
// Some callers cannot do that: code that runs while a caching allocator owns
// the whole device, solvers embedded in applications that forbid cudaMalloc
// after start-up, or host code that must not synchronise the device the way
// cudaMalloc/cudaFree can.  nair_block_inverse_noalloc does the same work with
// its status words in a fixed array that lives in this file's device memory.
// CUDA sets that array up on a GPU when it loads the library's device code
// there: at the first kernel call of the library on that GPU under lazy module
// loading (the default of recent CUDA releases), at start-up with
// CUDA_MODULE_LOADING=EAGER.  A caller whose caching allocator later takes the
// whole device should therefore make one warm-up call first.  The array stays
// until the process exits.
//
// The array holds one status word per thread block of the launch plus one
// result word, so one call handles at most kNoallocMaxCtas thread blocks
// (kNoallocMaxCtas * max(1, 256 / b) matrix blocks); larger calls are rejected
// with NAIR_ERR_INVALID_ARG before anything is launched.  The array keeps the
// last call's contents; every call writes each word it later reads (one status
// word per thread block it launches, then the result word), so nothing needs
// clearing between calls.  Calls that overlap on the GPU share the array and
// race; order them on one stream.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>

#include "common.cuh"

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxCtas = 8192;   // 8192 status words + 1 result word: 32 KB per GPU
constexpr int kNoallocMaxDevices = 64;

// status words of the thread blocks of the last call, then the result word
static __device__ __align__(256) int g_noalloc_scratch[kNoallocMaxCtas + 1];

// device address of the array per device; host threads may look it up at the
// same time (each stores the same value), so the cache is atomic
std::atomic<int *> g_scratch_ptr[kNoallocMaxDevices] = {};

// same Gauss-Jordan arithmetic as the allocating kernel (one thread per block
// row, partial pivoting, fma elimination, the pivot row multiplied by one
// correctly rounded reciprocal 1/d per step); each thread block stores 1 in
// its own status word if one of its blocks met a zero or NaN pivot, else 0
__global__ void k_block_inverse_noalloc(int nblk, int b, int bpc, const double *__restrict__ A,
                                        double *__restrict__ out, int *__restrict__ status) {
  extern __shared__ double sm[];
  int *piv = reinterpret_cast<int *>(sm + (size_t)bpc * b * b);
  __shared__ double rinv_s[256];
  __shared__ int cta_sing;
  const int lb = threadIdx.x / b, t = threadIdx.x % b;
  const long long blk = (long long)blockIdx.x * bpc + lb;
  const bool active = lb < bpc && blk < nblk;
  double *M = sm + (size_t)lb * b * b;
  if (threadIdx.x == 0) cta_sing = 0;
  if (active) {
    const double *src = A + (size_t)blk * b * b;
    for (int c = 0; c < b; ++c) M[t * b + c] = src[t * b + c];
  }
  __syncthreads();
  bool sing = false;
  for (int k = 0; k < b; ++k) {
    int p = k;
    if (active) {
      double best = fabs(M[k * b + k]);
      for (int r = k + 1; r < b; ++r) {
        double a = fabs(M[r * b + k]);
        if (a > best) { best = a; p = r; }
      }
      if (t == 0) piv[lb * 32 + k] = p;
    }
    __syncthreads();
    if (active && p != k) {
      double tmp = M[k * b + t];
      M[k * b + t] = M[p * b + t];
      M[p * b + t] = tmp;
    }
    __syncthreads();
    const double d = active ? M[k * b + k] : 1.0;
    if (active && (d == 0.0 || d != d)) sing = true;
    if (active && t == 0) rinv_s[lb] = __ddiv_rn(1.0, d);  // one division per step
    __syncthreads();
    if (active) {
      double v = (t == k) ? 1.0 : M[k * b + t];
      M[k * b + t] = __dmul_rn(v, rinv_s[lb]);
    }
    __syncthreads();
    if (active && t != k) {
      double l = M[t * b + k];
      M[t * b + k] = 0.0;
      for (int c = 0; c < b; ++c) M[t * b + c] = __fma_rn(-l, M[k * b + c], M[t * b + c]);
    }
    __syncthreads();
  }
  if (active) {
    for (int k = b - 1; k >= 0; --k) {
      int p = piv[lb * 32 + k];
      if (p != k) {
        double tmp = M[t * b + k];
        M[t * b + k] = M[t * b + p];
        M[t * b + p] = tmp;
      }
    }
    double *dst = out + (size_t)blk * b * b;
    for (int c = 0; c < b; ++c) dst[t * b + c] = M[t * b + c];
    if (sing) cta_sing = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) status[blockIdx.x] = cta_sing;
}

// result word = index of the first thread block that reported a zero pivot, or -1
__global__ void k_noalloc_first_bad(int nctas, const int *__restrict__ status, int *__restrict__ result) {
  __shared__ int best;
  if (threadIdx.x == 0) best = INT_MAX;
  __syncthreads();
  for (int c = threadIdx.x; c < nctas; c += blockDim.x)
    if (status[c]) atomicMin(&best, c);
  __syncthreads();
  if (threadIdx.x == 0) *result = best == INT_MAX ? -1 : best;
}

// address of the scratch array on the current device, looked up once per device
int *scratch_address(nair_status *st, const char **msg) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    cudaGetLastError();
    *st = NAIR_ERR_CUDA;
    *msg = "nair_block_inverse_noalloc: no usable current device";
    return nullptr;
  }
  int *cached = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!cached) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *st = NAIR_ERR_CUDA;
      *msg = "nair_block_inverse_noalloc: cudaGetSymbolAddress of the scratch array failed";
      return nullptr;
    }
    cached = static_cast<int *>(p);
    g_scratch_ptr[dev].store(cached, std::memory_order_release);
  }
  return cached;
}

}  // namespace

namespace nair {
nair_status noalloc_error(nair_status st, const char *msg);
}

nair_status nair_block_inverse_noalloc(int32_t nblk, int32_t b, const double *A, double *Ainv,
                                       void *stream) {
  using nair::noalloc_error;
  if (nblk < 0 || b < 1 || b > 32 || (nblk > 0 && (!A || !Ainv)))
    return noalloc_error(NAIR_ERR_INVALID_ARG, "nair_block_inverse_noalloc: bad arguments");
  if (nblk == 0) return NAIR_OK;
  const int bpc = b <= kNoallocThreads ? kNoallocThreads / b : 1;
  const long long nctas = ((long long)nblk + bpc - 1) / bpc;
  if (nctas > kNoallocMaxCtas) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "nair_block_inverse_noalloc: %d blocks of size %d need %lld thread blocks; the static "
             "scratch holds %d (at most %d blocks of this size per call)",
             nblk, b, nctas, kNoallocMaxCtas, kNoallocMaxCtas * bpc);
    return noalloc_error(NAIR_ERR_INVALID_ARG, buf);
  }
  nair_status st = NAIR_OK;
  const char *msg = nullptr;
  int *scratch = scratch_address(&st, &msg);
  if (!scratch) return noalloc_error(st, msg);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = (size_t)bpc * b * b * sizeof(double) + (size_t)bpc * 32 * sizeof(int);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_block_inverse_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_error(NAIR_ERR_CUDA, "nair_block_inverse_noalloc: shared-memory attribute failed");
  }
  k_block_inverse_noalloc<<<(int)nctas, bpc * b, smem, s>>>(nblk, b, bpc, A, Ainv, scratch);
  k_noalloc_first_bad<<<1, 256, 0, s>>>((int)nctas, scratch, scratch + kNoallocMaxCtas);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_error(NAIR_ERR_CUDA, cudaGetErrorString(e));
  int first_bad = -1;
  e = cudaMemcpyAsync(&first_bad, scratch + kNoallocMaxCtas, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_error(NAIR_ERR_CUDA, cudaGetErrorString(e));
  }
  if (first_bad >= 0) {
    char buf[160];
    long long lo = (long long)first_bad * bpc;
    long long hi = std::min<long long>(lo + bpc, nblk) - 1;
    snprintf(buf, sizeof(buf), "singular block among blocks %lld..%lld", lo, hi);
    return noalloc_error(NAIR_ERR_SINGULAR_BLOCK, buf);
  }
  return NAIR_OK;
}
