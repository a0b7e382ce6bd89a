// Shared host/device helpers of the nAIR GPU library: errors, device memory,
// canonical IEEE arithmetic, scans and small device utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/nair.h"

namespace nair {

// ---------------------------------------------------------------------------
// errors: internal code throws NairError; the C ABI converts it to a status
// ---------------------------------------------------------------------------
struct NairError {
  nair_status status;
  std::string msg;
};

[[noreturn]] void fail(nair_status st, const std::string &msg);
void ck_fail(cudaError_t e, const char *what, const char *file, int line);

#define NAIR_CK(x)                                              \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) ::nair::ck_fail(e_, #x, __FILE__, __LINE__); \
  } while (0)

// every kernel launch is followed by this check, which also counts the launch
void count_launch();
void add_launches(long long n);
long long launch_count();
long long thread_launch_count();  // this host thread's launches (graph capture counts)
#define NAIR_LAUNCH_CHECK()        \
  do {                             \
    ::nair::count_launch();        \
    NAIR_CK(cudaGetLastError());   \
  } while (0)

// ---------------------------------------------------------------------------
// device memory: stream-ordered allocations owned by one Mem until release
// ---------------------------------------------------------------------------
struct Mem {
  cudaStream_t s = nullptr;
  std::vector<void *> ptrs;
  void *raw(size_t bytes);
  template <class X>
  X *alloc(size_t n) {
    return static_cast<X *>(raw((n ? n : 1) * sizeof(X)));
  }
  void release(void *p);
  void release_all();
  ~Mem() { release_all(); }
};

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// canonical arithmetic: correctly rounded IEEE operations, never contracted
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// position of key in the sorted range a[lo, hi), or -1
__device__ __forceinline__ int find_sorted(const int *__restrict__ a, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// splitmix64 (Steele, Lea and Flood, 2014): tie-break hash of the C/F keys
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// optional per-kernel timing: when enabled, ProfScope records a CUDA event pair
// around the launches in its scope; the pairs are resolved into per-name totals
// ---------------------------------------------------------------------------
bool prof_on();
void prof_enable(bool on);
void prof_resolve();
int prof_count();
bool prof_entry(int idx, std::string &name, long long &launches, double &ms);

struct ProfScope {
  const char *name;
  int level;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(const char *name, cudaStream_t s, int level = -1);
  void end();  // close the scope early (the destructor then does nothing)
  ~ProfScope() { end(); }
};

// launch with programmatic dependent launch allowed: the kernel may start while
// its predecessor in the stream is still running; it must call griddepcontrol.wait
// (pdl_wait) before reading anything the predecessor writes
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  NAIR_CK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Programmatic dependent launch: let the next kernel of the stream be
// scheduled now, and wait for the previous kernel's results before reading them.
// Without the launch attribute both are no-ops.  The setup kernels call only
// pdl_wait (their successor is then scheduled as they finish): an early trigger
// let the successor's waiting thread blocks sit beside long-running kernels of
// the large-block workloads and slowed them, while the trigger at completion
// still hides the launch gap between the setup's many short kernels.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// exclusive scan of n ints into out[0..n]; out[n] = total; returns the total
// (synchronises the stream to read it back when want_total is set)
int exclusive_scan(const int *in, int *out, int n, cudaStream_t s, Mem &tmp, bool want_total = true);

// rows per thread block of the scalar-row sweep with G threads per scalar row
inline int sweep_rows_tpc(int b, int G) { return 256 / (b * G) > 1 ? 256 / (b * G) : 1; }

// read one int from device memory (synchronising)
int read_int(const int *p, cudaStream_t s);

}  // namespace nair
