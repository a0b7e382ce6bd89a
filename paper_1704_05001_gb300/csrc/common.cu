// Errors, stream-ordered device memory and the exclusive scan used to turn
// per-row counts into block-CSR row pointers.
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>

#include "common.cuh"

namespace nair {

void fail(nair_status st, const std::string &msg) { throw NairError{st, msg}; }

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // launches issued by this host thread
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
long long thread_launch_count() { return t_launches; }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void ck_fail(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
           cudaGetErrorString(e), what, file, line);
  throw NairError{e == cudaErrorMemoryAllocation ? NAIR_ERR_OOM : NAIR_ERR_CUDA, buf};
}

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
namespace {
struct Pending {
  std::string name;
  cudaEvent_t e0, e1;
};
struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<Pending> pending;
  std::map<std::string, std::pair<long long, double>> stats;
};
ProfState &prof() {
  static ProfState p;
  return p;
}
}  // namespace

bool prof_on() { return prof().on; }

void prof_enable(bool on) {
  prof_resolve();
  std::lock_guard<std::mutex> lk(prof().mu);
  prof().on = on;
  prof().stats.clear();
}

void prof_resolve() {
  std::lock_guard<std::mutex> lk(prof().mu);
  for (auto &p : prof().pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      auto &st = prof().stats[p.name];
      st.first += 1;
      st.second += ms;
    }
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  prof().pending.clear();
  cudaGetLastError();
}

int prof_count() {
  prof_resolve();
  std::lock_guard<std::mutex> lk(prof().mu);
  return (int)prof().stats.size();
}

bool prof_entry(int idx, std::string &name, long long &launches, double &ms) {
  std::lock_guard<std::mutex> lk(prof().mu);
  if (idx < 0 || idx >= (int)prof().stats.size()) return false;
  auto it = prof().stats.begin();
  std::advance(it, idx);
  name = it->first;
  launches = it->second.first;
  ms = it->second.second;
  return true;
}

ProfScope::ProfScope(const char *n, cudaStream_t st, int lvl) : name(n), level(lvl), s(st) {
  if (!prof().on) return;
  if (cudaEventCreate(&e0) != cudaSuccess) { e0 = nullptr; return; }
  cudaEventRecord(e0, s);
}

void ProfScope::end() {
  if (!e0) return;
  cudaEvent_t e1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); e0 = nullptr; return; }
  cudaEventRecord(e1, s);
  std::string nm = name;
  if (level >= 0) nm += "@L" + std::to_string(level);
  std::lock_guard<std::mutex> lk(prof().mu);
  prof().pending.push_back({nm, e0, e1});
  e0 = nullptr;
}

void *Mem::raw(size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed (%s)", bytes,
             cudaGetErrorName(e));
    fail(e == cudaErrorMemoryAllocation ? NAIR_ERR_OOM : NAIR_ERR_CUDA, buf);
  }
  ptrs.push_back(p);
  // the row kernels read rows with 16-byte loads from offsets that are
  // multiples of 16 bytes; they rely on the allocator's 256-byte alignment
  if ((uintptr_t)p & 255u) fail(NAIR_ERR_CUDA, "device allocation not 256-byte aligned");
  return p;
}

void Mem::release(void *p) {
  for (size_t i = 0; i < ptrs.size(); ++i)
    if (ptrs[i] == p) {
      cudaFreeAsync(p, s);
      ptrs[i] = ptrs.back();
      ptrs.pop_back();
      return;
    }
}

void Mem::release_all() {
  for (void *p : ptrs) cudaFreeAsync(p, s);
  ptrs.clear();
}

// ---------------------------------------------------------------------------
// exclusive scan: tiles of 2048 ints per CTA (256 threads x 8), tile sums
// scanned recursively, then added back
// ---------------------------------------------------------------------------
static constexpr int kScanThreads = 256;
static constexpr int kScanItems = 8;
static constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int cta_exclusive_scan(int v, int *warp_sums, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (kScanThreads / 32) ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (kScanThreads / 32)) warp_sums[lane] = wi - w;
    if (lane == (kScanThreads / 32) - 1) *total = wi;
  }
  __syncthreads();
  return inc - v + warp_sums[wid];
}

// writes the exclusive prefix of each tile, the tile sums, and (single-tile
// case) the total into out[n]
__global__ void k_scan_tiles(const int *__restrict__ in, int *__restrict__ out, int n,
                             int *__restrict__ tile_sums) {
  pdl_wait();
  __shared__ int warp_sums[kScanThreads / 32];
  __shared__ int total;
  const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + k;
    v[k] = (i < n) ? in[i] : 0;
    s += v[k];
  }
  int pre = cta_exclusive_scan(s, warp_sums, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + k;
    if (i < n) out[i] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) {
    if (tile_sums) tile_sums[blockIdx.x] = total;
    else out[n] = total;  // one tile: the total follows the prefixes
  }
}

// adds the scanned tile offsets; offs[tiles] is the total, copied to out[n]
__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ tile_off, int tiles) {
  pdl_wait();
  const long long base = (long long)blockIdx.x * kScanTile;
  const int add = tile_off[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    long long i = base + k;
    if (i < n) out[i] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[tiles];
}

__global__ void k_scan_zero(int *out) {
  pdl_wait(); out[0] = 0; }

// out[0..n) = exclusive prefix of in, out[n] = total
static void scan_rec(const int *in, int *out, int n, cudaStream_t s, Mem &tmp) {
  const int tiles = cdiv(n, kScanTile);
  if (tiles <= 1) {
    launch_pdl(k_scan_tiles, dim3(1), dim3(kScanThreads), 0, s, in, out, n, nullptr);
    NAIR_LAUNCH_CHECK();
    return;
  }
  int *sums = tmp.alloc<int>(tiles + 1);
  launch_pdl(k_scan_tiles, dim3(tiles), dim3(kScanThreads), 0, s, in, out, n, sums);
  NAIR_LAUNCH_CHECK();
  int *offs = tmp.alloc<int>(tiles + 1);
  scan_rec(sums, offs, tiles, s, tmp);
  launch_pdl(k_scan_add, dim3(tiles), dim3(kScanThreads), 0, s, out, n, offs, tiles);
  NAIR_LAUNCH_CHECK();
  tmp.release(offs);
  tmp.release(sums);
}

int exclusive_scan(const int *in, int *out, int n, cudaStream_t s, Mem &tmp, bool want_total) {
  if (n > 0) {
    scan_rec(in, out, n, s, tmp);
  } else {
    launch_pdl(k_scan_zero, dim3(1), dim3(1), 0, s, out);
    NAIR_LAUNCH_CHECK();
  }
  if (!want_total) return -1;
  return read_int(out + n, s);
}

int read_int(const int *p, cudaStream_t s) {
  // pinned staging word (one per host thread) keeps the read-back short
  static thread_local int *stage = nullptr;
  if (!stage) NAIR_CK(cudaMallocHost(&stage, sizeof(int)));
  NAIR_CK(cudaMemcpyAsync(stage, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
  return *stage;
}

}  // namespace nair
