// C ABI of the nAIR GPU library (declared in include/nair.h): handle life
// cycle, argument checking, the adjoint (transpose) hierarchy, hierarchy
// export, and the small parameter-dependent kernels of the transport problem.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <thread>

#include "solve.cuh"

namespace nair {
void validate_bsr(int E, int ncols, const int *rp, const int *ci, int nnzb, cudaStream_t s, Mem &tmp);
}

using namespace nair;

static thread_local std::string g_last_error;

struct nair_handle {
  Params P{};
  nair_params raw{};
  int b = 0, E = 0;
  long long n = 0;
  cudaStream_t s = nullptr;
  Mem mem;
  DBsr<double> A64;
  DBsr<float> A32;
  bool mixed = false, scalar = false;
  Hier<double> h64;
  Hier<float> h32;
  Outer fwd, bwd;  // FP64 operators of the forward (A) and adjoint (A^T) Krylov solves
  Krylov K;
  nair_handle *adj = nullptr;  // NAIR_ADJOINT_REBUILD: the hierarchy of A^T
  double setup_ms = 0.0;
  bool tbuilt = false;  // transposed form of the forward hierarchy (adjoint solves)
  double tsetup_ms = 0.0;
};

static nair_status set_error(nair_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

namespace nair {
// error reporting for the allocation-free entry point in noalloc.cu
nair_status noalloc_error(nair_status st, const char *msg) { return set_error(st, msg ? msg : ""); }
}  // namespace nair

#define NAIR_API_BEGIN try {
#define NAIR_API_END                                              \
  }                                                               \
  catch (const NairError &e) {                                    \
    return set_error(e.status, e.msg);                            \
  }                                                               \
  catch (const std::exception &e) {                               \
    return set_error(NAIR_ERR_CUDA, e.what());                    \
  }

static constexpr int kThreads = 256;
static inline int grid(long long n) { return std::max(1, cdiv(n, kThreads)); }

namespace nair {
Params resolve_params(const nair_params *p, int b) {
  Params P{};
  P.theta = p->strength_theta;
  P.filter_tol = p->filter_tol;
  P.filter_targets = p->filter_targets;
  P.k = p->neumann_degree;
  P.f_sweeps = p->f_sweeps > 0 ? p->f_sweeps : p->neumann_degree + 1;
  P.c_sweeps = p->c_sweeps < 0 ? 0 : p->c_sweeps;
  P.max_levels = p->max_levels;
  P.max_coarse = p->max_coarse > 0 ? p->max_coarse : std::max(2, 192 / b);
  P.max_dense = p->max_dense;
  P.seed = p->cf_seed;
  P.precision = p->precision;
  P.restart = p->gmres_restart;
  P.maxiter = p->maxiter;
  P.tol = p->tol;
  P.keep = p->keep_setup_data;
  P.use_graphs = p->use_graphs;
  P.sweep_timing = p->sweep_timing;
  P.cycle = p->cycle_type;
  P.scalar = p->scalar;
  return P;
}
}  // namespace nair

// ---------------------------------------------------------------------------
// small kernels of the API
// ---------------------------------------------------------------------------
template <typename A, typename B>
__global__ void k_cast_api(long long n, const A *__restrict__ in, B *__restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (B)in[i];
}

__global__ void k_assemble_sigma(int E, int b, const int *__restrict__ dpos, const double *__restrict__ v0,
                                 const double *__restrict__ M, const double *__restrict__ sigma,
                                 double *__restrict__ v) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = b * b;
  if (g >= (long long)E * bb) return;
  const int e = (int)(g / bb), rc = (int)(g - (long long)e * bb);
  const size_t o = (size_t)dpos[e] * bb + rc;
  v[o] = __dadd_rn(v0[o], __dmul_rn(sigma[e], M[g]));
}

__global__ void k_copy64(long long n, const double *__restrict__ a, double *__restrict__ b) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void k_mass_apply(int E, int b, const double *__restrict__ M, const double *__restrict__ q,
                             double *__restrict__ rhs) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)E * b) return;
  const int e = (int)(g / b), r = (int)(g - (long long)e * b);
  const double *m = M + (size_t)e * b * b + r * b;
  const double *qe = q + (size_t)e * b;
  double acc = 0.0;
  for (int c = 0; c < b; ++c) acc += m[c] * qe[c];
  rhs[g] = acc;
}

// gsigma_e = -lambda_e^T M_e x_e ; gq_e = M_e^T lambda_e
__global__ void k_gradients(int E, int b, const double *__restrict__ M, const double *__restrict__ lam,
                            const double *__restrict__ x, double *__restrict__ gs, double *__restrict__ gq) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double *Me = M + (size_t)e * b * b, *le = lam + (size_t)e * b, *xe = x + (size_t)e * b;
  double s = 0.0;
  for (int r = 0; r < b; ++r) {
    double mx = 0.0;
    for (int c = 0; c < b; ++c) mx += Me[r * b + c] * xe[c];
    s += le[r] * mx;
  }
  gs[e] = -s;
  for (int c = 0; c < b; ++c) {
    double t = 0.0;
    for (int r = 0; r < b; ++r) t += Me[r * b + c] * le[r];
    gq[(size_t)e * b + c] = t;
  }
}

// ---------------------------------------------------------------------------
// handle construction
// ---------------------------------------------------------------------------
// keep freed stream-ordered memory in the device's default pool (once per device)
static void init_pool_once() {
  static std::mutex m;
  static std::set<int> done;
  int dev = 0;
  NAIR_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  if (done.count(dev)) return;
  cudaMemPool_t pool;
  NAIR_CK(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  NAIR_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  done.insert(dev);
}

static void check_params(const nair_params *p, int b) {
  if (!(p->strength_theta >= 0.0) || !(p->strength_theta <= 1.0))
    fail(NAIR_ERR_INVALID_ARG, "strength_theta must lie in [0, 1]");
  if (!(p->filter_tol >= 0.0)) fail(NAIR_ERR_INVALID_ARG, "filter_tol must be >= 0");
  if (p->neumann_degree < 0 || p->neumann_degree > 64) fail(NAIR_ERR_INVALID_ARG, "neumann_degree must lie in 0..64");
  if (p->max_levels < 1 || p->max_levels > 64) fail(NAIR_ERR_INVALID_ARG, "max_levels must lie in 1..64");
  if (p->max_dense < b) fail(NAIR_ERR_INVALID_ARG, "max_dense smaller than one block");
  if (p->precision != NAIR_FP64 && p->precision != NAIR_MIXED) fail(NAIR_ERR_INVALID_ARG, "unknown precision");
  if (p->gmres_restart < 1 || p->gmres_restart > 1000) fail(NAIR_ERR_INVALID_ARG, "gmres_restart must lie in 1..1000");
  if (p->maxiter < 0) fail(NAIR_ERR_INVALID_ARG, "maxiter must be >= 0");
  if (!(p->tol >= 0.0)) fail(NAIR_ERR_INVALID_ARG, "tol must be >= 0");
  if (p->adjoint_mode != NAIR_ADJOINT_TRANSPOSED && p->adjoint_mode != NAIR_ADJOINT_REBUILD)
    fail(NAIR_ERR_INVALID_ARG, "unknown adjoint_mode");
  if (p->cycle_type != NAIR_CYCLE_V && p->cycle_type != NAIR_CYCLE_F) fail(NAIR_ERR_INVALID_ARG, "unknown cycle_type");
  if (p->scalar != 0 && p->scalar != 1) fail(NAIR_ERR_INVALID_ARG, "scalar must be 0 or 1");
}

static void setup_impl(nair_handle *h, const int *rp, const int *ci, const double *v, int E, int b,
                       long long nnzb, bool device_copy_done) {
  cudaStream_t s = h->s;
  Mem &mem = h->mem;
  mem.s = s;
  cudaEvent_t e0, e1;
  NAIR_CK(cudaEventCreate(&e0));
  NAIR_CK(cudaEventCreate(&e1));
  NAIR_CK(cudaEventRecord(e0, s));
  h->b = b;
  h->E = E;
  h->n = (long long)E * b;
  DBsr<double> &A = h->A64;
  if (!device_copy_done) {
    A.nrows = A.ncols = E;
    A.nnzb = (int)nnzb;
    A.rp = mem.alloc<int>(E + 1);
    A.ci = mem.alloc<int>(nnzb);
    A.v = mem.alloc<double>((size_t)nnzb * b * b);
    NAIR_CK(cudaMemcpyAsync(A.rp, rp, sizeof(int) * (E + 1), cudaMemcpyDefault, s));
    NAIR_CK(cudaMemcpyAsync(A.ci, ci, sizeof(int) * nnzb, cudaMemcpyDefault, s));
    NAIR_CK(cudaMemcpyAsync(A.v, v, sizeof(double) * nnzb * b * b, cudaMemcpyDefault, s));
  }
  {
    Mem tmp;
    tmp.s = s;
    int first = -1, last = -1;
    NAIR_CK(cudaMemcpyAsync(&first, A.rp, sizeof(int), cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaMemcpyAsync(&last, A.rp + E, sizeof(int), cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
    if (first != 0 || last != nnzb) fail(NAIR_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[E] must equal nnzb");
    validate_bsr(E, E, A.rp, A.ci, (int)nnzb, s, tmp);
  }
  h->mixed = h->P.precision == NAIR_MIXED;
  h->scalar = h->P.scalar != 0;
  h->fwd.A = A;
  h->fwd.b = b;
  // the matrix the hierarchy is built for: A, or for scalar nAIR D^{-1} A by
  // degree of freedom (block size 1)
  DBsr<double> M = A;
  int bm = b;
  double *Dsc = nullptr;
  if (h->scalar) {
    Mem tmp;
    tmp.s = s;
    int *diagA = mem.alloc<int>(E), *err = tmp.alloc<int>(1);
    NAIR_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    diag_positions(E, A.rp, A.ci, diagA, s);
    Dsc = mem.alloc<double>((size_t)E * b * b);
    block_inverses<double>(E, b, A.v, diagA, Dsc, err, s);
    if (read_int(err, s)) fail(NAIR_ERR_SINGULAR_BLOCK, "singular diagonal block");
    scalar_matrix(A, b, Dsc, diagA, M, s, mem);
    bm = 1;
    h->fwd.diag = diagA;
    build_l0comp<double>(A, diagA, b, s, mem, h->fwd.C);
  }
  if (h->mixed) {
    DBsr<float> &F = h->A32;
    F.nrows = F.ncols = M.nrows;
    F.nnzb = M.nnzb;
    F.rp = M.rp;
    F.ci = M.ci;
    F.v = mem.alloc<float>((size_t)M.nnzb * bm * bm);
    long long tot = (long long)M.nnzb * bm * bm;
    k_cast_api<double, float><<<grid(tot), kThreads, 0, s>>>(tot, M.v, F.v);
    NAIR_LAUNCH_CHECK();
    h->h32.b = bm;
    build_hierarchy<float>(F, h->P, s, mem, h->h32);
    if (h->scalar) {
      const long long nd = (long long)E * b * b;
      float *d32 = mem.alloc<float>((size_t)nd);
      k_cast_api<double, float><<<grid(nd), kThreads, 0, s>>>(nd, Dsc, d32);
      NAIR_LAUNCH_CHECK();
      h->h32.pre_dinv = d32;
      h->h32.pre_b = b;
      h->h32.pre_E = E;
    } else {
      h->fwd.diag = h->h32.lev[0].diag;
      if (!h->h32.lev[0].coarsest) build_l0comp<double>(A, h->fwd.diag, b, s, mem, h->fwd.C);
    }
  } else {
    h->h64.b = bm;
    build_hierarchy<double>(M, h->P, s, mem, h->h64);
    if (h->scalar) {
      h->h64.pre_dinv = Dsc;
      h->h64.pre_b = b;
      h->h64.pre_E = E;
    } else {
      h->fwd.diag = h->h64.lev[0].diag;
      h->fwd.C = h->h64.l0c;
    }
  }
  NAIR_CK(cudaEventRecord(e1, s));
  NAIR_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  NAIR_CK(cudaEventElapsedTime(&ms, e0, e1));
  h->setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// Definitions below take C linkage from their declarations in nair.h.

void nair_default_params(nair_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->strength_theta = 0.1;
  p->filter_tol = 1e-4;
  p->filter_targets = 3;
  p->neumann_degree = 1;
  p->f_sweeps = 0;
  p->c_sweeps = 1;
  p->max_levels = 25;
  p->max_coarse = 0;
  p->max_dense = 4096;
  p->cf_seed = 0;
  p->precision = NAIR_FP64;
  p->gmres_restart = 50;
  p->maxiter = 500;
  p->tol = 1e-10;
  p->stream = nullptr;
  p->keep_setup_data = 0;
  p->use_graphs = 1;
  p->sweep_timing = 0;
  p->adjoint_mode = NAIR_ADJOINT_TRANSPOSED;
  p->cycle_type = NAIR_CYCLE_V;
  p->scalar = 0;
}

const char *nair_last_error(void) { return g_last_error.c_str(); }

nair_status nair_sweep_timing(const nair_handle *h, int32_t level, int32_t cls, int64_t *sweeps,
                              double *total_ms) {
  NAIR_API_BEGIN
  if (!h || !sweeps || !total_ms || cls < 0) return set_error(NAIR_ERR_INVALID_ARG, "bad arguments");
  const SweepClock &c = h->mixed ? h->h32.clock : h->h64.clock;
  const int nl = h->mixed ? h->h32.nlev : h->h64.nlev;
  if (level < 0 || level >= nl) return set_error(NAIR_ERR_INVALID_ARG, "level out of range");
  const int S = h->P.f_sweeps + h->P.c_sweeps;
  if (cls > 1 + S) return set_error(NAIR_ERR_INVALID_ARG, "no such sweep");
  if (!c.dev) {
    *sweeps = 0;
    *total_ms = 0.0;
    return NAIR_OK;
  }
  if (cls >= 2) {  // sweep cls - 2 of the cycle
    *sweeps = c.site_count[(size_t)level * c.S + cls - 2];
    *total_ms = c.site_ms[(size_t)level * c.S + cls - 2];
    return NAIR_OK;
  }
  *sweeps = c.count[2 * level + cls];
  *total_ms = c.ms[2 * level + cls];
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_profile(int32_t enable) {
  NAIR_API_BEGIN
  prof_enable(enable != 0);
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_profile_entry(int32_t idx, char *name, size_t cap, int64_t *launches, double *total_ms) {
  NAIR_API_BEGIN
  if (idx == 0) prof_resolve();
  std::string nm;
  long long n = 0;
  double ms = 0.0;
  if (!prof_entry(idx, nm, n, ms)) return set_error(NAIR_ERR_INVALID_ARG, "no such profile entry");
  if (name && cap) {
    size_t k = std::min(cap - 1, nm.size());
    memcpy(name, nm.data(), k);
    name[k] = 0;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_kernel_launches(int64_t *count) {
  if (!count) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  *count = launch_count();
  return NAIR_OK;
}

// FP64 throughput probe.  mode 0: sixteen independent fma chains per thread;
// mode 1: four independent FP64 tensor-core chains per warp (mma.sync m8n8k4,
// 256 fused multiply-adds per warp instruction); mode 2: both in the same
// loop, to see whether the two paths add up.  Block 0's first thread records
// the SM clock cycles and the nanoseconds the block ran, from which the host
// derives the SM clock under this load.  The final test is never true for
// these inputs; it keeps the chains live.
__global__ void __launch_bounds__(256) k_fp64_rate(int mode, int iters, double a, double c, double *sink,
                                                   long long *clk) {
  long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  double x[16], acc[4][2];
  const double fa = 1.0 + 1e-3 * (threadIdx.x & 31), fb = 0.999;
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = 1e-3 * threadIdx.x + k;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
    if (mode != 1) {
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = fma(x[k], a, c);
    }
    if (mode != 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(acc[k][0]), "+d"(acc[k][1])
                     : "d"(fa), "d"(fb));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += x[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) s += acc[k][0] + acc[k][1];
  if (s == -1.0) *sink = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = clock64() - c0;
    clk[1] = t1 - t0;
  }
}

nair_status nair_fp64_peak(int32_t mode, int32_t iters, double *tflops, double *sm_mhz, void *stream) {
  NAIR_API_BEGIN
  if (!tflops || mode < 0 || mode > 2 || iters < 1 || iters > 1000000)
    return set_error(NAIR_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  NAIR_CK(cudaGetDevice(&dev));
  NAIR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Mem tmp;
  tmp.s = s;
  double *sink = tmp.alloc<double>(1);
  long long *clk = tmp.alloc<long long>(2);
  cudaEvent_t e0, e1;
  NAIR_CK(cudaEventCreate(&e0));
  NAIR_CK(cudaEventCreate(&e1));
  const int blocks = sms * 8;
  // fused multiply-adds per thread and iteration: 16 fma; 4 mma x 256 / 32 lanes
  const double per_thread = (mode != 1 ? 16.0 : 0.0) + (mode != 0 ? 32.0 : 0.0);
  double best = 0.0, mhz = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    NAIR_CK(cudaEventRecord(e0, s));
    k_fp64_rate<<<blocks, 256, 0, s>>>(mode, iters, 0.999999, 1e-6, sink, clk);
    NAIR_LAUNCH_CHECK();
    NAIR_CK(cudaEventRecord(e1, s));
    NAIR_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    NAIR_CK(cudaEventElapsedTime(&ms, e0, e1));
    long long hc[2] = {0, 0};
    NAIR_CK(cudaMemcpyAsync(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
    const double flops = 2.0 * per_thread * 256.0 * blocks * (double)iters;
    const double rate = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    if (rep > 0 && rate > best) {
      best = rate;
      mhz = hc[1] > 0 ? 1e3 * (double)hc[0] / (double)hc[1] : 0.0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  if (sm_mhz) *sm_mhz = mhz;
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_setup(const nair_bsr *A, const nair_params *p, nair_handle **out) {
  NAIR_API_BEGIN
  if (!A || !p || !out) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const int E = A->nb_rows, b = A->block_size;
  if (E <= 0) return set_error(NAIR_ERR_INVALID_ARG, "nb_rows must be positive");
  if (b < 1 || b > 32) return set_error(NAIR_ERR_UNSUPPORTED, "block_size must lie in 1..32");
  if (A->nnzb < E || A->nnzb > (int64_t)INT32_MAX || (long long)A->nnzb * b * b > (1LL << 40))
    return set_error(NAIR_ERR_INVALID_ARG, "nnzb out of range");
  if (!A->row_ptr || !A->col_idx || !A->vals) return set_error(NAIR_ERR_INVALID_ARG, "null matrix array");
  check_params(p, b);
  init_pool_once();
  nair_handle *h = new nair_handle();
  h->raw = *p;
  h->P = resolve_params(p, p->scalar ? 1 : b);
  h->s = (cudaStream_t)p->stream;
  h->K.mem.s = h->s;
  try {
    setup_impl(h, A->row_ptr, A->col_idx, A->vals, E, b, A->nnzb, false);
  } catch (...) {
    nair_free(h);
    throw;
  }
  *out = h;
  g_last_error.clear();
  return NAIR_OK;
  NAIR_API_END
}

static void fill_info(nair_handle *h, nair_info *info, int iters, double relres, double ms,
                      const std::vector<double> &hist, bool transposed) {
  if (!info) return;
  info->iterations = iters;
  info->rel_res = relres;
  info->solve_ms = ms;
  info->setup_ms = transposed ? h->tsetup_ms : h->setup_ms;
  if (h->mixed) {
    info->levels = h->h32.nlev;
    info->op_complexity = h->h32.op_complexity;
    info->cycle_complexity = h->h32.cycle_complexity;
  } else {
    info->levels = h->h64.nlev;
    info->op_complexity = h->h64.op_complexity;
    info->cycle_complexity = h->h64.cycle_complexity;
  }
  int nh = (int)hist.size();
  info->history_len = nh;
  if (info->history && info->history_cap > 0)
    for (int k = 0; k < std::min(nh, info->history_cap); ++k) info->history[k] = hist[k];
}

// FGMRES on A (or on A^T with the transposed cycle)
static nair_status solve_impl(nair_handle *h, const double *b, double *x, nair_info *info, bool transposed) {
  cudaEvent_t e0, e1;
  NAIR_CK(cudaEventCreate(&e0));
  NAIR_CK(cudaEventCreate(&e1));
  NAIR_CK(cudaEventRecord(e0, h->s));
  std::vector<double> hist;
  int iters = 0;
  double relres = 0.0;
  const Outer &op = transposed ? h->bwd : h->fwd;
  nair_status st = h->mixed ? fgmres<float>(op, h->h32, h->P, h->K, b, x, hist, &iters, &relres, h->s, transposed)
                            : fgmres<double>(op, h->h64, h->P, h->K, b, x, hist, &iters, &relres, h->s, transposed);
  NAIR_CK(cudaEventRecord(e1, h->s));
  NAIR_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  NAIR_CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fill_info(h, info, iters, relres, ms, hist, transposed);
  if (st == NAIR_ERR_NOT_CONVERGED) return set_error(st, "GMRES did not reach the tolerance within maxiter");
  if (st == NAIR_ERR_BREAKDOWN) return set_error(st, "non-finite value in the Krylov iteration");
  if (st == NAIR_OK) g_last_error.clear();
  return st;
}

// the row kernels read vectors with 16-byte loads where the block size
// allows it, so caller vectors must start on a 16-byte boundary
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
static const char *kAlignMsg = "device vectors must be 16-byte aligned";

nair_status nair_solve(nair_handle *h, const double *b, double *x, nair_info *info) {
  NAIR_API_BEGIN
  if (!h || !b || !x) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (!aligned16(b) || !aligned16(x)) return set_error(NAIR_ERR_INVALID_ARG, kAlignMsg);
  return solve_impl(h, b, x, info, false);
  NAIR_API_END
}

nair_status nair_vcycle(nair_handle *h, const double *f, double *x) {
  NAIR_API_BEGIN
  if (!h || !f || !x) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (!aligned16(f) || !aligned16(x)) return set_error(NAIR_ERR_INVALID_ARG, kAlignMsg);
  if (h->mixed) precond<float>(h->h32, h->P, f, x, h->s, h->n);
  else precond<double>(h->h64, h->P, f, x, h->s, h->n);
  NAIR_CK(cudaStreamSynchronize(h->s));
  return NAIR_OK;
  NAIR_API_END
}

// the transposed form of the forward hierarchy, and A^T in FP64
static void build_transposed_handle(nair_handle *h) {
  cudaStream_t s = h->s;
  cudaEvent_t e0, e1;
  NAIR_CK(cudaEventCreate(&e0));
  NAIR_CK(cudaEventCreate(&e1));
  NAIR_CK(cudaEventRecord(e0, s));
  if (h->mixed) build_transposed<float>(h->h32, h->P.f_sweeps, s, h->mem);
  else build_transposed<double>(h->h64, h->P.f_sweeps, s, h->mem);
  h->bwd.b = h->b;
  if (!h->mixed && !h->scalar) {  // level 0 of the transposed hierarchy is A^T itself
    h->bwd.A = h->h64.tlev[0].At;
    h->bwd.diag = h->h64.tlev[0].diag;
    h->bwd.C = h->h64.tl0c;
  } else {
    bsr_transpose<double>(h->A64, h->b, h->bwd.A, s, h->mem);
    int *diag = h->mem.alloc<int>(h->E);
    diag_positions(h->E, h->bwd.A.rp, h->bwd.A.ci, diag, s);
    h->bwd.diag = diag;
    build_l0comp<double>(h->bwd.A, diag, h->b, s, h->mem, h->bwd.C);
  }
  NAIR_CK(cudaEventRecord(e1, s));
  NAIR_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  NAIR_CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tsetup_ms = ms;
  h->tbuilt = true;
}

static void build_adjoint(nair_handle *h) {
  cudaStream_t s = h->s;
  nair_handle *a = new nair_handle();
  a->raw = h->raw;
  a->P = h->P;
  a->s = s;
  a->K.mem.s = s;
  a->mem.s = s;
  try {
    const int E = h->E, b = h->b, nnzb = h->A64.nnzb;
    bsr_transpose<double>(h->A64, b, a->A64, s, a->mem);
    setup_impl(a, nullptr, nullptr, nullptr, E, b, nnzb, true);
  } catch (...) {
    nair_free(a);
    throw;
  }
  h->adj = a;
}

nair_status nair_adjoint_solve(nair_handle *h, const double *w, double *lam, nair_info *info) {
  NAIR_API_BEGIN
  if (!h || !w || !lam) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (!aligned16(w) || !aligned16(lam)) return set_error(NAIR_ERR_INVALID_ARG, kAlignMsg);
  if (h->raw.adjoint_mode == NAIR_ADJOINT_REBUILD) {
    if (!h->adj) build_adjoint(h);
    return nair_solve(h->adj, w, lam, info);
  }
  if (!h->tbuilt) build_transposed_handle(h);
  return solve_impl(h, w, lam, info, true);
  NAIR_API_END
}

nair_status nair_adjoint_vcycle(nair_handle *h, const double *f, double *x) {
  NAIR_API_BEGIN
  if (!h || !f || !x) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (!aligned16(f) || !aligned16(x)) return set_error(NAIR_ERR_INVALID_ARG, kAlignMsg);
  if (!h->tbuilt) build_transposed_handle(h);
  if (h->mixed) precond<float>(h->h32, h->P, f, x, h->s, h->n, true);
  else precond<double>(h->h64, h->P, f, x, h->s, h->n, true);
  NAIR_CK(cudaStreamSynchronize(h->s));
  return NAIR_OK;
  NAIR_API_END
}

// ---------------------------------------------------------------------------
// batches of independent systems: one host thread per system, each issuing its
// system's work on that system's stream, so that the launch- and latency-bound
// parts (coarse levels, setup, Krylov read-backs) of the systems overlap
// ---------------------------------------------------------------------------
static constexpr int kMaxBatch = 256;

template <typename F>
static nair_status run_batch(int count, F fn) {
  int dev = 0;
  NAIR_CK(cudaGetDevice(&dev));
  std::vector<nair_status> st(count, NAIR_OK);
  std::vector<std::string> msg(count);
  std::vector<std::thread> th;
  th.reserve(count);
  for (int k = 0; k < count; ++k)
    th.emplace_back([&, k] {
      if (cudaSetDevice(dev) != cudaSuccess) {
        st[k] = NAIR_ERR_CUDA;
        msg[k] = "cudaSetDevice failed in a batch thread";
        return;
      }
      st[k] = fn(k);
      if (st[k] != NAIR_OK) msg[k] = g_last_error;
    });
  for (auto &t : th) t.join();
  for (int k = 0; k < count; ++k)
    if (st[k] != NAIR_OK) return set_error(st[k], "system " + std::to_string(k) + ": " + msg[k]);
  g_last_error.clear();
  return NAIR_OK;
}

nair_status nair_setup_batch(const nair_bsr *A, const nair_params *p, int32_t count, nair_handle **out) {
  NAIR_API_BEGIN
  if (!A || !p || !out) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (count < 1 || count > kMaxBatch) return set_error(NAIR_ERR_INVALID_ARG, "count must lie in 1..256");
  for (int k = 0; k < count; ++k) out[k] = nullptr;
  init_pool_once();
  nair_status st = run_batch(count, [&](int k) { return nair_setup(&A[k], &p[k], &out[k]); });
  if (st != NAIR_OK) {
    for (int k = 0; k < count; ++k) {
      nair_free(out[k]);
      out[k] = nullptr;
    }
  }
  return st;
  NAIR_API_END
}

nair_status nair_solve_batch(nair_handle *const *h, int32_t count, const double *const *b, double *const *x,
                             nair_info *info) {
  NAIR_API_BEGIN
  if (!h || !b || !x) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (count < 1 || count > kMaxBatch) return set_error(NAIR_ERR_INVALID_ARG, "count must lie in 1..256");
  for (int k = 0; k < count; ++k)
    for (int j = 0; j < k; ++j)
      if (h[j] == h[k]) return set_error(NAIR_ERR_INVALID_ARG, "a handle appears twice in the batch");
  return run_batch(count, [&](int k) { return nair_solve(h[k], b[k], x[k], info ? &info[k] : nullptr); });
  NAIR_API_END
}

nair_status nair_adjoint_solve_batch(nair_handle *const *h, int32_t count, const double *const *w,
                                     double *const *lam, nair_info *info) {
  NAIR_API_BEGIN
  if (!h || !w || !lam) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  if (count < 1 || count > kMaxBatch) return set_error(NAIR_ERR_INVALID_ARG, "count must lie in 1..256");
  for (int k = 0; k < count; ++k)
    for (int j = 0; j < k; ++j)
      if (h[j] == h[k]) return set_error(NAIR_ERR_INVALID_ARG, "a handle appears twice in the batch");
  return run_batch(count,
                   [&](int k) { return nair_adjoint_solve(h[k], w[k], lam[k], info ? &info[k] : nullptr); });
  NAIR_API_END
}

void nair_free(nair_handle *h) {
  if (!h) return;
  if (h->adj) nair_free(h->adj);
  cudaStreamSynchronize(h->s);
  release_graph(h->h64.graph);
  release_graph(h->h32.graph);
  release_graph(h->h64.tgraph);
  release_graph(h->h32.tgraph);
  release_clock(h->h64.clock);
  release_clock(h->h32.clock);
  h->K.mem.release_all();
  h->mem.release_all();
  cudaStreamSynchronize(h->s);
  delete h;
}

static const nair_handle *pick(const nair_handle *h, int adjoint) {
  if (!h) fail(NAIR_ERR_INVALID_ARG, "null handle");
  if (adjoint) {
    if (!h->adj) fail(NAIR_ERR_INVALID_ARG, "no adjoint hierarchy yet (call nair_adjoint_solve first)");
    return h->adj;
  }
  return h;
}

nair_status nair_num_levels(const nair_handle *h0, int32_t adjoint, int32_t *levels) {
  NAIR_API_BEGIN
  const nair_handle *h = pick(h0, adjoint);
  if (!levels) return set_error(NAIR_ERR_INVALID_ARG, "null argument");
  *levels = h->mixed ? h->h32.nlev : h->h64.nlev;
  return NAIR_OK;
  NAIR_API_END
}

template <typename T>
static void sizes_t(const Hier<T> &H, int l, int64_t *o) {
  const Level<T> &L = H.lev[l];
  o[0] = L.E;
  o[1] = L.A.nnzb;
  o[2] = L.nC;
  o[3] = L.nF;
  o[4] = L.L.nnzb;
  o[5] = L.Delta.nnzb;
  o[6] = L.R.nnzb;
  o[7] = 0;
  o[8] = L.coarsest;
  o[9] = L.cf_rounds;
}

template <typename T>
static void sweep_forms_t(const Hier<T> &H, bool transposed, int cap, int32_t *forms) {
  for (int l = 0; l < H.nlev && l < cap; ++l) {
    const Level<T> &L = H.lev[l];
    int f = 0;
    if (L.coarsest) {
      f = -1;
    } else if (!transposed) {
      if (l == 0 && H.l0c.W > 0) f = 1;
      else if (L.ymode) f = 3;
      else if (L.sr.srp) f = 2;
    } else {
      const TLevel<T> &TL = H.tlev[l];
      if (l == 0 && H.tl0c.W > 0) f = 1;
      else if (TL.ymode) f = 3;
      else if (TL.sr.srp) f = 2;
    }
    forms[l] = f;
  }
}

nair_status nair_sweep_forms(const nair_handle *h, int32_t transposed, int32_t cap, int32_t *forms) {
  NAIR_API_BEGIN
  if (!h || !forms || cap < 0) return set_error(NAIR_ERR_INVALID_ARG, "null handle or forms, or negative cap");
  if (transposed && !h->tbuilt) return set_error(NAIR_ERR_INVALID_ARG, "transposed cycle not built yet");
  if (h->mixed) sweep_forms_t(h->h32, transposed != 0, cap, forms);
  else sweep_forms_t(h->h64, transposed != 0, cap, forms);
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_level_sizes(const nair_handle *h0, int32_t adjoint, int32_t level, int64_t *sizes) {
  NAIR_API_BEGIN
  const nair_handle *h = pick(h0, adjoint);
  int nl = h->mixed ? h->h32.nlev : h->h64.nlev;
  if (level < 0 || level >= nl || !sizes) return set_error(NAIR_ERR_INVALID_ARG, "level out of range");
  if (h->mixed) sizes_t(h->h32, level, sizes);
  else sizes_t(h->h64, level, sizes);
  return NAIR_OK;
  NAIR_API_END
}

template <typename T>
static void copy_vals(const T *src, size_t count, void *out, cudaStream_t s) {
  if (!count) return;
  if constexpr (std::is_same<T, double>::value) {
    NAIR_CK(cudaMemcpyAsync(out, src, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
  } else {
    std::vector<T> tmp(count);
    NAIR_CK(cudaMemcpyAsync(tmp.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
    NAIR_CK(cudaStreamSynchronize(s));
    double *o = (double *)out;
    for (size_t i = 0; i < count; ++i) o[i] = (double)tmp[i];
  }
}

static void copy_raw(const void *src, size_t bytes, void *out, cudaStream_t s) {
  if (!bytes) return;
  if (!src) fail(NAIR_ERR_INVALID_ARG, "array not available (keep_setup_data not set, or coarsest level)");
  NAIR_CK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, s));
  NAIR_CK(cudaStreamSynchronize(s));
}

template <typename T>
static void get_level_t(const Hier<T> &H, int l, int which, void *out, size_t cap, size_t *need,
                        cudaStream_t s) {
  const Level<T> &L = H.lev[l];
  const size_t bb = (size_t)H.b * H.b;
  size_t bytes = 0;
  switch (which) {
    case NAIR_A_ROWPTR: bytes = sizeof(int) * (L.E + 1); break;
    case NAIR_A_COL: bytes = sizeof(int) * L.A.nnzb; break;
    case NAIR_A_VALS: bytes = sizeof(double) * bb * L.A.nnzb; break;
    case NAIR_DINV: bytes = sizeof(double) * bb * L.E; break;
    case NAIR_CF: bytes = L.cf ? (size_t)L.E : 0; break;
    case NAIR_P_MAP: bytes = L.ipc ? sizeof(int) * L.E : 0; break;
    case NAIR_DELTA_ROWPTR: bytes = L.Delta.rp ? sizeof(int) * (L.nF + 1) : 0; break;
    case NAIR_DELTA_COL: bytes = sizeof(int) * L.Delta.nnzb; break;
    case NAIR_DELTA_VALS: bytes = sizeof(double) * bb * L.Delta.nnzb; break;
    case NAIR_R_ROWPTR: bytes = L.R.rp ? sizeof(int) * (L.nC + 1) : 0; break;
    case NAIR_R_COL: bytes = sizeof(int) * L.R.nnzb; break;
    case NAIR_R_VALS: bytes = sizeof(double) * bb * L.R.nnzb; break;
    case NAIR_STRONG: bytes = L.strong ? (size_t)L.A.nnzb : 0; break;
    case NAIR_LAMBDA: bytes = L.lam ? sizeof(int) * L.E : 0; break;
    case NAIR_L_ROWPTR: bytes = L.L.rp ? sizeof(int) * (L.nF + 1) : 0; break;
    case NAIR_L_COL: bytes = sizeof(int) * L.L.nnzb; break;
    case NAIR_L_VALS: bytes = sizeof(double) * bb * L.L.nnzb; break;
    default: fail(NAIR_ERR_INVALID_ARG, "unknown level array");
  }
  if (need) *need = bytes;
  if (!out) return;
  if (cap < bytes) fail(NAIR_ERR_INVALID_ARG, "output buffer too small");
  switch (which) {
    case NAIR_A_ROWPTR: copy_raw(L.A.rp, bytes, out, s); break;
    case NAIR_A_COL: copy_raw(L.A.ci, bytes, out, s); break;
    case NAIR_A_VALS: copy_vals(L.A.v, bb * L.A.nnzb, out, s); break;
    case NAIR_DINV: copy_vals(L.dinv, bb * L.E, out, s); break;
    case NAIR_CF: copy_raw(L.cf, bytes, out, s); break;
    case NAIR_P_MAP: copy_raw(L.ipc, bytes, out, s); break;
    case NAIR_DELTA_ROWPTR: copy_raw(L.Delta.rp, bytes, out, s); break;
    case NAIR_DELTA_COL: copy_raw(L.Delta.ci, bytes, out, s); break;
    case NAIR_DELTA_VALS: copy_vals(L.Delta.v, bb * L.Delta.nnzb, out, s); break;
    case NAIR_R_ROWPTR: copy_raw(L.R.rp, bytes, out, s); break;
    case NAIR_R_COL: copy_raw(L.R_ci_f, bytes, out, s); break;
    case NAIR_R_VALS: copy_vals(L.R.v, bb * L.R.nnzb, out, s); break;
    case NAIR_STRONG: copy_raw(L.strong, bytes, out, s); break;
    case NAIR_LAMBDA: copy_raw(L.lam, bytes, out, s); break;
    case NAIR_L_ROWPTR: copy_raw(L.L.rp, bytes, out, s); break;
    case NAIR_L_COL: copy_raw(L.L.ci, bytes, out, s); break;
    case NAIR_L_VALS: copy_vals(L.L.v, bb * L.L.nnzb, out, s); break;
  }
}

nair_status nair_get_level(const nair_handle *h0, int32_t adjoint, int32_t level, int32_t which,
                           void *host_out, size_t cap, size_t *need) {
  NAIR_API_BEGIN
  const nair_handle *h = pick(h0, adjoint);
  int nl = h->mixed ? h->h32.nlev : h->h64.nlev;
  if (level < 0 || level >= nl) return set_error(NAIR_ERR_INVALID_ARG, "level out of range");
  if (h->mixed) get_level_t(h->h32, level, which, host_out, cap, need, h->s);
  else get_level_t(h->h64, level, which, host_out, cap, need, h->s);
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_block_inverse(int32_t nblk, int32_t b, const double *A, double *Ainv, void *stream) {
  NAIR_API_BEGIN
  if (nblk < 0 || b < 1 || b > 32 || (nblk > 0 && (!A || !Ainv)))
    return set_error(NAIR_ERR_INVALID_ARG, "bad block-inverse arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Mem tmp;
  tmp.s = s;
  int *err = tmp.alloc<int>(1);
  NAIR_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  block_inverses<double>(nblk, b, A, nullptr, Ainv, err, s);
  if (read_int(err, s)) return set_error(NAIR_ERR_SINGULAR_BLOCK, "singular block");
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_assemble_sigma(int32_t E, int32_t b, int64_t nnzb, const int32_t *diag_pos,
                                const double *vals0, const double *M, const double *sigma,
                                double *vals, void *stream) {
  NAIR_API_BEGIN
  if (E < 0 || b < 1 || b > 32 || nnzb < E || !diag_pos || !vals0 || !M || !sigma || !vals)
    return set_error(NAIR_ERR_INVALID_ARG, "bad assemble arguments");
  cudaStream_t s = (cudaStream_t)stream;
  long long tot = nnzb * b * b;
  if (vals != vals0) {
    k_copy64<<<grid(tot), kThreads, 0, s>>>(tot, vals0, vals);
    NAIR_LAUNCH_CHECK();
  }
  long long td = (long long)E * b * b;
  k_assemble_sigma<<<grid(td), kThreads, 0, s>>>(E, b, diag_pos, vals0, M, sigma, vals);
  NAIR_LAUNCH_CHECK();
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_mass_apply(int32_t E, int32_t b, const double *M, const double *q, double *rhs, void *stream) {
  NAIR_API_BEGIN
  if (E < 0 || b < 1 || b > 32 || !M || !q || !rhs) return set_error(NAIR_ERR_INVALID_ARG, "bad mass arguments");
  cudaStream_t s = (cudaStream_t)stream;
  k_mass_apply<<<grid((long long)E * b), kThreads, 0, s>>>(E, b, M, q, rhs);
  NAIR_LAUNCH_CHECK();
  return NAIR_OK;
  NAIR_API_END
}

nair_status nair_gradients(int32_t E, int32_t b, const double *M, const double *lambda, const double *x,
                           double *gsigma, double *gq, void *stream) {
  NAIR_API_BEGIN
  if (E < 0 || b < 1 || b > 32 || !M || !lambda || !x || !gsigma || !gq)
    return set_error(NAIR_ERR_INVALID_ARG, "bad gradient arguments");
  cudaStream_t s = (cudaStream_t)stream;
  k_gradients<<<grid(E), kThreads, 0, s>>>(E, b, M, lambda, x, gsigma, gq);
  NAIR_LAUNCH_CHECK();
  return NAIR_OK;
  NAIR_API_END
}

