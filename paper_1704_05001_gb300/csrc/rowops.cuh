// Block-row kernels of the solve phase (a10-a14): SpMV, residual, block
// Jacobi sweep (optionally reading its input through the one-point
// interpolation, which fuses x = P x_c into the first sweep) and restriction.
//
// A team of G x b threads owns one block row: thread (g, r) accumulates output
// component r over the row's blocks p = start + g, start + g + G, ...; the G
// partial sums are then added by a fixed pairwise tree.  b is a template
// parameter for the common DG block sizes so that the b loads of a block row
// and of x_j are issued back to back (no exposed latency per scalar), with a
// runtime-b fallback.  G > 1 is used on coarse levels, whose rows are long and
// few, to shorten the serial chain per thread and to fill the GPU.
#pragma once

#include "common.cuh"

namespace nair {

// OP_INTERP_T: out_i = f_i + sum_j v_ij x_j + (c2f[i] >= 0 ? x[c2f[i]] : 0), the
// interpolation x_fine += R^T x_c of the transposed cycle (c2f: own coarse index)
// OP_JACOBI_S (level-0 form only): the block-Jacobi sweep with the couplings
// scaled in advance, x_i = g_i - sum_{j != i} (D_ii^{-1} A_ij) x_j, g = D^{-1} f
// (a.f = g, a.ov = the scaled compressed blocks)
enum RowOp { OP_SPMV = 0, OP_RESID = 1, OP_JACOBI = 2, OP_RESTRICT = 3, OP_INTERP_T = 4, OP_JACOBI_S = 5 };

template <typename T>
struct RowArgs {
  int nrows, b, G, tpc;
  const int *rp, *ci;
  const T *v;
  const T *x;            // input vector; read as x[ipc[j]] (or 0) when ipc is set
  const int *ipc;
  const T *f;            // right-hand side (RESID, JACOBI) or fine vector (RESTRICT)
  const int *c2f;        // RESTRICT: coarse row -> fine element of its identity part
  const T *dinv;         // JACOBI: inverse diagonal blocks
  const int *list;       // rows to process (null: rows 0..nrows-1)
  T *out;
  // JACOBI copy segment: thread blocks comp_ctas.. copy rows copy_list[0..ncopy)
  // of the input (through ipc when set) into out and, if set, out2
  int comp_ctas, ncopy;
  const int *copy_list;
  T *out2;
  T *out2c;              // JACOBI: optional second output of the updated rows
  unsigned long long *stamp;  // optional: [0] earliest start, [ns] latest end (device clock)
  int ns;
  // level-0 column-compressed off-diagonal blocks (k_rowop_l0)
  const int *diag, *oci;
  const unsigned long long *ocols;
  const T *ov;
  // scalar-row form (k_scalar_rows): entries srp[i b + r] ..
  // srp[i b + r + 1] are the off-diagonal blocks of row i whose row r has a
  // nonzero, packed: sj[e] the block column, sv[e b ..] row r of the block;
  // perm orders each thread block's scalar rows by entry count
  const int *srp, *sj;
  const T *sv;
  const unsigned char *perm;
  // F sweeps with the C part of the F rows summed once (k_scalar_rows, OP_JACOBI):
  // the entries of an F row's scalar row list its C columns first, up to srs,
  // then its F columns.  fmode 1 (the first F sweep of a cycle): h = f - the C
  // part, stored, then the F part subtracted; fmode 2 (later F sweeps, x_C
  // unchanged): h read back and only the F part summed; fmode 0: every entry.
  // fmodes 3 and 4 are 1 and 2 with the F rows iterating on y = D x (no
  // D^{-1} applied; 4 reads sv = the right-scaled entries A_ij D_jj^{-1});
  // fmode 5 is the C sweep after them (sv = the scaled entries for its F
  // columns), whose copy part writes the F rows as x = D^{-1} y
  const int *srs;
  T *h;
  int fmode;
};

// B consecutive values from p into registers, as 16-byte loads where the
// row's size allows it (the callers' rows start on 16-byte boundaries then:
// every row offset is a multiple of B values and the arrays are allocated
// with 256-byte alignment)
template <typename T, int B>
__device__ __forceinline__ void load_row(const T *__restrict__ p, T (&o)[B]) {
  if constexpr (sizeof(T) == 8 && B % 2 == 0) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int c = 0; c < B / 2; ++c) {
      const double2 t = q[c];
      o[2 * c] = t.x;
      o[2 * c + 1] = t.y;
    }
  } else if constexpr (sizeof(T) == 4 && B % 4 == 0) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int c = 0; c < B / 4; ++c) {
      const float4 t = q[c];
      o[4 * c] = t.x;
      o[4 * c + 1] = t.y;
      o[4 * c + 2] = t.z;
      o[4 * c + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 4 && B % 2 == 0) {
    const float2 *q = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int c = 0; c < B / 2; ++c) {
      const float2 t = q[c];
      o[2 * c] = t.x;
      o[2 * c + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < B; ++c) o[c] = p[c];
  }
}

// the same values with scalar loads (prologue loads held across the
// dependency wait, where 16-byte loads cost registers)
template <typename T, int B>
__device__ __forceinline__ void load_row_scalar(const T *__restrict__ p, T (&o)[B]) {
#pragma unroll
  for (int c = 0; c < B; ++c) o[c] = p[c];
}

__device__ __forceinline__ unsigned long long global_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T, int B>
__device__ __forceinline__ T xval(const T *__restrict__ x, const int *__restrict__ ipc, int j, int c, int b) {
  const int bt = B > 0 ? B : b;
  if (ipc) {
    const int J = ipc[j];
    return J >= 0 ? x[(size_t)J * bt + c] : (T)0;
  }
  return x[(size_t)j * bt + c];
}


// partial sum of row i over the blocks p = p0, p0 + G, ... < p1; the first
// block's column, interpolation target and values (va0) were loaded before the
// dependency wait, because the matrix does not change during a V-cycle
template <typename T, int B>
__device__ __forceinline__ T row_partial(const RowArgs<T> &a, int p0, int p1, int r, int j0,
                                         const T *va0, int skip) {
  const int b = B > 0 ? B : a.b;
  const int bb = b * b;
  T acc = 0;
  if constexpr (B > 0) {
    if (p0 < p1 && j0 >= 0 && p0 != skip) {
      T vx[B];
      load_row<T, B>(a.x + (size_t)j0 * B, vx);
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(va0[c], vx[c], acc);
    }
#pragma unroll 2
    for (int p = p0 + a.G; p < p1; p += a.G) {
      if (p == skip) continue;
      int j = a.ci[p];
      if (a.ipc) {
        j = a.ipc[j];
        if (j < 0) continue;
      }
      T va[B], vx[B];
      load_row_scalar<T, B>(a.v + (size_t)p * bb + r * B, va);
      load_row_scalar<T, B>(a.x + (size_t)j * B, vx);
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(va[c], vx[c], acc);
    }
  } else {
    for (int p = p0; p < p1; p += a.G) {
      if (p == skip) continue;
      const int j = a.ci[p];
      const T *av = a.v + (size_t)p * bb + r * b;
#pragma unroll 4
      for (int c = 0; c < b; ++c) acc = fma(av[c], xval<T, 0>(a.x, a.ipc, j, c, b), acc);
    }
  }
  return acc;
}

template <typename T, int B, int OP>
__global__ void __launch_bounds__(256) k_rowop(RowArgs<T> a) {
  pdl_launch_dependents();
  if (OP == OP_JACOBI && (int)blockIdx.x >= a.comp_ctas) {
    // copy segment: rows of the class this sweep does not update
    const int bt = B > 0 ? B : a.b;
    const long long g = (long long)(blockIdx.x - a.comp_ctas) * blockDim.x + threadIdx.x;
    const bool in = g < (long long)a.ncopy * bt;
    const int row = in ? (int)(g / bt) : 0, r = in ? (int)(g - (long long)row * bt) : 0;
    const int i = in ? a.copy_list[row] : 0;
    const int J = (in && a.ipc) ? a.ipc[i] : i;
    pdl_wait();
    if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
    if (in) {
      const T v = a.ipc ? (J >= 0 ? a.x[(size_t)J * bt + r] : (T)0) : a.x[(size_t)i * bt + r];
      a.out[(size_t)i * bt + r] = v;
      if (a.out2) a.out2[(size_t)i * bt + r] = v;
    }
    if (a.stamp) {
      __syncthreads();
      if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
    }
    return;
  }
  extern __shared__ unsigned char smraw[];
  T *red = reinterpret_cast<T *>(smraw);             // [tpc][G][b]
  const int b = B > 0 ? B : a.b;
  const int tsz = a.G * b;
  T *sres = red + (size_t)a.tpc * tsz;               // [tpc][b]
  const int team = threadIdx.x / tsz, lt = threadIdx.x - team * tsz;
  const int g = lt / b, r = lt - g * b;
  const int idx = blockIdx.x * a.tpc + team;
  const bool active = team < a.tpc && idx < a.nrows;
  // ---- prologue on data that is constant during the V-cycle
  const int i = active ? (a.list ? a.list[idx] : idx) : 0;
  const int p0 = active ? a.rp[i] + g : 0, p1 = active ? a.rp[i + 1] : 0;
  int j0 = -1;
  T va0[B > 0 ? B : 1];
  T dv[(OP == OP_JACOBI && B > 0) ? B : 1];
  int ii = 0;
  if constexpr (B > 0) {
    if (p0 < p1) {
      j0 = a.ci[p0];
      if (a.ipc) j0 = a.ipc[j0];
      load_row_scalar<T, B>(a.v + (size_t)p0 * B * B + r * B, va0);
    }
    if constexpr (OP == OP_JACOBI) {
      if (active && g == 0) load_row_scalar<T, B>(a.dinv + (size_t)i * B * B + r * B, dv);
    }
  }
  // JACOBI works in the classical form x_i = D_ii^{-1} (f_i - sum_{j != i} A_ij x_j):
  // the diagonal block is skipped and x_i is not read
  const int skip = (OP == OP_JACOBI && active) ? a.diag[i] : -1;
  if ((OP == OP_RESTRICT || OP == OP_INTERP_T) && active && g == 0) ii = a.c2f[i];
  // ---- wait for the producer of x and f
  pdl_wait();
  if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
  T acc = 0;
  if (active) acc = row_partial<T, B>(a, p0, p1, r, j0, va0, skip);
  if (a.G > 1) {  // pairwise tree over the G partial sums (G is a power of two)
    T *tr = red + (size_t)team * tsz;
    if (team < a.tpc) tr[lt] = acc;
    __syncthreads();
    for (int h = a.G / 2; h > 0; h >>= 1) {
      if (team < a.tpc && g < h) tr[lt] += tr[lt + h * b];
      __syncthreads();
    }
    if (g == 0 && active) acc = tr[r];
  }
  if (OP == OP_SPMV) {
    if (active && g == 0) a.out[(size_t)i * b + r] = acc;
  } else if (OP == OP_RESID) {
    if (active && g == 0) a.out[(size_t)i * b + r] = a.f[(size_t)i * b + r] - acc;
  } else if (OP == OP_RESTRICT) {
    if (active && g == 0) a.out[(size_t)i * b + r] = a.f[(size_t)ii * b + r] + acc;
  } else if (OP == OP_INTERP_T) {
    if (active && g == 0) {
      T v = a.f[(size_t)i * b + r] + acc;
      if (ii >= 0) v += a.x[(size_t)ii * b + r];
      a.out[(size_t)i * b + r] = v;
    }
  } else {  // OP_JACOBI
    if (active && g == 0) sres[(size_t)team * b + r] = a.f[(size_t)i * b + r] - acc;
    __syncthreads();
    if (active && g == 0) {
      const T *sr = sres + (size_t)team * b;
      T s = 0;
      if constexpr (B > 0) {
#pragma unroll
        for (int c = 0; c < B; ++c) s = fma(dv[c], sr[c], s);
      } else {
        const T *d = a.dinv + (size_t)i * b * b + r * b;
        for (int c = 0; c < b; ++c) s = fma(d[c], sr[c], s);
      }
      a.out[(size_t)i * b + r] = s;
      if (a.out2c) a.out2c[(size_t)i * b + r] = s;
    }
  }
  if (a.stamp) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
  }
}

// Scalar-row form of the coarse-level row kernels (levels >= 1, whose
// off-diagonal blocks -- and the blocks of R_cf -- keep about half of their
// rows zero): thread block c owns rows list[c tpc ..] (rows c tpc .. when list
// is null), and its tpc x B scalar rows (i, r) are assigned, G threads each,
// in the order perm gives -- sorted by entry count, so that the threads of a
// warp run loops of nearly equal length and the FP64 pipe is not spent on the
// zero rows of the blocks.  Thread g of scalar row (i, r) accumulates
// sum_e sv_e . x_{sj_e} over its packed entries g, g + G, ... in ascending
// block order; the G partial sums are added by the pairwise tree of the row
// kernels.  Then each thread of the natural layout finishes component r of
// row i:
//   OP_JACOBI: row r of D_ii^{-1} applied to f_i - sum (from shared memory);
//     in the F sweeps of the y form (FM 3, 4) the result is y_i = h_i - sum
//     itself, written by the thread that summed it when G = 1 (no exchange);
//   OP_RESTRICT: f_c = f_{c2f[i]} + sum, the restriction f_c = f_C + R_cf f_F.
// Six thread blocks per SM (register cap 40): these sweeps wait on memory, and
// the extra resident warps gained more than the few spilled registers cost
// (C5 FP64, Neumann degree 6: solve 145.9 -> 140.8 ms)
template <typename T, int B, int OP, int FM = 0>
__global__ void __launch_bounds__(256, 6) k_scalar_rows(RowArgs<T> a) {
  pdl_launch_dependents();
  if (OP == OP_JACOBI && (int)blockIdx.x >= a.comp_ctas) {  // copy segment, as in k_rowop
    const long long g = (long long)(blockIdx.x - a.comp_ctas) * blockDim.x + threadIdx.x;
    const bool in = g < (long long)a.ncopy * B;
    const int row = in ? (int)(g / B) : 0, r = in ? (int)(g - (long long)row * B) : 0;
    const int i = in ? a.copy_list[row] : 0;
    const int J = (in && a.ipc) ? a.ipc[i] : i;
    pdl_wait();
    if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
    if (in) {
      T v;
      if constexpr (FM == 5) {  // an F row's x = D^{-1} y from the scaled iterate
        const T *d = a.dinv + ((size_t)i * B + r) * B;
        const T *y = a.x + (size_t)i * B;
        v = 0;
#pragma unroll
        for (int c = 0; c < B; ++c) v = fma(d[c], y[c], v);
      } else {
        v = a.ipc ? (J >= 0 ? a.x[(size_t)J * B + r] : (T)0) : a.x[(size_t)i * B + r];
      }
      a.out[(size_t)i * B + r] = v;
      if (a.out2) a.out2[(size_t)i * B + r] = v;
    }
    if (a.stamp) {
      __syncthreads();
      if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
    }
    return;
  }
  // F sweep modes: 1, 3 the first (h = f - C part stored, then the F part),
  // 2, 4 the later ones (h - F part); 3, 4 leave the result in y = D x (no
  // D^{-1}); 5 is the C sweep after them (D^{-1} applied to its rows, the F
  // rows copied as x = D^{-1} y)
  constexpr bool kFirst = FM == 1 || FM == 3, kLater = FM == 2 || FM == 4, kNoInv = FM == 3 || FM == 4;
  __shared__ T sres[256];
  __shared__ T red[256];
  const int G = a.G;
  const int base = blockIdx.x * a.tpc;
  const int nact = min(a.tpc, a.nrows - base);  // rows of this thread block
  const int t = threadIdx.x;
  // sorted layout: this thread's scalar row and its share g of the entries
  const int slot = t / G, g = t - slot * G;
  const bool act = slot < nact * B;
  const int enc = act ? (int)a.perm[(size_t)base * B + slot] : 0;
  const int team = enc / B, r = enc - team * B;
  const int i = act ? (a.list ? a.list[base + team] : base + team) : 0;
  // entry ranges: A = every entry (fmode 0), the C part (1) or the F part (2);
  // B = the F part in fmode 1, else empty
  int s0 = 0, sm = 0, s1 = 0;
  if (act) {
    const size_t q = (size_t)i * B + r;
    s0 = a.srp[q];
    s1 = a.srp[q + 1];
    sm = FM ? a.srs[q] : s0;
  }
  const int e0 = (kLater ? sm : s0) + g, e1 = kFirst ? sm : s1;
  // natural layout: the row and component this thread finishes.  For the
  // sweep with B <= 10 the thread block's D^{-1} blocks are staged in shared
  // memory before the dependency wait; larger blocks are read after the loop
  const int team2 = t / B, r2 = t - team2 * B;
  const bool act2 = team2 < nact;
  const int i2 = act2 ? (a.list ? a.list[base + team2] : base + team2) : 0;
  const int own = (OP == OP_RESTRICT && act2) ? a.c2f[i2] : i2;  // row of f this component takes
  constexpr bool kStage = OP == OP_JACOBI && B <= 10 && !kNoInv;
  __shared__ T sd[kStage ? (256 / B) * B * B : 1];
  if constexpr (kStage) {
    for (int q = t; q < nact * B * B; q += blockDim.x) {
      const int tm = q / (B * B);
      sd[q] = a.dinv[(size_t)a.list[base + tm] * B * B + (q - tm * B * B)];
    }
  }
  // the first entry's values and the first two columns do not change during
  // the cycle: loaded before the dependency wait
  int j0 = -1, jn = 0;
  T va0[B];
  if (e0 < e1) {
    j0 = a.sj[e0];
    if (a.ipc) j0 = a.ipc[j0];
    load_row_scalar<T, B>(a.sv + (size_t)e0 * B, va0);
    if (e0 + G < e1) jn = a.sj[e0 + G];
  }
  pdl_wait();
  if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
  T acc = 0;
  if (e0 < e1 && j0 >= 0) {
    T vx[B];
    load_row<T, B>(a.x + (size_t)j0 * B, vx);
#pragma unroll
    for (int c = 0; c < B; ++c) acc = fma(va0[c], vx[c], acc);
  }
  // each entry's column was loaded one entry ahead, so the gather of x starts
  // at once and the next column's load overlaps it
#pragma unroll 2
  for (int e = e0 + G; e < e1; e += G) {
    int j = jn;
    if (e + G < e1) jn = a.sj[e + G];
    if (a.ipc) {
      j = a.ipc[j];
      if (j < 0) continue;
    }
    T va[B], vx[B];
    if constexpr (B >= 10) {  // 16-byte loads; for smaller rows they cost spills
      load_row<T, B>(a.sv + (size_t)e * B, va);
      load_row<T, B>(a.x + (size_t)j * B, vx);
    } else {
      load_row_scalar<T, B>(a.sv + (size_t)e * B, va);
      load_row_scalar<T, B>(a.x + (size_t)j * B, vx);
    }
#pragma unroll
    for (int c = 0; c < B; ++c) acc = fma(va[c], vx[c], acc);
  }
  T accB = 0;
  if constexpr (OP == OP_JACOBI && kFirst) {  // the F part of the first F sweep
#pragma unroll 2
    for (int e = sm + g; e < s1; e += G) {
      int j = a.sj[e];
      if (a.ipc) {
        j = a.ipc[j];
        if (j < 0) continue;
      }
      T va[B], vx[B];
      if constexpr (B >= 10) {
        load_row<T, B>(a.sv + (size_t)e * B, va);
        load_row<T, B>(a.x + (size_t)j * B, vx);
      } else {
        load_row_scalar<T, B>(a.sv + (size_t)e * B, va);
        load_row_scalar<T, B>(a.x + (size_t)j * B, vx);
      }
#pragma unroll
      for (int c = 0; c < B; ++c) accB = fma(va[c], vx[c], accB);
    }
  }
  // f_i - the row's sum: with the C part kept in h (stored in fmode 1, read
  // back in fmode 2)
  auto residual = [&](int row, int comp, T sumA, T sumB) -> T {
    const size_t q = (size_t)row * B + comp;
    if constexpr (kFirst) {
      const T hv = a.f[q] - sumA;
      a.h[q] = hv;
      return hv - sumB;
    } else if constexpr (kLater) {
      return a.h[q] - sumA;
    } else {
      return a.f[q] - sumA;
    }
  };
  if (G > 1) {  // pairwise tree over the G partial sums of each scalar row
    if (act) red[enc * G + g] = acc;
    __syncthreads();
    for (int h = G / 2; h > 0; h >>= 1) {
      if (act && g < h) red[enc * G + g] += red[enc * G + g + h];
      __syncthreads();
    }
    T sumB = 0;
    if (OP == OP_JACOBI && kFirst) {  // the same tree for the F part
      const T sumA = (t < nact * B) ? red[t * G] : (T)0;
      __syncthreads();
      if (act) red[enc * G + g] = accB;
      __syncthreads();
      for (int h = G / 2; h > 0; h >>= 1) {
        if (act && g < h) red[enc * G + g] += red[enc * G + g + h];
        __syncthreads();
      }
      if (t < nact * B) sres[t] = residual(i2, r2, sumA, red[t * G]);
    } else if (OP == OP_RESTRICT) {
      if (act2) a.out[(size_t)i2 * B + r2] = a.f[(size_t)own * B + r2] + red[t * G];
    } else if (t < nact * B) {
      sres[t] = residual(i2, r2, red[t * G], sumB);
    }
  } else if (act) {
    if (OP == OP_RESTRICT) {
      a.out[(size_t)i * B + r] = a.f[(size_t)a.c2f[i] * B + r] + acc;
    } else if (kNoInv) {  // y of this scalar row: no exchange needed
      const T y = residual(i, r, acc, accB);
      a.out[(size_t)i * B + r] = y;
      if (a.out2c) a.out2c[(size_t)i * B + r] = y;
    } else {
      sres[enc] = residual(i, r, acc, accB);
    }
  }
  if constexpr (OP == OP_JACOBI && kNoInv) {
    if (G > 1) {
      __syncthreads();
      if (act2) {
        a.out[(size_t)i2 * B + r2] = sres[t];
        if (a.out2c) a.out2c[(size_t)i2 * B + r2] = sres[t];
      }
    }
  } else if constexpr (OP == OP_JACOBI) {
    __syncthreads();
    if (act2) {
      const T *d = kStage ? sd + (size_t)team2 * B * B + r2 * B : a.dinv + (size_t)i2 * B * B + r2 * B;
      T s2 = 0;
#pragma unroll
      for (int c = 0; c < B; ++c) s2 = fma(d[c], sres[team2 * B + c], s2);
      a.out[(size_t)i2 * B + r2] = s2;
      if (a.out2c) a.out2c[(size_t)i2 * B + r2] = s2;
    }
  }
  if (a.stamp) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
  }
}

// host launcher of the scalar-row kernels (OP_JACOBI, OP_RESTRICT) with G
// threads per scalar row and tpc = max(1, 256 / (b G)) rows per thread block
// (b in 3, 6, 10, 15, 21, 28); false if there is no kernel for b
template <typename T, int OP>
bool launch_scalar_rows(RowArgs<T> a, int G, cudaStream_t s);

// Level-0 form of the row kernel: the diagonal block from the BSR values, the
// off-diagonal blocks from their W nonzero columns (one team of B threads per
// row).  Same operations as k_rowop for OP_SPMV, OP_RESID and OP_JACOBI.
template <typename T, int B, int W, int OP>
__global__ void __launch_bounds__(256) k_rowop_l0(RowArgs<T> a) {
  pdl_launch_dependents();
  if ((OP == OP_JACOBI || OP == OP_JACOBI_S) && (int)blockIdx.x >= a.comp_ctas) {
    const long long g = (long long)(blockIdx.x - a.comp_ctas) * blockDim.x + threadIdx.x;
    const bool in = g < (long long)a.ncopy * B;
    const int row = in ? (int)(g / B) : 0, r = in ? (int)(g - (long long)row * B) : 0;
    const int i = in ? a.copy_list[row] : 0;
    const int J = (in && a.ipc) ? a.ipc[i] : i;
    pdl_wait();
    if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
    if (in) {
      const T v = a.ipc ? (J >= 0 ? a.x[(size_t)J * B + r] : (T)0) : a.x[(size_t)i * B + r];
      a.out[(size_t)i * B + r] = v;
      if (a.out2) a.out2[(size_t)i * B + r] = v;
    }
    if (a.stamp) {
      __syncthreads();
      if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
    }
    return;
  }
  __shared__ T sres[256];
  const int team = threadIdx.x / B, r = threadIdx.x - team * B;
  const int idx = blockIdx.x * a.tpc + team;
  const bool active = team < a.tpc && idx < a.nrows;
  // ---- prologue on data that is constant during the V-cycle
  const int i = active ? (a.list ? a.list[idx] : idx) : 0;
  const int q0 = active ? a.rp[i] - i : 0, q1 = active ? a.rp[i + 1] - i - 1 : 0;
  // JACOBI: the classical form x_i = D_ii^{-1} (f_i - sum_{j != i} A_ij x_j)
  // needs neither the diagonal block nor x_i
  constexpr bool kDiag = OP != OP_JACOBI && OP != OP_JACOBI_S;
  T dv[kDiag ? B : 1], drow[OP == OP_JACOBI ? B : 1], ov0[W];
  int j0 = -1;
  unsigned long long cols0 = 0;
  if (active) {
    if constexpr (kDiag) load_row_scalar<T, B>(a.v + (size_t)a.diag[i] * B * B + r * B, dv);
    if constexpr (OP == OP_JACOBI) load_row_scalar<T, B>(a.dinv + (size_t)i * B * B + r * B, drow);
    if (q0 < q1) {
      j0 = a.oci[q0];
      if (a.ipc) j0 = a.ipc[j0];
      cols0 = a.ocols[q0];
      load_row_scalar<T, W>(a.ov + (size_t)q0 * B * W + r * W, ov0);
    }
  }
  // ---- wait for the producer of x and f
  pdl_wait();
  if (a.stamp && threadIdx.x == 0) atomicMin(a.stamp, global_clock());
  T acc = 0;
  if (active) {
    if constexpr (kDiag) {  // SPMV / RESID: x is never read through ipc
      T xv[B];
      load_row<T, B>(a.x + (size_t)i * B, xv);
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(dv[c], xv[c], acc);
    }
    if (q0 < q1 && j0 >= 0) {
      const T *xj = a.x + (size_t)j0 * B;
#pragma unroll
      for (int w = 0; w < W; ++w) acc = fma(ov0[w], xj[(cols0 >> (8 * w)) & 255u], acc);
    }
    for (int q = q0 + 1; q < q1; ++q) {
      int j = a.oci[q];
      if (a.ipc) {
        j = a.ipc[j];
        if (j < 0) continue;
      }
      const unsigned long long cols = a.ocols[q];
      const T *xj = a.x + (size_t)j * B;
      T ovq[W], xq[W];
      if constexpr (OP == OP_JACOBI) load_row_scalar<T, W>(a.ov + (size_t)q * B * W + r * W, ovq);
      else load_row<T, W>(a.ov + (size_t)q * B * W + r * W, ovq);
#pragma unroll
      for (int w = 0; w < W; ++w) xq[w] = xj[(cols >> (8 * w)) & 255u];
#pragma unroll
      for (int w = 0; w < W; ++w) acc = fma(ovq[w], xq[w], acc);
    }
  }
  if (OP == OP_SPMV) {
    if (active) a.out[(size_t)i * B + r] = acc;
  } else if (OP == OP_RESID) {
    if (active) a.out[(size_t)i * B + r] = a.f[(size_t)i * B + r] - acc;
  } else if (OP == OP_JACOBI_S) {
    if (active) {
      const T v = a.f[(size_t)i * B + r] - acc;
      a.out[(size_t)i * B + r] = v;
      if (a.out2c) a.out2c[(size_t)i * B + r] = v;
    }
  } else {
    if (active) sres[team * B + r] = a.f[(size_t)i * B + r] - acc;
    __syncthreads();
    if (active) {
      T s2 = 0;
#pragma unroll
      for (int c = 0; c < B; ++c) s2 = fma(drow[c], sres[team * B + c], s2);
      a.out[(size_t)i * B + r] = s2;
      if (a.out2c) a.out2c[(size_t)i * B + r] = s2;
    }
  }
  if (a.stamp) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(a.stamp + a.ns, global_clock());
  }
}

// host launcher of the level-0 form (b must have a compressed width W)
template <typename T, int OP>
void launch_rowop_l0(RowArgs<T> a, int W, cudaStream_t s);

// host launcher: picks the team shape from the average row length; for JACOBI,
// a.nrows / a.list are the rows to update and a.ncopy / a.copy_list the rows to copy
template <typename T, int OP>
void launch_rowop(RowArgs<T> a, double avg_blocks, cudaStream_t s);

}  // namespace nair
