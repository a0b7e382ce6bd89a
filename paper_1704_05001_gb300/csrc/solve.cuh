// Solve-phase declarations: Krylov workspace, FP64 SpMV and flexible GMRES.
#pragma once

#include <type_traits>
#include <vector>

#include "hier.cuh"

namespace nair {

// FGMRES(m) workspace: basis V (m + 1 vectors), preconditioned vectors Z (m),
// one work vector, Arnoldi partial sums, a pinned host staging buffer and two
// pinned read-back slots (with their events) for the Hessenberg columns of
// two consecutive iterations, which are in flight together
struct Krylov {
  Mem mem;
  long long n = 0;
  int m = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *partial = nullptr, *hdev = nullptr,
         *ydev = nullptr, *hhost = nullptr;
  double *slot[2] = {};
  cudaEvent_t ev[2] = {};
  void ensure(long long n, int m, cudaStream_t s);
  ~Krylov();
};

void spmv64(const DBsr<double> &A, int b, const double *x, const double *bvec, double *y, cudaStream_t s,
            const L0Comp<double> *C = nullptr, const int *diag = nullptr);

// the operator of the Krylov solve (A, or A^T for the adjoint) in FP64 with its
// block size, diagonal-block positions and level-0 column compression
struct Outer {
  DBsr<double> A;
  int b = 0;
  const int *diag = nullptr;
  L0Comp<double> C;
};

template <typename T>
void precond(const Hier<T> &H, const Params &P, const double *v, double *z, cudaStream_t s, long long n,
             bool transposed = false);

template <typename T>
nair_status fgmres(const Outer &op, const Hier<T> &H, const Params &P, Krylov &K, const double *bvec,
                   double *x, std::vector<double> &hist, int *iters, double *relres, cudaStream_t s,
                   bool transposed = false);

}  // namespace nair
