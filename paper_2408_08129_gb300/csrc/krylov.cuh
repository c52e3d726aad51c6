// Restarted GMRES(m) on the device for the pressure Helmholtz problem of the
// implicit stage (Sec. 3.2: a non-symmetric linear system solved by GMRES
// inside the pressure fixed-point loop).
//
// Arnoldi with classical Gram-Schmidt applied twice; Hessenberg matrix, Givens
// rotations and the residual estimate live on the device and are updated by
// one single-thread kernel per iteration, so no iteration needs the host.  A
// device flag `done` turns the remaining kernels of a restart cycle into
// no-ops once the estimate meets the tolerance; the host reads the residual
// once per cycle.  Dot products accumulate in FP64 with a fixed reduction
// order, whatever the vector type, so results are bitwise reproducible.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int kDotBlocks = 160;
constexpr int kDotThreads = 256;

// device scalars and small arrays of one GMRES instance
struct GmresDev {
  double* H;        // [(m+1)*m] column-major: H[k*(m+1) + j]
  double* cs;       // [m]
  double* sn;       // [m]
  double* g;        // [m+1]
  double* h1;       // [m+1] first Gram-Schmidt coefficients of the current column
  double* h2;       // [m+1] second pass
  double* y;        // [m]
  double* partial;  // [(m+1)*kDotBlocks]
  double* scal;     // [8]: 0 bnorm^2, 1 beta^2, 2 resid, 3 1/h, 4 w.w, 5 tol
  int* iflag;       // [4]: 0 done, 1 kdone (iterations in this cycle), 2 zero rhs
};

struct GmresResult {
  int iters = 0;
  double rel = 0.0;
  bool converged = false;
};

template <typename Tv>
struct Gmres {
  int m = 30;
  int64_t n = 0;
  Tv* Q = nullptr;  // [(m+1)][n]
  Tv* w = nullptr;  // [n]
  GmresDev d{};
  void* block = nullptr;

  int init(int64_t n_, int m_);
  void release();
  // Solve A x = b; x holds the initial guess on entry.  apply(in, out, skip)
  // enqueues out = A in on stream s (skip: device flag making it a no-op).
  int solve(dg_ctx* ctx, const std::function<int(const Tv*, Tv*, const int*)>& apply, const Tv* b, Tv* x,
            double tol, int max_iters, cudaStream_t s, GmresResult* res);
};

// FP64 deterministic dot product of two vectors (any of float/double) into out[0].
template <typename Ta, typename Tb>
int dot_into(const Ta* a, const Tb* b, int64_t n, double* partial, double* out, cudaStream_t s,
             const int* skip);

}  // namespace dg
