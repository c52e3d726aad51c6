// One persistent cooperative kernel per Helmholtz solve: restarted GMRES(m)
// with the matrix-free Helmholtz mat-vec inlined (Sec. 3.2: GMRES on the
// pressure system inside the fixed-point loop).
//
// The whole solve -- restart cycles, Arnoldi with classical Gram-Schmidt
// applied twice, Givens rotations, convergence test and the solution update
// -- runs in a single launch.  Phases are separated by grid-wide barriers of a
// cooperative launch (all blocks co-resident), so no host round trip or extra
// launch sits inside the Krylov loop.  Every block keeps an identical copy of
// the small Hessenberg/Givens state in shared memory, computed from the same
// global partial sums in the same order, so the decisions (convergence,
// restart) agree across blocks and the result is bitwise reproducible.
//
// The basis is stored unnormalised: Q_j holds the orthogonalised vector and
// sigma_j = 1/||Q_j||, so q_j = sigma_j Q_j.  A q_j = sigma_j A Q_j is formed
// by scaling the mat-vec output.  Dot products accumulate in FP64 for both
// the FP64 solve and the FP32 inner solve of the refined form.
//
// Loops are bounded by max_iters; there is no spin-wait of our own (the grid
// barrier is the cooperative-groups one, valid because the launch is
// cooperative and every block executes the same sequence of barriers).
#pragma once

#include <cooperative_groups.h>

#include "k_implicit.cuh"

namespace dg {

template <typename T>
struct GmresPArgs {
  MeshView<T> mv;
  const T* h;        // enthalpy at nodes
  const T* b;        // right-hand side
  T* x;              // initial guess in, solution out
  T* Q;              // [(m+1)][n] unnormalised Krylov basis
  T* w;              // [n] mat-vec output
  T* Gh;             // face scratch [dim][nf*NF]
  T* gv;             // [dim][n] scaled-gradient scratch
  double* partial;   // >= gridDim.x doubles
  double* out;       // [4]: iterations, relative residual, converged (0/1), ||b||
  T alpha;           // (a_ii dt)^2
  double tol;
  int m;
  int max_iters;
  int64_t n;
};

__device__ __forceinline__ double block_sum(double v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sred[i];
  return r;
}

// w = scale * A p, A the Helmholtz operator (four phases, four grid barriers)
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void pmatvec(const GmresPArgs<T>& a, const T* p, T scale, T* out,
                                        cooperative_groups::grid_group& grid, T* scell, const T* sD, const T* sDw,
                                        const T* sIt) {
  using S = Shape<DIM, DEG>;
  const int64_t nfi = (int64_t)(a.mv.nconf + a.mv.nsub) * S::NF;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = (a.mv.n_cells + S::CPB - 1) / S::CPB;
  for (int64_t t = tid; t < nfi; t += stride) grad_face_item<DIM, DEG, T>(a.mv, p, a.Gh, t);
  grid.sync();
  for (int64_t bt = blockIdx.x; bt < nb; bt += gridDim.x)
    grad_cell_batch<DIM, DEG, T>(a.mv, p, a.h, a.Gh, a.gv, bt, scell, sD, sIt);
  grid.sync();
  for (int64_t t = tid; t < nfi; t += stride) div_face_item<DIM, DEG, T>(a.mv, a.gv, a.Gh, t);
  grid.sync();
  for (int64_t bt = blockIdx.x; bt < nb; bt += gridDim.x)
    div_cell_batch<DIM, DEG, T, true>(a.mv, a.gv, a.Gh, p, a.alpha, scale, out, bt, scell, sDw, sIt);
  grid.sync();
}

// partial[j*C + c] = sum over chunk c of Q_j . w, for j < nv (C chunks per vector)
template <typename T>
__device__ __forceinline__ void pdots(const T* Q, int64_t n, const T* w, int nv, int C, double* partial,
                                      double* sred) {
  const int64_t chunk = (n + C - 1) / C;
  for (int it = blockIdx.x; it < nv * C; it += gridDim.x) {
    const int j = it / C, c = it % C;
    const int64_t lo = (int64_t)c * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    const T* q = Q + (int64_t)j * n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += (double)q[i] * (double)w[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) partial[it] = s;
  }
}

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(256) gmres_persistent_kernel(GmresPArgs<T> a) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  // shared layout: doubles first, then T tables and the cell tile
  double* sigma = (double*)smem_raw;          // [m+1]
  double* h1 = sigma + (m + 1);               // [m+1]
  double* h2 = h1 + (m + 1);                  // [m+1]
  double* R = h2 + (m + 1);                   // [(m+1)*m], column k at R[k*(m+1)]
  double* cs = R + (m + 1) * m;               // [m]
  double* sn = cs + m;                        // [m]
  double* gg = sn + m;                         // [m+1]
  double* y = gg + (m + 1);                   // [m]
  double* sred = y + m;                       // [32]
  double* sc = sred + 32;                     // [8] scalars: 0 bn, 1 resid, 2 beta
  int* sflag = (int*)(sc + 8);                // [4]: 0 stop inner, 1 converged, 2 kd
  T* tabs = (T*)(sflag + 4);
  T* sD = tabs;
  T* sDw = sD + N * N;
  T* sIt = sDw + N * N;
  T* scell = sIt + 2 * N * N;

  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    sD[q] = a.mv.tab[S::T_D + q];
    sDw[q] = a.mv.tab[S::T_DW + q];
  }
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = a.mv.tab[S::T_IT + q];
  __syncthreads();

  const int64_t n = a.n;
  const int G = gridDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;  // one chunk per block for single-vector passes

  // ||b||^2
  {
    const int64_t lo = (int64_t)blockIdx.x * chunk1;
    const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += (double)a.b[i] * (double)a.b[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
  }
  grid.sync();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < G; ++i) s += a.partial[i];
    sc[0] = sqrt(s);
    sflag[1] = 0;
  }
  __syncthreads();
  const double bn = sc[0];
  if (bn == 0.0) {
    for (int64_t i = tid; i < n; i += gstride) a.x[i] = T(0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.out[0] = 0;
      a.out[1] = 0;
      a.out[2] = 1;
      a.out[3] = 0;
    }
    return;
  }
  grid.sync();  // everyone has read partial before it is reused

  int total = 0;
  double rel = 1.0;
  bool converged = false;
  while (total < a.max_iters) {
    // r = b - A x  -> Q_0 (unnormalised), beta = ||r||
    pmatvec<DIM, DEG, T>(a, a.x, T(1), a.w, grid, scell, sD, sDw, sIt);
    {
      const int64_t lo = (int64_t)blockIdx.x * chunk1;
      const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
      double acc = 0.0;
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const T r = a.b[i] - a.w[i];
        a.Q[i] = r;
        acc += (double)r * (double)r;
      }
      const double s = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
    }
    grid.sync();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < G; ++i) s += a.partial[i];
      const double beta = sqrt(s);
      sc[2] = beta;
      sflag[1] = (beta <= a.tol * bn) ? 1 : 0;
      sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
      for (int j = 0; j <= m; ++j) gg[j] = 0.0;
      gg[0] = beta;
      sflag[0] = 0;
      sflag[2] = 0;
    }
    __syncthreads();
    rel = sc[2] / bn;
    if (sflag[1]) {
      converged = true;
      break;
    }
    grid.sync();  // partial reused below
    int kd = 0;
    for (int k = 0; k < m; ++k) {
      const T* qk = a.Q + (int64_t)k * n;
      pmatvec<DIM, DEG, T>(a, qk, (T)sigma[k], a.w, grid, scell, sD, sDw, sIt);
      // first Gram-Schmidt pass
      int C = G / (k + 1);
      if (C < 1) C = 1;
      pdots<T>(a.Q, n, a.w, k + 1, C, a.partial, sred);
      grid.sync();
      if (threadIdx.x <= k) {
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += a.partial[threadIdx.x * C + c];
        h1[threadIdx.x] = s * sigma[threadIdx.x];
      }
      __syncthreads();
      for (int64_t i = tid; i < n; i += gstride) {
        double acc = 0.0;
        for (int j = 0; j <= k; ++j) acc += h1[j] * sigma[j] * (double)a.Q[(int64_t)j * n + i];
        a.w[i] = (T)((double)a.w[i] - acc);
      }
      grid.sync();
      // second pass
      pdots<T>(a.Q, n, a.w, k + 1, C, a.partial, sred);
      grid.sync();
      if (threadIdx.x <= k) {
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += a.partial[threadIdx.x * C + c];
        h2[threadIdx.x] = s * sigma[threadIdx.x];
      }
      __syncthreads();
      {
        T* qn = a.Q + (int64_t)(k + 1) * n;
        const int64_t lo = (int64_t)blockIdx.x * chunk1;
        const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
        double acc2 = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
          double acc = 0.0;
          for (int j = 0; j <= k; ++j) acc += h2[j] * sigma[j] * (double)a.Q[(int64_t)j * n + i];
          const T v = (T)((double)a.w[i] - acc);
          qn[i] = v;
          acc2 += (double)v * (double)v;
        }
        const double s = block_sum(acc2, sred);
        // the partials of pass 2 were consumed above by every block before this
        // barrier-free write? No: other blocks may still read them -- use a
        // separate slot range past the dot items.
        if (threadIdx.x == 0) a.partial[G + blockIdx.x] = s;
      }
      grid.sync();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < G; ++i) s += a.partial[G + i];
        const double hn = sqrt(s);
        double* col = R + (int64_t)k * (m + 1);
        for (int j = 0; j <= k; ++j) col[j] = h1[j] + h2[j];
        col[k + 1] = hn;
        for (int j = 0; j < k; ++j) {
          const double t = cs[j] * col[j] + sn[j] * col[j + 1];
          col[j + 1] = -sn[j] * col[j] + cs[j] * col[j + 1];
          col[j] = t;
        }
        const double den = hypot(col[k], col[k + 1]);
        const double c = den > 0.0 ? col[k] / den : 1.0;
        const double sg = den > 0.0 ? col[k + 1] / den : 0.0;
        cs[k] = c;
        sn[k] = sg;
        col[k] = den;
        col[k + 1] = 0.0;
        gg[k + 1] = -sg * gg[k];
        gg[k] = c * gg[k];
        const double resid = fabs(gg[k + 1]);
        sc[1] = resid;
        sigma[k + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
        const bool conv = resid <= a.tol * bn;
        sflag[1] = conv ? 1 : 0;
        sflag[0] = (conv || hn == 0.0 || total + 1 >= a.max_iters) ? 1 : 0;
      }
      __syncthreads();
      ++total;
      kd = k + 1;
      rel = sc[1] / bn;
      if (sflag[0]) break;
    }
    // y = R^-1 g over the kd columns, x += sum_j y_j q_j
    if (threadIdx.x == 0) {
      for (int i = kd - 1; i >= 0; --i) {
        double s = gg[i];
        for (int j = i + 1; j < kd; ++j) s -= R[(int64_t)j * (m + 1) + i] * y[j];
        y[i] = s / R[(int64_t)i * (m + 1) + i];
      }
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += gstride) {
      double acc = 0.0;
      for (int j = 0; j < kd; ++j) acc += y[j] * sigma[j] * (double)a.Q[(int64_t)j * n + i];
      a.x[i] = (T)((double)a.x[i] + acc);
    }
    grid.sync();
    if (sflag[1]) {
      converged = true;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = rel;
    a.out[2] = converged ? 1.0 : 0.0;
    a.out[3] = bn;
  }
}

template <int DIM, int DEG, typename T>
inline size_t gmres_smem_bytes(int m) {
  constexpr int N = DEG + 1;
  const size_t dbl = (size_t)3 * (m + 1) + (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m + 32 + 8;
  return dbl * sizeof(double) + 4 * sizeof(int) + (size_t)(4 * N * N + Shape<DIM, DEG>::CPB * Shape<DIM, DEG>::NC) * sizeof(T) + 16;
}

}  // namespace dg
