// One persistent cooperative kernel per Helmholtz solve: restarted GMRES(m)
// with the matrix-free Helmholtz mat-vec inlined (Sec. 3.2: GMRES on the
// pressure system inside the fixed-point loop).
//
// The whole solve -- FP64 residual at every restart, Arnoldi cycles, Givens
// rotations, convergence test and the FP64 solution update -- runs in one
// launch.  Phases are separated by grid-wide barriers of a cooperative
// launch (all blocks co-resident), so no host round trip or extra launch
// sits inside the Krylov loop.  Every block keeps an identical copy of the
// small Hessenberg/Givens state in shared memory, computed from the same
// global partial sums in the same order, so all blocks take the same
// decisions and the result is bitwise reproducible.
//
// Krylov type TK:
//  * double: plain FP64 GMRES (x, b, basis and mat-vec in FP64).
//  * float:  the mixed form.  The basis and the Arnoldi mat-vecs are FP32
//    (FP32 per-thread and per-warp accumulation of the dots, FP64 across
//    warps and blocks); each cycle reduces the residual by inner_tol, then
//    the next restart recomputes the residual b - A x with the FP64
//    operator and FP64 x: iterative refinement inside one kernel.
//
// Orthogonalisation: classical Gram-Schmidt with the norm of w computed in
// the same pass; ||w - Q h||^2 = ||w||^2 - ||h||^2 unless more than half of
// ||w||^2 cancels, in which case a second Gram-Schmidt pass is made
// ("twice is enough").  The new basis vector is written normalised.
//
// Loops are bounded by max_iters; there is no spin-wait of our own (the grid
// barrier is the cooperative-groups one, valid because the launch is
// cooperative and every block executes the same sequence of barriers).
#pragma once

#include <cooperative_groups.h>

#include <algorithm>

#include "k_implicit.cuh"

namespace dg {

template <typename TK>
struct GmresPArgs {
  MeshView<double> mv64;  // FP64 residual mat-vec
  MeshView<TK> mvk;       // Arnoldi mat-vec
  const double* h64;      // enthalpy at nodes (FP64)
  const TK* hk;           // the same in TK
  const double* b;        // right-hand side
  double* x;              // initial guess in, solution out
  TK* Q;                  // [(m+1)][n] Krylov basis (q_0 unnormalised, scale sigma_0)
  TK* w;                  // [n] Arnoldi mat-vec output
  double* w64;            // [n] FP64 residual mat-vec output (may alias w when TK = double)
  double* gv;             // [dim][n] gradient scratch (doubles), reused as TK
  double* partial;        // >= 2 x (CTAs of the solve) doubles
  double* out;            // [4]: iterations, relative residual, converged (0/1), ||b||
  unsigned long long* phase;  // optional [16] ns per phase accumulated by block 0, then per CTA
                              // [512] gradient-pass ns, [512] divergence-pass ns and [512] flags
                              // (batch holds a coarse side) of the Chebyshev solve (NULL = off)
  double alpha;           // (a_ii dt)^2
  double tol;             // target ||b - A x|| / ||b|| (checked on the FP64 residual)
  double inner_tol;       // TK = float: residual reduction per cycle
  int m;
  int max_iters;
  int64_t n;
  int method;  // 0: GMRES(m), one reduction per step; 1: conjugate gradients in the M inner
              // product (needs m >= 2); 2: GMRES(m) with classical Gram-Schmidt twice per step;
              // 3: Chebyshev iteration on [1/(gamma-1), lmax] (needs m >= 1)
  double* lmax;  // [2] device: Chebyshev upper bound (0 = not estimated yet) and the alpha it belongs to
};

enum GmresPhase {
  PH_GRAD_CELL = 1, PH_DIV_CELL = 3, PH_DOTS, PH_UPDATE, PH_REORTH, PH_RESIDUAL,
  PH_SOLUTION, PH_DOTS_WORK = 9, PH_SUMS, PH_GIVENS, PH_COEFS, PH_LINCOMB, PH_ITERS = 15
};

struct PhaseClock {
  unsigned long long* acc;  // NULL = off; set only on the CTA that records
  unsigned long long last;
  __device__ __forceinline__ static unsigned long long now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
  }
  __device__ __forceinline__ void mark(int p) {
    if (acc && threadIdx.x == 0) {
      const unsigned long long t = now();
      acc[p] += t - last;
      last = t;
    }
  }
};

// Barrier over the CTAs working on one solve.  GridSync: the whole grid of a
// cooperative launch (cooperative-groups barrier).  SubSync: the CTAs of one
// member of a batched launch (a generation barrier on two global counters;
// all CTAs of a cooperative launch are co-resident, so it cannot deadlock).
// Its wait is bounded: after limit_ns (a launch parameter, 2 s by default) it
// raises the launch's error flag and every barrier of the launch returns at
// once from then on, so a fault can only end the kernel early, never hang it.
struct GridSync {
  cooperative_groups::grid_group grid;
  int rank, size;
  __device__ GridSync() : grid(cooperative_groups::this_grid()), rank(blockIdx.x), size(gridDim.x) {}
  __device__ __forceinline__ void sync() { grid.sync(); }
  // the barrier in two halves (whole block each): arrive after this CTA's
  // writes of the phase, wait before its first read of other CTAs' writes
  __device__ __forceinline__ unsigned int arrive() { return grid.barrier_arrive(); }
  __device__ __forceinline__ void wait(unsigned int token) { grid.barrier_wait(std::move(token)); }
  __device__ __forceinline__ bool failed() const { return false; }
};

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s, the default limit

struct SubSync {
  int rank, size;
  unsigned int* count;  // arrivals at the current barrier
  unsigned int* gen;    // barrier generation
  int* err;             // launch-wide error flag
  int* sfail;           // shared-memory copy of err, read by every thread
  unsigned long long limit_ns;  // bound of one wait
  __device__ __forceinline__ void sync() {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!*(volatile int*)err && size > 1) {
        __threadfence();
        const unsigned int g = *(volatile unsigned int*)gen;
        const unsigned int arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == (unsigned int)size) {
          atomicExch(count, 0u);
          __threadfence();
          atomicAdd(gen, 1u);
        } else {
          const unsigned long long t0 = PhaseClock::now();
          while (*(volatile unsigned int*)gen == g) {
            if (*(volatile int*)err) break;
            if (PhaseClock::now() - t0 > limit_ns) {
              atomicExch(err, 1);
              break;
            }
            __nanosleep(32);
          }
        }
        __threadfence();
      }
      *sfail = *(volatile int*)err;
    }
    __syncthreads();
  }
  // no split form: arrive is the whole barrier
  __device__ __forceinline__ unsigned int arrive() {
    sync();
    return 0u;
  }
  __device__ __forceinline__ void wait(unsigned int) {}
  __device__ __forceinline__ bool failed() const { return *(volatile int*)sfail != 0; }
};

// On this part an FP64 instruction costs a whole warp issue slot on a pipe
// with a few lanes per SM, so a chain of FP64 operations in one thread is
// slow: every reduction below is a shuffle tree over the lanes (fixed order,
// so the sums are bitwise reproducible), never a serial loop.

// sum over the lanes of the values of warp 0 at lanes < cnt (<= 32); the result in lane 0
__device__ __forceinline__ double warp0_tree(double r, int cnt) {
  int top = 1;
  while (top < cnt) top <<= 1;
  for (int o = top >> 1; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  return r;
}

// FP64 sum over the block; the result in thread 0
__device__ __forceinline__ double block_sum(double v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int nw = (int)(blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) r = warp0_tree(threadIdx.x < nw ? sred[threadIdx.x] : 0.0, nw);
  return r;
}

// FP32 sum over the block (shuffle tree per warp, then over the warp sums);
// the result in thread 0; sred is used as float storage
__device__ __forceinline__ float block_sum_f(float v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int nw = (int)(blockDim.x + 31) >> 5;
  float* sf = (float*)sred;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sf[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.0f;
  if (threadIdx.x < 32) {
    r = threadIdx.x < nw ? sf[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

// the same, returned to every thread
__device__ __forceinline__ float block_allsum_f(float v, double* sred) {
  const float r = block_sum_f(v, sred);
  if (threadIdx.x == 0) ((float*)sred)[0] = r;
  __syncthreads();
  return ((float*)sred)[0];
}

// FP64 sum over the block, returned to every thread
__device__ __forceinline__ double block_allsum(double v, double* sred) {
  const double r = block_sum(v, sred);
  if (threadIdx.x == 0) sred[0] = r;
  __syncthreads();
  return sred[0];
}

// sum of cnt partial sums in global memory (written by the CTAs before the
// last barrier), returned to every thread of the block
__device__ __forceinline__ double gather_allsum(const double* part, int cnt, double* sred) {
  double v = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) v += part[i];
  return block_allsum(v, sred);
}

// square root of the same sum, taken by thread 0 and returned to every thread
__device__ __forceinline__ double gather_allnorm(const double* part, int cnt, double* sred) {
  double v = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) v += part[i];
  const double r = block_sum(v, sred);
  if (threadIdx.x == 0) sred[0] = sqrt(r);
  __syncthreads();
  return sred[0];
}

// the same for the strided sub-array part[off], part[off + stride], ... (cnt entries)
__device__ __forceinline__ double gather_allsum_strided(const double* part, int cnt, int stride, int off,
                                                        double* sred) {
  double v = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) v += part[(int64_t)i * stride + off];
  return block_allsum(v, sred);
}


// three FP64 sums over the block with one pair of block barriers; the results
// in thread 0 (sred holds 3 x 32 doubles)
__device__ __forceinline__ void block_sum3(double& x, double& y, double& z, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
    z += __shfl_down_sync(0xffffffffu, z, o);
  }
  const int nw = (int)(blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sred[threadIdx.x >> 5] = x;
    sred[32 + (threadIdx.x >> 5)] = y;
    sred[64 + (threadIdx.x >> 5)] = z;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = (int)threadIdx.x < nw;
    x = warp0_tree(in ? sred[threadIdx.x] : 0.0, nw);
    y = warp0_tree(in ? sred[32 + threadIdx.x] : 0.0, nw);
    z = warp0_tree(in ? sred[64 + threadIdx.x] : 0.0, nw);
  }
}

// copy cnt global partial sums (no more than the staging area holds) into
// shared memory with all threads
// (one parallel round trip instead of a serial chain of loads)
__device__ __forceinline__ void stage_partials(const double* partial, int cnt, double* spart) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) spart[i] = partial[i];
  __syncthreads();
}

// warp-level sum in TK, then FP64 across warps; the result in thread 0
template <typename TK>
__device__ __forceinline__ double block_sum_k(TK v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int nw = (int)(blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) r = warp0_tree(threadIdx.x < nw ? sred[threadIdx.x] : 0.0, nw);
  return r;
}

// Stores the mat-vec result (the default epilogue of pmatvec).
template <typename T>
struct StoreEpi {
  T* out;
  __device__ __forceinline__ void operator()(int64_t i, T v) const { out[i] = v; }
};
struct NoFin {
  __device__ __forceinline__ void operator()() const {}
};

// The Chebyshev step's update fused into the divergence pass: x += d,
// r -= A d, d = c1 d + c2 r, and the stop test's sum of (r / beta)^2.  pre()
// loads the node's d, r and x (or the cycle's correction) before the pass's
// first barrier, so that their latency is off the pass's critical path.
template <typename TK>
struct ChebStepEpi {
  TK* d;
  TK* r;
  TK* dx;
  double* x;
  bool fold;  // TK = float: the correction is summed in dx, added to x once per cycle
  TK c1, c2;
  bool want;  // this step's residual is tested
  float ibeta;
  float* racc;
  TK di, ri0, dxi;
  double xi;
  __device__ __forceinline__ void pre(int64_t i) {
    di = d[i];
    ri0 = r[i];
    if (fold)
      dxi = dx[i];
    else
      xi = x[i];
  }
  __device__ __forceinline__ void operator()(int64_t i, TK ad) {
    const TK ri = ri0 - ad;
    r[i] = ri;
    if (fold)
      dx[i] = dxi + di;
    else
      x[i] = xi + (double)di;
    d[i] = c1 * di + c2 * ri;
    if (want) {
      const float rs = (float)ri * ibeta;  // FP32: no FP64 instruction for the stop test
      *racc += rs * rs;
    }
  }
};

// scale * (ident p/(gamma-1) - alpha div(h grad p)) (two phases, two grid
// barriers, the first split; the face terms are computed inside the cell passes), handed node
// by node to epi(i, value); fin() runs on every thread of every CTA after its
// last divergence batch, before the closing barrier.
template <int DIM, int DEG, typename T, class Sync, class Epi, class Fin, bool AFF = false>
__device__ __forceinline__ void pmatvec_epi(const MeshView<T>& mv, const T* h, T alpha, T ident, const T* p,
                                            T scale, Epi& epi, Fin& fin, T* gv, Sync& sg, T* scell, T* sJ,
                                            const T* sD, const T* sDw, const T* sII, PhaseClock& pc) {
  const int64_t nb = mv.nbat;
  for (int64_t bt = sg.rank; bt < nb; bt += sg.size)
    grad_cell_batch<DIM, DEG, T, false, AFF>(mv, p, h, gv, batch_range(mv, bt), scell, sJ, sD, sII);
  // split barrier: arrive after the gradient's writes, wait inside the divergence pass once its
  // own loads are in flight
  unsigned int token = sg.arrive();
  bool pending = true;
  pc.mark(PH_GRAD_CELL);
  auto wait = [&]() {
    if (pending) sg.wait(token);
    pending = false;
  };
  for (int64_t bt = sg.rank; bt < nb; bt += sg.size)
    div_cell_batch<DIM, DEG, T, true, Epi, false, AFF, decltype(wait)>(
        mv, gv, p, alpha, scale, ident, epi, batch_range(mv, bt), scell, sJ, sDw, sII, nullptr, nullptr, nullptr, wait);
  if (pending) sg.wait(token);  // a CTA without a batch still meets the barrier
  fin();
  sg.sync();
  pc.mark(PH_DIV_CELL);
}

// out = scale * (ident p/(gamma-1) - alpha div(h grad p))
template <int DIM, int DEG, typename T, class Sync, bool AFF = false>
__device__ __forceinline__ void pmatvec(const MeshView<T>& mv, const T* h, T alpha, T ident, const T* p, T scale,
                                        T* out, T* gv, Sync& sg, T* scell, T* sJ, const T* sD, const T* sDw,
                                        const T* sII, PhaseClock& pc) {
  StoreEpi<T> epi{out};
  NoFin fin;
  pmatvec_epi<DIM, DEG, T, Sync, StoreEpi<T>, NoFin, AFF>(mv, h, alpha, ident, p, scale, epi, fin, gv, sg, scell, sJ, sD,
                                                          sDw, sII, pc);
}

// partial[j*C + c] = sum over chunk c of v_j . w for j < nv, where v_j = Q_j for
// j < nv-1 and v_{nv-1} = w itself (so the last entry is ||w||^2 by chunks)
template <typename TK>
__device__ __forceinline__ void pdots(const TK* Q, int64_t n, const TK* w, int nv, int C, double* partial,
                                      double* sred, int rank, int size) {
  const int64_t chunk = (n + C - 1) / C;
  for (int it = rank; it < nv * C; it += size) {
    const int j = it / C, c = it % C;
    const int64_t lo = (int64_t)c * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    const TK* q = (j < nv - 1) ? Q + (int64_t)j * n : w;
    // four independent accumulators so that four pairs of loads are in flight
    TK a0 = TK(0), a1 = TK(0), a2 = TK(0), a3 = TK(0);
    const int64_t bd = blockDim.x;
    int64_t i = lo + threadIdx.x;
    for (; i + 3 * bd < hi; i += 4 * bd) {
      const TK q0 = q[i], q1 = q[i + bd], q2 = q[i + 2 * bd], q3 = q[i + 3 * bd];
      const TK w0 = w[i], w1 = w[i + bd], w2 = w[i + 2 * bd], w3 = w[i + 3 * bd];
      a0 += q0 * w0;
      a1 += q1 * w1;
      a2 += q2 * w2;
      a3 += q3 * w3;
    }
    for (; i < hi; i += bd) a0 += q[i] * w[i];
    const double s = block_sum_k<TK>((a0 + a1) + (a2 + a3), sred);
    if (threadIdx.x == 0) partial[it] = s;
  }
}

// sum_{j<cnt} coef[j] Q_j[i] accumulated in TK, with the loads of eight basis
// vectors in flight at once
template <typename TK>
__device__ __forceinline__ TK lincomb(const TK* __restrict__ Q, int64_t n, int64_t i,
                                      const double* __restrict__ coef, int cnt) {
  TK acc = TK(0);
  int j = 0;
  for (; j + 8 <= cnt; j += 8) {
    TK q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = Q[(int64_t)(j + u) * n + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += (TK)coef[j + u] * q[u];
  }
  for (; j < cnt; ++j) acc += (TK)coef[j] * Q[(int64_t)j * n + i];
  return acc;
}

// partial[2 (j C + c) + {0, 1}] = sum over chunk c of V_j . u and V_j . w for
// j < nv, where V_j = Q_j and u = Q_{nv-1} (so the last pair is u.u, u.w)
template <typename TK>
__device__ __forceinline__ void pdots2(const TK* Q, int64_t n, const TK* w, int nv, int C, double* partial,
                                       double* sred, int rank, int size) {
  const TK* u = Q + (int64_t)(nv - 1) * n;
  const int64_t chunk = (n + C - 1) / C;
  for (int it = rank; it < nv * C; it += size) {
    const int j = it / C, c = it % C;
    const int64_t lo = (int64_t)c * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    const TK* q = Q + (int64_t)j * n;
    // four nodes per thread per round: twelve loads in flight
    TK su[4] = {TK(0), TK(0), TK(0), TK(0)}, sw[4] = {TK(0), TK(0), TK(0), TK(0)};
    const int64_t bd = blockDim.x;
    int64_t i = lo + threadIdx.x;
    for (; i + 3 * bd < hi; i += 4 * bd) {
      TK qv[4], uv[4], wv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        qv[r] = q[i + r * bd];
        uv[r] = u[i + r * bd];
        wv[r] = w[i + r * bd];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        su[r] += qv[r] * uv[r];
        sw[r] += qv[r] * wv[r];
      }
    }
    for (; i < hi; i += bd) {
      const TK qv = q[i];
      su[0] += qv * u[i];
      sw[0] += qv * w[i];
    }
    const double du = block_sum_k<TK>((su[0] + su[1]) + (su[2] + su[3]), sred);
    const double dw = block_sum_k<TK>((sw[0] + sw[1]) + (sw[2] + sw[3]), sred);
    if (threadIdx.x == 0) {
      partial[2 * it] = du;
      partial[2 * it + 1] = dw;
    }
  }
}

// o1 = sum_{j<cnt} c1[j] Q_j[i], o2 = sum_{j<cnt} c2[j] Q_j[i] in TK, reading
// each basis vector once with eight loads in flight
template <typename TK>
__device__ __forceinline__ void lincomb2(const TK* __restrict__ Q, int64_t n, int64_t i,
                                         const double* __restrict__ c1, const double* __restrict__ c2, int cnt,
                                         TK& o1, TK& o2) {
  TK a1 = TK(0), a2 = TK(0);
  int j = 0;
  for (; j + 8 <= cnt; j += 8) {
    TK q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = Q[(int64_t)(j + u) * n + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a1 += (TK)c1[j + u] * q[u];
      a2 += (TK)c2[j + u] * q[u];
    }
  }
  for (; j < cnt; ++j) {
    const TK q = Q[(int64_t)j * n + i];
    a1 += (TK)c1[j] * q;
    a2 += (TK)c2[j] * q;
  }
  o1 = a1;
  o2 = a2;
}

// 1D tables of the mesh's degree into shared memory, FP64 and TK copies:
// D, Dw, then I (2 N^2) followed by It (2 N^2)
template <int DIM, int DEG, typename TK>
__device__ __forceinline__ void load_tables(const GmresPArgs<TK>& a, double* sD64, double* sDw64, double* sII64,
                                            TK* sDk, TK* sDwk, TK* sIIk) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    sD64[q] = a.mv64.tab[S::T_D + q];
    sDw64[q] = a.mv64.tab[S::T_DW + q];
    sDk[q] = a.mvk.tab[S::T_D + q];
    sDwk[q] = a.mvk.tab[S::T_DW + q];
  }
  for (int q = threadIdx.x; q < 4 * N * N; q += blockDim.x) {
    sII64[q] = a.mv64.tab[S::T_I + q];
    sIIk[q] = a.mvk.tab[S::T_I + q];
  }
  __syncthreads();
}

// Restarted GMRES(m) with one global reduction per Arnoldi step: classical
// Gram-Schmidt with the second (re-orthogonalisation) pass of each vector
// delayed into the next step, in the manner of the low-synchronisation DCGS2
// Arnoldi of Swirydowicz et al. (2020) and Bielich et al. (2022); the
// derivation below is our own.  Step k has u_k = B q_{k-1} - Q_k hf (one
// Gram-Schmidt pass, not normalised; u_0 = r) in basis slot k and
//   1. v = B u_k                                   (mat-vec, two phases)
//   2. a = Q_k^T u_k, b = Q_k^T v, u_k.u_k, u_k.v   (ONE reduction)
//   3. rho^2 = u_k.u_k - |a|^2, q_k = (u_k - Q_k a)/rho;  column k-1 of H is
//      hf + a with subdiagonal rho (Givens update, residual estimate);
//      B q_k = (v - Q_{k+1} z)/rho with z = H a (Arnoldi relation), so the
//      first pass of column k is hf'_i = (b_i - z_i)/rho (i < k),
//      hf'_k = ((u_k.v - a.b)/rho - z_k)/rho, and
//      u_{k+1} = v/rho - c u_k - Q_k d,  c = (z_k/rho + hf'_k)/rho,
//      d = z/rho + hf' - c a                          (no further reduction)
//   4. one pass writes q_k and u_{k+1}.
// Four grid barriers per step (two in the mat-vec), two passes over the basis.
// Arnoldi runs on B = A - I/(gamma-1) (same Krylov space; the Hessenberg of A
// adds 1/(gamma-1) on the diagonal).  Each cycle ends one mat-vec after its
// last column (the step that completes it).  TK = float: FP32 basis and
// mat-vecs, FP64 residual recomputed at every restart (iterative refinement).
template <int DIM, int DEG, typename TK, class Sync>
__device__ __forceinline__ void gmres_body(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw,
                                           bool record) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  const int m = a.m;
  double* Hb = (double*)smem_raw;    // [(m+1)*m] Hessenberg of B, column j at Hb[j*(m+1)]
  double* R = Hb + (m + 1) * m;      // [(m+1)*m] rotated Hessenberg of A
  double* cs = R + (m + 1) * m;      // [m]
  double* sn = cs + m;               // [m]
  double* gg = sn + m;               // [m+1]
  double* y = gg + (m + 1);          // [m]
  double* av = y + m;                // [m+1] a (second pass), then u.u in [k]; solution weights at the end
  double* bv = av + (m + 1);         // [m+1] b, then u.v in [k]
  double* hf = bv + (m + 1);         // [m+1] first-pass coefficients of the newest column
  double* zc = hf + (m + 1);         // [m+1] z = H a
  double* dv = zc + (m + 1);         // [m+1] d
  double* sred = dv + (m + 1);       // [32]
  double* sc = sred + 32;            // [8]: 1 resid, 3 rho, 4 c, 5 1/rho
  int* sflag = (int*)(sc + 8);       // [4]: 0 stop cycle, 1 converged
  double* t64 = (double*)(sflag + 4);  // FP64 tables D, Dw, I|It
  double* sD64 = t64;
  double* sDw64 = sD64 + N * N;
  double* sII64 = sDw64 + N * N;
  double* scell64 = sII64 + 4 * N * N;      // cell tile, DIM*CPB*NC doubles (reused as TK)
  double* sJ64 = scell64 + DIM * S::CPB * S::NC;  // coarse-pass buffer (reused as TK)
  TK* tk = (TK*)(sJ64 + coarse_buffer<DIM, DEG, DIM>());
  TK* sDk = tk;
  TK* sDwk = sDk + N * N;
  TK* sIIk = sDwk + N * N;
  TK* scellk = (TK*)scell64;
  TK* sJk = (TK*)sJ64;
  load_tables<DIM, DEG, TK>(a, sD64, sDw64, sII64, sDk, sDwk, sIIk);
  PhaseClock pc{record ? a.phase : nullptr, PhaseClock::now()};

  const int64_t n = a.n;
  const int G = sg.size;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;
  const bool mixed = sizeof(TK) != sizeof(double);
  const double shift = 1.0 / (kGamma - 1.0);
  TK* gvk = (TK*)a.gv;

  // ||b||
  {
    const int64_t lo = (int64_t)sg.rank * chunk1;
    const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += a.b[i] * a.b[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[sg.rank] = s;
  }
  sg.sync();
  const double bn = gather_allnorm(a.partial, G, sred);
  if (bn == 0.0) {
    for (int64_t i = tid; i < n; i += gstride) a.x[i] = 0.0;
    if (sg.rank == 0 && threadIdx.x == 0) {
      a.out[0] = 0;
      a.out[1] = 0;
      a.out[2] = 1;
      a.out[3] = 0;
    }
    return;
  }
  sg.sync();  // partial reused below

  int total = 0;
  double rel = 1.0;
  bool converged = false;
  while (true) {
    // r = b - A x with the FP64 operator -> u_0 in slot 0, beta
    pmatvec<DIM, DEG, double, Sync>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.gv, sg, scell64, sJ64, sD64,
                                    sDw64, sII64, pc);
    {
      const int64_t lo = (int64_t)sg.rank * chunk1;
      const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
      double acc = 0.0;
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double r = a.b[i] - a.w64[i];
        a.Q[i] = (TK)r;
        acc += r * r;
      }
      const double s = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[sg.rank] = s;
    }
    sg.sync();
    pc.mark(PH_RESIDUAL);
    const double beta = gather_allnorm(a.partial, G, sred);
    if (threadIdx.x == 0) {
      sflag[1] = (beta <= a.tol * bn) ? 1 : 0;
      sflag[0] = 0;
    }
    __syncthreads();
    rel = beta / bn;
    if (sg.failed()) break;
    if (sflag[1]) {
      converged = true;
      break;
    }
    if (total >= a.max_iters) break;
    const double cycle_floor = fmax(a.tol * bn, (mixed ? a.inner_tol : 0.0) * beta);
    int kd = 0;
    for (int k = 0; k <= m; ++k) {
      TK* uk = a.Q + (int64_t)k * n;
      // 1. v = B u_k
      pmatvec<DIM, DEG, TK, Sync>(a.mvk, a.hk, (TK)a.alpha, TK(0), uk, TK(1), a.w, gvk, sg, scellk, sJk, sDk, sDwk,
                                  sIIk, pc);
      // 2. a = Q_k^T u_k, b = Q_k^T v, u.u, u.v: one reduction
      const int nv = k + 1;
      int C = G / nv;
      if (C < 1) C = 1;
      pdots2<TK>(a.Q, n, a.w, nv, C, a.partial, sred, sg.rank, sg.size);
      pc.mark(PH_DOTS_WORK);
      sg.sync();
      pc.mark(PH_DOTS);
      if (sg.failed()) break;
      // sums of the chunk partials: warp w takes the pairs p = w, w + 8, ... (a_j for even
      // p, b_j for odd), its lanes split the chunks (all loads issued first), and a
      // shuffle tree adds them
      {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
        constexpr int PG = 4;  // pairs per warp whose loads are in flight together
        for (int q0 = 0; warp + q0 * nw < 2 * nv; q0 += PG) {
          double v[PG];
#pragma unroll
          for (int q = 0; q < PG; ++q) {
            const int pr = warp + (q0 + q) * nw;
            v[q] = 0.0;
            if (pr < 2 * nv)
              for (int c = lane; c < C; c += 32) v[q] += a.partial[2 * ((pr >> 1) * C + c) + (pr & 1)];
          }
#pragma unroll
          for (int q = 0; q < PG; ++q) {
            const int pr = warp + (q0 + q) * nw;
            if (pr < 2 * nv) {  // warp-uniform
              double t = v[q];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
              if (lane == 0) (pr & 1 ? bv : av)[pr >> 1] = t;
            }
          }
        }
      }
      __syncthreads();
      pc.mark(PH_SUMS);
      // 3. warp 0: |a|^2 and a.b by lanes, the new column hf + a (+ shift on the diagonal)
      // by lanes, the products cs_j col_{j+1} of the earlier rotations by lanes; then lane 0
      // runs the rotation chain x_{j+1} = cs_j col_{j+1} - sn_j x_j (one FMA per link), the
      // new rotation and the stop test.  Threads 32..32+k-1 meanwhile form z = H a, taking
      // the new column as hf + a directly.
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double s1 = 0.0, s2 = 0.0;
        for (int j = lane; j < k; j += 32) {
          s1 += av[j] * av[j];
          s2 += av[j] * bv[j];
        }
        s1 = warp0_tree(s1, 32);
        s2 = warp0_tree(s2, 32);
        double* hb = Hb + (int64_t)(k > 0 ? k - 1 : 0) * (m + 1);
        double* col = R + (int64_t)(k > 0 ? k - 1 : 0) * (m + 1);
        if (k > 0) {
          for (int j = lane; j < k; j += 32) {
            const double hj = hf[j] + av[j];
            hb[j] = hj;
            col[j] = hj + (j == k - 1 ? shift : 0.0);
          }
          __syncwarp();
          for (int j = lane; j < k - 1; j += 32) y[j] = cs[j] * col[j + 1];  // y: scratch until the cycle ends
          __syncwarp();
        }
        if (lane == 0) {
          const double uu = av[k];
          const double rho2 = uu - s1;
          // breakdown (u_k in the span of Q_k to working precision) ends the cycle
          const bool ok = rho2 > 1e-24 * uu && rho2 > 0.0;
          const double irho = ok ? rsqrt64(rho2) : 0.0;
          const double rho = ok ? rho2 * irho : 0.0;
          sc[3] = rho;
          sc[5] = irho;
          // first-pass entry k of the new column and the weight c of u_k in u_{k+1}
          const double zk = k > 0 ? rho * av[k - 1] : 0.0;
          const double hk = ((bv[k] - s2) * irho - zk) * irho;
          hf[k] = hk;
          sc[4] = (zk * irho + hk) * irho;
          int stop = 0;
          if (k == 0) {
            gg[0] = rho;
            for (int j = 1; j <= m; ++j) gg[j] = 0.0;
            if (!ok) stop = 1;
          } else {
            hb[k] = rho;
            // chain: x_0 = col_0, x_{j+1} = cs_j col_{j+1} - sn_j x_j; the rotated entries
            // R_j = cs_j x_j + sn_j col_{j+1} are written back off the chain
            double x = col[0];
            for (int j = 0; j < k - 1; ++j) {
              const double xn = fma(-sn[j], x, y[j]);
              col[j] = fma(cs[j], x, sn[j] * col[j + 1]);
              x = xn;
            }
            const double x1 = rho;
            const double r2 = x * x + x1 * x1;
            const double ir = r2 > 0.0 ? rsqrt64(r2) : 0.0;
            const double c = r2 > 0.0 ? x * ir : 1.0;
            const double sgn = r2 > 0.0 ? x1 * ir : 0.0;
            cs[k - 1] = c;
            sn[k - 1] = sgn;
            col[k - 1] = r2 * ir;
            col[k] = 0.0;
            gg[k] = -sgn * gg[k - 1];
            gg[k - 1] = c * gg[k - 1];
            const double resid = fabs(gg[k]);
            sc[1] = resid;
            sflag[1] = resid <= a.tol * bn ? 1 : 0;
            stop = (resid <= cycle_floor || !ok || total + 1 >= a.max_iters || k == m) ? 1 : 0;
          }
          sflag[0] = stop;
        }
      } else if ((int)threadIdx.x < 32 + k) {
        const int i = threadIdx.x - 32;
        double z = (hf[i] + av[i]) * av[k - 1];
        for (int j = (i > 0 ? i - 1 : 0); j < k - 1; ++j) z += Hb[(int64_t)j * (m + 1) + i] * av[j];
        zc[i] = z;
      }
      __syncthreads();
      pc.mark(PH_GIVENS);
      if (k > 0) {
        ++total;
        rel = sc[1] / bn;
      }
      kd = k;
      if (sflag[0]) break;
      // first pass of column k and the weights of u_{k+1} (the scalars from lane 0)
      const double irho = sc[5];
      const double cu = sc[4];
      if ((int)threadIdx.x < k) {
        const int i = threadIdx.x;
        const double h = (bv[i] - zc[i]) * irho;
        hf[i] = h;
        dv[i] = zc[i] * irho + h - cu * av[i];
      }
      __syncthreads();
      pc.mark(PH_COEFS);
      // 4. q_k = (u_k - Q_k a)/rho and u_{k+1} = v/rho - c u_k - Q_k d, one pass
      {
        const TK irk = (TK)irho, cuk = (TK)cu;
        TK* un = a.Q + (int64_t)(k + 1) * n;
        for (int64_t i = tid; i < n; i += gstride) {
          const TK u = uk[i], v = a.w[i];
          TK sa, sd;
          lincomb2(a.Q, n, i, av, dv, k, sa, sd);
          uk[i] = (u - sa) * irk;
          un[i] = v * irk - cuk * u - sd;
        }
      }
      pc.mark(PH_LINCOMB);
      sg.sync();
      pc.mark(PH_UPDATE);
      if (sg.failed()) break;
    }
    // x += sum_j y_j q_j over the kd completed columns
    if (threadIdx.x == 0) {
      for (int i = kd - 1; i >= 0; --i) {
        double s = gg[i];
        for (int j = i + 1; j < kd; ++j) s -= R[(int64_t)j * (m + 1) + i] * y[j];
        y[i] = s / R[(int64_t)i * (m + 1) + i];
      }
      for (int j = 0; j < kd; ++j) av[j] = y[j];
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += gstride) a.x[i] += (double)lincomb(a.Q, n, i, av, kd);
    sg.sync();
    pc.mark(PH_SOLUTION);
    // plain FP64 GMRES trusts its residual estimate; the mixed form re-checks
    // with the FP64 residual at the next restart
    if (!mixed && sflag[1]) {
      converged = true;
      break;
    }
    if (kd == 0 || total >= a.max_iters || sg.failed()) break;  // kd = 0: no progress possible
  }
  if (sg.rank == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = rel;
    a.out[2] = (converged && !sg.failed()) ? 1.0 : 0.0;
    a.out[3] = bn;
    if (pc.acc) a.phase[PH_ITERS] += (unsigned long long)total;
  }
}

template <int DIM, int DEG, typename TK, class Sync>
__device__ __forceinline__ void gmres_cgs2_body(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw,
                                                bool record) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  const int m = a.m;
  double* sigma = (double*)smem_raw;  // [m+1] scale of q_j (1/beta for j = 0, else 1)
  double* hh = sigma + (m + 1);       // [m+2] Gram-Schmidt coefficients (+ ||w||^2 in [k+1])
  double* h2 = hh + (m + 2);          // [m+2] second pass
  double* R = h2 + (m + 2);           // [(m+1)*m] rotated Hessenberg, column k at R[k*(m+1)]
  double* cs = R + (m + 1) * m;       // [m]
  double* sn = cs + m;                // [m]
  double* gg = sn + m;                // [m+1]
  double* y = gg + (m + 1);           // [m]
  double* coef = y + m;               // [m+1]
  double* sred = coef + (m + 1);      // [32]
  double* sc = sred + 32;             // [8]: 0 ||b||, 1 resid, 2 beta, 3 1/hn, 4 ||w||^2 after
  double* spart = sc + 8;             // [512] staged block partials
  int* sflag = (int*)(spart + 512);   // [4]: 0 stop cycle, 1 converged, 2 reorth
  double* t64 = (double*)(sflag + 4);  // FP64 tables D, Dw, I|It
  double* sD64 = t64;
  double* sDw64 = sD64 + N * N;
  double* sII64 = sDw64 + N * N;
  double* scell64 = sII64 + 4 * N * N;  // cell tile, DIM*CPB*NC doubles (reused as TK)
  double* sJ64 = scell64 + DIM * S::CPB * S::NC;  // coarse-pass buffer (reused as TK)
  TK* tk = (TK*)(sJ64 + coarse_buffer<DIM, DEG, DIM>());
  TK* sDk = tk;
  TK* sDwk = sDk + N * N;
  TK* sIIk = sDwk + N * N;
  TK* scellk = (TK*)scell64;
  TK* sJk = (TK*)sJ64;
  load_tables<DIM, DEG, TK>(a, sD64, sDw64, sII64, sDk, sDwk, sIIk);
  PhaseClock pc{record ? a.phase : nullptr, PhaseClock::now()};

  const int64_t n = a.n;
  const int G = sg.size;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;
  const bool mixed = sizeof(TK) != sizeof(double);
  TK* gvk = (TK*)a.gv;

  // ||b||
  {
    const int64_t lo = (int64_t)sg.rank * chunk1;
    const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += a.b[i] * a.b[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[sg.rank] = s;
  }
  sg.sync();
  const double bn = gather_allnorm(a.partial, G, sred);
  if (bn == 0.0) {
    for (int64_t i = tid; i < n; i += gstride) a.x[i] = 0.0;
    if (sg.rank == 0 && threadIdx.x == 0) {
      a.out[0] = 0;
      a.out[1] = 0;
      a.out[2] = 1;
      a.out[3] = 0;
    }
    return;
  }
  sg.sync();  // partial reused below

  int total = 0;
  double rel = 1.0;
  bool converged = false;
  while (true) {
    // r = b - A x with the FP64 operator -> q_0 (unnormalised), beta
    pmatvec<DIM, DEG, double, Sync>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.gv, sg, scell64, sJ64, sD64,
                                    sDw64, sII64, pc);
    {
      const int64_t lo = (int64_t)sg.rank * chunk1;
      const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
      double acc = 0.0;
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double r = a.b[i] - a.w64[i];
        a.Q[i] = (TK)r;
        acc += r * r;
      }
      const double s = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[sg.rank] = s;
    }
    sg.sync();
    pc.mark(PH_RESIDUAL);
    const double beta = gather_allnorm(a.partial, G, sred);
    if (threadIdx.x == 0) {
      sc[2] = beta;
      sflag[1] = (beta <= a.tol * bn) ? 1 : 0;
      sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
      for (int j = 1; j <= m; ++j) sigma[j] = 1.0;
      for (int j = 0; j <= m; ++j) gg[j] = 0.0;
      gg[0] = beta;
      sflag[0] = 0;
    }
    __syncthreads();
    rel = sc[2] / bn;
    if (sg.failed()) break;
    if (sflag[1]) {
      converged = true;
      break;
    }
    if (total >= a.max_iters) break;
    const double cycle_floor = fmax(a.tol * bn, (mixed ? a.inner_tol : 0.0) * sc[2]);
    int kd = 0;
    for (int k = 0; k < m; ++k) {
      const TK* qk = a.Q + (int64_t)k * n;
      // Arnoldi on B = A - I/(gamma-1): same Krylov space, Hessenberg of A = that of B
      // plus 1/(gamma-1) on the diagonal; w = B q_k has no large component along q_k
      pmatvec<DIM, DEG, TK, Sync>(a.mvk, a.hk, (TK)a.alpha, TK(0), qk, (TK)sigma[k], a.w, gvk, sg, scellk, sJk,
                                  sDk, sDwk, sIIk, pc);
      // h_j = q_j . w (j <= k) and ||w||^2, one pass
      const int nv = k + 2;
      int C = G / nv;
      if (C < 1) C = 1;
      pdots<TK>(a.Q, n, a.w, nv, C, a.partial, sred, sg.rank, sg.size);
      sg.sync();
      pc.mark(PH_DOTS);
      stage_partials(a.partial, nv * C, spart);
      if (threadIdx.x < nv) {
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += spart[threadIdx.x * C + c];
        hh[threadIdx.x] = (threadIdx.x < nv - 1) ? s * sigma[threadIdx.x] : s;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double ss = 0.0;
        for (int j = 0; j <= k; ++j) {
          ss += hh[j] * hh[j];
          coef[j] = hh[j] * sigma[j];
        }
        const double ww = hh[k + 1];
        const double after = ww - ss;
        sflag[2] = (after < 0.5 * ww) ? 1 : 0;
        sc[4] = after;
        sc[3] = after > 0.0 ? 1.0 / sqrt(after) : 0.0;
      }
      __syncthreads();
      TK* qn = a.Q + (int64_t)(k + 1) * n;
      if (!sflag[2]) {
        const double inv = sc[3];
        const TK invk = (TK)inv;
        for (int64_t i = tid; i < n; i += gstride) qn[i] = (a.w[i] - lincomb(a.Q, n, i, coef, k + 1)) * invk;
      } else {
        // second Gram-Schmidt pass
        if (pc.acc && threadIdx.x == 0) a.phase[14] += 1;
        for (int64_t i = tid; i < n; i += gstride) a.w[i] -= lincomb(a.Q, n, i, coef, k + 1);
        sg.sync();
        pdots<TK>(a.Q, n, a.w, nv, C, a.partial, sred, sg.rank, sg.size);
        sg.sync();
        pc.mark(PH_REORTH);
        stage_partials(a.partial, nv * C, spart);
        if (threadIdx.x < nv) {
          double s = 0.0;
          for (int c = 0; c < C; ++c) s += spart[threadIdx.x * C + c];
          h2[threadIdx.x] = (threadIdx.x < nv - 1) ? s * sigma[threadIdx.x] : s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double ss = 0.0;
          for (int j = 0; j <= k; ++j) {
            ss += h2[j] * h2[j];
            coef[j] = h2[j] * sigma[j];
            hh[j] += h2[j];
          }
          const double after = h2[k + 1] - ss;
          sc[4] = after;
          sc[3] = after > 0.0 ? 1.0 / sqrt(after) : 0.0;
        }
        __syncthreads();
        const double inv = sc[3];
        const TK invk = (TK)inv;
        for (int64_t i = tid; i < n; i += gstride) qn[i] = (a.w[i] - lincomb(a.Q, n, i, coef, k + 1)) * invk;
      }
      // Givens update of column k (every block, identical)
      if (threadIdx.x == 0) {
        const double hn = sc[4] > 0.0 ? sqrt(sc[4]) : 0.0;
        double* col = R + (int64_t)k * (m + 1);
        for (int j = 0; j <= k; ++j) col[j] = hh[j];
        col[k] += 1.0 / (kGamma - 1.0);
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
        sflag[1] = resid <= a.tol * bn ? 1 : 0;
        sflag[0] = (resid <= cycle_floor || hn == 0.0 || total + 1 >= a.max_iters) ? 1 : 0;
      }
      sg.sync();
      pc.mark(PH_UPDATE);
      ++total;
      kd = k + 1;
      rel = sc[1] / bn;
      if (sflag[0] || sg.failed()) break;
    }
    // x += sum_j y_j q_j, y from the rotated Hessenberg system
    if (threadIdx.x == 0) {
      for (int i = kd - 1; i >= 0; --i) {
        double s = gg[i];
        for (int j = i + 1; j < kd; ++j) s -= R[(int64_t)j * (m + 1) + i] * y[j];
        y[i] = s / R[(int64_t)i * (m + 1) + i];
      }
      for (int j = 0; j < kd; ++j) coef[j] = y[j] * sigma[j];
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += gstride) a.x[i] += (double)lincomb(a.Q, n, i, coef, kd);
    sg.sync();
    pc.mark(PH_SOLUTION);
    // plain FP64 GMRES trusts its residual estimate; the mixed form re-checks
    // with the FP64 residual at the next restart
    if (!mixed && sflag[1]) {
      converged = true;
      break;
    }
    if (total >= a.max_iters || sg.failed()) break;
  }
  if (sg.rank == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = rel;
    a.out[2] = (converged && !sg.failed()) ? 1.0 : 0.0;
    a.out[3] = bn;
    if (pc.acc) a.phase[PH_ITERS] += (unsigned long long)total;
  }
}

// Conjugate gradients on the same Helmholtz system.  With the strong gradient
// and weak divergence, M A is symmetric positive definite (M = diag(w J)), so
// A is self-adjoint in the inner product <x, y>_M = sum w J x y and CG in that
// inner product applies.  Chronopoulos-Gear form: one mat-vec and ONE fused
// reduction (<r, r>_M, <A r, r>_M, ||r||^2) per iteration, then one vector
// update pass -- six barriers per iteration against GMRES's eight, and no
// orthogonalisation against a growing basis.  The stopping test is on the
// Euclidean residual ||b - A x|| / ||b||, checked at the end with the FP64
// operator (restarting the recurrence if the recursive residual drifted);
// TK = float runs the recurrence in FP32 and restarts from the FP64 residual
// whenever the residual has dropped by inner_tol (iterative refinement).
template <int DIM, int DEG, typename TK, class Sync>
__device__ __forceinline__ void cg_body(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw, bool record) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  double* sred = (double*)smem_raw;  // [96]
  double* sc = sred + 96;            // [16]
  double* sD64 = sc + 16;
  double* sDw64 = sD64 + N * N;
  double* sII64 = sDw64 + N * N;
  double* scell64 = sII64 + 4 * N * N;
  double* sJ64 = scell64 + DIM * S::CPB * S::NC;
  TK* sDk = (TK*)(sJ64 + coarse_buffer<DIM, DEG, DIM>());
  TK* sDwk = sDk + N * N;
  TK* sIIk = sDwk + N * N;
  TK* scellk = (TK*)scell64;
  TK* sJk = (TK*)sJ64;
  load_tables<DIM, DEG, TK>(a, sD64, sDw64, sII64, sDk, sDwk, sIIk);
  PhaseClock pc{record ? a.phase : nullptr, PhaseClock::now()};
  const int64_t n = a.n;
  const int G = sg.size;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;
  const int64_t lo = (int64_t)sg.rank * chunk1;
  const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
  const bool mixed = sizeof(TK) != sizeof(double);
  TK* r = a.Q;
  TK* p = a.Q + n;
  TK* s = a.Q + 2 * n;
  TK* w = a.w;
  const TK* wJ = a.mvk.wJ;
  TK* gvk = (TK*)a.gv;

  {
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += a.b[i] * a.b[i];
    const double t = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[sg.rank] = t;
  }
  sg.sync();
  const double bn = gather_allnorm(a.partial, G, sred);
  if (bn == 0.0) {
    for (int64_t i = tid; i < n; i += gstride) a.x[i] = 0.0;
    if (sg.rank == 0 && threadIdx.x == 0) {
      a.out[0] = 0;
      a.out[1] = 0;
      a.out[2] = 1;
      a.out[3] = 0;
    }
    return;
  }
  sg.sync();
  int total = 0;
  double rel = 1.0;
  bool converged = false;
  while (true) {
    // true residual with the FP64 operator
    pmatvec<DIM, DEG, double, Sync>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.gv, sg, scell64, sJ64, sD64,
                                    sDw64, sII64, pc);
    {
      double acc = 0.0;
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double ri = a.b[i] - a.w64[i];
        r[i] = (TK)ri;
        acc += ri * ri;
      }
      const double t = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[sg.rank] = t;
    }
    sg.sync();
    pc.mark(PH_RESIDUAL);
    const double beta0 = gather_allnorm(a.partial, G, sred);
    rel = beta0 / bn;
    if (sg.failed()) break;
    if (beta0 <= a.tol * bn) {
      converged = true;
      break;
    }
    if (total >= a.max_iters) break;
    const double floor = fmax(a.tol * bn, (mixed ? a.inner_tol : 0.0) * beta0);
    double alpha = 1.0, gamma = 1.0;
    bool first = true;
    for (;;) {
      pmatvec<DIM, DEG, TK, Sync>(a.mvk, a.hk, (TK)a.alpha, TK(1), r, TK(1), w, gvk, sg, scellk, sJk, sDk, sDwk,
                                  sIIk, pc);
      {
        TK g0 = TK(0), d0 = TK(0), e0 = TK(0);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
          const TK ri = r[i], mi = wJ[i] * ri;
          g0 += mi * ri;
          d0 += mi * w[i];
          e0 += ri * ri;
        }
        // warp sums in TK, FP64 across the warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          g0 += __shfl_down_sync(0xffffffffu, g0, o);
          d0 += __shfl_down_sync(0xffffffffu, d0, o);
          e0 += __shfl_down_sync(0xffffffffu, e0, o);
        }
        double tg = (threadIdx.x & 31) == 0 ? (double)g0 : 0.0;
        double td = (threadIdx.x & 31) == 0 ? (double)d0 : 0.0;
        double te = (threadIdx.x & 31) == 0 ? (double)e0 : 0.0;
        block_sum3(tg, td, te, sred);
        if (threadIdx.x == 0) {
          a.partial[3 * sg.rank] = tg;
          a.partial[3 * sg.rank + 1] = td;
          a.partial[3 * sg.rank + 2] = te;
        }
      }
      sg.sync();
      pc.mark(PH_DOTS);
      // the three sums of the G block partials in one block reduction; thread 0 evaluates
      // the square root, the divisions and the stop test and broadcasts them through sc
      {
        double gs = 0.0, ds = 0.0, es = 0.0;
        for (int c = threadIdx.x; c < G; c += blockDim.x) {
          gs += a.partial[3 * c];
          ds += a.partial[3 * c + 1];
          es += a.partial[3 * c + 2];
        }
        block_sum3(gs, ds, es, sred);
        if (threadIdx.x == 0) {
          const double rn = sqrt(es);
          const bool stop = rn <= floor || total + 1 >= a.max_iters || !(ds > 0.0) || !(gs > 0.0);
          double beta = 0.0, al = alpha;
          if (!stop) {
            if (first) {
              al = gs / ds;
            } else {
              beta = gs / gamma;
              al = gs / (ds - beta * gs / alpha);
            }
          }
          sc[0] = rn / bn;
          sc[1] = stop ? 1.0 : 0.0;
          sc[2] = beta;
          sc[3] = al;
          sc[4] = gs;
        }
        __syncthreads();
      }
      ++total;
      rel = sc[0];
      if (sg.failed() || sc[1] != 0.0) break;
      const double beta = first ? 0.0 : sc[2];
      alpha = sc[3];
      gamma = sc[4];
      first = false;
      const TK bk = (TK)beta, ak = (TK)alpha;
      for (int64_t i = tid; i < n; i += gstride) {
        const TK pi = r[i] + bk * p[i];
        const TK si = w[i] + bk * s[i];
        p[i] = pi;
        s[i] = si;
        a.x[i] += alpha * (double)pi;
        r[i] -= ak * si;
      }
      sg.sync();
      pc.mark(PH_UPDATE);
    }
    sg.sync();  // x complete before the residual mat-vec reads it
    if (total >= a.max_iters || sg.failed()) {
      // report the last residual estimate
      break;
    }
  }
  if (sg.rank == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = rel;
    a.out[2] = (converged && !sg.failed()) ? 1.0 : 0.0;
    a.out[3] = bn;
    if (pc.acc) a.phase[PH_ITERS] += (unsigned long long)total;
  }
}

// Chebyshev iteration on the Helmholtz system.  A is self-adjoint in the w J
// inner product and A >= I/(gamma-1) (the operator -div h grad is positive
// semi-definite there, with the constants in its null space), so its
// spectrum is real and lies in [1/(gamma-1), lmax].  With these bounds the
// Chebyshev recurrence (Saad, Iterative Methods for Sparse Linear Systems,
// Alg. 12.1) needs no inner product: one step is one mat-vec whose epilogue
// updates x, r and the direction in the same pass, two grid barriers in all;
// the residual norm for the stopping test comes from block partial sums read
// during the next step's gradient pass.  lmax is estimated in the kernel by power iteration in the
// w J norm (the ratio ||A p|| / ||p|| approaches lmax from below), widened by
// kLmaxMargin, and kept in a.lmax for later solves with the same alpha.  If
// the residual grows (an estimate too low), the bound is cleared and the solve
// finishes with GMRES from the current iterate.  The FP64 residual is
// recomputed at every restart; TK = float restarts whenever the residual has
// dropped by inner_tol (iterative refinement).
constexpr int kPowerIters = 24;
constexpr int kCtaClocks = 512;  // CTAs with a per-CTA pass clock
constexpr double kLmaxMargin = 1.05;

// The GMRES fallback of the Chebyshev solve, kept out of line: inlined, its
// register needs would be imposed on the Chebyshev loop as well.
template <int DIM, int DEG, typename TK, class Sync>
__device__ __noinline__ void gmres_fallback(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw, bool record) {
  gmres_body<DIM, DEG, TK, Sync>(a, sg, smem_raw, record);
}

// AFF: the mesh is horizontally affine (MeshView::aff), known at compile time
// for the Chebyshev steps' passes (the vanishing metric terms drop out).
template <int DIM, int DEG, typename TK, class Sync, bool AFF = false>
__device__ __forceinline__ void cheb_body(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw, bool record) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  double* sred = (double*)smem_raw;  // [32]
  double* sc = sred + 32;            // [16]
  double* sD64 = sc + 16;
  double* sDw64 = sD64 + N * N;
  double* sII64 = sDw64 + N * N;
  double* scell64 = sII64 + 4 * N * N;
  double* sJ64 = scell64 + DIM * S::CPB * S::NC;
  TK* sDk = (TK*)(sJ64 + coarse_buffer<DIM, DEG, DIM>());
  TK* sDwk = sDk + N * N;
  TK* sIIk = sDwk + N * N;
  TK* scellk = (TK*)scell64;
  TK* sJk = (TK*)sJ64;
  // the CTA's own batch for the Chebyshev steps (16-byte aligned, after the tables)
  auto* bcache = (BatchCache<DIM, DEG, TK>*)(((uintptr_t)(sIIk + 4 * N * N) + 15) & ~(uintptr_t)15);
  load_tables<DIM, DEG, TK>(a, sD64, sDw64, sII64, sDk, sDwk, sIIk);
  PhaseClock pc{record ? a.phase : nullptr, PhaseClock::now()};
  const int64_t n = a.n;
  const int G = sg.size;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;
  const int64_t lo = (int64_t)sg.rank * chunk1;
  const int64_t hi = lo + chunk1 < n ? lo + chunk1 : n;
  const bool mixed = sizeof(TK) != sizeof(double);
  TK* r = a.Q;          // residual (recurrence)
  TK* d = a.Q + n;      // direction
  TK* w = a.w;          // power-iteration partner
  // TK = float: the cycle's correction is summed in TK and added to the FP64 x
  // once per cycle (no FP64 work in the steps themselves)
  const bool fold = mixed && a.m >= 2;
  TK* dx = a.Q + 2 * n;
  const TK* wJ = a.mvk.wJ;
  TK* gvk = (TK*)a.gv;
  // sum of the G block partials, the same in every CTA
  auto gather_sum = [&]() -> double { return gather_allsum(a.partial, G, sred); };

  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += a.b[i] * a.b[i];
  {
    const double t = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[sg.rank] = t;
  }
  sg.sync();
  // Scalar functions of block-uniform values (square roots, divisions, logarithms) are
  // evaluated by thread 0 and read by the others from sc[3..15]: evaluated by every warp,
  // each would occupy the FP64 pipe once per warp.  Every slot is read right after the
  // barrier that follows its write, and rewritten only after further block barriers.
  {
    const double bsum = gather_sum();
    if (threadIdx.x == 0) sc[13] = sqrt(bsum);
    __syncthreads();
  }
  const double bn = sc[13];
  if (bn == 0.0) {
    for (int64_t i = tid; i < n; i += gstride) a.x[i] = 0.0;
    if (sg.rank == 0 && threadIdx.x == 0) {
      a.out[0] = 0;
      a.out[1] = 0;
      a.out[2] = 1;
      a.out[3] = 0;
    }
    return;
  }
  sg.sync();  // partial reused below

  // upper spectral bound: stored, or estimated here by power iteration
  const double lmin = 1.0 / (kGamma - 1.0);
  double lmax = a.lmax[0];
  if (!(lmax > lmin) || fabs(a.lmax[1] - a.alpha) > 1e-12 * a.alpha) {
    // deterministic start vector with every mode present; TK buffers r (p) and w
    acc = 0.0;
    for (int64_t i = tid; i < n; i += gstride) {
      unsigned int hsh = (unsigned int)i * 2654435761u + 0x9e3779b9u;
      hsh ^= hsh >> 16;
      hsh *= 0x85ebca6bu;
      hsh ^= hsh >> 13;
      const TK v = (TK)((double)(hsh & 0xffffffu) / 8388608.0 - 1.0);
      r[i] = v;
      acc += (double)wJ[i] * (double)v * (double)v;
    }
    {
      const double t = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[sg.rank] = t;
    }
    sg.sync();
    {
      const double s0 = gather_sum();
      if (threadIdx.x == 0) sc[14] = 1.0 / sqrt(s0);
      __syncthreads();
    }
    double inv = sc[14];
    TK* pin = r;
    TK* pout = w;
    double est = 0.0;
    for (int it = 0; it < kPowerIters; ++it) {
      double nacc = 0.0;
      auto epi = [&](int64_t i, TK v) {
        pout[i] = v;
        nacc += (double)wJ[i] * (double)v * (double)v;
      };
      auto fin = [&]() {
        const double t = block_sum(nacc, sred);
        if (threadIdx.x == 0) a.partial[sg.rank] = t;
      };
      pmatvec_epi<DIM, DEG, TK, Sync, decltype(epi), decltype(fin), AFF>(a.mvk, a.hk, (TK)a.alpha, TK(1), pin, (TK)inv, epi,
                                                                        fin, gvk, sg, scellk, sJk,
                                      sDk, sDwk, sIIk, pc);
      {
        const double s1 = gather_sum();
        if (threadIdx.x == 0) {
          const double e = sqrt(s1);  // ||A p^|| with ||p^|| = 1 in the w J norm
          sc[15] = e;
          sc[14] = e > 0.0 ? 1.0 / e : 0.0;
        }
        __syncthreads();
      }
      est = sc[15];
      inv = sc[14];
      TK* t = pin;
      pin = pout;
      pout = t;
      if (sg.failed()) break;
    }
    lmax = kLmaxMargin * est;
    if (!(lmax > lmin)) lmax = 2.0 * lmin;
    if (sg.rank == 0 && threadIdx.x == 0) {
      a.lmax[0] = lmax;
      a.lmax[1] = a.alpha;
    }
  }
  // theta, delta: centre and half width of [lmin, lmax]; sigma1 = theta / delta; q the
  // Chebyshev convergence factor (sqrt(kappa) - 1) / (sqrt(kappa) + 1)
  if (threadIdx.x == 0) {
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sk = sqrt(lmax / lmin);
    sc[8] = theta / delta;
    sc[9] = 1.0 / theta;
    sc[10] = 2.0 / delta;
    sc[11] = delta / theta;
    sc[12] = log((sk - 1.0) / (sk + 1.0));
  }
  __syncthreads();
  const double sigma1 = sc[8], itheta = sc[9], two_idelta = sc[10], rho0 = sc[11], logq = sc[12];

  int total = 0;
  double rel = 1.0;
  bool converged = false, diverged = false;
  while (!sg.failed()) {
    // FP64 residual r = b - A x; d = r / theta in the same pass
    pmatvec<DIM, DEG, double, Sync, AFF>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.gv, sg, scell64, sJ64, sD64,
                                    sDw64, sII64, pc);
    acc = 0.0;
    const TK ith = (TK)itheta;
    for (int64_t i = tid; i < n; i += gstride) {
      const double ri = a.b[i] - a.w64[i];
      r[i] = (TK)ri;
      d[i] = (TK)ri * ith;
      if (fold) dx[i] = TK(0);
      acc += ri * ri;
    }
    {
      const double t = block_sum(acc, sred);
      if (threadIdx.x == 0) a.partial[sg.rank] = t;
    }
    sg.sync();
    pc.mark(PH_RESIDUAL);
    {
      const double rsum = gather_sum();
      if (threadIdx.x == 0) {
        const double beta = sqrt(rsum);
        const double floor = fmax(a.tol * bn, (mixed ? a.inner_tol : 0.0) * beta);
        const double ib = 1.0 / beta, fr = floor * ib;
        sc[3] = beta;
        // steps the Chebyshev bound 2 q^k needs to reach the floor; well past that, the
        // residual has stalled or grows slowly (a bound a little low).  The stop test starts
        // after 3/4 of those steps: the residual norms before that are not needed (a bound
        // far too low makes that count small, so growth is still caught early)
        const double kpred = ceil(log(0.5 * fr) / logq);
        sc[4] = fmin(2.0 * kpred + 20.0, 1e9);
        sc[7] = fmin(fmax(trunc(0.75 * kpred) - 1.0, 0.0), 1e9);
        sc[5] = ib;
        sc[6] = fr * fr;
        rel = beta / bn;  // reported by thread 0
      }
      __syncthreads();
    }
    const double beta = sc[3];
    if (beta <= a.tol * bn) {
      converged = true;
      break;
    }
    if (total >= a.max_iters) break;
    const int cycle_cap = (int)sc[4];
    const int kskip = (int)sc[7];
    int cycle_its = 0;
    const float ibeta = (float)sc[5];
    // the stop test compares (||r|| / beta)^2 with squared limits (no square root per step);
    // the floor is kept above FP32 underflow (a cycle then ends at a 1e-15 reduction and the
    // FP64 restart decides)
    const float floor2 = fmaxf((float)sc[6], 1e-30f);
    constexpr float kGrowth2 = 1e8f;  // (1e4)^2
    double rho = rho0;
    const int64_t nb = a.mvk.nbat;
    bool have_prev = false;  // residual partials of the previous step are waiting in a.partial
    unsigned int token = 0u;  // the split grid barrier's arrival
    bool pending = false;
    // with at most one cell batch per CTA (the usual case on meshes that fit the launch), the
    // CTA's batch range is read once for the whole cycle (kept in shared memory: registers are
    // the scarce resource of this loop)
    const bool one = nb <= sg.size;
    __shared__ int4 s_mine;
    if (threadIdx.x == 0) s_mine = one && sg.rank < nb ? a.mvk.bdesc[sg.rank] : make_int4(0, 0, 0, 0);
    __syncthreads();
    // ... and its face links and coarse-side entries (BatchCache)
    const BatchCache<DIM, DEG, TK>* bc = nullptr;
    if (one && sg.rank < nb) {
      batch_cache_fill<DIM, DEG, TK>(a.mvk, BatchRange{s_mine.x, s_mine.y, s_mine.z, s_mine.w}, bcache);
      bc = bcache;
    }
    // per-CTA pass clocks (profiling): own gradient and divergence work, before the grid barriers
    unsigned long long* cta_clock = a.phase ? a.phase + 16 : nullptr;
    if (cta_clock && sg.rank < kCtaClocks && threadIdx.x == 0) {
      const bool cm = sg.rank < nb && a.mvk.bdesc[sg.rank].w > a.mvk.bdesc[sg.rank].z;
      cta_clock[2 * kCtaClocks + sg.rank] = cm ? 1ull : 0ull;
    }
    while (true) {
      // the next step's recurrence coefficients, by one thread, while the others start the
      // gradient pass (the FP64 division is off the critical path); read after the grid
      // barrier, and rewritten only after the divergence pass's block barriers
      if (threadIdx.x == blockDim.x - 1) {
        const double rho1 = 1.0 / (2.0 * sigma1 - rho);
        sc[0] = rho1;
        sc[1] = rho1 * rho;
        sc[2] = rho1 * two_idelta;
      }
      // gradient pass of A d_k; the grid barrier after the previous divergence pass is split:
      // this CTA arrived after its own writes, and waits inside the pass once its own loads
      // are in flight (pending: an arrival not yet waited for; the same in every CTA)
      unsigned long long tg0 = 0ull;
      auto wait_div = [&]() {
        if (pending) sg.wait(token);
        pending = false;
        if (cta_clock) tg0 = PhaseClock::now();
      };
      for (int64_t bt = sg.rank; bt < nb; bt += sg.size)
        grad_cell_batch<DIM, DEG, TK, false, AFF, decltype(wait_div)>(
            a.mvk, d, a.hk, gvk, one ? BatchRange{s_mine.x, s_mine.y, s_mine.z, s_mine.w} : batch_range(a.mvk, bt),
            scellk, sJk, sDk, sIIk, nullptr, bc, wait_div);
      if (pending) {  // a CTA without a batch still meets the barrier
        sg.wait(token);
        pending = false;
      }
      if (cta_clock && threadIdx.x == 0 && sg.rank < kCtaClocks && tg0) cta_clock[sg.rank] += PhaseClock::now() - tg0;
      if (have_prev) {
        // the previous step's residual norm.  The stop test needs it to a few digits only: its
        // sums run in FP32 on the residual scaled by 1/beta (no FP64 shuffle trees on the step's
        // critical path)
        float pv = 0.0f;
        for (int i = threadIdx.x; i < G; i += blockDim.x) pv += ((const float*)a.partial)[i];
        const float rn2 = block_allsum_f(pv, sred);  // (||r|| / beta)^2
        pc.mark(PH_UPDATE);
        if (!(rn2 <= kGrowth2) || (cycle_its > cycle_cap && rn2 > floor2)) {  // growth, stall or NaN: bound too low
          diverged = true;
          break;
        }
        if (rn2 <= floor2 || total >= a.max_iters || sg.failed()) break;  // same decision in every CTA
      } else if (total >= a.max_iters || sg.failed()) {
        break;
      }
      token = sg.arrive();
      pending = true;
      pc.mark(PH_GRAD_CELL);
      // whether the next step tests this step's residual (the same in every CTA)
      const bool want = cycle_its + 1 >= kskip;
      // divergence pass with the update: x += d, r -= A d, d = c1 d + c2 r
      const double rho1 = sc[0];
      const TK c1 = (TK)sc[1], c2 = (TK)sc[2];
      float racc = 0.0f;
      ChebStepEpi<TK> epi{d, r, dx, a.x, fold, c1, c2, want, ibeta, &racc};
      unsigned long long td0 = 0ull;
      auto wait_grad = [&]() {
        if (pending) sg.wait(token);
        pending = false;
        if (cta_clock) td0 = PhaseClock::now();
      };
      for (int64_t bt = sg.rank; bt < nb; bt += sg.size)
        div_cell_batch<DIM, DEG, TK, true, ChebStepEpi<TK>, false, AFF, decltype(wait_grad)>(
            a.mvk, gvk, d, (TK)a.alpha, TK(1), TK(1), epi,
            one ? BatchRange{s_mine.x, s_mine.y, s_mine.z, s_mine.w} : batch_range(a.mvk, bt), scellk, sJk, sDwk,
            sIIk, nullptr, nullptr, bc, wait_grad);
      if (pending) {
        sg.wait(token);
        pending = false;
      }
      if (cta_clock && threadIdx.x == 0 && sg.rank < kCtaClocks && td0)
        cta_clock[kCtaClocks + sg.rank] += PhaseClock::now() - td0;
      if (want) {
        const float t = block_sum_f(racc, sred);
        if (threadIdx.x == 0) ((float*)a.partial)[sg.rank] = t;  // FP32 partials for the stop test
      }
      token = sg.arrive();
      pending = true;
      pc.mark(PH_DIV_CELL);
      rho = rho1;
      ++total;
      ++cycle_its;
      have_prev = want;
    }
    if (pending) {  // (the loop leaves only after a gradient pass, which has waited)
      sg.wait(token);
      pending = false;
    }
    if (fold)
      for (int64_t i = tid; i < n; i += gstride) a.x[i] += (double)dx[i];
    // CTAs may leave the loop inside a gradient pass (whose scratch aliases the
    // FP64 residual's): meet before the next pass.  At max_iters the loop still
    // goes round once more, so that the reported residual is the final one.
    sg.sync();
    if (diverged) break;
  }
  if (diverged) {
    if (sg.rank == 0 && threadIdx.x == 0) a.lmax[0] = 0.0;  // re-estimate on the next solve
    sg.sync();
    gmres_fallback<DIM, DEG, TK, Sync>(a, sg, smem_raw, record);
    if (sg.rank == 0 && threadIdx.x == 0) a.out[0] += total;
    return;
  }
  if (sg.rank == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = rel;
    a.out[2] = (converged && !sg.failed()) ? 1.0 : 0.0;
    a.out[3] = bn;
    if (pc.acc) a.phase[PH_ITERS] += (unsigned long long)total;
  }
}

// One kernel per method (each allocates registers for its own body only; the
// Chebyshev one holds the GMRES body too, its fallback); AFF: the Chebyshev
// form for horizontally affine meshes.
template <int DIM, int DEG, typename TK, int METHOD, bool AFF = false>
__global__ void __launch_bounds__(256, 2) gmres_persistent_kernel(GmresPArgs<TK> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GridSync sg;
  if (METHOD == 1)
    cg_body<DIM, DEG, TK, GridSync>(a, sg, smem_raw, blockIdx.x == 0);
  else if (METHOD == 2)
    gmres_cgs2_body<DIM, DEG, TK, GridSync>(a, sg, smem_raw, blockIdx.x == 0);
  else if (METHOD == 3)
    cheb_body<DIM, DEG, TK, GridSync, AFF>(a, sg, smem_raw, blockIdx.x == 0);
  else
    gmres_body<DIM, DEG, TK, GridSync>(a, sg, smem_raw, blockIdx.x == 0);
}

// Many independent solves in one cooperative launch: CTA b works on member
// cta_member[b] as its rank cta_rank[b] of member_ctas[member] CTAs, with the
// member's own barrier; members progress and finish independently.
struct BatchMap {
  const int* cta_member;
  const int* cta_rank;
  const int* member_ctas;
  unsigned int* bar_count;  // [members]
  unsigned int* bar_gen;    // [members]
  int* err;                 // [1]
  unsigned long long timeout_ns;  // bound of every barrier wait
};

template <int DIM, int DEG, typename TK>
__global__ void __launch_bounds__(256, 2) gmres_batched_kernel(const GmresPArgs<TK>* __restrict__ args, BatchMap map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sfail;
  const int mem = map.cta_member[blockIdx.x];
  if (threadIdx.x == 0) sfail = 0;
  __syncthreads();
  SubSync sg{map.cta_rank[blockIdx.x], map.member_ctas[mem], map.bar_count + mem, map.bar_gen + mem, map.err,
             &sfail, map.timeout_ns};
  const GmresPArgs<TK> a = args[mem];
  if (a.method == 1)
    cg_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
  else if (a.method == 2)
    gmres_cgs2_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
  else if (a.method == 3)
    cheb_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
  else
    gmres_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
}

template <int DIM, int DEG, typename TK>
inline size_t gmres_smem_bytes(int m) {
  constexpr int N = DEG + 1;
  using S = Shape<DIM, DEG>;
  const size_t dbl = (size_t)(m + 1) + 2 * (size_t)(m + 2) + (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m +
                     (m + 1) + 32 + 8 + 512;
  const size_t tabs = (size_t)(6 * N * N + DIM * S::CPB * S::NC + coarse_buffer<DIM, DEG, DIM>()) * sizeof(double) +
                      (size_t)(6 * N * N) * sizeof(TK) + sizeof(BatchCache<DIM, DEG, TK>) + 16;
  const size_t gm = dbl * sizeof(double) + 4 * sizeof(int) + tabs + 64;
  const size_t d1 = 2 * (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m + 5 * (size_t)(m + 1) + 32 + 8;
  const size_t g1 = d1 * sizeof(double) + 4 * sizeof(int) + tabs + 64;
  const size_t cg = (size_t)(96 + 16) * sizeof(double) + tabs + 64;
  return std::max(gm, std::max(g1, cg));
}

}  // namespace dg
