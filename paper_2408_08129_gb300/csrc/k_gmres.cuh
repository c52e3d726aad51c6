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
  double* Gh;             // face scratch (dim*nf*NF doubles), reused as TK
  double* gv;             // [dim][n] gradient scratch (doubles), reused as TK
  double* partial;        // >= 2 x (CTAs of the solve) doubles
  double* out;            // [4]: iterations, relative residual, converged (0/1), ||b||
  unsigned long long* phase;  // optional [16] ns per phase accumulated by block 0 (NULL = off)
  double alpha;           // (a_ii dt)^2
  double tol;             // target ||b - A x|| / ||b|| (checked on the FP64 residual)
  double inner_tol;       // TK = float: residual reduction per cycle
  int m;
  int max_iters;
  int64_t n;
  int method;  // 0: GMRES(m); 1: conjugate gradients in the M inner product (needs m >= 2)
};

enum GmresPhase {
  PH_GRAD_FACE = 0, PH_GRAD_CELL, PH_DIV_FACE, PH_DIV_CELL, PH_DOTS, PH_UPDATE, PH_REORTH, PH_RESIDUAL,
  PH_SOLUTION, PH_ITERS = 15
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
// Its wait is bounded: after kBarrierTimeoutNs it raises the launch's error
// flag and every barrier of the launch returns at once from then on, so a
// fault can only end the kernel early, never hang it.
struct GridSync {
  cooperative_groups::grid_group grid;
  int rank, size;
  __device__ GridSync() : grid(cooperative_groups::this_grid()), rank(blockIdx.x), size(gridDim.x) {}
  __device__ __forceinline__ void sync() { grid.sync(); }
  __device__ __forceinline__ bool failed() const { return false; }
};

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s

struct SubSync {
  int rank, size;
  unsigned int* count;  // arrivals at the current barrier
  unsigned int* gen;    // barrier generation
  int* err;             // launch-wide error flag
  int* sfail;           // shared-memory copy of err, read by every thread
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
            if (PhaseClock::now() - t0 > kBarrierTimeoutNs) {
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
  __device__ __forceinline__ bool failed() const { return *(volatile int*)sfail != 0; }
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

// copy cnt (<= 512) global partial sums into shared memory with all threads
// (one parallel round trip instead of a serial chain of loads)
__device__ __forceinline__ void stage_partials(const double* partial, int cnt, double* spart) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) spart[i] = partial[i];
  __syncthreads();
}

// warp-level sum in TK, then FP64 across warps
template <typename TK>
__device__ __forceinline__ double block_sum_k(TK v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sred[i];
  return r;
}

// out = scale * (ident p/(gamma-1) - alpha div(h grad p)) (four phases, four grid barriers)
template <int DIM, int DEG, typename T, class Sync>
__device__ __forceinline__ void pmatvec(const MeshView<T>& mv, const T* h, T alpha, T ident, const T* p, T scale,
                                        T* out, T* Gh, T* gv, Sync& sg, T* scell, const T* sD, const T* sDw,
                                        const T* sIt, PhaseClock& pc) {
  using S = Shape<DIM, DEG>;
  const int64_t nfi = (int64_t)(mv.nconf + mv.nsub) * S::NF;
  const int64_t stride = (int64_t)sg.size * blockDim.x;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t nb = (mv.n_cells + S::CPB - 1) / S::CPB;
  for (int64_t t = tid; t < nfi; t += stride) grad_face_item<DIM, DEG, T>(mv, p, Gh, t);
  sg.sync();
  pc.mark(PH_GRAD_FACE);
  for (int64_t bt = sg.rank; bt < nb; bt += sg.size) grad_cell_batch<DIM, DEG, T>(mv, p, h, Gh, gv, bt, scell, sD, sIt);
  sg.sync();
  pc.mark(PH_GRAD_CELL);
  for (int64_t t = tid; t < nfi; t += stride) div_face_item<DIM, DEG, T>(mv, gv, Gh, t);
  sg.sync();
  pc.mark(PH_DIV_FACE);
  for (int64_t bt = sg.rank; bt < nb; bt += sg.size)
    div_cell_batch<DIM, DEG, T, true>(mv, gv, Gh, p, alpha, scale, ident, out, bt, scell, sDw, sIt);
  sg.sync();
  pc.mark(PH_DIV_CELL);
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

template <int DIM, int DEG, typename TK, class Sync>
__device__ __forceinline__ void gmres_body(const GmresPArgs<TK>& a, Sync& sg, unsigned char* smem_raw,
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
  double* t64 = (double*)(sflag + 4);  // FP64 tables D, Dw, It
  double* sD64 = t64;
  double* sDw64 = sD64 + N * N;
  double* sIt64 = sDw64 + N * N;
  double* scell64 = sIt64 + 2 * N * N;  // cell tile, CPB*NC doubles (reused as TK)
  TK* tk = (TK*)(scell64 + S::CPB * S::NC);
  TK* sDk = tk;
  TK* sDwk = sDk + N * N;
  TK* sItk = sDwk + N * N;
  TK* scellk = (TK*)scell64;

  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    sD64[q] = a.mv64.tab[S::T_D + q];
    sDw64[q] = a.mv64.tab[S::T_DW + q];
    sDk[q] = a.mvk.tab[S::T_D + q];
    sDwk[q] = a.mvk.tab[S::T_DW + q];
  }
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) {
    sIt64[q] = a.mv64.tab[S::T_IT + q];
    sItk[q] = a.mvk.tab[S::T_IT + q];
  }
  __syncthreads();
  PhaseClock pc{record ? a.phase : nullptr, PhaseClock::now()};

  const int64_t n = a.n;
  const int G = sg.size;
  const int64_t tid = (int64_t)sg.rank * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)G * blockDim.x;
  const int64_t chunk1 = (n + G - 1) / G;
  const bool mixed = sizeof(TK) != sizeof(double);
  TK* Ghk = (TK*)a.Gh;
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
  stage_partials(a.partial, G, spart);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < G; ++i) s += spart[i];
    sc[0] = sqrt(s);
  }
  __syncthreads();
  const double bn = sc[0];
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
    pmatvec<DIM, DEG, double, Sync>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.Gh, a.gv, sg, scell64, sD64,
                                    sDw64, sIt64, pc);
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
    stage_partials(a.partial, G, spart);
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < G; ++i) s += spart[i];
      const double beta = sqrt(s);
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
      pmatvec<DIM, DEG, TK, Sync>(a.mvk, a.hk, (TK)a.alpha, TK(0), qk, (TK)sigma[k], a.w, Ghk, gvk, sg, scellk,
                                  sDk, sDwk, sItk, pc);
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
  double* sred = (double*)smem_raw;  // [32]
  double* sc = sred + 32;            // [16]
  double* spart = sc + 16;           // [3*512]
  double* sD64 = spart + 3 * 512;
  double* sDw64 = sD64 + N * N;
  double* sIt64 = sDw64 + N * N;
  double* scell64 = sIt64 + 2 * N * N;
  TK* sDk = (TK*)(scell64 + S::CPB * S::NC);
  TK* sDwk = sDk + N * N;
  TK* sItk = sDwk + N * N;
  TK* scellk = (TK*)scell64;
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    sD64[q] = a.mv64.tab[S::T_D + q];
    sDw64[q] = a.mv64.tab[S::T_DW + q];
    sDk[q] = a.mvk.tab[S::T_D + q];
    sDwk[q] = a.mvk.tab[S::T_DW + q];
  }
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) {
    sIt64[q] = a.mv64.tab[S::T_IT + q];
    sItk[q] = a.mvk.tab[S::T_IT + q];
  }
  __syncthreads();
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
  TK* Ghk = (TK*)a.Gh;
  TK* gvk = (TK*)a.gv;

  {
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += a.b[i] * a.b[i];
    const double t = block_sum(acc, sred);
    if (threadIdx.x == 0) a.partial[sg.rank] = t;
  }
  sg.sync();
  stage_partials(a.partial, G, spart);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < G; ++i) t += spart[i];
    sc[0] = sqrt(t);
  }
  __syncthreads();
  const double bn = sc[0];
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
    pmatvec<DIM, DEG, double, Sync>(a.mv64, a.h64, a.alpha, 1.0, a.x, 1.0, a.w64, a.Gh, a.gv, sg, scell64, sD64,
                                    sDw64, sIt64, pc);
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
    stage_partials(a.partial, G, spart);
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < G; ++i) t += spart[i];
      sc[1] = sqrt(t);
    }
    __syncthreads();
    const double beta0 = sc[1];
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
      pmatvec<DIM, DEG, TK, Sync>(a.mvk, a.hk, (TK)a.alpha, TK(1), r, TK(1), w, Ghk, gvk, sg, scellk, sDk, sDwk,
                                  sItk, pc);
      {
        TK g0 = TK(0), d0 = TK(0), e0 = TK(0);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
          const TK ri = r[i], mi = wJ[i] * ri;
          g0 += mi * ri;
          d0 += mi * w[i];
          e0 += ri * ri;
        }
        const double tg = block_sum_k<TK>(g0, sred);
        const double td = block_sum_k<TK>(d0, sred);
        const double te = block_sum_k<TK>(e0, sred);
        if (threadIdx.x == 0) {
          a.partial[3 * sg.rank] = tg;
          a.partial[3 * sg.rank + 1] = td;
          a.partial[3 * sg.rank + 2] = te;
        }
      }
      sg.sync();
      pc.mark(PH_DOTS);
      stage_partials(a.partial, 3 * G, spart);
      if (threadIdx.x == 0) {
        double tg = 0.0, td = 0.0, te = 0.0;
        for (int i = 0; i < G; ++i) {
          tg += spart[3 * i];
          td += spart[3 * i + 1];
          te += spart[3 * i + 2];
        }
        sc[2] = tg;
        sc[3] = td;
        sc[4] = sqrt(te);
      }
      __syncthreads();
      const double gnew = sc[2], delta = sc[3], rn = sc[4];
      ++total;
      rel = rn / bn;
      if (sg.failed() || rn <= floor || total >= a.max_iters || !(delta > 0.0) || !(gnew > 0.0)) break;
      double beta;
      if (first) {
        beta = 0.0;
        alpha = gnew / delta;
        first = false;
      } else {
        beta = gnew / gamma;
        alpha = gnew / (delta - beta * gnew / alpha);
      }
      gamma = gnew;
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

template <int DIM, int DEG, typename TK>
__global__ void __launch_bounds__(256, 2) gmres_persistent_kernel(GmresPArgs<TK> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GridSync sg;
  if (a.method == 1)
    cg_body<DIM, DEG, TK, GridSync>(a, sg, smem_raw, blockIdx.x == 0);
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
};

template <int DIM, int DEG, typename TK>
__global__ void __launch_bounds__(256, 3) gmres_batched_kernel(const GmresPArgs<TK>* __restrict__ args, BatchMap map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sfail;
  const int mem = map.cta_member[blockIdx.x];
  if (threadIdx.x == 0) sfail = 0;
  __syncthreads();
  SubSync sg{map.cta_rank[blockIdx.x], map.member_ctas[mem], map.bar_count + mem, map.bar_gen + mem, map.err,
             &sfail};
  const GmresPArgs<TK> a = args[mem];
  if (a.method == 1)
    cg_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
  else
    gmres_body<DIM, DEG, TK, SubSync>(a, sg, smem_raw, false);
}

template <int DIM, int DEG, typename TK>
inline size_t gmres_smem_bytes(int m) {
  constexpr int N = DEG + 1;
  using S = Shape<DIM, DEG>;
  const size_t dbl = (size_t)(m + 1) + 2 * (size_t)(m + 2) + (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m +
                     (m + 1) + 32 + 8 + 512;
  const size_t tabs = (size_t)(4 * N * N + S::CPB * S::NC) * sizeof(double) + (size_t)(4 * N * N) * sizeof(TK);
  const size_t gm = dbl * sizeof(double) + 4 * sizeof(int) + tabs + 64;
  const size_t cg = (size_t)(32 + 16 + 3 * 512) * sizeof(double) + tabs + 64;
  return gm > cg ? gm : cg;
}

}  // namespace dg
