// Operators of the implicit pressure stage (Sec. 2 IMEX split; Sec. 3.2
// pressure loop), centred traces, in two passes each:
//
//  gradient (strong form):  g_b = [ sum_a Ja^a_b (D_a p) + Gh_b / w_end ] / J,
//      face value Gh_b = 1/2 |N| n_b (p+ - p-), added with + on both sides
//      and through It on the coarse side; zero on walls (p^ = p-).
//  divergence (weak form):  div = [ -sum_a sum_k Dw[i_a][k] (Ja^a.f)(k) + Dh/w_end ] / J,
//      face value Dh = |N| {f}.n, + on the minus side, - on the plus and
//      coarse sides; zero on walls.
//  Helmholtz:  A p = p/(gamma-1) - alpha div(h grad p), as grad(h-scaled)
//      followed by the divergence with the Helmholtz epilogue.
//
// The per-item work is written as device functions so that the standalone
// kernels below and the persistent GMRES kernel (k_gmres.cuh) share it.
#pragma once

#include "dg_device.cuh"
#include "k_explicit.cuh"

namespace dg {

// Interpolated coarse value of an NV-component field at fine face node k of subface f.
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void coarse_at(const MeshView<T>& mv, const T* __restrict__ X, int64_t Nn, int f,
                                          int k, T* out) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC;
  const int cp = mv.face_p[f], lfp = mv.face_lfp[f], s = mv.face_s[f];
  const T* I = mv.tab + S::T_I;
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = T(0);
  if (DIM == 2) {
    const T* Is = I + s * N * N + k * N;
    for (int j = 0; j < N; ++j) {
      const int64_t ic = (int64_t)cp * NC + face_node<DIM, DEG>(lfp, j);
#pragma unroll
      for (int v = 0; v < NV; ++v) out[v] += Is[j] * X[(int64_t)v * Nn + ic];
    }
  } else {
    const int k1 = k % N, k2 = k / N;
    const T* I1 = I + (s & 1) * N * N + k1 * N;
    const T* I2 = I + ((s >> 1) & 1) * N * N + k2 * N;
    for (int j2 = 0; j2 < N; ++j2)
      for (int j1 = 0; j1 < N; ++j1) {
        const int64_t ic = (int64_t)cp * NC + face_node<DIM, DEG>(lfp, j1 + N * j2);
        const T wgt = I1[j1] * I2[j2];
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] += wgt * X[(int64_t)v * Nn + ic];
      }
  }
}

// ---------------------------------------------------------------- gradient

// face node t (< (nconf+nsub)*NF): Gh_b = 1/2 |N| n_b (p+ - p-)
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void grad_face_item(const MeshView<T>& mv, const T* __restrict__ p, T* __restrict__ Gh,
                                               int64_t t) {
  using S = Shape<DIM, DEG>;
  constexpr int NC = S::NC, NF = S::NF;
  const int64_t total = (int64_t)mv.nf * NF;
  const int f = (int)(t / NF), k = (int)(t % NF);
  const T pm = p[mv.fnode_m[t]];
  T pp;
  if (f < mv.nconf)
    pp = p[mv.fnode_p[t]];
  else
    coarse_at<DIM, DEG, T, 1>(mv, p, mv.n_nodes, f, k, &pp);
  const T jmp = T(0.5) * mv.fsj[t] * (pp - pm);
#pragma unroll
  for (int b = 0; b < DIM; ++b) Gh[(int64_t)b * total + t] = jmp * mv.fn[(int64_t)b * total + t];
}

// Cells [batch*CPB, batch*CPB + CPB): g_b = h [sum_a Ja^a_b (D_a p) + Gh_b / w_end] / J.
// Called by a whole block with blockDim >= CPB*NC; contains __syncthreads.
// Every global load that does not depend on the face values is issued before
// the barrier so that the loads' latencies overlap.
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void grad_cell_batch(const MeshView<T>& mv, const T* __restrict__ p,
                                                const T* __restrict__ h, const T* __restrict__ Gh,
                                                T* __restrict__ g, int64_t batch, T* sp, const T* sD,
                                                const T* sIt) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, CPB = S::CPB;
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int64_t c = batch * CPB + lc;
  const bool active = (lc < CPB) && (c < mv.n_cells);
  const int64_t Nn = mv.n_nodes;
  const int64_t idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  int codes[DIM];
  T Jl[DIM][DIM];
  T scale = T(0);
  if (active) {
    sp[lc * NC + i] = p[idx];
    load_face_codes<DIM, DEG, T>(mv, c, id, codes);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) Jl[a][b] = mv.Ja[(int64_t)(a * DIM + b) * Nn + idx];
    scale = mv.invJ[idx] * (h ? h[idx] : T(1));
  }
  __syncthreads();
  if (active) {
    T dp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int i0 = lc * NC + i - id[a] * stride;
      const T* D = sD + id[a] * N;
      T s = T(0);
#pragma unroll
      for (int kk = 0; kk < N; ++kk) s += D[kk] * sp[i0 + kk * stride];
      dp[a] = s;
    }
    T facc[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) facc[b] = T(0);
    gather_faces_codes<DIM, DEG, T, DIM>(mv, Gh, codes, id, sIt, T(1), T(1), true, facc);
    const T iwend = mv.tab[S::T_IWEND];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T s = facc[b] * iwend;
#pragma unroll
      for (int a = 0; a < DIM; ++a) s += Jl[a][b] * dp[a];
      g[(int64_t)b * Nn + idx] = s * scale;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- divergence

// face node t (< (nconf+nsub)*NF): Dh = |N| {f}.n
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void div_face_item(const MeshView<T>& mv, const T* __restrict__ fld, T* __restrict__ Dh,
                                              int64_t t) {
  using S = Shape<DIM, DEG>;
  constexpr int NC = S::NC, NF = S::NF;
  const int64_t total = (int64_t)mv.nf * NF;
  const int f = (int)(t / NF), k = (int)(t % NF);
  const int64_t Nn = mv.n_nodes;
  const int64_t im = mv.fnode_m[t];
  T fp[DIM];
  if (f < mv.nconf) {
    const int64_t ip = mv.fnode_p[t];
#pragma unroll
    for (int b = 0; b < DIM; ++b) fp[b] = fld[(int64_t)b * Nn + ip];
  } else {
    coarse_at<DIM, DEG, T, DIM>(mv, fld, Nn, f, k, fp);
  }
  T s = T(0);
#pragma unroll
  for (int b = 0; b < DIM; ++b) s += (fld[(int64_t)b * Nn + im] + fp[b]) * mv.fn[(int64_t)b * total + t];
  Dh[t] = T(0.5) * mv.fsj[t] * s;
}

// Cells of one batch: out = HELM ? scale * (ident p/(gamma-1) - alpha div) : div.
// Called by a whole block with blockDim >= CPB*NC; contains __syncthreads.
template <int DIM, int DEG, typename T, bool HELM>
__device__ __forceinline__ void div_cell_batch(const MeshView<T>& mv, const T* __restrict__ fld,
                                               const T* __restrict__ Dh, const T* __restrict__ p, T alpha, T scale,
                                               T ident, T* __restrict__ out, int64_t batch, T* sF, const T* sDw,
                                               const T* sIt) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, CPB = S::CPB;
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int64_t c = batch * CPB + lc;
  const bool active = (lc < CPB) && (c < mv.n_cells);
  const int64_t Nn = mv.n_nodes;
  const int64_t idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  int codes[DIM];
  T ft[DIM];  // Ja^a . f for each axis a
  T ij = T(0), pv = T(0);
  if (active) {
    T fv[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) fv[b] = fld[(int64_t)b * Nn + idx];
    load_face_codes<DIM, DEG, T>(mv, c, id, codes);
    ij = mv.invJ[idx];
    if (HELM) pv = p[idx];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < DIM; ++b) s += mv.Ja[(int64_t)(a * DIM + b) * Nn + idx] * fv[b];
      ft[a] = s;
    }
  }
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (active) sF[lc * NC + i] = ft[a];
    __syncthreads();
    if (active) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int i0 = lc * NC + i - id[a] * stride;
      const T* Dw = sDw + id[a] * N;
#pragma unroll
      for (int kk = 0; kk < N; ++kk) acc -= Dw[kk] * sF[i0 + kk * stride];
    }
    __syncthreads();
  }
  if (active) {
    T facc = T(0);
    gather_faces_codes<DIM, DEG, T, 1>(mv, Dh, codes, id, sIt, T(1), T(-1), true, &facc);
    const T dv = (acc + facc * mv.tab[S::T_IWEND]) * ij;
    if (HELM)
      out[idx] = scale * (ident * pv / gm1<T>() - alpha * dv);
    else
      out[idx] = dv;
  }
}

// ---------------------------------------------------------------- standalone kernels

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(256) grad_face_kernel(MeshView<T> mv, const T* __restrict__ p,
                                                        T* __restrict__ Gh, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(mv.nconf + mv.nsub) * Shape<DIM, DEG>::NF) return;
  grad_face_item<DIM, DEG, T>(mv, p, Gh, t);
}

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) grad_cell_kernel(MeshView<T> mv,
                                                                             const T* __restrict__ p,
                                                                             const T* __restrict__ h,
                                                                             const T* __restrict__ Gh,
                                                                             T* __restrict__ g,
                                                                             const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sp[S::CPB * S::NC];
  __shared__ T sD[N * N];
  __shared__ T sIt[2 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sD[q] = mv.tab[S::T_D + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  grad_cell_batch<DIM, DEG, T>(mv, p, h, Gh, g, blockIdx.x, sp, sD, sIt);
}

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(256) div_face_kernel(MeshView<T> mv, const T* __restrict__ fld,
                                                       T* __restrict__ Dh, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(mv.nconf + mv.nsub) * Shape<DIM, DEG>::NF) return;
  div_face_item<DIM, DEG, T>(mv, fld, Dh, t);
}

template <int DIM, int DEG, typename T, bool HELM>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) div_cell_kernel(MeshView<T> mv,
                                                                            const T* __restrict__ fld,
                                                                            const T* __restrict__ Dh,
                                                                            const T* __restrict__ p, T alpha,
                                                                            T* __restrict__ out,
                                                                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sF[S::CPB * S::NC];
  __shared__ T sDw[N * N];
  __shared__ T sIt[2 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sDw[q] = mv.tab[S::T_DW + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  div_cell_batch<DIM, DEG, T, HELM>(mv, fld, Dh, p, alpha, T(1), T(1), out, blockIdx.x, sF, sDw, sIt);
}

}  // namespace dg
