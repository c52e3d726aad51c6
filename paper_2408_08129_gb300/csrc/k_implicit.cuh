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

// Gh_b = 1/2 |N| n_b (p+ - p-) on conforming faces and subfaces (walls skipped).
template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(256) grad_face_kernel(MeshView<T> mv, const T* __restrict__ p,
                                                        T* __restrict__ Gh, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int NC = S::NC, NF = S::NF;
  const int64_t total = (int64_t)mv.nf * NF;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(mv.nconf + mv.nsub) * NF) return;
  const int f = (int)(t / NF), k = (int)(t % NF);
  const int64_t Nn = mv.n_nodes;
  const T pm = p[(int64_t)mv.face_m[f] * NC + face_node<DIM, DEG>(mv.face_lfm[f], k)];
  T pp;
  if (f < mv.nconf)
    pp = p[(int64_t)mv.face_p[f] * NC + face_node<DIM, DEG>(mv.face_lfp[f], k)];
  else
    coarse_at<DIM, DEG, T, 1>(mv, p, Nn, f, k, &pp);
  const T jmp = T(0.5) * mv.fsj[t] * (pp - pm);
#pragma unroll
  for (int b = 0; b < DIM; ++b) Gh[(int64_t)b * total + t] = jmp * mv.fn[(int64_t)b * total + t];
}

// g_b = h * [sum_a Ja^a_b (D_a p) + gathered Gh_b / w_end] / J   (h optional)
template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) grad_cell_kernel(MeshView<T> mv,
                                                                             const T* __restrict__ p,
                                                                             const T* __restrict__ h,
                                                                             const T* __restrict__ Gh,
                                                                             T* __restrict__ g, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, CPB = S::CPB;
  __shared__ T sp[CPB * NC];
  __shared__ T sD[N * N];
  __shared__ T sIt[2 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sD[q] = mv.tab[S::T_D + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int64_t c = (int64_t)blockIdx.x * CPB + lc;
  const bool active = (lc < CPB) && (c < mv.n_cells);
  const int64_t Nn = mv.n_nodes;
  const int64_t idx = c * NC + i;
  if (active) sp[lc * NC + i] = p[idx];
  __syncthreads();
  if (!active) return;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
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
  gather_faces<DIM, DEG, T, DIM>(mv, Gh, c, id, sIt, T(1), T(1), true, facc);
  const T iwend = mv.tab[S::T_IWEND];
  const T scale = mv.invJ[idx] * (h ? h[idx] : T(1));
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    T s = facc[b] * iwend;
#pragma unroll
    for (int a = 0; a < DIM; ++a) s += mv.Ja[(int64_t)(a * DIM + b) * Nn + idx] * dp[a];
    g[(int64_t)b * Nn + idx] = s * scale;
  }
}

// Dh = |N| {f}.n on conforming faces and subfaces (walls skipped).
template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(256) div_face_kernel(MeshView<T> mv, const T* __restrict__ fld,
                                                       T* __restrict__ Dh, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int NC = S::NC, NF = S::NF;
  const int64_t total = (int64_t)mv.nf * NF;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(mv.nconf + mv.nsub) * NF) return;
  const int f = (int)(t / NF), k = (int)(t % NF);
  const int64_t Nn = mv.n_nodes;
  const int64_t im = (int64_t)mv.face_m[f] * NC + face_node<DIM, DEG>(mv.face_lfm[f], k);
  T fp[DIM];
  if (f < mv.nconf) {
    const int64_t ip = (int64_t)mv.face_p[f] * NC + face_node<DIM, DEG>(mv.face_lfp[f], k);
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

// out = HELM ? p/(gamma-1) - alpha*div : div
template <int DIM, int DEG, typename T, bool HELM>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) div_cell_kernel(MeshView<T> mv,
                                                                            const T* __restrict__ fld,
                                                                            const T* __restrict__ Dh,
                                                                            const T* __restrict__ p, T alpha,
                                                                            T* __restrict__ out, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, CPB = S::CPB;
  __shared__ T sF[CPB * NC];
  __shared__ T sDw[N * N];
  __shared__ T sIt[2 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sDw[q] = mv.tab[S::T_DW + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int64_t c = (int64_t)blockIdx.x * CPB + lc;
  const bool active = (lc < CPB) && (c < mv.n_cells);
  const int64_t Nn = mv.n_nodes;
  const int64_t idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  T fv[DIM];
  if (active) {
#pragma unroll
    for (int b = 0; b < DIM; ++b) fv[b] = fld[(int64_t)b * Nn + idx];
  }
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (active) {
      T ft = T(0);
#pragma unroll
      for (int b = 0; b < DIM; ++b) ft += mv.Ja[(int64_t)(a * DIM + b) * Nn + idx] * fv[b];
      sF[lc * NC + i] = ft;
    }
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
  if (!active) return;
  T facc = T(0);
  gather_faces<DIM, DEG, T, 1>(mv, Dh, c, id, sIt, T(1), T(-1), true, &facc);
  const T dv = (acc + facc * mv.tab[S::T_IWEND]) * mv.invJ[idx];
  if (HELM)
    out[idx] = p[idx] / gm1<T>() - alpha * dv;
  else
    out[idx] = dv;
}

}  // namespace dg
