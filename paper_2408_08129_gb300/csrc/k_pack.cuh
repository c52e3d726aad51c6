// Member packs: one launch of an operator kernel over the cells (or face
// nodes) of many meshes of the same dimension and degree, for the ensemble
// step (many uneven members advanced together, one launch per phase instead of
// one per member).  The pack travels as a kernel parameter (__grid_constant__,
// a few KB), so a launch needs no argument upload and can be captured into a
// CUDA graph as it is.  CTA b works on member j with start[j] <= b < start[j+1],
// as CTA b - start[j] of that member's own launch shape.
#pragma once

#include "k_explicit.cuh"
#include "k_implicit.cuh"
#include "ops.h"

namespace dg {

// member of this CTA (linear scan of at most kPack starts in parameter space)
template <typename T>
__device__ __forceinline__ int pack_member(const OpPack<T>& P) {
  int j = 0;
  while (j + 1 < P.n && (int)blockIdx.x >= P.start[j + 1]) ++j;
  return j;
}

template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__global__ void __launch_bounds__(256) explicit_face_pack_kernel(const __grid_constant__ OpPack<T> P) {
  const int j = pack_member(P);
  const MeshView<T>& mv = P.mv[j];
  const int64_t t = (int64_t)(blockIdx.x - P.start[j]) * blockDim.x + threadIdx.x;
  if (t >= (int64_t)mv.nf * Shape<DIM, DEG>::NF) return;
  explicit_face_item<DIM, DEG, T, FULL, PERT>(mv, P.in[j], P.scratch[j], t);
}

template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) explicit_cell_pack_kernel(
    const __grid_constant__ OpPack<T> P) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sF[S::V][S::CPB * S::NC];
  __shared__ T sDw[N * N];
  __shared__ T sIt[2 * N * N];
  const int j = pack_member(P);
  const MeshView<T>& mv = P.mv[j];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sDw[q] = mv.tab[S::T_DW + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  explicit_cell_batch<DIM, DEG, T, FULL, PERT>(mv, P.in[j], P.scratch[j], P.out[j], blockIdx.x - P.start[j], sF,
                                               sDw, sIt);
}

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) grad_pack_kernel(const __grid_constant__ OpPack<T> P) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sp[S::CPB * S::NC];
  __shared__ T sJ[coarse_buffer<DIM, DEG, DIM>()];
  __shared__ T sD[N * N];
  __shared__ T sII[4 * N * N];
  const int j = pack_member(P);
  const MeshView<T>& mv = P.mv[j];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sD[q] = mv.tab[S::T_D + q];
  for (int q = threadIdx.x; q < 4 * N * N; q += blockDim.x) sII[q] = mv.tab[S::T_I + q];
  __syncthreads();  // the fine-side traces read the interpolation tables before the batch's first barrier
  const BatchRange br = batch_range(mv, blockIdx.x - P.start[j]);
  if (mv.aff)  // block-uniform: the horizontally affine form without the vanishing metric terms
    grad_cell_batch<DIM, DEG, T, false, true>(mv, P.in[j], P.aux[j], P.out[j], br, sp, sJ, sD, sII);
  else
    grad_cell_batch<DIM, DEG, T, false, false>(mv, P.in[j], P.aux[j], P.out[j], br, sp, sJ, sD, sII);
}

template <int DIM, int DEG, typename T>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) div_pack_kernel(const __grid_constant__ OpPack<T> P) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sF[DIM * S::CPB * S::NC];
  __shared__ T sJ[coarse_buffer<DIM, DEG, 1>()];
  __shared__ T sDw[N * N];
  __shared__ T sII[4 * N * N];
  const int j = pack_member(P);
  const MeshView<T>& mv = P.mv[j];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sDw[q] = mv.tab[S::T_DW + q];
  for (int q = threadIdx.x; q < 4 * N * N; q += blockDim.x) sII[q] = mv.tab[S::T_I + q];
  __syncthreads();
  StoreOut<T> epi{P.out[j]};
  const BatchRange br = batch_range(mv, blockIdx.x - P.start[j]);
  if (mv.aff)
    div_cell_batch<DIM, DEG, T, false, StoreOut<T>, false, true>(mv, P.in[j], nullptr, T(0), T(1), T(1), epi, br,
                                                                 sF, sJ, sDw, sII);
  else
    div_cell_batch<DIM, DEG, T, false, StoreOut<T>, false, false>(mv, P.in[j], nullptr, T(0), T(1), T(1), epi, br,
                                                                  sF, sJ, sDw, sII);
}

}  // namespace dg
