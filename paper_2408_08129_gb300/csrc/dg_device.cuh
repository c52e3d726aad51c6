// Device-side helpers shared by the DG kernels: compile-time sizes, node and
// face-node indexing, table layout, and the pointwise Euler physics of Eq. (1)
// written in perturbation form about the hydrostatic background.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"

namespace dg {

__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

template <int DIM, int DEG>
struct Shape {
  static constexpr int N = DEG + 1;             // nodes per axis
  static constexpr int NC = cpow(N, DIM);       // nodes per cell
  static constexpr int NF = cpow(N, DIM - 1);   // nodes per face
  static constexpr int V = DIM + 2;             // conserved variables
  static constexpr int NSUB = 1 << (DIM - 1);   // subfaces of a 2:1 face
  // cells per CTA for the one-thread-per-node cell kernels: fill 256 threads
  static constexpr int CPB = NC >= 256 ? 1 : 256 / NC;
  static constexpr int THREADS = ((CPB * NC + 31) / 32) * 32;
  // table offsets (see Tables1D)
  static constexpr int T_D = 0, T_DW = N * N, T_I = 2 * N * N, T_IT = 4 * N * N, T_W = 6 * N * N,
                       T_IWEND = 6 * N * N + N, T_XI = 6 * N * N + N + 1, T_SIZE = 6 * N * N + 2 * N + 1;
};

// node index inside the cell of face node k on local face lf = 2*axis + side
template <int DIM, int DEG>
__device__ __forceinline__ int face_node(int lf, int k) {
  constexpr int N = DEG + 1;
  const int a = lf >> 1;
  const int fix = (lf & 1) ? DEG : 0;
  if (DIM == 2) {
    return a == 0 ? fix + N * k : k + N * fix;
  } else {
    const int k1 = k % N, k2 = k / N;
    if (a == 0) return fix + N * k1 + N * N * k2;
    if (a == 1) return k1 + N * fix + N * N * k2;
    return k1 + N * k2 + N * N * fix;
  }
}

// Tangential face index of a cell node lying on a face normal to axis a.
template <int DIM, int DEG>
__device__ __forceinline__ int tangential_index(int a, const int* idx) {
  constexpr int N = DEG + 1;
  if (DIM == 2) return a == 0 ? idx[1] : idx[0];
  if (a == 0) return idx[1] + N * idx[2];
  if (a == 1) return idx[0] + N * idx[2];
  return idx[0] + N * idx[1];
}

template <typename T>
__device__ __forceinline__ T gm1() {
  return T(0.4);
}
// 1/sqrt(x) for finite x > 0 in the FP32 range, in FP64: FP32 seed (relative
// error ~1e-7), then two Newton steps y <- y (3 - x y^2) / 2, each of which
// squares the relative error (1e-7 -> 1e-14 -> below FP64 rounding)
__device__ __forceinline__ double rsqrt64(double x) {
  double y = (double)rsqrtf((float)x);
  const double hx = 0.5 * x;
#pragma unroll
  for (int i = 0; i < 2; ++i) y = y * fma(-hx, y * y, 1.5);
  return y;
}

// 2^-l for a refinement level 0 <= l < 127, built from its IEEE-754 fields
template <typename T>
__device__ __forceinline__ T pow2_neg(int l);
template <>
__device__ __forceinline__ float pow2_neg<float>(int l) {
  return __int_as_float((127 - l) << 23);
}
template <>
__device__ __forceinline__ double pow2_neg<double>(int l) {
  return __longlong_as_double((long long)(1023 - l) << 52);
}
// correctly rounded 1/x (the value of 1 / x), through CUDA's reciprocal intrinsics
template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) {
  return __frcp_rn(x);
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return __drcp_rn(x);
}

// Metric terms of node id of a cell whose x (and y) are affine, from the
// heights above the computational coordinates in shared memory (sz: the
// cell's NC values) and the cell's half widths (hb * 2^-level per axis):
//   2D: Ja = [[z_z, 0], [-z_x, ax]],  J = ax z_z
//   3D: Ja = [[ay z_z, 0, 0], [0, ax z_z, 0], [-ay z_x, -ax z_y, ax ay]],  J = ax ay z_z
// with z_a = d z / d xi^a (the vertical one includes the computational half
// width).  These equal the cofactors of the nodal-derivative Jacobian that the
// stored metric terms hold.
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void metric_from_z(const MeshView<T>& mv, int64_t c, const T* sz, const int* id,
                                              const T* sD, T (&Ja)[DIM][DIM], T& invJ) {
  constexpr int N = DEG + 1;
  const T scale = pow2_neg<T>(mv.cell_level[c]);
  T zd[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
    const int node = id[0] + N * id[1] + (DIM == 3 ? N * N * id[2] : 0);
    const T* zc = sz + node - id[a] * stride;
    const T* D = sD + id[a] * N;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < N; ++k) s += D[k] * zc[k * stride];
    zd[a] = s;
  }
  zd[DIM - 1] += mv.hb[DIM - 1] * scale;
  const T ax = mv.hb[0] * scale;
  if (DIM == 2) {
    Ja[0][0] = zd[1];
    Ja[0][1] = T(0);
    Ja[1][0] = -zd[0];
    Ja[1][1] = ax;
    invJ = recip<T>(ax * zd[1]);
  } else {
    const T ay = mv.hb[1] * scale;
    Ja[0][0] = ay * zd[DIM - 1];
    Ja[0][1] = T(0);
    Ja[0][DIM - 1] = T(0);
    Ja[1][0] = T(0);
    Ja[1][1] = ax * zd[DIM - 1];
    Ja[1][DIM - 1] = T(0);
    Ja[DIM - 1][0] = -ay * zd[0];
    Ja[DIM - 1][1] = -ax * zd[1];
    Ja[DIM - 1][DIM - 1] = ax * ay;
    invJ = recip<T>(ax * ay * zd[DIM - 1]);
  }
}

// Hydrostatic background (rho_bar, p_bar) at height z from the mesh's cubic
// Hermite table (heights outside the table clamp to its ends)
template <typename T>
__device__ __forceinline__ void background_at(const MeshView<T>& mv, T z, T& rb, T& pb) {
  T s = (z - mv.bg_z0) * mv.bg_idz;
  s = s < T(0) ? T(0) : (s > T(mv.bg_m) ? T(mv.bg_m) : s);
  int k = (int)s;
  if (k >= mv.bg_m) k = mv.bg_m - 1;
  s -= T(k);
  const T s2 = s * s, s3 = s2 * s;
  const T h00 = T(2) * s3 - T(3) * s2 + T(1), h10 = s3 - T(2) * s2 + s, h01 = T(3) * s2 - T(2) * s3,
          h11 = s3 - s2;
  const T* e = mv.bg_tab + 4 * k;
  pb = h00 * e[0] + h10 * e[1] + h01 * e[4] + h11 * e[5];
  rb = h00 * e[2] + h10 * e[3] + h01 * e[6] + h11 * e[7];
}

// 1/(gamma-1) = 2.5 exactly: a multiplication instead of a division sequence
template <typename T>
__device__ __forceinline__ T inv_gm1() {
  return T(2.5);
}

// Load a state at node `idx` in perturbation form u' = u - u_bg.  FP64 arrays
// hold the full state (the background is subtracted here); FP32 arrays hold
// the perturbation already.
template <int V, typename T, bool PERT>
__device__ __forceinline__ void load_pert(const T* __restrict__ U, int64_t Nn, int64_t idx, const T* rhob,
                                          const T* pb, T* u) {
#pragma unroll
  for (int v = 0; v < V; ++v) u[v] = U[(int64_t)v * Nn + idx];
  if (!PERT) {
    u[0] -= rhob[idx];
    u[V - 1] -= pb[idx] * inv_gm1<T>();
  }
}

// Normal flux F(U).n and the dissipation speed for a state given as a
// perturbation u' about (rho_b, p_b):  rho = rho_b + rho', rho E = p_b/(g-1) + E',
// p' = (g-1)(E' - |m|^2/(2 rho)), p = p_b + p'.
template <int DIM, typename T, bool FULL>
__device__ __forceinline__ void normal_flux(const T* u, T rb, T pb, const T* n, T* F, T& lam) {
  constexpr int V = DIM + 2;
  const T rho = rb + u[0];
  const T irho = T(1) / rho;
  T mn = T(0), m2 = T(0);
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    mn += u[1 + b] * n[b];
    m2 += u[1 + b] * u[1 + b];
  }
  const T un = mn * irho;
  F[0] = mn;
  if (FULL) {
    const T pp = gm1<T>() * (u[V - 1] - T(0.5) * m2 * irho);
#pragma unroll
    for (int b = 0; b < DIM; ++b) F[1 + b] = u[1 + b] * un + pp * n[b];
    // rho E + p = E' + p' + gamma/(gamma-1) p_b
    F[V - 1] = (u[V - 1] + pp + pb * (T(1.4) / gm1<T>())) * un;
    const T p = pb + pp;
    lam = fabs(un) + sqrt(T(1.4) * p * irho);
  } else {
#pragma unroll
    for (int b = 0; b < DIM; ++b) F[1 + b] = u[1 + b] * un;
    F[V - 1] = T(0.5) * m2 * irho * irho * mn;
    lam = fabs(un);
  }
}

}  // namespace dg
