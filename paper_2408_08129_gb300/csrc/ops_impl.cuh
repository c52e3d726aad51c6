// Launcher bodies; included once per (dimension, precision) translation unit.
#pragma once

#include <type_traits>

#include "k_explicit.cuh"
#include "k_gmres.cuh"
#include "k_implicit.cuh"
#include "ops.h"

namespace dg {

namespace {

inline int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return DG_OK;
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

template <int DIM, int DEG, typename T>
int run_explicit(const dg_mesh* m, const T* U, T* R, T* Fh, bool full, cudaStream_t s, const int* skip) {
  using S = Shape<DIM, DEG>;
  constexpr bool PERT = std::is_same<T, float>::value;
  const MeshView<T>& mv = view<T>(m);
  const int64_t tf = (int64_t)mv.nf * S::NF;
  const unsigned cb = blocks_for(mv.n_cells, S::CPB);
  count_launches(m->ctx, tf ? 2 : 1);
  if (full) {
    if (tf) explicit_face_kernel<DIM, DEG, T, true, PERT><<<blocks_for(tf, 256), 256, 0, s>>>(mv, U, Fh, skip);
    explicit_cell_kernel<DIM, DEG, T, true, PERT><<<cb, S::THREADS, 0, s>>>(mv, U, Fh, R, skip);
  } else {
    if (tf) explicit_face_kernel<DIM, DEG, T, false, PERT><<<blocks_for(tf, 256), 256, 0, s>>>(mv, U, Fh, skip);
    explicit_cell_kernel<DIM, DEG, T, false, PERT><<<cb, S::THREADS, 0, s>>>(mv, U, Fh, R, skip);
  }
  return check_launch("explicit operator launch");
}

template <int DIM, int DEG, typename T>
int run_grad(const dg_mesh* m, const T* p, const T* h, T* g, T* Gh, cudaStream_t s, const int* skip) {
  using S = Shape<DIM, DEG>;
  const MeshView<T>& mv = view<T>(m);
  const int64_t tf = (int64_t)(mv.nconf + mv.nsub) * S::NF;
  count_launches(m->ctx, tf ? 2 : 1);
  if (tf) grad_face_kernel<DIM, DEG, T><<<blocks_for(tf, 256), 256, 0, s>>>(mv, p, Gh, skip);
  grad_cell_kernel<DIM, DEG, T><<<blocks_for(mv.n_cells, S::CPB), S::THREADS, 0, s>>>(mv, p, h, Gh, g, skip);
  return check_launch("gradient launch");
}

template <int DIM, int DEG, typename T, bool HELM>
int run_div(const dg_mesh* m, const T* f, const T* p, T alpha, T* out, T* Dh, cudaStream_t s, const int* skip) {
  using S = Shape<DIM, DEG>;
  const MeshView<T>& mv = view<T>(m);
  const int64_t tf = (int64_t)(mv.nconf + mv.nsub) * S::NF;
  count_launches(m->ctx, tf ? 2 : 1);
  if (tf) div_face_kernel<DIM, DEG, T><<<blocks_for(tf, 256), 256, 0, s>>>(mv, f, Dh, skip);
  div_cell_kernel<DIM, DEG, T, HELM><<<blocks_for(mv.n_cells, S::CPB), S::THREADS, 0, s>>>(mv, f, Dh, p, alpha,
                                                                                           out, skip);
  return check_launch("divergence launch");
}

template <int DIM, int DEG, typename TK>
int run_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
              double tol, double inner_tol, int restart, int max_iters, TK* Q, TK* w, double* w64, double* partial,
              int npartial, double* out, unsigned long long* phase, cudaStream_t s) {
  GmresPArgs<TK> a;
  a.mv64 = m->v64;
  a.mvk = view<TK>(m);
  a.h64 = h64;
  a.hk = hk;
  a.b = b;
  a.x = x;
  a.Q = Q;
  a.w = w;
  a.w64 = w64;
  a.Gh = m->d_face_scratch64;
  a.gv = m->d_vec_scratch64;
  a.partial = partial;
  a.out = out;
  a.phase = phase;
  a.alpha = alpha;
  a.tol = tol;
  a.inner_tol = inner_tol;
  a.m = restart;
  a.max_iters = max_iters;
  a.n = m->Nn;
  auto kern = gmres_persistent_kernel<DIM, DEG, TK>;
  const size_t smem = gmres_smem_bytes<DIM, DEG, TK>(restart);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "gmres smem attribute");
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return cuda_fail(e, "gmres occupancy");
  if (per_sm < 1) return fail(DG_ECUDA, "persistent GMRES kernel does not fit on an SM");
  int G = m->ctx->sm_count * (per_sm < 2 ? per_sm : 2);
  if (G > npartial) G = npartial;
  if (G > 512) G = 512;  // staged partial sums in shared memory
  if (G < 1) return fail(DG_EINVAL, "GMRES partial buffer too small");
  count_launches(m->ctx, 1);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(256), args, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "persistent GMRES launch");
  return DG_OK;
}

}  // namespace

#define DG_DEGREE_SWITCH(deg, ...)                         \
  switch (deg) {                                           \
    case 1: { constexpr int DEG = 1; __VA_ARGS__; }        \
    case 2: { constexpr int DEG = 2; __VA_ARGS__; }        \
    case 3: { constexpr int DEG = 3; __VA_ARGS__; }        \
    case 4: { constexpr int DEG = 4; __VA_ARGS__; }        \
    case 5: { constexpr int DEG = 5; __VA_ARGS__; }        \
    default: return fail(DG_EINVAL, "unsupported degree"); \
  }

template <int DIM, typename T>
int launch_explicit(const dg_mesh* m, const T* U, T* R, T* fs, bool full, cudaStream_t s, const int* skip) {
  DG_DEGREE_SWITCH(m->degree, return (run_explicit<DIM, DEG, T>(m, U, R, fs, full, s, skip)))
}

template <int DIM, typename T>
int launch_grad(const dg_mesh* m, const T* p, const T* h, T* g, T* fs, cudaStream_t s, const int* skip) {
  DG_DEGREE_SWITCH(m->degree, return (run_grad<DIM, DEG, T>(m, p, h, g, fs, s, skip)))
}

template <int DIM, typename T>
int launch_div(const dg_mesh* m, const T* f, T* out, T* fs, cudaStream_t s, const int* skip) {
  DG_DEGREE_SWITCH(m->degree, return (run_div<DIM, DEG, T, false>(m, f, nullptr, T(0), out, fs, s, skip)))
}

template <int DIM, typename T>
int launch_helmholtz(const dg_mesh* m, const T* h, const T* p, T* Ap, T alpha, T* fs, T* vs, cudaStream_t s,
                     const int* skip) {
  DG_DEGREE_SWITCH(m->degree, {
    int st = run_grad<DIM, DEG, T>(m, p, h, vs, fs, s, skip);
    if (st != DG_OK) return st;
    return (run_div<DIM, DEG, T, true>(m, vs, p, alpha, Ap, fs, s, skip));
  })
}

template <int DIM, typename TK>
int launch_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
                 double tol, double inner_tol, int restart, int max_iters, TK* Q, TK* w, double* w64,
                 double* partial, int npartial, double* out, unsigned long long* phase, cudaStream_t s) {
  DG_DEGREE_SWITCH(m->degree, return (run_gmres<DIM, DEG, TK>(m, h64, hk, b, x, alpha, tol, inner_tol, restart,
                                                               max_iters, Q, w, w64, partial, npartial, out, phase,
                                                               s)))
}

#define DG_INSTANTIATE_OPS(DIM, T)                                                                              \
  template int launch_explicit<DIM, T>(const dg_mesh*, const T*, T*, T*, bool, cudaStream_t, const int*);      \
  template int launch_grad<DIM, T>(const dg_mesh*, const T*, const T*, T*, T*, cudaStream_t, const int*);      \
  template int launch_div<DIM, T>(const dg_mesh*, const T*, T*, T*, cudaStream_t, const int*);                 \
  template int launch_helmholtz<DIM, T>(const dg_mesh*, const T*, const T*, T*, T, T*, T*, cudaStream_t,       \
                                        const int*);                                                            \
  template int launch_gmres<DIM, T>(const dg_mesh*, const double*, const T*, const double*, double*, double,     \
                                    double, double, int, int, T*, T*, double*, double*, int, double*,            \
                                    unsigned long long*, cudaStream_t);

}  // namespace dg
