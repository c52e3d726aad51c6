// Host-side launchers of the DG operator kernels, one explicit instantiation
// per (dimension, precision) translation unit.  All launchers enqueue on
// `stream` and return a dg_status; `skip` (device int, may be NULL) turns every
// launched kernel into a no-op when it is non-zero (used by GMRES after
// convergence inside a restart cycle).
#pragma once

#include "dg_internal.h"

namespace dg {

template <typename T>
inline const MeshView<T>& view(const dg_mesh* m);
template <>
inline const MeshView<double>& view<double>(const dg_mesh* m) {
  return m->v64;
}
template <>
inline const MeshView<float>& view<float>(const dg_mesh* m) {
  return m->v32;
}

template <int DIM, typename T>
int launch_explicit(const dg_mesh* m, const T* U, T* R, T* face_scratch, bool full, cudaStream_t s,
                    const int* skip);
template <int DIM, typename T>
int launch_grad(const dg_mesh* m, const T* p, const T* h, T* g, cudaStream_t s, const int* skip);
template <int DIM, typename T>
int launch_div(const dg_mesh* m, const T* f, T* out, cudaStream_t s, const int* skip);
// vec_scratch: the h-scaled gradient between the two launches, dim * n_nodes elements
template <int DIM, typename T>
int launch_helmholtz(const dg_mesh* m, const T* h, const T* p, T* Ap, T alpha, T* vec_scratch, cudaStream_t s,
                     const int* skip);

// One cooperative launch solving A(h) x = b by restarted GMRES(restart) to
// relative residual tol (k_gmres.cuh).  TK = double: FP64 GMRES; TK = float:
// FP32 Arnoldi with FP64 residual and solution (iterative refinement inside
// the kernel, inner_tol = residual reduction per cycle).  x, b: FP64.  hk: h
// in TK (may equal h64 when TK = double).  Q: (restart+1)*n TK, w: n TK, w64:
// n doubles (may alias w when TK = double), partial: npartial doubles, out: 4
// doubles (iterations, rel. residual, converged, ||b||), phase: optional
// per-phase ns accumulators (16, or NULL).
template <int DIM, typename TK>
int launch_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
                 double tol, double inner_tol, int restart, int max_iters, int method, TK* Q, TK* w, double* w64,
                 double* partial, int npartial, double* out, double* lmax, unsigned long long* phase,
                 cudaStream_t s);
// One member of a batched solve (see launch_gmres_batched).
template <typename TK>
struct GmresItem {
  const dg_mesh* m;
  const double* h64;
  const TK* hk;
  const double* b;
  double* x;
  double alpha, tol, inner_tol;
  int max_iters;
  int method;  // dg_krylov
  TK* Q;
  TK* w;
  double* w64;
  double* partial;
  int npartial;
  double* out;
  double* lmax;  // [2] Chebyshev bound of this member (device)
};

// Member packs (k_pack.cuh): one launch of an operator over many meshes of the
// same dimension and degree, the pack passed as a kernel parameter.
constexpr int kPack = 32;  // members per packed launch
template <typename T>
struct OpPack {
  MeshView<T> mv[kPack];
  const T* in[kPack];   // U (explicit), p (gradient), f (divergence)
  const T* aux[kPack];  // h of the gradient (may be NULL)
  T* out[kPack];        // R, g, div
  T* scratch[kPack];    // face buffer (explicit)
  int start[kPack + 1]; // first CTA of each member (filled by the launchers)
  int n;
};
// FP64 operators over a pack (members of one dimension and degree)
int op_explicit_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, bool full, cudaStream_t s);
int op_grad_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, cudaStream_t s);
int op_div_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, cudaStream_t s);

// upper bound of one member's entry in a batched launch's argument table
constexpr size_t kBatchArgBytes = 1024;

// Solve every item's Helmholtz system in ONE cooperative launch (more if the
// items outnumber the co-resident CTAs).  All items share dimension, degree
// and TK, and no two share a mesh (the mesh holds the mat-vec scratch).  The
// CTAs are split among the items in proportion to their node counts; each
// item's solve runs on its own CTAs with its own barrier.  *err (device int)
// is set if a barrier wait ran out.
template <int DIM, typename TK>
int launch_gmres_batched(dg_ctx* ctx, const GmresItem<TK>* items, int n_items, int restart, int* err,
                         cudaStream_t s);
template <typename TK>
inline int op_gmres_batched(dg_ctx* ctx, int dim, const GmresItem<TK>* items, int n_items, int restart, int* err,
                            cudaStream_t s) {
  return dim == 2 ? launch_gmres_batched<2, TK>(ctx, items, n_items, restart, err, s)
                  : launch_gmres_batched<3, TK>(ctx, items, n_items, restart, err, s);
}

template <typename TK>
inline int op_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
                    double tol, double inner_tol, int restart, int max_iters, int method, TK* Q, TK* w, double* w64,
                    double* partial, int npartial, double* out, double* lmax, unsigned long long* phase,
                    cudaStream_t s) {
  return m->dim == 2 ? launch_gmres<2, TK>(m, h64, hk, b, x, alpha, tol, inner_tol, restart, max_iters, method, Q,
                                           w, w64, partial, npartial, out, lmax, phase, s)
                     : launch_gmres<3, TK>(m, h64, hk, b, x, alpha, tol, inner_tol, restart, max_iters, method, Q,
                                           w, w64, partial, npartial, out, lmax, phase, s);
}

// dimension dispatch (with optional event timing per operator category)
template <typename T>
inline int op_explicit(const dg_mesh* m, const T* U, T* R, T* fs, bool full, cudaStream_t s, const int* skip) {
  ProfScope ps(m->ctx, DG_PROF_EXPLICIT, s);
  return m->dim == 2 ? launch_explicit<2, T>(m, U, R, fs, full, s, skip)
                     : launch_explicit<3, T>(m, U, R, fs, full, s, skip);
}
template <typename T>
inline int op_grad(const dg_mesh* m, const T* p, const T* h, T* g, cudaStream_t s, const int* skip) {
  ProfScope ps(m->ctx, DG_PROF_GRAD, s);
  return m->dim == 2 ? launch_grad<2, T>(m, p, h, g, s, skip) : launch_grad<3, T>(m, p, h, g, s, skip);
}
template <typename T>
inline int op_div(const dg_mesh* m, const T* f, T* out, cudaStream_t s, const int* skip) {
  ProfScope ps(m->ctx, DG_PROF_DIV, s);
  return m->dim == 2 ? launch_div<2, T>(m, f, out, s, skip) : launch_div<3, T>(m, f, out, s, skip);
}
template <typename T>
inline int op_helmholtz(const dg_mesh* m, const T* h, const T* p, T* Ap, T alpha, T* vs, cudaStream_t s,
                        const int* skip) {
  ProfScope ps(m->ctx, DG_PROF_HELMHOLTZ, s);
  return m->dim == 2 ? launch_helmholtz<2, T>(m, h, p, Ap, alpha, vs, s, skip)
                     : launch_helmholtz<3, T>(m, h, p, Ap, alpha, vs, s, skip);
}

}  // namespace dg
