// Declarations of the per-degree launcher bodies defined in ops_impl.cuh
// (compiled and instantiated elsewhere), for the run-time degree dispatch.
#pragma once

#include "ops.h"

namespace dg {

template <int DIM, int DEG, typename T>
int run_explicit(const dg_mesh* m, const T* U, T* R, T* Fh, bool full, cudaStream_t s, const int* skip);
template <int DIM, int DEG, typename T>
int run_grad(const dg_mesh* m, const T* p, const T* h, T* g, cudaStream_t s, const int* skip);
template <int DIM, int DEG, typename T, bool HELM>
int run_div(const dg_mesh* m, const T* f, const T* p, T alpha, T* out, cudaStream_t s, const int* skip);
template <int DIM, int DEG, typename TK>
int run_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
              double tol, double inner_tol, int restart, int max_iters, int method, TK* Q, TK* w, double* w64,
              double* partial, int npartial, double* out, double* lmax, unsigned long long* phase,
              cudaStream_t s);
template <int DIM, int DEG, typename TK>
int run_gmres_batched(dg_ctx* ctx, const GmresItem<TK>* items, int n_items, int restart, int* err,
                      cudaStream_t s);

template <int DIM, int DEG, typename T>
int run_explicit_pack(dg_ctx* ctx, OpPack<T>& P, bool full, cudaStream_t s);
template <int DIM, int DEG, typename T>
int run_grad_pack(dg_ctx* ctx, OpPack<T>& P, cudaStream_t s);
template <int DIM, int DEG, typename T>
int run_div_pack(dg_ctx* ctx, OpPack<T>& P, cudaStream_t s);

}  // namespace dg
