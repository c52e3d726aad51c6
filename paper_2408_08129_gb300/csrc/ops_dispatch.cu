// Run-time choice of the degree: the operator launchers of ops.h call the
// per-degree launcher bodies (ops_impl.cuh), which are compiled in
// translation units of their own.
#include "ops_run.h"

namespace dg {

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
int launch_grad(const dg_mesh* m, const T* p, const T* h, T* g, cudaStream_t s, const int* skip) {
  DG_DEGREE_SWITCH(m->degree, return (run_grad<DIM, DEG, T>(m, p, h, g, s, skip)))
}

template <int DIM, typename T>
int launch_div(const dg_mesh* m, const T* f, T* out, cudaStream_t s, const int* skip) {
  DG_DEGREE_SWITCH(m->degree, return (run_div<DIM, DEG, T, false>(m, f, nullptr, T(0), out, s, skip)))
}

template <int DIM, typename T>
int launch_helmholtz(const dg_mesh* m, const T* h, const T* p, T* Ap, T alpha, T* vs, cudaStream_t s,
                     const int* skip) {
  DG_DEGREE_SWITCH(m->degree, {
    int st = run_grad<DIM, DEG, T>(m, p, h, vs, s, skip);
    if (st != DG_OK) return st;
    return (run_div<DIM, DEG, T, true>(m, vs, p, alpha, Ap, s, skip));
  })
}

template <int DIM, typename TK>
int launch_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
                 double tol, double inner_tol, int restart, int max_iters, int method, TK* Q, TK* w, double* w64,
                 double* partial, int npartial, double* out, double* lmax, unsigned long long* phase,
                 cudaStream_t s) {
  DG_DEGREE_SWITCH(m->degree, return (run_gmres<DIM, DEG, TK>(m, h64, hk, b, x, alpha, tol, inner_tol, restart,
                                                               max_iters, method, Q, w, w64, partial, npartial, out,
                                                               lmax, phase, s)))
}

template <int DIM, typename TK>
int launch_gmres_batched(dg_ctx* ctx, const GmresItem<TK>* items, int n_items, int restart, int* err,
                         cudaStream_t s) {
  if (n_items <= 0) return DG_OK;
  DG_DEGREE_SWITCH(items[0].m->degree, return (run_gmres_batched<DIM, DEG, TK>(ctx, items, n_items, restart, err, s)))
}

#define DG_INSTANTIATE_OPS(DIM, T)                                                                              \
  template int launch_explicit<DIM, T>(const dg_mesh*, const T*, T*, T*, bool, cudaStream_t, const int*);      \
  template int launch_grad<DIM, T>(const dg_mesh*, const T*, const T*, T*, cudaStream_t, const int*);          \
  template int launch_div<DIM, T>(const dg_mesh*, const T*, T*, cudaStream_t, const int*);                     \
  template int launch_helmholtz<DIM, T>(const dg_mesh*, const T*, const T*, T*, T, T*, cudaStream_t,           \
                                        const int*);                                                            \
  template int launch_gmres<DIM, T>(const dg_mesh*, const double*, const T*, const double*, double*, double,     \
                                    double, double, int, int, int, T*, T*, double*, double*, int, double*,       \
                                    double*, unsigned long long*, cudaStream_t);                                \
  template int launch_gmres_batched<DIM, T>(dg_ctx*, const GmresItem<T>*, int, int, int*, cudaStream_t);

int op_explicit_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, bool full, cudaStream_t s) {
  ProfScope ps(ctx, DG_PROF_EXPLICIT, s);
  if (dim == 2) {
    DG_DEGREE_SWITCH(degree, return (run_explicit_pack<2, DEG, double>(ctx, P, full, s)))
  }
  DG_DEGREE_SWITCH(degree, return (run_explicit_pack<3, DEG, double>(ctx, P, full, s)))
}

int op_grad_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, cudaStream_t s) {
  ProfScope ps(ctx, DG_PROF_GRAD, s);
  if (dim == 2) {
    DG_DEGREE_SWITCH(degree, return (run_grad_pack<2, DEG, double>(ctx, P, s)))
  }
  DG_DEGREE_SWITCH(degree, return (run_grad_pack<3, DEG, double>(ctx, P, s)))
}

int op_div_pack(dg_ctx* ctx, int dim, int degree, OpPack<double>& P, cudaStream_t s) {
  ProfScope ps(ctx, DG_PROF_DIV, s);
  if (dim == 2) {
    DG_DEGREE_SWITCH(degree, return (run_div_pack<2, DEG, double>(ctx, P, s)))
  }
  DG_DEGREE_SWITCH(degree, return (run_div_pack<3, DEG, double>(ctx, P, s)))
}

DG_INSTANTIATE_OPS(2, double)
DG_INSTANTIATE_OPS(2, float)
DG_INSTANTIATE_OPS(3, double)
DG_INSTANTIATE_OPS(3, float)

}  // namespace dg
