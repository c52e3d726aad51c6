// IMEX-RK2 time step on the device (Sec. 2 scheme; Sec. 3.2 pressure loop).
//
// Readings of the scheme (the paper cites the method, not its details):
//  * ARK2(2,3,2) tableau (Giraldo, Kelly, Constantinescu 2013): gamma = 1-1/sqrt2,
//    delta = 1/(2 sqrt2), a32 = (3+2 sqrt2)/6; implicit tableau stiffly accurate,
//    so U^{n+1} = U^(3) + dt sum_j (b_j - A[2][j]) E_j.
//  * Explicit terms E: continuity, momentum advection, kinetic-energy flux and
//    the energy gravity work (DG_TERMS_IMEX_EXPLICIT).  Implicit terms I:
//    momentum -grad p' - rho' g k, energy -div(h m), h = gamma p/((gamma-1) rho).
//  * Implicit stage: rho from the explicit continuity update; momentum
//    mhat = known part - dt a_ii rho' g k; Picard loop (fixed count) with h and
//    the kinetic energy lagged:  p'/(g-1) - (dt a_ii)^2 div(h grad p') =
//    Ehat - p_bar/(g-1) - rho k - dt a_ii div(h mhat), solved by GMRES from the
//    previous iterate; m = mhat - dt a_ii grad p'; rho E = p/(g-1) + rho k.
#include <cmath>

#include "krylov.cuh"
#include "ops.h"

struct dg_state {
  dg_ctx* ctx = nullptr;
  const dg_mesh* mesh = nullptr;
  int64_t Nn = 0;
  int V = 0, dim = 0;
  void* block = nullptr;
  double* U = nullptr;  // [V][Nn]
  double* E[3] = {nullptr, nullptr, nullptr};
  double* I[2] = {nullptr, nullptr};
  double* Ui = nullptr;
  double* rho = nullptr;
  double* mhat = nullptr;  // [dim][Nn]
  double* Ehat = nullptr;
  double* p = nullptr;
  double* p_prev = nullptr;
  double* h = nullptr;
  double* mk = nullptr;   // [dim][Nn]
  double* rhs = nullptr;
  double* tmpv = nullptr; // [dim][Nn]
  double* tmps = nullptr;
  double* g = nullptr;    // [dim][Nn]
  double* r64 = nullptr;  // FP64 outer residual
  double* solve_out = nullptr;  // [64][4] per-solve results of one step
  float* f32 = nullptr;   // FP32 Krylov: h, rhs, delta [3 Nn]
  int* flag = nullptr;    // non-finite flag
  dg::Gmres<double> gm64;
  dg::Gmres<float> gm32;
  bool has32 = false;
  int restart = 30;
  cudaStream_t stream = nullptr;
};

namespace dg {

namespace {

constexpr double kSq2 = 1.41421356237309504880;
const double kG = 1.0 - 1.0 / kSq2;
const double kDl = 1.0 / (2.0 * kSq2);
const double kA32 = (3.0 + 2.0 * kSq2) / 6.0;
const double AEX[3][3] = {{0, 0, 0}, {2 * kG, 0, 0}, {1 - kA32, kA32, 0}};
const double AIM[3][3] = {{0, 0, 0}, {kG, kG, 0}, {kDl, kDl, kG}};
const double BW[3] = {kDl, kDl, kG};

inline unsigned gridn(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

#define GRID_LOOP(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// p' = (g-1)(rho E - |m|^2/(2 rho)) - p_bar and h = gamma p / ((gamma-1) rho)
__global__ void pressure_kernel(const double* __restrict__ U, const double* __restrict__ pb, int64_t Nn, int dim,
                                double* __restrict__ pp, double* __restrict__ h) {
  const int V = dim + 2;
  GRID_LOOP(i, Nn) {
    const double rho = U[i];
    double m2 = 0.0;
    for (int b = 0; b < dim; ++b) m2 += U[(1 + b) * Nn + i] * U[(1 + b) * Nn + i];
    const double p = (kGamma - 1.0) * (U[(V - 1) * Nn + i] - 0.5 * m2 / rho);
    pp[i] = p - pb[i];
    h[i] = kGamma * p / ((kGamma - 1.0) * rho);
  }
}

// out[b] = h * m[b]
__global__ void hm_kernel(const double* __restrict__ h, const double* __restrict__ m, int64_t Nn, int dim,
                          double* __restrict__ out) {
  GRID_LOOP(i, Nn) {
    for (int b = 0; b < dim; ++b) out[b * Nn + i] = h[i] * m[b * Nn + i];
  }
}

// implicit tendencies: I = (0, -g - rho' grav k, -divhm)
__global__ void implicit_terms_kernel(const double* __restrict__ rho, const double* __restrict__ rhob,
                                      const double* __restrict__ g, const double* __restrict__ divhm, double grav,
                                      int64_t Nn, int dim, double* __restrict__ I) {
  const int V = dim + 2;
  GRID_LOOP(i, Nn) {
    I[i] = 0.0;
    for (int b = 0; b < dim; ++b) I[(1 + b) * Nn + i] = -g[b * Nn + i];
    I[dim * Nn + i] -= (rho[i] - rhob[i]) * grav;
    I[(V - 1) * Nn + i] = -divhm[i];
  }
}

struct StageCoef {
  double ae[2], ai[2];
  int nprev;
};

// rho, mhat, Ehat of an implicit stage from U^n and the earlier tendencies
__global__ void stage_combine_kernel(const double* __restrict__ U, const double* __restrict__ E0,
                                     const double* __restrict__ E1, const double* __restrict__ I0,
                                     const double* __restrict__ I1, StageCoef c, double dt, double dt_aii,
                                     const double* __restrict__ rhob, double grav, int64_t Nn, int dim,
                                     double* __restrict__ rho, double* __restrict__ mhat, double* __restrict__ Ehat) {
  const int V = dim + 2;
  GRID_LOOP(i, Nn) {
    double r = c.ae[0] * E0[i];
    if (c.nprev > 1) r += c.ae[1] * E1[i];
    const double rh = U[i] + dt * r;
    rho[i] = rh;
    for (int b = 0; b < dim; ++b) {
      const int64_t o = (int64_t)(1 + b) * Nn + i;
      double s = c.ae[0] * E0[o] + c.ai[0] * I0[o];
      if (c.nprev > 1) s += c.ae[1] * E1[o] + c.ai[1] * I1[o];
      double mh = U[o] + dt * s;
      if (b == dim - 1) mh -= dt_aii * (rh - rhob[i]) * grav;
      mhat[b * Nn + i] = mh;
    }
    const int64_t o = (int64_t)(V - 1) * Nn + i;
    double s = c.ae[0] * E0[o] + c.ai[0] * I0[o];
    if (c.nprev > 1) s += c.ae[1] * E1[o] + c.ai[1] * I1[o];
    Ehat[i] = U[o] + dt * s;
  }
}

// Picard preparation: h = gamma (p_bar + p')/((g-1) rho);  rhs0 = Ehat - p_bar/(g-1) - |mk|^2/(2 rho);
// hm = h * mhat
__global__ void picard_prep_kernel(const double* __restrict__ pp, const double* __restrict__ pb,
                                   const double* __restrict__ rho, const double* __restrict__ mk,
                                   const double* __restrict__ mhat, const double* __restrict__ Ehat, int64_t Nn,
                                   int dim, double* __restrict__ h, double* __restrict__ rhs0,
                                   double* __restrict__ hm) {
  GRID_LOOP(i, Nn) {
    const double r = rho[i];
    const double hh = kGamma * (pb[i] + pp[i]) / ((kGamma - 1.0) * r);
    h[i] = hh;
    double m2 = 0.0;
    for (int b = 0; b < dim; ++b) {
      m2 += mk[b * Nn + i] * mk[b * Nn + i];
      hm[b * Nn + i] = hh * mhat[b * Nn + i];
    }
    rhs0[i] = Ehat[i] - pb[i] / (kGamma - 1.0) - 0.5 * m2 / r;
  }
}

// ax = b - ax (in place)
__global__ void sub_from_kernel(const double* b, double* ax, int64_t n) {
  GRID_LOOP(i, n) { ax[i] = b[i] - ax[i]; }
}

// y += c * x
__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, double c, int64_t n) {
  GRID_LOOP(i, n) { y[i] += c * x[i]; }
}

// mk = mhat - c * g
__global__ void momentum_kernel(const double* __restrict__ mhat, const double* __restrict__ g, double c, int64_t n,
                                double* __restrict__ mk) {
  GRID_LOOP(i, n) { mk[i] = mhat[i] - c * g[i]; }
}

// stage state: (rho, mk, (p_bar + p')/(g-1) + |mk|^2/(2 rho))
__global__ void stage_state_kernel(const double* __restrict__ rho, const double* __restrict__ mk,
                                   const double* __restrict__ pp, const double* __restrict__ pb, int64_t Nn, int dim,
                                   double* __restrict__ Ui) {
  const int V = dim + 2;
  GRID_LOOP(i, Nn) {
    const double r = rho[i];
    double m2 = 0.0;
    Ui[i] = r;
    for (int b = 0; b < dim; ++b) {
      const double mb = mk[b * Nn + i];
      Ui[(1 + b) * Nn + i] = mb;
      m2 += mb * mb;
    }
    Ui[(V - 1) * Nn + i] = (pb[i] + pp[i]) / (kGamma - 1.0) + 0.5 * m2 / r;
  }
}

// U = Ui + dt sum_j c_j E_j ; flag non-finite values
__global__ void final_kernel(const double* __restrict__ Ui, const double* __restrict__ E0,
                             const double* __restrict__ E1, const double* __restrict__ E2, double c0, double c1,
                             double c2, int64_t n, double* __restrict__ U, int* __restrict__ flag) {
  GRID_LOOP(i, n) {
    const double v = Ui[i] + c0 * E0[i] + c1 * E1[i] + c2 * E2[i];
    U[i] = v;
    if (!isfinite(v)) *flag = 1;
  }
}

__global__ void to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  GRID_LOOP(i, n) { y[i] = (float)x[i]; }
}
__global__ void add_f32_kernel(double* __restrict__ x, const float* __restrict__ d, int64_t n) {
  GRID_LOOP(i, n) { x[i] += (double)d[i]; }
}
__global__ void zero_f32_kernel(float* __restrict__ x, int64_t n) {
  GRID_LOOP(i, n) { x[i] = 0.0f; }
}

int check(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : cuda_fail(e, what);
}

// Helmholtz solve A(h) p = rhs (p holds the initial guess), FP64 or FP32-refined.
// The fused FP64 path leaves its (iterations, residual, converged, ||b||) in
// out[0..3] on the device and does not wait; the caller reads them later.
int helmholtz_solve(dg_state* S, const dg_solver_opts* o, double alpha, dg_step_stats* st, double* out,
                    cudaStream_t s) {
  const dg_mesh* m = S->mesh;
  const int64_t Nn = S->Nn;
  const int restart = std::min(o->restart, S->restart);
  auto A64 = [&](const double* x, double* y, const int* skip) {
    return op_helmholtz<double>(m, S->h, x, y, alpha, m->d_face_scratch64, m->d_vec_scratch64, s, skip);
  };
  GmresResult res;
  int rc;
  unsigned long long* phase = S->ctx->prof ? S->ctx->d_phase : nullptr;
  const int npart = (restart + 1) * kDotBlocks;
  if (o->fused) {
    ProfScope ps(S->ctx, DG_PROF_GMRES, s);
    if (o->precision == DG_FP64)
      return op_gmres<double>(m, S->h, S->h, S->rhs, S->p, alpha, o->tol, 0.0, restart, o->max_iters, S->gm64.Q,
                              S->gm64.w, S->gm64.w, S->gm64.d.partial, npart, out, phase, s);
    float* h32 = S->f32;
    to_f32_kernel<<<gridn(Nn), 256, 0, s>>>(S->h, h32, Nn);
    count_launches(S->ctx, 1);
    return op_gmres<float>(m, S->h, h32, S->rhs, S->p, alpha, o->tol, o->inner_tol, restart, o->max_iters,
                           S->gm32.Q, S->gm32.w, S->r64, S->gm32.d.partial, npart, out, phase, s);
  }
  if (o->precision == DG_FP64) {
    rc = S->gm64.solve(S->ctx, A64, S->rhs, S->p, o->tol, o->max_iters, s, &res);
    if (rc != DG_OK) return rc;
    const double host[4] = {(double)res.iters, res.rel, res.converged ? 1.0 : 0.0, 0.0};
    DG_CUDA(cudaMemcpyAsync(out, host, sizeof(host), cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaStreamSynchronize(s));
    return DG_OK;
  }
  // FP32 inner GMRES inside FP64 iterative refinement: p += A32^-1 (rhs - A64 p)
  float* h32 = S->f32;
  float* r32 = S->f32 + Nn;
  float* d32 = S->f32 + 2 * Nn;
  to_f32_kernel<<<gridn(Nn), 256, 0, s>>>(S->h, h32, Nn);
  count_launches(S->ctx, 1);
  auto A32 = [&](const float* x, float* y, const int* skip) {
    return op_helmholtz<float>(m, h32, x, y, (float)alpha, (float*)m->d_face_scratch64,
                               (float*)m->d_vec_scratch64, s, skip);
  };
  double bn2 = 0.0, rn2 = 0.0;
  double* scal = S->gm64.d.scal;  // reuse: [6] = ||b||^2, [7] = ||r||^2
  if ((rc = dot_into<double, double>(S->rhs, S->rhs, Nn, S->gm64.d.partial, scal + 6, s, nullptr)) != DG_OK)
    return rc;
  count_launches(S->ctx, 2);
  DG_CUDA(cudaMemcpyAsync(&bn2, scal + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  const double bn = std::sqrt(bn2);
  double rel = 0.0;
  int inner = 0, refine = 0;
  for (int k = 0; k <= o->max_refine; ++k) {
    if ((rc = A64(S->p, S->r64, nullptr)) != DG_OK) return rc;
    sub_from_kernel<<<gridn(Nn), 256, 0, s>>>(S->rhs, S->r64, Nn);
    count_launches(S->ctx, 1);
    if ((rc = dot_into<double, double>(S->r64, S->r64, Nn, S->gm64.d.partial, scal + 7, s, nullptr)) != DG_OK)
      return rc;
    count_launches(S->ctx, 2);
    DG_CUDA(cudaMemcpyAsync(&rn2, scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    rel = bn > 0 ? std::sqrt(rn2) / bn : 0.0;
    if (rel <= o->tol || k == o->max_refine) break;
    to_f32_kernel<<<gridn(Nn), 256, 0, s>>>(S->r64, r32, Nn);
    zero_f32_kernel<<<gridn(Nn), 256, 0, s>>>(d32, Nn);
    count_launches(S->ctx, 2);
    if ((rc = S->gm32.solve(S->ctx, A32, r32, d32, o->inner_tol, o->max_iters, s, &res)) != DG_OK) return rc;
    inner += res.iters;
    add_f32_kernel<<<gridn(Nn), 256, 0, s>>>(S->p, d32, Nn);
    count_launches(S->ctx, 1);
    ++refine;
  }
  const double host[4] = {(double)inner, rel, rel <= o->tol ? 1.0 : 0.0, bn};
  DG_CUDA(cudaMemcpyAsync(out, host, sizeof(host), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));
  st->refine_steps += refine;
  return DG_OK;
}

// The explicit tendencies, gradients and divergences of the step enter the
// new state directly, with no correction step after them, so they stay in
// FP64 in both precision modes; the FP32 form puts the Krylov mat-vecs (the
// bulk of the work) in FP32 and recovers FP64 accuracy by the FP64 residual.
int step_explicit(dg_state* S, const double* U, double* E, cudaStream_t s) {
  return op_explicit<double>(S->mesh, U, E, S->mesh->d_face_scratch64, false, s, nullptr);
}
int step_grad(dg_state* S, const double* p, double* g, cudaStream_t s) {
  return op_grad<double>(S->mesh, p, nullptr, g, S->mesh->d_face_scratch64, s, nullptr);
}
int step_div(dg_state* S, const double* f, double* out, cudaStream_t s) {
  return op_div<double>(S->mesh, f, out, S->mesh->d_face_scratch64, s, nullptr);
}

}  // namespace

}  // namespace dg

using namespace dg;

extern "C" void dg_solver_opts_default(dg_solver_opts* o) {
  if (!o) return;
  o->picard = 3;
  o->restart = 30;
  o->max_iters = 2000;
  o->tol = 1e-12;
  o->precision = DG_FP64;
  o->inner_tol = 1e-4;
  o->max_refine = 20;
  o->fused = 1;
}

extern "C" int dg_state_create(dg_ctx* ctx, const dg_mesh* m, const dg_solver_opts* opts, dg_state** out) {
  if (!ctx || !m || !out) return fail(DG_EINVAL, "null argument");
  dg_solver_opts o;
  dg_solver_opts_default(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > kMaxRestart) return fail(DG_EINVAL, "restart must be in 1..64");
  dg_state* S = new (std::nothrow) dg_state();
  if (!S) return fail(DG_ENOMEM, "host allocation failed");
  S->ctx = ctx;
  S->mesh = m;
  S->Nn = m->Nn;
  S->V = m->V;
  S->dim = m->dim;
  S->restart = o.restart;
  const int64_t Nn = S->Nn;
  const int V = S->V, dim = S->dim;
  // every buffer is rounded up to 32 doubles (256 bytes); 20 buffers in all
  auto rup = [](size_t n) { return (n + 31) & ~(size_t)31; };
  const size_t nd = 7 * rup((size_t)V * Nn) + 4 * rup((size_t)dim * Nn) + 8 * rup((size_t)Nn) + rup(8) + rup(256);
  cudaError_t e = cudaSetDevice(ctx->device);
  const size_t nf32 = (size_t)Nn * 3 + 256;
  if (e == cudaSuccess) e = cudaMalloc(&S->block, nd * sizeof(double) + nf32 * sizeof(float) + 1024);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "state allocation");
  }
  double* p = (double*)S->block;
  auto take = [&](size_t n) {
    double* r = p;
    p += (n + 31) & ~(size_t)31;
    return r;
  };
  S->U = take((size_t)V * Nn);
  for (int j = 0; j < 3; ++j) S->E[j] = take((size_t)V * Nn);
  for (int j = 0; j < 2; ++j) S->I[j] = take((size_t)V * Nn);
  S->Ui = take((size_t)V * Nn);
  S->mhat = take((size_t)dim * Nn);
  S->mk = take((size_t)dim * Nn);
  S->tmpv = take((size_t)dim * Nn);
  S->g = take((size_t)dim * Nn);
  S->rho = take(Nn);
  S->Ehat = take(Nn);
  S->p = take(Nn);
  S->p_prev = take(Nn);
  S->h = take(Nn);
  S->rhs = take(Nn);
  S->tmps = take(Nn);
  S->r64 = take(Nn);
  S->flag = (int*)take(8);
  S->solve_out = take(256);
  S->f32 = (float*)p;
  int rc = S->gm64.init(Nn, o.restart);
  if (rc == DG_OK) rc = S->gm32.init(Nn, o.restart);
  if (rc != DG_OK) {
    dg_state_destroy(S);
    return rc;
  }
  S->has32 = true;
  e = cudaMemset(S->block, 0, nd * sizeof(double));
  if (e != cudaSuccess) {
    dg_state_destroy(S);
    return cuda_fail(e, "state memset");
  }
  *out = S;
  return DG_OK;
}

extern "C" int dg_state_destroy(dg_state* S) {
  if (!S) return DG_OK;
  S->gm64.release();
  S->gm32.release();
  if (S->block) cudaFree(S->block);
  delete S;
  return DG_OK;
}

extern "C" double* dg_state_data(dg_state* S) { return S ? S->U : nullptr; }

extern "C" int dg_state_upload(dg_state* S, const double* host_U) {
  if (!S || !host_U) return fail(DG_EINVAL, "null argument");
  DG_CUDA(cudaMemcpyAsync(S->U, host_U, (size_t)S->V * S->Nn * sizeof(double), cudaMemcpyHostToDevice, S->stream));
  DG_CUDA(cudaStreamSynchronize(S->stream));
  return DG_OK;
}

extern "C" int dg_state_download(dg_state* S, double* host_U) {
  if (!S || !host_U) return fail(DG_EINVAL, "null argument");
  DG_CUDA(cudaMemcpyAsync(host_U, S->U, (size_t)S->V * S->Nn * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  DG_CUDA(cudaStreamSynchronize(S->stream));
  return DG_OK;
}

extern "C" int imex_rk2_step(dg_ctx* ctx, const dg_mesh* m, dg_state* S, double dt, const dg_solver_opts* opts,
                             dg_step_stats* stats, void* stream) {
  if (!ctx || !m || !S || S->mesh != m) return fail(DG_EINVAL, "bad arguments");
  if (!(dt > 0.0)) return fail(DG_EINVAL, "dt must be positive");
  dg_solver_opts o;
  dg_solver_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != DG_FP64 && o.precision != DG_FP32) return fail(DG_EINVAL, "bad precision");
  if (o.picard < 1) return fail(DG_EINVAL, "picard must be >= 1");
  dg_step_stats st{};
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Nn = S->Nn;
  const int V = S->V, dim = S->dim;
  const unsigned gb = gridn(Nn);
  const double grav = m->desc.gravity;
  const MeshView<double>& mv = m->v64;

  int rc = DG_OK;
  int status = DG_OK;
  ProfScope step_scope(ctx, DG_PROF_STEP, s);
  int nsolve = 0;
#define RUN(x)                     \
  do {                             \
    if ((rc = (x)) != DG_OK) return rc; \
  } while (0)
  // stage 1: U^(1) = U^n
  pressure_kernel<<<gb, 256, 0, s>>>(S->U, mv.pb, Nn, dim, S->p_prev, S->h);
  count_launches(S->ctx, 1);
  RUN(step_explicit(S, S->U, S->E[0], s));
  RUN(step_grad(S, S->p_prev, S->g, s));
  hm_kernel<<<gb, 256, 0, s>>>(S->h, S->U + Nn, Nn, dim, S->tmpv);
  count_launches(S->ctx, 1);
  RUN(step_div(S, S->tmpv, S->tmps, s));
  implicit_terms_kernel<<<gb, 256, 0, s>>>(S->U, mv.rhob, S->g, S->tmps, grav, Nn, dim, S->I[0]);
  count_launches(S->ctx, 1);
  RUN(check("stage 1"));
  for (int i = 1; i <= 2; ++i) {
    const double aii = AIM[i][i];
    const double dta = dt * aii;
    StageCoef c{};
    c.nprev = i;
    for (int j = 0; j < i; ++j) {
      c.ae[j] = AEX[i][j];
      c.ai[j] = AIM[i][j];
    }
    stage_combine_kernel<<<gb, 256, 0, s>>>(S->U, S->E[0], S->E[1], S->I[0], S->I[1], c, dt, dta, mv.rhob, grav, Nn,
                                            dim, S->rho, S->mhat, S->Ehat);
    count_launches(S->ctx, 1);
    DG_CUDA(cudaMemcpyAsync(S->p, S->p_prev, Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(S->mk, S->mhat, (size_t)dim * Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < o.picard; ++it) {
      picard_prep_kernel<<<gb, 256, 0, s>>>(S->p, mv.pb, S->rho, S->mk, S->mhat, S->Ehat, Nn, dim, S->h, S->rhs,
                                            S->tmpv);
      count_launches(S->ctx, 1);
      RUN(step_div(S, S->tmpv, S->tmps, s));
      axpy_kernel<<<gb, 256, 0, s>>>(S->rhs, S->tmps, -dta, Nn);
      count_launches(S->ctx, 1);
      RUN(check("picard"));
      if (nsolve >= 64) return fail(DG_EINVAL, "too many Picard iterations per step (at most 32)");
      RUN(helmholtz_solve(S, &o, dta * dta, &st, S->solve_out + 4 * nsolve, s));
      ++nsolve;
      RUN(step_grad(S, S->p, S->g, s));
      momentum_kernel<<<gb, 256, 0, s>>>(S->mhat, S->g, dta, (int64_t)dim * Nn, S->mk);
      count_launches(S->ctx, 1);
    }
    stage_state_kernel<<<gb, 256, 0, s>>>(S->rho, S->mk, S->p, mv.pb, Nn, dim, S->Ui);
    count_launches(S->ctx, 1);
    RUN(step_explicit(S, S->Ui, S->E[i], s));
    if (i == 1) {
      hm_kernel<<<gb, 256, 0, s>>>(S->h, S->mk, Nn, dim, S->tmpv);
      count_launches(S->ctx, 1);
      RUN(step_div(S, S->tmpv, S->tmps, s));
      implicit_terms_kernel<<<gb, 256, 0, s>>>(S->Ui, mv.rhob, S->g, S->tmps, grav, Nn, dim, S->I[1]);
      count_launches(S->ctx, 1);
    }
    std::swap(S->p, S->p_prev);
  }
  DG_CUDA(cudaMemsetAsync(S->flag, 0, sizeof(int), s));
  final_kernel<<<gb, 256, 0, s>>>(S->Ui, S->E[0], S->E[1], S->E[2], dt * (BW[0] - AEX[2][0]),
                                  dt * (BW[1] - AEX[2][1]), dt * (BW[2] - AEX[2][2]), (int64_t)V * Nn, S->U,
                                  S->flag);
  count_launches(S->ctx, 1);
  RUN(check("final combination"));
  int flag = 0;
  double sol[256];
  DG_CUDA(cudaMemcpyAsync(&flag, S->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaMemcpyAsync(sol, S->solve_out, 4 * nsolve * sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
#undef RUN
  for (int k = 0; k < nsolve; ++k) {
    st.gmres_iters += (int)sol[4 * k];
    st.max_rel_residual = std::max(st.max_rel_residual, sol[4 * k + 1]);
    if (sol[4 * k + 2] == 0.0) status = fail(DG_ENOTCONV, "a Helmholtz solve missed its tolerance");
  }
  st.solves = nsolve;
  if (stats) *stats = st;
  if (flag) return fail(DG_ENONFINITE, "non-finite value in the new state");
  return status;
}
