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
#include <algorithm>
#include <cmath>
#include <vector>

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
  double* p_save = nullptr;     // initial guess kept while the autotuner tries both solver forms
  double* lmax = nullptr;       // [2] Chebyshev upper spectral bound and the alpha it was estimated for
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

// Rayleigh damping layer: E -= tau (U - U_ref), U_ref = background with the
// uniform x-velocity u0 (rho_b, rho_b u0, 0.., p_b/(gamma-1) + rho_b u0^2/2)
__global__ void sponge_kernel(const double* __restrict__ U, const double* __restrict__ tau,
                              const double* __restrict__ rhob, const double* __restrict__ pb, double u0, int64_t n,
                              int dim, double* __restrict__ E) {
  GRID_LOOP(i, n) {
    const double t = tau[i];
    if (t == 0.0) continue;
    const double rb = rhob[i];
    E[i] -= t * (U[i] - rb);
    E[n + i] -= t * (U[n + i] - rb * u0);
    for (int b = 1; b < dim; ++b) E[(int64_t)(1 + b) * n + i] -= t * U[(int64_t)(1 + b) * n + i];
    const int64_t ie = (int64_t)(dim + 1) * n + i;
    E[ie] -= t * (U[ie] - (pb[i] / (kGamma - 1.0) + 0.5 * rb * u0 * u0));
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

// Krylov forms that exist only as persistent kernels
inline bool persistent_only(int krylov) { return krylov == DG_KRYLOV_CG || krylov == DG_KRYLOV_CHEBYSHEV; }

// Helmholtz solve A(h) p = rhs (p holds the initial guess), FP64 or FP32-refined.
// The fused FP64 path leaves its (iterations, residual, converged, ||b||) in
// out[0..3] on the device and does not wait; the caller reads them later.
int helmholtz_solve(dg_state* S, const dg_solver_opts* o, double alpha, dg_step_stats* st, double* out,
                    cudaStream_t s) {
  const dg_mesh* m = S->mesh;
  const int64_t Nn = S->Nn;
  const int restart = std::min(o->restart, S->restart);
  auto A64 = [&](const double* x, double* y, const int* skip) {
    return op_helmholtz<double>(m, S->h, x, y, alpha, m->d_vec_scratch64, s, skip);
  };
  GmresResult res;
  int rc;
  unsigned long long* phase = S->ctx->prof ? S->ctx->d_phase : nullptr;
  const int npart = (restart + 1) * kDotBlocks;
  if (o->fused || persistent_only(o->krylov)) {
    ProfScope ps(S->ctx, DG_PROF_GMRES, s);
    if (o->precision == DG_FP64)
      return op_gmres<double>(m, S->h, S->h, S->rhs, S->p, alpha, o->tol, 0.0, restart, o->max_iters, o->krylov,
                              S->gm64.Q, S->gm64.w, S->gm64.w, S->gm64.d.partial, npart, out, S->lmax, phase, s);
    float* h32 = S->f32;  // converted by phase_picard_pre
    return op_gmres<float>(m, S->h, h32, S->rhs, S->p, alpha, o->tol, o->inner_tol, restart, o->max_iters,
                           o->krylov, S->gm32.Q, S->gm32.w, S->r64, S->gm32.d.partial, npart, out, S->lmax,
                           phase, s);
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
    return op_helmholtz<float>(m, h32, x, y, (float)alpha, (float*)m->d_vec_scratch64, s, skip);
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
  const dg_mesh* m = S->mesh;
  int rc = op_explicit<double>(m, U, E, m->d_face_scratch64, false, s, nullptr);
  if (rc != DG_OK || !m->d_tau) return rc;
  sponge_kernel<<<gridn(S->Nn), 256, 0, s>>>(U, m->d_tau, m->v64.rhob, m->v64.pb, m->desc.sponge_u0, S->Nn, S->dim, E);
  count_launches(S->ctx, 1);
  return check("sponge layer");
}
int step_grad(dg_state* S, const double* p, double* g, cudaStream_t s) {
  return op_grad<double>(S->mesh, p, nullptr, g, s, nullptr);
}
int step_div(dg_state* S, const double* f, double* out, cudaStream_t s) {
  return op_div<double>(S->mesh, f, out, s, nullptr);
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
  o->inner_tol = 1e-6;
  o->max_refine = 20;
  o->fused = -1;
  o->krylov = DG_KRYLOV_AUTO;
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
  // every buffer is rounded up to 32 doubles (256 bytes); 21 buffers in all
  auto rup = [](size_t n) { return (n + 31) & ~(size_t)31; };
  const size_t nd = 7 * rup((size_t)V * Nn) + 4 * rup((size_t)dim * Nn) + 9 * rup((size_t)Nn) + 2 * rup(8) + rup(256);
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
  S->p_save = take(Nn);
  S->lmax = take(8);
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

extern "C" int dg_state_chebyshev_bound(dg_state* S, double* get, const double* set) {
  if (!S) return fail(DG_EINVAL, "null argument");
  DG_CUDA(cudaDeviceSynchronize());
  if (get) DG_CUDA(cudaMemcpy(get, S->lmax, 2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (set) {
    double v[2] = {set[0], set[1]};
    if (!(v[0] > 1.0 / (kGamma - 1.0))) v[0] = v[1] = 0.0;
    DG_CUDA(cudaMemcpy(S->lmax, v, 2 * sizeof(double), cudaMemcpyHostToDevice));
  }
  return DG_OK;
}

namespace dg {
namespace {

// One member of a step: the state, its step size and options, and what the
// phases below accumulate.  imex_rk2_step runs the phases for one member;
// dg_batch_step runs each phase for every member and solves all members'
// Helmholtz systems of a Picard iteration in one batched launch.
struct Member {
  dg_state* S = nullptr;
  const dg_mesh* m = nullptr;
  double dt = 0.0;
  dg_solver_opts o{};
  dg_step_stats st{};
  int nsolve = 0;
  int flag = 0;
};

inline double stage_dta(const Member& M, int i) { return M.dt * AIM[i][i]; }

int phase_stage1(Member& M, cudaStream_t s) {
  dg_state* S = M.S;
  const int64_t Nn = S->Nn;
  const int dim = S->dim;
  const unsigned gb = gridn(Nn);
  const MeshView<double>& mv = M.m->v64;
  int rc;
  pressure_kernel<<<gb, 256, 0, s>>>(S->U, mv.pb, Nn, dim, S->p_prev, S->h);
  count_launches(S->ctx, 1);
  if ((rc = step_explicit(S, S->U, S->E[0], s)) != DG_OK) return rc;
  if ((rc = step_grad(S, S->p_prev, S->g, s)) != DG_OK) return rc;
  hm_kernel<<<gb, 256, 0, s>>>(S->h, S->U + Nn, Nn, dim, S->tmpv);
  count_launches(S->ctx, 1);
  if ((rc = step_div(S, S->tmpv, S->tmps, s)) != DG_OK) return rc;
  implicit_terms_kernel<<<gb, 256, 0, s>>>(S->U, mv.rhob, S->g, S->tmps, M.m->desc.gravity, Nn, dim, S->I[0]);
  count_launches(S->ctx, 1);
  return check("stage 1");
}

int phase_stage_begin(Member& M, int i, cudaStream_t s) {
  dg_state* S = M.S;
  const int64_t Nn = S->Nn;
  const int dim = S->dim;
  StageCoef c{};
  c.nprev = i;
  for (int j = 0; j < i; ++j) {
    c.ae[j] = AEX[i][j];
    c.ai[j] = AIM[i][j];
  }
  stage_combine_kernel<<<gridn(Nn), 256, 0, s>>>(S->U, S->E[0], S->E[1], S->I[0], S->I[1], c, M.dt,
                                                 stage_dta(M, i), M.m->v64.rhob, M.m->desc.gravity, Nn, dim, S->rho,
                                                 S->mhat, S->Ehat);
  count_launches(S->ctx, 1);
  DG_CUDA(cudaMemcpyAsync(S->p, S->p_prev, Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaMemcpyAsync(S->mk, S->mhat, (size_t)dim * Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return check("stage begin");
}

// right-hand side of the Helmholtz problem for the current Picard iterate
int phase_picard_pre(Member& M, int i, cudaStream_t s) {
  dg_state* S = M.S;
  const int64_t Nn = S->Nn;
  const unsigned gb = gridn(Nn);
  int rc;
  if (M.nsolve >= 64) return fail(DG_EINVAL, "too many Picard iterations per step (at most 32)");
  picard_prep_kernel<<<gb, 256, 0, s>>>(S->p, M.m->v64.pb, S->rho, S->mk, S->mhat, S->Ehat, Nn, S->dim, S->h,
                                        S->rhs, S->tmpv);
  count_launches(S->ctx, 1);
  if ((rc = step_div(S, S->tmpv, S->tmps, s)) != DG_OK) return rc;
  axpy_kernel<<<gb, 256, 0, s>>>(S->rhs, S->tmps, -stage_dta(M, i), Nn);
  count_launches(S->ctx, 1);
  if (M.o.precision == DG_FP32) {
    to_f32_kernel<<<gb, 256, 0, s>>>(S->h, S->f32, Nn);  // h for the FP32 Arnoldi mat-vecs
    count_launches(S->ctx, 1);
  }
  return check("picard");
}

// Solver forms the autotuner chooses among
enum SolverForm { FORM_GMRES_MULTI = 0, FORM_GMRES_PERSISTENT = 1, FORM_CHEBYSHEV = 2, N_FORMS = 3 };

inline void apply_form(dg_solver_opts& o, int form) {
  o.krylov = form == FORM_CHEBYSHEV ? DG_KRYLOV_CHEBYSHEV : DG_KRYLOV_GMRES;
  o.fused = form == FORM_GMRES_MULTI ? 0 : 1;
}

// Autotuner.  With krylov = AUTO the first solve of a (mesh, precision) is
// run as GMRES in both forms (one persistent launch; one launch per Krylov
// kernel) and as Chebyshev; with krylov = GMRES and fused = -1, as GMRES in
// both forms.  Every candidate starts from the same initial guess, in two
// rounds (the first pays the one-off costs -- lazy module loading, occupancy
// queries, the Chebyshev bound -- and is not timed; the second is), and the
// fastest is kept for every later solve on that mesh.  The persistent forms
// win on small meshes, where launch latency dominates; the multi-kernel form
// can win on large FP64 meshes, where full occupancy hides the FP64 pipe's
// latency; Chebyshev needs no inner products.
int phase_solve_single(Member& M, int i, cudaStream_t s) {
  const double dta = stage_dta(M, i);
  double* out = M.S->solve_out + 4 * M.nsolve;
  ++M.nsolve;
  const bool auto_k = M.o.krylov == DG_KRYLOV_AUTO;
  if (!auto_k && (M.o.fused >= 0 || persistent_only(M.o.krylov)))
    return helmholtz_solve(M.S, &M.o, dta * dta, &M.st, out, s);
  const int pi = M.o.precision == DG_FP32 ? 1 : 0;
  const int ncand = auto_k ? 3 : 2;
  float* ms = M.m->tuned_ms[pi];
  bool timed = true;
  for (int f = 0; f < ncand; ++f) timed = timed && ms[f] > 0.0f;
  dg_solver_opts o = M.o;
  if (timed) {
    int best = 0;
    for (int f = 1; f < ncand; ++f)
      if (ms[f] < ms[best]) best = f;
    M.m->tuned_form[pi] = best;
    apply_form(o, best);
    return helmholtz_solve(M.S, &o, dta * dta, &M.st, out, s);
  }
  dg_state* S = M.S;
  DG_CUDA(cudaMemcpyAsync(S->p_save, S->p, S->Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e[N_FORMS + 1];
  for (auto& ev : e) DG_CUDA(cudaEventCreate(&ev));
  int rc = DG_OK;
  bool first = true;
  const dg_step_stats st0 = M.st;  // only the last (kept) solve counts in the step's statistics
  // candidates in the order persistent GMRES, Chebyshev, multi-kernel GMRES (the last one's result is kept)
  int order[N_FORMS], no = 0;
  order[no++] = FORM_GMRES_PERSISTENT;
  if (auto_k) order[no++] = FORM_CHEBYSHEV;
  order[no++] = FORM_GMRES_MULTI;
  for (int round = 0; round < 2 && rc == DG_OK; ++round) {
    for (int c = 0; c < no && rc == DG_OK; ++c) {
      M.st = st0;
      if (!first) DG_CUDA(cudaMemcpyAsync(S->p, S->p_save, S->Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      first = false;
      apply_form(o, order[c]);
      if (round == 1) DG_CUDA(cudaEventRecord(e[c], s));
      rc = helmholtz_solve(S, &o, dta * dta, &M.st, out, s);
    }
  }
  if (rc == DG_OK) {
    DG_CUDA(cudaEventRecord(e[no], s));
    DG_CUDA(cudaEventSynchronize(e[no]));
    int best = -1;
    for (int c = 0; c < no; ++c) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, e[c], e[c + 1]);
      ms[order[c]] = t > 0.0f ? t : 1e-6f;
      if (best < 0 || ms[order[c]] < ms[best]) best = order[c];
    }
    M.m->tuned_form[pi] = best;
  }
  for (auto& ev : e) cudaEventDestroy(ev);
  return rc;
}

int phase_picard_post(Member& M, int i, cudaStream_t s) {
  dg_state* S = M.S;
  int rc;
  if ((rc = step_grad(S, S->p, S->g, s)) != DG_OK) return rc;
  momentum_kernel<<<gridn(S->Nn), 256, 0, s>>>(S->mhat, S->g, stage_dta(M, i), (int64_t)S->dim * S->Nn, S->mk);
  count_launches(S->ctx, 1);
  return check("momentum update");
}

int phase_stage_end(Member& M, int i, cudaStream_t s) {
  dg_state* S = M.S;
  const int64_t Nn = S->Nn;
  const int dim = S->dim;
  const unsigned gb = gridn(Nn);
  int rc;
  stage_state_kernel<<<gb, 256, 0, s>>>(S->rho, S->mk, S->p, M.m->v64.pb, Nn, dim, S->Ui);
  count_launches(S->ctx, 1);
  if ((rc = step_explicit(S, S->Ui, S->E[i], s)) != DG_OK) return rc;
  if (i == 1) {
    hm_kernel<<<gb, 256, 0, s>>>(S->h, S->mk, Nn, dim, S->tmpv);
    count_launches(S->ctx, 1);
    if ((rc = step_div(S, S->tmpv, S->tmps, s)) != DG_OK) return rc;
    implicit_terms_kernel<<<gb, 256, 0, s>>>(S->Ui, M.m->v64.rhob, S->g, S->tmps, M.m->desc.gravity, Nn, dim,
                                             S->I[1]);
    count_launches(S->ctx, 1);
  }
  std::swap(S->p, S->p_prev);
  return check("stage end");
}

int phase_final(Member& M, cudaStream_t s) {
  dg_state* S = M.S;
  const double dt = M.dt;
  DG_CUDA(cudaMemsetAsync(S->flag, 0, sizeof(int), s));
  final_kernel<<<gridn(S->Nn), 256, 0, s>>>(S->Ui, S->E[0], S->E[1], S->E[2], dt * (BW[0] - AEX[2][0]),
                                            dt * (BW[1] - AEX[2][1]), dt * (BW[2] - AEX[2][2]),
                                            (int64_t)S->V * S->Nn, S->U, S->flag);
  count_launches(S->ctx, 1);
  return check("final combination");
}

// after the stream has been synchronised: solve results and the non-finite flag
int member_finish(Member& M, const double* sol, int flag) {
  int status = DG_OK;
  for (int k = 0; k < M.nsolve; ++k) {
    M.st.gmres_iters += (int)sol[4 * k];
    M.st.max_rel_residual = std::max(M.st.max_rel_residual, sol[4 * k + 1]);
    if (sol[4 * k + 2] == 0.0) status = fail(DG_ENOTCONV, "a Helmholtz solve missed its tolerance");
  }
  M.st.solves = M.nsolve;
  if (flag) status = fail(DG_ENONFINITE, "non-finite value in the new state");
  return status;
}

int prepare_member(Member& M, dg_ctx* ctx, const dg_mesh* m, dg_state* S, double dt, const dg_solver_opts* opts) {
  if (!ctx || !m || !S || S->mesh != m) return fail(DG_EINVAL, "bad arguments");
  if (!(dt > 0.0)) return fail(DG_EINVAL, "dt must be positive");
  dg_solver_opts_default(&M.o);
  if (opts) M.o = *opts;
  if (M.o.precision != DG_FP64 && M.o.precision != DG_FP32) return fail(DG_EINVAL, "bad precision");
  if (M.o.picard < 1 || M.o.picard > 32) return fail(DG_EINVAL, "picard must be in 1..32");
  if (M.o.krylov < DG_KRYLOV_AUTO || M.o.krylov > DG_KRYLOV_CHEBYSHEV) return fail(DG_EINVAL, "bad Krylov method");
  M.S = S;
  M.m = m;
  M.dt = dt;
  return DG_OK;
}

}  // namespace
}  // namespace dg

extern "C" int imex_rk2_step(dg_ctx* ctx, const dg_mesh* m, dg_state* S, double dt, const dg_solver_opts* opts,
                             dg_step_stats* stats, void* stream) {
  Member M;
  int rc = prepare_member(M, ctx, m, S, dt, opts);
  if (rc != DG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope step_scope(ctx, DG_PROF_STEP, s);
#define RUN(x)                          \
  do {                                  \
    if ((rc = (x)) != DG_OK) return rc; \
  } while (0)
  RUN(phase_stage1(M, s));
  for (int i = 1; i <= 2; ++i) {
    RUN(phase_stage_begin(M, i, s));
    for (int it = 0; it < M.o.picard; ++it) {
      RUN(phase_picard_pre(M, i, s));
      RUN(phase_solve_single(M, i, s));
      RUN(phase_picard_post(M, i, s));
    }
    RUN(phase_stage_end(M, i, s));
  }
  RUN(phase_final(M, s));
#undef RUN
  int flag = 0;
  double sol[256];
  DG_CUDA(cudaMemcpyAsync(&flag, S->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaMemcpyAsync(sol, S->solve_out, 4 * M.nsolve * sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  const int status = member_finish(M, sol, flag);
  if (stats) *stats = M.st;
  return status;
}

namespace dg {
namespace {

// Parallel branches for the per-member phases of a captured batch step: each
// segment of member work forks from the main stream, member i runs on branch
// i mod K, and the branches join before the next batched solve.
struct Branches {
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

// Krylov method of a member's solves inside a batched launch: krylov = AUTO
// takes the mesh's tuned persistent form, else Chebyshev (a batch cannot time
// candidates one by one).
int batch_method(const Member& M) {
  if (M.o.krylov != DG_KRYLOV_AUTO) return M.o.krylov;
  const int pi = M.o.precision == DG_FP32 ? 1 : 0;
  return M.m->tuned_form[pi] == FORM_GMRES_PERSISTENT ? DG_KRYLOV_GMRES : DG_KRYLOV_CHEBYSHEV;
}
// Members that run alone (one launch per Krylov kernel) instead of batched
bool batch_alone(const Member& M) {
  return M.o.krylov != DG_KRYLOV_AUTO && M.o.fused == 0 && !persistent_only(M.o.krylov);
}

// Batched Helmholtz solves of one Picard iteration: the persistent solves
// grouped by (dim, degree, precision), one batched launch per group; members
// that asked for the one-launch-per-kernel form are solved alone.
int solve_all(dg_ctx* ctx, std::vector<Member>& M, const dg_solver_opts& o, int stage, int* err,
              cudaStream_t s) {
  const int n = (int)M.size();
  const int restart = std::min(o.restart, kMaxRestart);
  int rc;
  std::vector<int> rest;
  std::vector<std::vector<int>> groups;
  std::vector<std::pair<std::pair<int, int>, int>> keys;
  for (int i = 0; i < n; ++i) {
    // members of a batch use the batched persistent solve unless told otherwise
    if (batch_alone(M[i])) {
      rest.push_back(i);
      continue;
    }
    const std::pair<int, int> key{M[i].m->dim * 16 + M[i].m->degree, M[i].o.precision};
    size_t g = 0;
    for (; g < keys.size(); ++g)
      if (keys[g].first == key) break;
    if (g == keys.size()) {
      keys.push_back({key, (int)g});
      groups.emplace_back();
    }
    groups[g].push_back(i);
  }
  for (size_t g = 0; g < groups.size(); ++g) {
    ProfScope ps(ctx, DG_PROF_GMRES, s);
    const int dim = M[groups[g][0]].m->dim;
    const bool f32 = keys[g].first.second == DG_FP32;
    if (!f32) {
      std::vector<GmresItem<double>> items;
      for (int i : groups[g]) {
        dg_state* S = M[i].S;
        const double dta = stage_dta(M[i], stage);
        items.push_back({M[i].m, S->h, S->h, S->rhs, S->p, dta * dta, o.tol, 0.0, o.max_iters, batch_method(M[i]),
                         S->gm64.Q,
                         S->gm64.w, S->gm64.w, S->gm64.d.partial, (restart + 1) * kDotBlocks,
                         S->solve_out + 4 * M[i].nsolve, S->lmax});
      }
      if ((rc = op_gmres_batched<double>(ctx, dim, items.data(), (int)items.size(), restart, err, s)) != DG_OK)
        return rc;
    } else {
      std::vector<GmresItem<float>> items;
      for (int i : groups[g]) {
        dg_state* S = M[i].S;
        const double dta = stage_dta(M[i], stage);
        items.push_back({M[i].m, S->h, S->f32, S->rhs, S->p, dta * dta, o.tol, o.inner_tol, o.max_iters,
                         batch_method(M[i]), S->gm32.Q, S->gm32.w, S->r64, S->gm32.d.partial, (restart + 1) * kDotBlocks,
                         S->solve_out + 4 * M[i].nsolve, S->lmax});
      }
      if ((rc = op_gmres_batched<float>(ctx, dim, items.data(), (int)items.size(), restart, err, s)) != DG_OK)
        return rc;
    }
    for (int i : groups[g]) ++M[i].nsolve;
  }
  for (int i : rest)
    if ((rc = phase_solve_single(M[i], stage, s)) != DG_OK) return rc;
  return DG_OK;
}

// One IMEX-RK2 step of every member: the per-member phases (on branches if
// given) between the batched solves of each Picard iteration.
int batch_phases(dg_ctx* ctx, std::vector<Member>& M, const dg_solver_opts& o, int* err, cudaStream_t s,
                 const Branches* br) {
  int rc;
  // run body(member, stream) for every member, forked over the branches
  auto segment = [&](auto&& body) -> int {
    const int K = br ? (int)br->st.size() : 0;
    if (K == 0) {
      for (auto& mm : M)
        if ((rc = body(mm, s)) != DG_OK) return rc;
      return DG_OK;
    }
    DG_CUDA(cudaEventRecord(br->fork, s));
    for (int k = 0; k < K; ++k) DG_CUDA(cudaStreamWaitEvent(br->st[k], br->fork, 0));
    for (size_t i = 0; i < M.size(); ++i)
      if ((rc = body(M[i], br->st[i % K])) != DG_OK) return rc;
    for (int k = 0; k < K; ++k) {
      DG_CUDA(cudaEventRecord(br->join[k], br->st[k]));
      DG_CUDA(cudaStreamWaitEvent(s, br->join[k], 0));
    }
    return DG_OK;
  };
#define RUN(x)                          \
  do {                                  \
    if ((rc = (x)) != DG_OK) return rc; \
  } while (0)
  RUN(segment([&](Member& mm, cudaStream_t t) {
    int r;
    if ((r = phase_stage1(mm, t)) != DG_OK) return r;
    if ((r = phase_stage_begin(mm, 1, t)) != DG_OK) return r;
    return phase_picard_pre(mm, 1, t);
  }));
  for (int i = 1; i <= 2; ++i) {
    for (int it = 0; it < o.picard; ++it) {
      RUN(solve_all(ctx, M, o, i, err, s));
      const bool last = it == o.picard - 1;
      RUN(segment([&](Member& mm, cudaStream_t t) {
        int r;
        if ((r = phase_picard_post(mm, i, t)) != DG_OK) return r;
        if (!last) return phase_picard_pre(mm, i, t);
        if ((r = phase_stage_end(mm, i, t)) != DG_OK) return r;
        if (i == 1) {
          if ((r = phase_stage_begin(mm, 2, t)) != DG_OK) return r;
          return phase_picard_pre(mm, 2, t);
        }
        return phase_final(mm, t);
      }));
    }
  }
#undef RUN
  return DG_OK;
}

int prepare_batch(dg_ctx* ctx, int n, const dg_mesh* const* meshes, dg_state* const* states, const double* dt,
                  const dg_solver_opts* opts, std::vector<Member>& M) {
  if (!ctx || n < 0 || (n > 0 && (!meshes || !states || !dt))) return fail(DG_EINVAL, "null argument");
  M.assign(n, Member{});
  int rc;
  for (int i = 0; i < n; ++i) {
    if ((rc = prepare_member(M[i], ctx, meshes[i], states[i], dt[i], opts)) != DG_OK) return rc;
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return fail(DG_EINVAL, "members of a batch must not share a mesh");
  }
  if (n > 0) {
    const int restart = std::min(M[0].o.restart, kMaxRestart);
    for (int i = 0; i < n; ++i)
      if (M[i].S->restart < restart) return fail(DG_EINVAL, "a state was created with a shorter restart length");
  }
  if (!ctx->d_batch_err) DG_CUDA(cudaMalloc(&ctx->d_batch_err, sizeof(int)));
  return DG_OK;
}

// statuses and statistics of every member from the flags and solve results read back after the step
int finish_batch(std::vector<Member>& M, const int* flags, const double* sol, int herr, dg_step_stats* stats,
                 int* statuses) {
  int worst = DG_OK;
  for (size_t i = 0; i < M.size(); ++i) {
    int st = member_finish(M[i], &sol[i * 256], flags[i]);
    if (herr) st = fail(DG_ETIMEOUT, "a barrier of the batched GMRES launch ran out of time");
    if (stats) stats[i] = M[i].st;
    if (statuses) statuses[i] = st;
    if (st != DG_OK && worst == DG_OK) worst = st;
  }
  return worst;
}

}  // namespace
}  // namespace dg

extern "C" int dg_batch_step(dg_ctx* ctx, int n, const dg_mesh* const* meshes, dg_state* const* states,
                             const double* dt, const dg_solver_opts* opts, dg_step_stats* stats, int* statuses,
                             void* stream) {
  std::vector<Member> M;
  int rc = prepare_batch(ctx, n, meshes, states, dt, opts, M);
  if (rc != DG_OK || n == 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope step_scope(ctx, DG_PROF_STEP, s);
  int* err = ctx->d_batch_err;
  DG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if ((rc = batch_phases(ctx, M, M[0].o, err, s, nullptr)) != DG_OK) return rc;
  // read every member's flag and solve results with one synchronisation
  std::vector<int> flags(n, 0);
  std::vector<double> sol((size_t)n * 256, 0.0);
  int herr = 0;
  for (int i = 0; i < n; ++i) {
    DG_CUDA(cudaMemcpyAsync(&flags[i], M[i].S->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaMemcpyAsync(&sol[(size_t)i * 256], M[i].S->solve_out, 4 * M[i].nsolve * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
  }
  DG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return finish_batch(M, flags.data(), sol.data(), herr, stats, statuses);
}

// ---- batch plans: one captured CUDA graph per ensemble step ----

struct dg_batch_plan {
  dg_ctx* ctx = nullptr;
  std::vector<dg::Member> M;
  int n = 0;
  cudaStream_t cs = nullptr;  // capture stream
  dg::Branches br;
  dg::BatchArena arena;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;       // kernels in one replay
  int* h_flags = nullptr;      // pinned: [n] flags, then the timeout flag
  double* h_sol = nullptr;     // pinned: [n*256] solve results
};

extern "C" int dg_batch_plan_destroy(dg_batch_plan* P) {
  if (!P) return DG_OK;
  cudaSetDevice(P->ctx->device);
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (auto st : P->br.st) cudaStreamDestroy(st);
  for (auto ev : P->br.join) cudaEventDestroy(ev);
  if (P->br.fork) cudaEventDestroy(P->br.fork);
  if (P->cs) cudaStreamDestroy(P->cs);
  if (P->arena.dev) cudaFree(P->arena.dev);
  if (P->h_flags) cudaFreeHost(P->h_flags);
  if (P->h_sol) cudaFreeHost(P->h_sol);
  delete P;
  return DG_OK;
}

extern "C" int dg_batch_plan_create(dg_ctx* ctx, int n, const dg_mesh* const* meshes, dg_state* const* states,
                                    const double* dt, const dg_solver_opts* opts, dg_batch_plan** out) {
  if (!out) return fail(DG_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1) return fail(DG_EINVAL, "a batch plan needs at least one member");
  dg_batch_plan* P = new (std::nothrow) dg_batch_plan();
  if (!P) return fail(DG_ENOMEM, "host allocation failed");
  P->ctx = ctx;
  P->n = n;
  int rc = prepare_batch(ctx, n, meshes, states, dt, opts, P->M);
  if (rc != DG_OK) {
    delete P;
    return rc;
  }
  for (auto& mm : P->M)
    if (batch_alone(mm)) {
      delete P;
      return fail(DG_EINVAL, "a batch plan needs the persistent solve (fused != 0)");
    }
  const dg_solver_opts& o = P->M[0].o;
  auto bail = [&](int r) {
    dg_batch_plan_destroy(P);
    return r;
  };
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking);
  const int K = std::min(n, 16);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) P->br.st.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) P->br.join.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->br.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&P->h_flags, (n + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&P->h_sol, (size_t)n * 256 * sizeof(double));
  // argument tables of the batched launches: per launch at most one table of
  // n members and a CTA map of 2 x (2 CTAs per SM) entries; one launch per
  // group (at most n) in each of the 2 x picard Picard iterations
  const size_t per_member = kBatchArgBytes;
  const size_t per_launch = (size_t)(2 * 2 * ctx->sm_count) * sizeof(int) + 4 * 256;
  const size_t arena_bytes = (size_t)2 * o.picard * ((per_member + 3 * sizeof(int) + 16) * n + per_launch * n);
  if (e == cudaSuccess) e = cudaMalloc(&P->arena.dev, arena_bytes);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch plan resources"));
  P->arena.host.assign(arena_bytes, 0);

  // capture one step; nothing runs while the capture is open
  const bool prof = ctx->prof;
  const long long launches0 = ctx->launches;
  ctx->prof = false;
  ctx->arena = &P->arena;
  int* err = ctx->d_batch_err;
  e = cudaStreamBeginCapture(P->cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = DG_OK;
    e = cudaMemsetAsync(err, 0, sizeof(int), P->cs);
    if (e != cudaSuccess) rc = cuda_fail(e, "batch plan capture");
    if (rc == DG_OK) rc = batch_phases(ctx, P->M, o, err, P->cs, &P->br);
    for (int i = 0; i < n && rc == DG_OK; ++i) {
      e = cudaMemcpyAsync(&P->h_flags[i], P->M[i].S->flag, sizeof(int), cudaMemcpyDeviceToHost, P->cs);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&P->h_sol[(size_t)i * 256], P->M[i].S->solve_out, 4 * P->M[i].nsolve * sizeof(double),
                            cudaMemcpyDeviceToHost, P->cs);
      if (e != cudaSuccess) rc = cuda_fail(e, "batch plan capture");
    }
    if (rc == DG_OK) {
      e = cudaMemcpyAsync(&P->h_flags[n], err, sizeof(int), cudaMemcpyDeviceToHost, P->cs);
      if (e != cudaSuccess) rc = cuda_fail(e, "batch plan capture");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cs, &g);  // ends the capture whether or not the phases succeeded
    P->graph = g;
    if (rc == DG_OK && e != cudaSuccess) rc = cuda_fail(e, "batch plan capture");
  } else {
    rc = cuda_fail(e, "batch plan capture");
  }
  ctx->arena = nullptr;
  ctx->prof = prof;
  P->kernels = ctx->launches - launches0;
  ctx->launches = launches0;
  if (rc != DG_OK) return bail(rc);
  e = cudaMemcpy(P->arena.dev, P->arena.host.data(), P->arena.used, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch plan instantiation"));
  *out = P;
  return DG_OK;
}

extern "C" int dg_batch_plan_step(dg_batch_plan* P, dg_step_stats* stats, int* statuses, void* stream) {
  if (!P) return fail(DG_EINVAL, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope step_scope(P->ctx, DG_PROF_STEP, s);
  DG_CUDA(cudaGraphLaunch(P->exec, s));
  count_launches(P->ctx, (int)P->kernels);
  DG_CUDA(cudaStreamSynchronize(s));
  for (auto& mm : P->M) mm.st = dg_step_stats{};
  return finish_batch(P->M, P->h_flags, P->h_sol, P->h_flags[P->n], stats, statuses);
}
