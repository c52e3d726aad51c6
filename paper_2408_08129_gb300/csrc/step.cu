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

// ---- the step's pointwise work, as operations on member views ----------------
//
// Each operation works on one node (or one entry of a multi-variable array) of
// one member; pack_kernel runs it over the nodes of up to kPack members in one
// launch (the pack is a kernel parameter), so that an ensemble step launches
// every pointwise phase once, and a single step uses the same code with one
// member.

// what the pointwise operations of the step read and write of one member
struct StepView {
  double *U, *E0, *E1, *E2, *I0, *I1, *Ui, *rho, *mhat, *Ehat, *p, *p_prev, *h, *mk, *rhs, *tmpv, *tmps, *g;
  float* f32;
  int* flag;
  const double *rhob, *pb, *tau;
  int64_t Nn;
  int dim;
  double dt, grav, u0;
};

struct StepPack {
  StepView m[kPack];
  int64_t start[kPack + 1];  // first CTA of each member
  int n;
};

__device__ __forceinline__ double* e_of(const StepView& M, int j) { return j == 0 ? M.E0 : (j == 1 ? M.E1 : M.E2); }

template <class Op>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ StepPack P, const Op op) {
  int j = 0;
  while (j + 1 < P.n && (int64_t)blockIdx.x >= P.start[j + 1]) ++j;
  const StepView& M = P.m[j];
  const int64_t len = M.Nn * op.width(M.dim);
  const int64_t stride = (P.start[j + 1] - P.start[j]) * blockDim.x;
  for (int64_t i = (int64_t)(blockIdx.x - P.start[j]) * blockDim.x + threadIdx.x; i < len; i += stride) op(M, i);
}

// p' = (g-1)(rho E - |m|^2/(2 rho)) - p_bar and h = gamma p / ((gamma-1) rho) of U; the step's
// first operation also clears the member's non-finite flag
struct OpPressure {
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const int64_t Nn = M.Nn;
    const int V = M.dim + 2;
    if (i == 0) *M.flag = 0;
    const double rho = M.U[i];
    double m2 = 0.0;
    for (int b = 0; b < M.dim; ++b) m2 += M.U[(1 + b) * Nn + i] * M.U[(1 + b) * Nn + i];
    const double p = (kGamma - 1.0) * (M.U[(V - 1) * Nn + i] - 0.5 * m2 / rho);
    M.p_prev[i] = p - M.pb[i];
    M.h[i] = kGamma * p / ((kGamma - 1.0) * rho);
  }
};

// tmpv[b] = h * m[b], m the momentum of U (from_mk = 0) or mk (1)
struct OpHm {
  int from_mk;
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const double* m = from_mk ? M.mk : M.U + M.Nn;
    for (int b = 0; b < M.dim; ++b) M.tmpv[b * M.Nn + i] = M.h[i] * m[b * M.Nn + i];
  }
};

// implicit tendencies I_k = (0, -g - rho' grav k, -div(h m)) with rho from U (k = 0) or Ui (k = 1)
struct OpImplicitTerms {
  int k;
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const int64_t Nn = M.Nn;
    const int V = M.dim + 2;
    const double* rho = k ? M.Ui : M.U;
    double* I = k ? M.I1 : M.I0;
    I[i] = 0.0;
    for (int b = 0; b < M.dim; ++b) I[(1 + b) * Nn + i] = -M.g[b * Nn + i];
    I[M.dim * Nn + i] -= (rho[i] - M.rhob[i]) * M.grav;
    I[(V - 1) * Nn + i] = -M.tmps[i];
  }
};

// rho, mhat, Ehat of implicit stage `stage` from U^n and the earlier tendencies; p = p_prev
// (the Picard loop starts from the previous stage's pressure) and mk = mhat
struct OpStageCombine {
  int stage;
  double ae[2], ai[2], aii;  // tableau rows (times dt in the operation)
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const int64_t Nn = M.Nn;
    const int V = M.dim + 2;
    const double dt = M.dt, dta = dt * aii;
    double r = ae[0] * M.E0[i];
    if (stage > 1) r += ae[1] * M.E1[i];
    const double rh = M.U[i] + dt * r;
    M.rho[i] = rh;
    for (int b = 0; b < M.dim; ++b) {
      const int64_t o = (int64_t)(1 + b) * Nn + i;
      double s = ae[0] * M.E0[o] + ai[0] * M.I0[o];
      if (stage > 1) s += ae[1] * M.E1[o] + ai[1] * M.I1[o];
      double mh = M.U[o] + dt * s;
      if (b == M.dim - 1) mh -= dta * (rh - M.rhob[i]) * M.grav;
      M.mhat[b * Nn + i] = mh;
      M.mk[b * Nn + i] = mh;
    }
    const int64_t o = (int64_t)(V - 1) * Nn + i;
    double s = ae[0] * M.E0[o] + ai[0] * M.I0[o];
    if (stage > 1) s += ae[1] * M.E1[o] + ai[1] * M.I1[o];
    M.Ehat[i] = M.U[o] + dt * s;
    M.p[i] = M.p_prev[i];
  }
};

// Picard preparation: h = gamma (p_bar + p')/((g-1) rho); rhs = Ehat - p_bar/(g-1) - |mk|^2/(2 rho);
// tmpv = h * mhat
struct OpPicardPrep {
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const int64_t Nn = M.Nn;
    const double r = M.rho[i];
    const double hh = kGamma * (M.pb[i] + M.p[i]) / ((kGamma - 1.0) * r);
    M.h[i] = hh;
    double m2 = 0.0;
    for (int b = 0; b < M.dim; ++b) {
      m2 += M.mk[b * Nn + i] * M.mk[b * Nn + i];
      M.tmpv[b * Nn + i] = hh * M.mhat[b * Nn + i];
    }
    M.rhs[i] = M.Ehat[i] - M.pb[i] / (kGamma - 1.0) - 0.5 * m2 / r;
  }
};

// rhs -= dt a_ii div(h mhat); FP32 forms also get h in FP32 for their Krylov mat-vecs
struct OpRhsFinish {
  double aii;
  int f32;
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    M.rhs[i] += -(M.dt * aii) * M.tmps[i];
    if (f32) M.f32[i] = (float)M.h[i];
  }
};

// mk = mhat - dt a_ii grad p'
struct OpMomentum {
  double aii;
  __host__ __device__ int width(int dim) const { return dim; }
  __device__ void operator()(const StepView& M, int64_t i) const { M.mk[i] = M.mhat[i] - (M.dt * aii) * M.g[i]; }
};

// stage state: (rho, mk, (p_bar + p')/(g-1) + |mk|^2/(2 rho))
struct OpStageState {
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const int64_t Nn = M.Nn;
    const int V = M.dim + 2;
    const double r = M.rho[i];
    double m2 = 0.0;
    M.Ui[i] = r;
    for (int b = 0; b < M.dim; ++b) {
      const double mb = M.mk[b * Nn + i];
      M.Ui[(1 + b) * Nn + i] = mb;
      m2 += mb * mb;
    }
    M.Ui[(V - 1) * Nn + i] = (M.pb[i] + M.p[i]) / (kGamma - 1.0) + 0.5 * m2 / r;
  }
};

// Rayleigh damping layer: E_k -= tau (X - U_ref), X = U (k = 0) or Ui, U_ref = the background with
// the uniform x-velocity u0 (rho_b, rho_b u0, 0.., p_b/(gamma-1) + rho_b u0^2/2); no-op without a layer
struct OpSponge {
  int k;
  __host__ __device__ int width(int) const { return 1; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    if (!M.tau) return;
    const double t = M.tau[i];
    if (t == 0.0) return;
    const int64_t n = M.Nn;
    const double* X = k ? M.Ui : M.U;
    double* E = e_of(M, k);
    const double rb = M.rhob[i], u0 = M.u0;
    E[i] -= t * (X[i] - rb);
    E[n + i] -= t * (X[n + i] - rb * u0);
    for (int b = 1; b < M.dim; ++b) E[(int64_t)(1 + b) * n + i] -= t * X[(int64_t)(1 + b) * n + i];
    const int64_t ie = (int64_t)(M.dim + 1) * n + i;
    E[ie] -= t * (X[ie] - (M.pb[i] / (kGamma - 1.0) + 0.5 * rb * u0 * u0));
  }
};

// U = Ui + dt sum_j c_j E_j; flag non-finite values
struct OpFinal {
  double c[3];  // b_j - A[2][j]
  __host__ __device__ int width(int dim) const { return dim + 2; }
  __device__ void operator()(const StepView& M, int64_t i) const {
    const double v = M.Ui[i] + (M.dt * c[0]) * M.E0[i] + (M.dt * c[1]) * M.E1[i] + (M.dt * c[2]) * M.E2[i];
    M.U[i] = v;
    if (!isfinite(v)) *M.flag = 1;
  }
};


// ax = b - ax (in place)
__global__ void sub_from_kernel(const double* b, double* ax, int64_t n) {
  GRID_LOOP(i, n) { ax[i] = b[i] - ax[i]; }
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
  unsigned long long* phase = S->ctx->prof_clocks ? S->ctx->d_phase : nullptr;
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

// ---- the step's phases over a list of members ----

StepView step_view(const Member& M) {
  const dg_state* S = M.S;
  StepView v;
  v.U = S->U;
  v.E0 = S->E[0];
  v.E1 = S->E[1];
  v.E2 = S->E[2];
  v.I0 = S->I[0];
  v.I1 = S->I[1];
  v.Ui = S->Ui;
  v.rho = S->rho;
  v.mhat = S->mhat;
  v.Ehat = S->Ehat;
  v.p = S->p;
  v.p_prev = S->p_prev;
  v.h = S->h;
  v.mk = S->mk;
  v.rhs = S->rhs;
  v.tmpv = S->tmpv;
  v.tmps = S->tmps;
  v.g = S->g;
  v.f32 = S->f32;
  v.flag = S->flag;
  v.rhob = M.m->v64.rhob;
  v.pb = M.m->v64.pb;
  v.tau = M.m->d_tau;
  v.Nn = S->Nn;
  v.dim = S->dim;
  v.dt = M.dt;
  v.grav = M.m->desc.gravity;
  v.u0 = M.m->desc.sponge_u0;
  return v;
}

// one launch of a pointwise operation over the members (one per kPack members)
template <class Op>
int launch_pack(dg_ctx* ctx, std::vector<Member>& M, const Op& op, cudaStream_t s) {
  for (size_t first = 0; first < M.size(); first += kPack) {
    StepPack P;
    P.n = (int)std::min(M.size() - first, (size_t)kPack);
    int64_t nb = 0;
    for (int j = 0; j < P.n; ++j) {
      P.m[j] = step_view(M[first + j]);
      P.start[j] = nb;
      const int64_t len = P.m[j].Nn * op.width(P.m[j].dim);
      nb += std::max<int64_t>(1, std::min<int64_t>((len + 255) / 256, 2048));
    }
    P.start[P.n] = nb;
    pack_kernel<Op><<<(unsigned)nb, 256, 0, s>>>(P, op);
    count_launches(ctx, 1);
  }
  return check("pointwise step operation");
}

// members grouped by (dimension, degree): the packed FP64 operators need one shape
std::vector<std::vector<Member*>> shape_groups(std::vector<Member>& M) {
  std::vector<std::vector<Member*>> g;
  std::vector<int> key;
  for (auto& mm : M) {
    const int k = mm.m->dim * 16 + mm.m->degree;
    size_t j = 0;
    for (; j < key.size(); ++j)
      if (key[j] == k) break;
    if (j == key.size()) {
      key.push_back(k);
      g.emplace_back();
    }
    g[j].push_back(&mm);
  }
  return g;
}

// one FP64 operator over every member: kind 0 explicit (U -> E0, or Ui -> E_k for k > 0),
// 1 gradient (p_prev, or p if k = 1, -> g), 2 divergence (tmpv -> tmps)
int launch_dg(dg_ctx* ctx, std::vector<Member>& M, int kind, int k, cudaStream_t s) {
  int rc;
  for (auto& grp : shape_groups(M)) {
    for (size_t first = 0; first < grp.size(); first += kPack) {
      OpPack<double> P;
      P.n = (int)std::min(grp.size() - first, (size_t)kPack);
      for (int j = 0; j < P.n; ++j) {
        const Member& mm = *grp[first + j];
        dg_state* S = mm.S;
        P.mv[j] = mm.m->v64;
        P.aux[j] = nullptr;
        P.scratch[j] = mm.m->d_face_scratch64;
        if (kind == 0) {
          P.in[j] = k == 0 ? S->U : S->Ui;
          P.out[j] = S->E[k];
        } else if (kind == 1) {
          P.in[j] = k == 0 ? S->p_prev : S->p;
          P.out[j] = S->g;
        } else {
          P.in[j] = S->tmpv;
          P.out[j] = S->tmps;
        }
      }
      const int dim = grp[first]->m->dim, deg = grp[first]->m->degree;
      rc = kind == 0 ? op_explicit_pack(ctx, dim, deg, P, false, s)
                     : (kind == 1 ? op_grad_pack(ctx, dim, deg, P, s) : op_div_pack(ctx, dim, deg, P, s));
      if (rc != DG_OK) return rc;
    }
  }
  return DG_OK;
}

bool any_layer(const std::vector<Member>& M) {
  for (const auto& mm : M)
    if (mm.m->d_tau) return true;
  return false;
}

// the explicit tendency E_k of U (k = 0) or of the stage state Ui, with the damping layer
int phase_explicit(dg_ctx* ctx, std::vector<Member>& M, int k, cudaStream_t s) {
  int rc = launch_dg(ctx, M, 0, k, s);
  if (rc != DG_OK || !any_layer(M)) return rc;
  return launch_pack(ctx, M, OpSponge{k}, s);
}

// stage 1: tendencies of U^n (explicit, and the implicit ones with the pressure of U^n)
int phase_stage1(dg_ctx* ctx, std::vector<Member>& M, cudaStream_t s) {
  int rc;
  if ((rc = launch_pack(ctx, M, OpPressure{}, s)) != DG_OK) return rc;
  if ((rc = phase_explicit(ctx, M, 0, s)) != DG_OK) return rc;
  if ((rc = launch_dg(ctx, M, 1, 0, s)) != DG_OK) return rc;
  if ((rc = launch_pack(ctx, M, OpHm{0}, s)) != DG_OK) return rc;
  if ((rc = launch_dg(ctx, M, 2, 0, s)) != DG_OK) return rc;
  return launch_pack(ctx, M, OpImplicitTerms{0}, s);
}

int phase_stage_begin(dg_ctx* ctx, std::vector<Member>& M, int i, cudaStream_t s) {
  OpStageCombine op{};
  op.stage = i;
  for (int j = 0; j < i; ++j) {
    op.ae[j] = AEX[i][j];
    op.ai[j] = AIM[i][j];
  }
  op.aii = AIM[i][i];
  return launch_pack(ctx, M, op, s);
}

// right-hand side of the Helmholtz problem for the current Picard iterate
int phase_picard_pre(dg_ctx* ctx, std::vector<Member>& M, int i, cudaStream_t s) {
  int rc;
  for (auto& mm : M)
    if (mm.nsolve >= 64) return fail(DG_EINVAL, "too many Picard iterations per step (at most 32)");
  if ((rc = launch_pack(ctx, M, OpPicardPrep{}, s)) != DG_OK) return rc;
  if ((rc = launch_dg(ctx, M, 2, 0, s)) != DG_OK) return rc;
  return launch_pack(ctx, M, OpRhsFinish{AIM[i][i], M[0].o.precision == DG_FP32 ? 1 : 0}, s);
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
  const int pi = M.o.precision == DG_FP32 ? 1 : 0;
  if (!auto_k && (M.o.fused >= 0 || persistent_only(M.o.krylov))) {
    set_partition(M.m, M.m->tuned_part[pi]);
    return helmholtz_solve(M.S, &M.o, dta * dta, &M.st, out, s);
  }
  const int ncand = auto_k ? 3 : 2;
  const int nparts = M.m->n_parts;
  float* ms[2] = {M.m->tuned_ms[pi], M.m->tuned_ms_balanced[pi]};
  bool timed = true;
  for (int pt = 0; pt < nparts; ++pt)
    for (int f = 0; f < ncand; ++f) timed = timed && ms[pt][f] > 0.0f;
  dg_solver_opts o = M.o;
  if (timed) {
    int best = 0, bpart = 0;
    for (int pt = 0; pt < nparts; ++pt)
      for (int f = 0; f < ncand; ++f)
        if (ms[pt][f] < ms[bpart][best]) {
          best = f;
          bpart = pt;
        }
    M.m->tuned_form[pi] = best;
    M.m->tuned_part[pi] = bpart;
    set_partition(M.m, bpart);
    apply_form(o, best);
    return helmholtz_solve(M.S, &o, dta * dta, &M.st, out, s);
  }
  dg_state* S = M.S;
  DG_CUDA(cudaMemcpyAsync(S->p_save, S->p, S->Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  constexpr int kMaxCand = 2 * N_FORMS;
  cudaEvent_t e[kMaxCand + 1];
  for (auto& ev : e) DG_CUDA(cudaEventCreate(&ev));
  int rc = DG_OK;
  bool first = true;
  const dg_step_stats st0 = M.st;  // only the last (kept) solve counts in the step's statistics
  // candidates: per cell partition, persistent GMRES, Chebyshev, multi-kernel GMRES (the last
  // one's result is kept: multi-kernel GMRES on the uniform partition)
  int order[kMaxCand], opart[kMaxCand], no = 0;
  for (int pt = nparts - 1; pt >= 0; --pt) {
    order[no] = FORM_GMRES_PERSISTENT;
    opart[no++] = pt;
    if (auto_k) {
      order[no] = FORM_CHEBYSHEV;
      opart[no++] = pt;
    }
    order[no] = FORM_GMRES_MULTI;
    opart[no++] = pt;
  }
  for (int round = 0; round < 2 && rc == DG_OK; ++round) {
    for (int c = 0; c < no && rc == DG_OK; ++c) {
      M.st = st0;
      if (!first) DG_CUDA(cudaMemcpyAsync(S->p, S->p_save, S->Nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      first = false;
      apply_form(o, order[c]);
      set_partition(M.m, opart[c]);
      if (round == 1) DG_CUDA(cudaEventRecord(e[c], s));
      rc = helmholtz_solve(S, &o, dta * dta, &M.st, out, s);
    }
  }
  if (rc == DG_OK) {
    DG_CUDA(cudaEventRecord(e[no], s));
    DG_CUDA(cudaEventSynchronize(e[no]));
    int best = -1, bpart = 0;
    for (int c = 0; c < no; ++c) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, e[c], e[c + 1]);
      ms[opart[c]][order[c]] = t > 0.0f ? t : 1e-6f;
      if (best < 0 || ms[opart[c]][order[c]] < ms[bpart][best]) {
        best = order[c];
        bpart = opart[c];
      }
    }
    M.m->tuned_form[pi] = best;
    M.m->tuned_part[pi] = bpart;
  }
  set_partition(M.m, M.m->tuned_part[pi]);
  for (auto& ev : e) cudaEventDestroy(ev);
  return rc;
}

int phase_picard_post(dg_ctx* ctx, std::vector<Member>& M, int i, cudaStream_t s) {
  int rc;
  if ((rc = launch_dg(ctx, M, 1, 1, s)) != DG_OK) return rc;
  return launch_pack(ctx, M, OpMomentum{AIM[i][i]}, s);
}

int phase_stage_end(dg_ctx* ctx, std::vector<Member>& M, int i, cudaStream_t s) {
  int rc;
  if ((rc = launch_pack(ctx, M, OpStageState{}, s)) != DG_OK) return rc;
  if ((rc = phase_explicit(ctx, M, i, s)) != DG_OK) return rc;
  if (i == 1) {
    if ((rc = launch_pack(ctx, M, OpHm{1}, s)) != DG_OK) return rc;
    if ((rc = launch_dg(ctx, M, 2, 0, s)) != DG_OK) return rc;
    if ((rc = launch_pack(ctx, M, OpImplicitTerms{1}, s)) != DG_OK) return rc;
  }
  for (auto& mm : M) std::swap(mm.S->p, mm.S->p_prev);
  return DG_OK;
}

int phase_final(dg_ctx* ctx, std::vector<Member>& M, cudaStream_t s) {
  OpFinal op{};
  for (int j = 0; j < 3; ++j) op.c[j] = BW[j] - AEX[2][j];
  return launch_pack(ctx, M, op, s);
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
  set_partition(m, m->tuned_part[M.o.precision == DG_FP32 ? 1 : 0]);
  return DG_OK;
}

}  // namespace
}  // namespace dg

extern "C" int imex_rk2_step(dg_ctx* ctx, const dg_mesh* m, dg_state* S, double dt, const dg_solver_opts* opts,
                             dg_step_stats* stats, void* stream) {
  std::vector<Member> M(1);
  int rc = prepare_member(M[0], ctx, m, S, dt, opts);
  if (rc != DG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope step_scope(ctx, DG_PROF_STEP, s);
#define RUN(x)                          \
  do {                                  \
    if ((rc = (x)) != DG_OK) return rc; \
  } while (0)
  RUN(phase_stage1(ctx, M, s));
  for (int i = 1; i <= 2; ++i) {
    RUN(phase_stage_begin(ctx, M, i, s));
    for (int it = 0; it < M[0].o.picard; ++it) {
      RUN(phase_picard_pre(ctx, M, i, s));
      RUN(phase_solve_single(M[0], i, s));
      RUN(phase_picard_post(ctx, M, i, s));
    }
    RUN(phase_stage_end(ctx, M, i, s));
  }
  RUN(phase_final(ctx, M, s));
#undef RUN
  int flag = 0;
  double sol[256];
  DG_CUDA(cudaMemcpyAsync(&flag, S->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaMemcpyAsync(sol, S->solve_out, 4 * M[0].nsolve * sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  const int status = member_finish(M[0], sol, flag);
  if (stats) *stats = M[0].st;
  return status;
}

namespace dg {
namespace {

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

// One IMEX-RK2 step of every member: each phase is one packed launch per
// operation over all members (per (dimension, degree) group for the DG
// operators), between the batched solves of each Picard iteration.
int batch_phases(dg_ctx* ctx, std::vector<Member>& M, const dg_solver_opts& o, int* err, cudaStream_t s) {
  int rc;
#define RUN(x)                          \
  do {                                  \
    if ((rc = (x)) != DG_OK) return rc; \
  } while (0)
  RUN(phase_stage1(ctx, M, s));
  for (int i = 1; i <= 2; ++i) {
    RUN(phase_stage_begin(ctx, M, i, s));
    for (int it = 0; it < o.picard; ++it) {
      RUN(phase_picard_pre(ctx, M, i, s));
      RUN(solve_all(ctx, M, o, i, err, s));
      RUN(phase_picard_post(ctx, M, i, s));
    }
    RUN(phase_stage_end(ctx, M, i, s));
  }
  RUN(phase_final(ctx, M, s));
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
  if ((rc = batch_phases(ctx, M, M[0].o, err, s)) != DG_OK) return rc;
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
  const bool prof = ctx->prof, prof_clocks = ctx->prof_clocks;
  const long long launches0 = ctx->launches;
  ctx->prof = false;
  ctx->prof_clocks = false;
  ctx->arena = &P->arena;
  int* err = ctx->d_batch_err;
  e = cudaStreamBeginCapture(P->cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = DG_OK;
    e = cudaMemsetAsync(err, 0, sizeof(int), P->cs);
    if (e != cudaSuccess) rc = cuda_fail(e, "batch plan capture");
    if (rc == DG_OK) rc = batch_phases(ctx, P->M, o, err, P->cs);
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
  ctx->prof_clocks = prof_clocks;
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
