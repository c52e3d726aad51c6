// Context, error reporting and the operator entry points of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_device.cuh"
#include "ops.h"

namespace dg {

namespace {
thread_local std::string g_last_error;
// profiling words on the device: 16 phase accumulators, then 3 x 512 per-CTA pass clocks
constexpr size_t kPhaseWords = 16 + 3 * 512;
}

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(DG_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Deterministic FP64 sums of w J rho and w J rho E: fixed grid, per-block tree,
// then one block adds the block partials in index order.
constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) conservation_partial(const double* __restrict__ U,
                                                                   const double* __restrict__ wJ, int64_t Nn,
                                                                   int V, double* __restrict__ partial) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double w = wJ[i];
    a += w * U[i];
    b += w * U[(int64_t)(V - 1) * Nn + i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s0[threadIdx.x] += s0[threadIdx.x + st];
      s1[threadIdx.x] += s1[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0[0];
    partial[gridDim.x + blockIdx.x] = s1[0];
  }
}

__global__ void __launch_bounds__(kRedThreads) conservation_final(const double* __restrict__ partial, int nblk,
                                                                 double* __restrict__ out) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += partial[i];
    b += partial[nblk + i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s0[threadIdx.x] += s0[threadIdx.x + st];
      s1[threadIdx.x] += s1[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

size_t prof_begin(dg_ctx* c, cudaStream_t s) {
  if (!c || !c->prof) return SIZE_MAX;
  if (c->ev_next + 2 > c->ev_pool.size()) prof_resolve(c);
  const size_t i = c->ev_next;
  c->ev_next += 2;
  cudaEventRecord(c->ev_pool[i], s);
  return i;
}

void prof_end(dg_ctx* c, int cat, size_t tok, cudaStream_t s) {
  if (!c || tok == SIZE_MAX) return;
  cudaEventRecord(c->ev_pool[tok + 1], s);
  c->ev_pending.emplace_back(cat, tok);
}

void prof_resolve(dg_ctx* c) {
  cudaDeviceSynchronize();
  for (const auto& pr : c->ev_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[pr.second], c->ev_pool[pr.second + 1]) == cudaSuccess) {
      c->prof_ms[pr.first] += ms;
      c->prof_n[pr.first] += 1;
    }
  }
  c->ev_pending.clear();
  c->ev_next = 0;
}

int conservation(const dg_mesh* m, const double* U, double* out, double* partial, cudaStream_t s) {
  count_launches(m->ctx, 2);
  conservation_partial<<<kRedBlocks, kRedThreads, 0, s>>>(U, m->v64.wJ, m->Nn, m->V, partial);
  conservation_final<<<1, kRedThreads, 0, s>>>(partial, kRedBlocks, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "conservation launch");
  return DG_OK;
}

// Host evaluation of the background and the initial states (setup only).
void host_background(const dg_mesh* m, std::vector<double>& Ubg) {
  const int64_t Nn = m->Nn;
  const int V = m->V;
  Ubg.assign((size_t)V * Nn, 0.0);
  std::vector<double> rb(Nn), pb(Nn);
  cudaMemcpy(rb.data(), m->v64.rhob, Nn * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(pb.data(), m->v64.pb, Nn * sizeof(double), cudaMemcpyDeviceToHost);
  for (int64_t i = 0; i < Nn; ++i) {
    Ubg[i] = rb[i];
    Ubg[(size_t)(V - 1) * Nn + i] = pb[i] / (kGamma - 1.0);
  }
}

}  // namespace dg

using namespace dg;

extern "C" const char* dg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* dg_version(void) { return "dg_atmo 0.1 (sm_103a)"; }

extern "C" int dg_ctx_create(int device, dg_ctx** out) {
  if (!out) return fail(DG_EINVAL, "null argument");
  int n = 0;
  DG_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(DG_EINVAL, "no such CUDA device");
  DG_CUDA(cudaSetDevice(device));
  dg_ctx* c = new (std::nothrow) dg_ctx();
  if (!c) return fail(DG_ENOMEM, "host allocation failed");
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return DG_OK;
}

extern "C" int dg_ctx_destroy(dg_ctx* c) {
  if (!c) return DG_OK;
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->d_phase) cudaFree(c->d_phase);
  if (c->d_batch) cudaFree(c->d_batch);
  if (c->d_batch_err) cudaFree(c->d_batch_err);
  delete c;
  return DG_OK;
}

extern "C" int dg_profile_enable(dg_ctx* c, int on) {
  if (!c) return fail(DG_EINVAL, "null context");
  if (on && c->ev_pool.empty()) {
    c->ev_pool.resize(8192);
    for (auto& e : c->ev_pool) DG_CUDA(cudaEventCreate(&e));
  }
  if (on && !c->d_phase) {
    DG_CUDA(cudaMalloc(&c->d_phase, kPhaseWords * sizeof(unsigned long long)));
    DG_CUDA(cudaMemset(c->d_phase, 0, kPhaseWords * sizeof(unsigned long long)));
  }
  if (!on && c->prof) prof_resolve(c);
  c->prof = on != 0;
  c->prof_clocks = on >= 2;
  return DG_OK;
}

extern "C" int dg_profile_read(dg_ctx* c, double* ms, long long* counts) {
  if (!c) return fail(DG_EINVAL, "null context");
  prof_resolve(c);
  for (int i = 0; i < DG_PROF_N; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (counts) counts[i] = c->prof_n[i];
  }
  return DG_OK;
}

extern "C" int dg_batch_barrier_test(dg_ctx* c, double barrier_limit_s, int missing_cta_member) {
  if (!c) return fail(DG_EINVAL, "null context");
  if (!(barrier_limit_s >= 1e-3 && barrier_limit_s <= 10.0)) return fail(DG_EINVAL, "barrier limit must be in 1e-3..10 s");
  if (missing_cta_member < -1) return fail(DG_EINVAL, "missing_cta_member must be >= -1");
  c->batch_timeout_ns = (unsigned long long)(barrier_limit_s * 1e9);
  c->batch_missing_cta_member = missing_cta_member;
  return DG_OK;
}

extern "C" int dg_launch_count(const dg_ctx* c, long long* out) {
  if (!c || !out) return fail(DG_EINVAL, "null argument");
  *out = c->launches;
  return DG_OK;
}

extern "C" int dg_profile_read_gmres_phases(dg_ctx* c, double* ns) {
  if (!c || !ns) return fail(DG_EINVAL, "null argument");
  unsigned long long h[16] = {0};
  if (c->d_phase) {
    DG_CUDA(cudaDeviceSynchronize());
    DG_CUDA(cudaMemcpy(h, c->d_phase, sizeof(h), cudaMemcpyDeviceToHost));
  }
  for (int i = 0; i < 16; ++i) ns[i] = (double)h[i];
  return DG_OK;
}

extern "C" int dg_profile_read_cta_passes(dg_ctx* c, double* grad_ns, double* div_ns, int* coarse, int max_ctas) {
  if (!c || max_ctas < 0 || (max_ctas > 0 && (!grad_ns || !div_ns || !coarse))) return fail(DG_EINVAL, "bad arguments");
  std::vector<unsigned long long> h(kPhaseWords, 0ull);
  if (c->d_phase) {
    DG_CUDA(cudaDeviceSynchronize());
    DG_CUDA(cudaMemcpy(h.data(), c->d_phase, kPhaseWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  }
  const int n = std::min(max_ctas, 512);
  for (int i = 0; i < n; ++i) {
    grad_ns[i] = (double)h[16 + i];
    div_ns[i] = (double)h[16 + 512 + i];
    coarse[i] = (int)h[16 + 1024 + i];
  }
  return DG_OK;
}

extern "C" int dg_profile_reset(dg_ctx* c) {
  if (!c) return fail(DG_EINVAL, "null context");
  prof_resolve(c);
  if (c->d_phase) DG_CUDA(cudaMemset(c->d_phase, 0, kPhaseWords * sizeof(unsigned long long)));
  for (int i = 0; i < DG_PROF_N; ++i) {
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return DG_OK;
}

extern "C" int dg_apply_explicit(dg_ctx* ctx, const dg_mesh* m, const void* U, void* R, int precision, int terms,
                                 void* stream) {
  if (!ctx || !m || !U || !R) return fail(DG_EINVAL, "null argument");
  if (terms != DG_TERMS_FULL && terms != DG_TERMS_IMEX_EXPLICIT) return fail(DG_EINVAL, "bad terms");
  cudaStream_t s = (cudaStream_t)stream;
  const bool full = terms == DG_TERMS_FULL;
  if (precision == DG_FP64)
    return op_explicit<double>(m, (const double*)U, (double*)R, m->d_face_scratch64, full, s, nullptr);
  if (precision == DG_FP32)
    return op_explicit<float>(m, (const float*)U, (float*)R, (float*)m->d_face_scratch64, full, s, nullptr);
  return fail(DG_EINVAL, "bad precision");
}

extern "C" int dg_apply_grad(dg_ctx* ctx, const dg_mesh* m, const void* p, const void* h, void* g, int precision,
                             void* stream) {
  if (!ctx || !m || !p || !g) return fail(DG_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == DG_FP64)
    return op_grad<double>(m, (const double*)p, (const double*)h, (double*)g, s, nullptr);
  if (precision == DG_FP32)
    return op_grad<float>(m, (const float*)p, (const float*)h, (float*)g, s, nullptr);
  return fail(DG_EINVAL, "bad precision");
}

extern "C" int dg_apply_div(dg_ctx* ctx, const dg_mesh* m, const void* f, void* out, int precision, void* stream) {
  if (!ctx || !m || !f || !out) return fail(DG_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == DG_FP64)
    return op_div<double>(m, (const double*)f, (double*)out, s, nullptr);
  if (precision == DG_FP32)
    return op_div<float>(m, (const float*)f, (float*)out, s, nullptr);
  return fail(DG_EINVAL, "bad precision");
}

extern "C" int dg_apply_implicit(dg_ctx* ctx, const dg_mesh* m, const void* h, const void* p, void* Ap,
                                 double alpha, int precision, void* stream) {
  if (!ctx || !m || !h || !p || !Ap) return fail(DG_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == DG_FP64)
    return op_helmholtz<double>(m, (const double*)h, (const double*)p, (double*)Ap, alpha, m->d_vec_scratch64, s,
                                nullptr);
  if (precision == DG_FP32)
    return op_helmholtz<float>(m, (const float*)h, (const float*)p, (float*)Ap, (float)alpha,
                               (float*)m->d_vec_scratch64, s, nullptr);
  return fail(DG_EINVAL, "bad precision");
}

extern "C" int dg_conservation(dg_ctx* ctx, const dg_mesh* m, const double* U, double* out, void* stream) {
  if (!ctx || !m || !U || !out) return fail(DG_EINVAL, "null argument");
  return conservation(m, U, out, m->d_red_scratch, (cudaStream_t)stream);
}

extern "C" int dg_background(dg_ctx* ctx, const dg_mesh* m, double* Ubg, void* stream) {
  if (!ctx || !m || !Ubg) return fail(DG_EINVAL, "null argument");
  std::vector<double> h;
  host_background(m, h);
  DG_CUDA(cudaMemcpyAsync(Ubg, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return DG_OK;
}

extern "C" int dg_init_state(dg_ctx* ctx, const dg_mesh* m, int kind, const double* params, int n_params,
                             double* U, void* stream) {
  if (!ctx || !m || !U) return fail(DG_EINVAL, "null argument");
  std::vector<double> h;
  host_background(m, h);
  const int64_t Nn = m->Nn, K = m->K;
  const int V = m->V, dim = m->dim, nc = m->nc;
  const dg_mesh_desc& d = m->desc;
  if (kind == DG_INIT_REST) {
  } else if (kind == DG_INIT_BUBBLE) {
    if (n_params < 4 || !params) return fail(DG_EINVAL, "bubble needs amp, radius, xc, zc");
    if (d.atm_kind == DG_ATM_NONE) return fail(DG_EINVAL, "bubble needs a background atmosphere");
    const double amp = params[0], R = params[1], xc = params[2], zc = params[3];
    const double yc = n_params > 4 ? params[4] : 0.5 * d.extent[1];
    const double pi = 3.14159265358979323846;
    for (int64_t c = 0; c < K; ++c)
      for (int q = 0; q < nc; ++q) {
        const int64_t i = c * nc + q;
        const double x = m->X[(size_t)c * nc + q];
        const double z = m->X[((size_t)(dim - 1) * K + c) * nc + q];
        double r2 = (x - xc) * (x - xc) + (z - zc) * (z - zc);
        if (dim == 3) {
          const double y = m->X[((size_t)K + c) * nc + q];
          r2 += (y - yc) * (y - yc);
        }
        const double r = std::sqrt(r2);
        if (r >= R) continue;
        const double cc = std::cos(0.5 * pi * r / R);
        const double dth = amp * cc * cc;
        const double rho_b = h[i];
        const double p_b = h[(size_t)(V - 1) * Nn + i] * (kGamma - 1.0);
        const double exner = std::pow(p_b / d.atm_p_ref, (kGamma - 1.0) / kGamma);
        const double T = p_b / (kRgas * rho_b) + dth * exner;
        h[i] = p_b / (kRgas * T);
      }
  } else if (kind == DG_INIT_INFLOW) {
    const double u0 = (params && n_params > 0) ? params[0] : 10.0;
    for (int64_t i = 0; i < Nn; ++i) {
      const double rho = h[i];
      h[(size_t)Nn + i] = rho * u0;
      h[(size_t)(V - 1) * Nn + i] += 0.5 * rho * u0 * u0;
    }
  } else {
    return fail(DG_EINVAL, "unknown initial state kind");
  }
  DG_CUDA(cudaMemcpyAsync(U, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return DG_OK;
}

__global__ void dg_newton_selftest_kernel(int op, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (op == 0) y[i] = dg::rsqrt64(x[i]);
}

extern "C" int dg_math_selftest(int op, const double* x, double* y, int64_t n, void* stream) {
  if (op != 0 || n < 0 || (n > 0 && (!x || !y))) return dg::fail(DG_EINVAL, "bad arguments");
  if (n == 0) return DG_OK;
  dg_newton_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(op, x, y, n);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}
