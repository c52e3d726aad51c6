// Device GMRES(m): kernels and the host loop over restart cycles.
#include <cmath>

#include "krylov.cuh"

namespace dg {

namespace {

__device__ __forceinline__ bool skipped(const int* f) { return f && *f; }

// partial[j*kDotBlocks + bx] = sum over this block's chunk of Q_j . w
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(kDotThreads) multi_dot_kernel(const Ta* __restrict__ Q, int64_t ld,
                                                               const Tb* __restrict__ w, int64_t n,
                                                               double* __restrict__ partial, const int* skip) {
  if (skipped(skip)) return;
  __shared__ double sm[kDotThreads];
  const int j = blockIdx.y;
  const Ta* q = Q + (int64_t)j * ld;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)q[i] * (double)w[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = sm[0];
}

// out[j] = sum_b partial[j*nb + b], one block per j, fixed order
__global__ void __launch_bounds__(kDotThreads) finalize_kernel(const double* __restrict__ partial, int nb,
                                                              double* __restrict__ out, const int* skip) {
  if (skipped(skip)) return;
  __shared__ double sm[kDotThreads];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[(int64_t)j * nb + i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sm[0];
}

// w += sign * sum_{j<nvec} c[j] Q_j ; nvec from the host, or from *nvec_dev when >= 0 is not given
template <typename Tv>
__global__ void multi_axpy_kernel(Tv* __restrict__ w, const Tv* __restrict__ Q, int64_t ld, int64_t n,
                                  const double* __restrict__ c, int nvec, const int* nvec_dev, double sign,
                                  const int* skip) {
  if (skipped(skip)) return;
  const int nv = nvec_dev ? *nvec_dev : nvec;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < nv; ++j) acc += c[j] * (double)Q[(int64_t)j * ld + i];
    w[i] = (Tv)((double)w[i] + sign * acc);
  }
}

// out = a * (b - in)  with a from a device scalar (or 1)
template <typename Tv>
__global__ void residual_kernel(const Tv* __restrict__ b, const Tv* __restrict__ Ax, Tv* __restrict__ r, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Ax[i];
}

template <typename Tv>
__global__ void scale_kernel(const Tv* __restrict__ in, Tv* __restrict__ out, int64_t n,
                             const double* __restrict__ factor, const int* skip) {
  if (skipped(skip)) return;
  const double f = *factor;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (Tv)((double)in[i] * f);
}

template <typename Tv>
__global__ void zero_if_kernel(Tv* __restrict__ x, int64_t n, const int* flag) {
  if (!*flag) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = Tv(0);
}

// start of a restart cycle: beta = ||r||, g = (beta, 0, ...), 1/beta for Q_0
__global__ void cycle_start_kernel(GmresDev d, int m) {
  const double bn = sqrt(d.scal[0]);
  const double beta = sqrt(d.scal[1]);
  const double tol = d.scal[5];
  d.iflag[1] = 0;
  d.iflag[2] = 0;
  for (int j = 0; j <= m; ++j) d.g[j] = 0.0;
  d.g[0] = beta;
  d.scal[2] = beta;
  if (bn == 0.0) {
    d.iflag[0] = 1;
    d.iflag[2] = 1;
    d.scal[2] = 0.0;
    return;
  }
  d.iflag[0] = (beta <= tol * bn || beta == 0.0) ? 1 : 0;
  d.scal[3] = d.iflag[0] ? 0.0 : 1.0 / beta;
}

// column k of H from the two Gram-Schmidt passes and ||w||; Givens update
__global__ void arnoldi_finish_kernel(GmresDev d, int m, int kmax, int k) {
  if (d.iflag[0]) return;
  const int ld = m + 1;
  double* col = d.H + (int64_t)k * ld;
  for (int j = 0; j <= k; ++j) col[j] = d.h1[j] + d.h2[j];
  const double hn = sqrt(d.scal[4]);
  col[k + 1] = hn;
  for (int j = 0; j < k; ++j) {
    const double t = d.cs[j] * col[j] + d.sn[j] * col[j + 1];
    col[j + 1] = -d.sn[j] * col[j] + d.cs[j] * col[j + 1];
    col[j] = t;
  }
  const double den = hypot(col[k], col[k + 1]);
  const double c = den > 0.0 ? col[k] / den : 1.0;
  const double s = den > 0.0 ? col[k + 1] / den : 0.0;
  d.cs[k] = c;
  d.sn[k] = s;
  col[k] = den;
  col[k + 1] = 0.0;
  d.g[k + 1] = -s * d.g[k];
  d.g[k] = c * d.g[k];
  d.iflag[1] = k + 1;
  const double resid = fabs(d.g[k + 1]);
  d.scal[2] = resid;
  const double bn = sqrt(d.scal[0]);
  if (resid <= d.scal[5] * bn || hn == 0.0 || k + 1 == kmax) {
    d.iflag[0] = 1;
    d.scal[3] = 0.0;
  } else {
    d.scal[3] = 1.0 / hn;
  }
}

// back substitution for y over the kdone iterations of this cycle
__global__ void solve_y_kernel(GmresDev d, int m) {
  const int kd = d.iflag[1];
  const int ld = m + 1;
  for (int i = kd - 1; i >= 0; --i) {
    double s = d.g[i];
    for (int j = i + 1; j < kd; ++j) s -= d.H[(int64_t)j * ld + i] * d.y[j];
    d.y[i] = s / d.H[(int64_t)i * ld + i];
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

template <typename Ta, typename Tb>
int dot_into(const Ta* a, const Tb* b, int64_t n, double* partial, double* out, cudaStream_t s, const int* skip) {
  multi_dot_kernel<Ta, Tb><<<dim3(kDotBlocks, 1), kDotThreads, 0, s>>>(a, n, b, n, partial, skip);
  finalize_kernel<<<1, kDotThreads, 0, s>>>(partial, kDotBlocks, out, skip);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "dot launch");
}
template int dot_into<double, double>(const double*, const double*, int64_t, double*, double*, cudaStream_t,
                                      const int*);
template int dot_into<float, float>(const float*, const float*, int64_t, double*, double*, cudaStream_t,
                                    const int*);

template <typename Tv>
int Gmres<Tv>::init(int64_t n_, int m_) {
  n = n_;
  m = m_;
  const size_t vec_bytes = ((size_t)(m + 2) * n + 64) * sizeof(Tv);
  const size_t small = ((size_t)(m + 1) * m + 2 * m + 4 * (m + 1) + (size_t)(m + 1) * kDotBlocks + 8) * sizeof(double) +
                       16 * sizeof(int);
  DG_CUDA(cudaMalloc(&block, vec_bytes + small + 256));
  char* p = (char*)block;
  Q = (Tv*)p;
  w = Q + (size_t)(m + 1) * n;
  p += (vec_bytes + 255) & ~(size_t)255;
  double* dp = (double*)p;
  d.H = dp;
  dp += (size_t)(m + 1) * m;
  d.cs = dp;
  dp += m;
  d.sn = dp;
  dp += m;
  d.g = dp;
  dp += m + 1;
  d.h1 = dp;
  dp += m + 1;
  d.h2 = dp;
  dp += m + 1;
  d.y = dp;
  dp += m + 1;
  d.partial = dp;
  dp += (size_t)(m + 1) * kDotBlocks;
  d.scal = dp;
  dp += 8;
  d.iflag = (int*)dp;
  DG_CUDA(cudaMemset(d.iflag, 0, 16 * sizeof(int)));
  return DG_OK;
}

template <typename Tv>
void Gmres<Tv>::release() {
  if (block) cudaFree(block);
  block = nullptr;
}

template <typename Tv>
int Gmres<Tv>::solve(dg_ctx* ctx, const std::function<int(const Tv*, Tv*, const int*)>& apply, const Tv* b, Tv* x,
                     double tol, int max_iters, cudaStream_t s, GmresResult* res) {
  int st;
  const unsigned gb = grid_for(n);
  int* done = d.iflag;
  int total = 0;
  double hbuf[3];
  int ibuf[3];
  // ||b||^2 and the tolerance
  if ((st = dot_into<Tv, Tv>(b, b, n, d.partial, d.scal + 0, s, nullptr)) != DG_OK) return st;
  count_launches(ctx, 2);
  DG_CUDA(cudaMemcpyAsync(d.scal + 5, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
  res->converged = false;
  for (int cycle = 0;; ++cycle) {
    // r = b - A x -> Q_0 (unnormalised), beta^2
    if ((st = apply(x, w, nullptr)) != DG_OK) return st;
    residual_kernel<Tv><<<gb, 256, 0, s>>>(b, w, Q, n);
    count_launches(ctx, 6);
    if ((st = dot_into<Tv, Tv>(Q, Q, n, d.partial, d.scal + 1, s, nullptr)) != DG_OK) return st;
    cycle_start_kernel<<<1, 1, 0, s>>>(d, m);
    zero_if_kernel<Tv><<<gb, 256, 0, s>>>(x, n, d.iflag + 2);
    scale_kernel<Tv><<<gb, 256, 0, s>>>(Q, Q, n, d.scal + 3, done);
    const int kmax = std::min(m, std::max(1, max_iters - total));
    for (int k = 0; k < kmax; ++k) {
      Tv* qk = Q + (size_t)k * n;
      if ((st = apply(qk, w, done)) != DG_OK) return st;
      ProfScope ps(ctx, DG_PROF_KRYLOV, s);
      count_launches(ctx, 10);
      multi_dot_kernel<Tv, Tv><<<dim3(kDotBlocks, k + 1), kDotThreads, 0, s>>>(Q, n, w, n, d.partial, done);
      finalize_kernel<<<k + 1, kDotThreads, 0, s>>>(d.partial, kDotBlocks, d.h1, done);
      multi_axpy_kernel<Tv><<<gb, 256, 0, s>>>(w, Q, n, n, d.h1, k + 1, nullptr, -1.0, done);
      multi_dot_kernel<Tv, Tv><<<dim3(kDotBlocks, k + 1), kDotThreads, 0, s>>>(Q, n, w, n, d.partial, done);
      finalize_kernel<<<k + 1, kDotThreads, 0, s>>>(d.partial, kDotBlocks, d.h2, done);
      multi_axpy_kernel<Tv><<<gb, 256, 0, s>>>(w, Q, n, n, d.h2, k + 1, nullptr, -1.0, done);
      if ((st = dot_into<Tv, Tv>(w, w, n, d.partial, d.scal + 4, s, done)) != DG_OK) return st;
      arnoldi_finish_kernel<<<1, 1, 0, s>>>(d, m, kmax, k);
      scale_kernel<Tv><<<gb, 256, 0, s>>>(w, Q + (size_t)(k + 1) * n, n, d.scal + 3, done);
    }
    solve_y_kernel<<<1, 1, 0, s>>>(d, m);
    count_launches(ctx, 2);
    multi_axpy_kernel<Tv><<<gb, 256, 0, s>>>(x, Q, n, n, d.y, 0, d.iflag + 1, 1.0, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gmres launch");
    DG_CUDA(cudaMemcpyAsync(hbuf, d.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaMemcpyAsync(ibuf, d.iflag, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    total += ibuf[1];
    const double bn = std::sqrt(hbuf[0]);
    res->iters = total;
    res->rel = bn > 0 ? hbuf[2] / bn : 0.0;
    if (ibuf[2] || res->rel <= tol) {
      res->converged = true;
      res->rel = ibuf[2] ? 0.0 : res->rel;
      return DG_OK;
    }
    if (total >= max_iters || (ibuf[1] == 0 && cycle > 0)) return DG_OK;
  }
}

template struct Gmres<double>;
template struct Gmres<float>;

}  // namespace dg
