// Launcher bodies of the operator kernels, one function per (dimension,
// degree, precision).  The build compiles this header once per combination,
// in translation units of its own (generated by build.py) that instantiate
// them with DG_INSTANTIATE_DEGREE; ops_dispatch.cu picks among them at run
// time by the mesh's degree.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "k_explicit.cuh"
#include "k_gmres.cuh"
#include "k_implicit.cuh"
#include "k_pack.cuh"
#include "ops.h"

namespace dg {

namespace {

inline int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return DG_OK;
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

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

// Gradient and divergence, one launch each, face terms computed by the cells
// (k_implicit.cuh, standalone one-pass kernels); FP32 on meshes affine in x
// and y recomputes the metric terms from the nodal heights.
template <int DIM, int DEG, typename T>
int run_grad(const dg_mesh* m, const T* p, const T* h, T* g, cudaStream_t s, const int* skip) {
  using S = Shape<DIM, DEG>;
  const MeshView<T>& mv = view<T>(m);
  const unsigned nb = (unsigned)mv.nbat;
  count_launches(m->ctx, 1);
  if (std::is_same<T, float>::value && mv.geo_z)
    grad_cell_kernel<DIM, DEG, T, true, true><<<nb, S::THREADS, 0, s>>>(mv, p, h, g, skip);
  else if (mv.aff)
    grad_cell_kernel<DIM, DEG, T, false, true><<<nb, S::THREADS, 0, s>>>(mv, p, h, g, skip);
  else
    grad_cell_kernel<DIM, DEG, T, false, false><<<nb, S::THREADS, 0, s>>>(mv, p, h, g, skip);
  return check_launch("gradient launch");
}

template <int DIM, int DEG, typename T, bool HELM>
int run_div(const dg_mesh* m, const T* f, const T* p, T alpha, T* out, cudaStream_t s, const int* skip) {
  using S = Shape<DIM, DEG>;
  const MeshView<T>& mv = view<T>(m);
  const unsigned nb = (unsigned)mv.nbat;
  count_launches(m->ctx, 1);
  if (std::is_same<T, float>::value && mv.geo_z)
    div_cell_kernel<DIM, DEG, T, HELM, true, true><<<nb, S::THREADS, 0, s>>>(mv, f, p, alpha, out, skip);
  else if (mv.aff)
    div_cell_kernel<DIM, DEG, T, HELM, false, true><<<nb, S::THREADS, 0, s>>>(mv, f, p, alpha, out, skip);
  else
    div_cell_kernel<DIM, DEG, T, HELM, false, false><<<nb, S::THREADS, 0, s>>>(mv, f, p, alpha, out, skip);
  return check_launch("divergence launch");
}

// Packed operators: the CTA ranges of the members, then one launch per pass.
template <int DIM, int DEG, typename T>
int run_explicit_pack(dg_ctx* ctx, OpPack<T>& P, bool full, cudaStream_t s) {
  using S = Shape<DIM, DEG>;
  int nb = 0;
  for (int j = 0; j < P.n; ++j) {
    P.start[j] = nb;
    nb += (int)blocks_for((int64_t)P.mv[j].nf * S::NF, 256);
  }
  P.start[P.n] = nb;
  if (nb > 0) {
    if (full)
      explicit_face_pack_kernel<DIM, DEG, T, true, false><<<nb, 256, 0, s>>>(P);
    else
      explicit_face_pack_kernel<DIM, DEG, T, false, false><<<nb, 256, 0, s>>>(P);
    count_launches(ctx, 1);
  }
  nb = 0;
  for (int j = 0; j < P.n; ++j) {
    P.start[j] = nb;
    nb += (int)blocks_for(P.mv[j].n_cells, S::CPB);
  }
  P.start[P.n] = nb;
  if (full)
    explicit_cell_pack_kernel<DIM, DEG, T, true, false><<<nb, S::THREADS, 0, s>>>(P);
  else
    explicit_cell_pack_kernel<DIM, DEG, T, false, false><<<nb, S::THREADS, 0, s>>>(P);
  count_launches(ctx, 1);
  return check_launch("packed explicit operator launch");
}

template <int DIM, int DEG, typename T>
int run_grad_pack(dg_ctx* ctx, OpPack<T>& P, cudaStream_t s) {
  using S = Shape<DIM, DEG>;
  int nb = 0;
  for (int j = 0; j < P.n; ++j) {
    P.start[j] = nb;
    nb += P.mv[j].nbat;
  }
  P.start[P.n] = nb;
  grad_pack_kernel<DIM, DEG, T><<<nb, S::THREADS, 0, s>>>(P);
  count_launches(ctx, 1);
  return check_launch("packed gradient launch");
}

template <int DIM, int DEG, typename T>
int run_div_pack(dg_ctx* ctx, OpPack<T>& P, cudaStream_t s) {
  using S = Shape<DIM, DEG>;
  int nb = 0;
  for (int j = 0; j < P.n; ++j) {
    P.start[j] = nb;
    nb += P.mv[j].nbat;
  }
  P.start[P.n] = nb;
  div_pack_kernel<DIM, DEG, T><<<nb, S::THREADS, 0, s>>>(P);
  count_launches(ctx, 1);
  return check_launch("packed divergence launch");
}

template <int DIM, int DEG, typename TK>
int run_gmres(const dg_mesh* m, const double* h64, const TK* hk, const double* b, double* x, double alpha,
              double tol, double inner_tol, int restart, int max_iters, int method, TK* Q, TK* w, double* w64,
              double* partial, int npartial, double* out, double* lmax, unsigned long long* phase,
              cudaStream_t s) {
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
  a.gv = m->d_vec_scratch64;
  a.partial = partial;
  a.out = out;
  a.lmax = lmax;
  a.lmax = lmax;
  a.phase = phase;
  a.alpha = alpha;
  a.tol = tol;
  a.inner_tol = inner_tol;
  a.m = restart;
  a.max_iters = max_iters;
  a.n = m->Nn;
  a.method = method;
  if (method == 1 && restart < 2) return fail(DG_EINVAL, "CG needs restart >= 2 (three work vectors)");
  if (method == 3 && !lmax) return fail(DG_EINVAL, "Chebyshev needs a bound buffer");
  const bool aff = a.mvk.aff && a.mv64.aff;
  void (*kern)(GmresPArgs<TK>) = method == 1   ? gmres_persistent_kernel<DIM, DEG, TK, 1>
                                 : method == 2 ? gmres_persistent_kernel<DIM, DEG, TK, 2>
                                 : method == 3 ? (aff ? gmres_persistent_kernel<DIM, DEG, TK, 3, true>
                                                      : gmres_persistent_kernel<DIM, DEG, TK, 3>)
                                               : gmres_persistent_kernel<DIM, DEG, TK, 0>;
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
  if (G > npartial / 3) G = npartial / 3;  // CG stores three partial sums per CTA
  if (G > 512) G = 512;  // staged partial sums in shared memory
  if (G < 1) return fail(DG_EINVAL, "GMRES partial buffer too small");
  count_launches(m->ctx, 1);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(256), args, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "persistent GMRES launch");
  return DG_OK;
}

template <int DIM, int DEG, typename TK>
int run_gmres_batched(dg_ctx* ctx, const GmresItem<TK>* items, int n_items, int restart, int* err,
                      cudaStream_t s) {
  static_assert(sizeof(GmresPArgs<TK>) <= kBatchArgBytes, "argument table entry larger than planned");
  auto kern = gmres_batched_kernel<DIM, DEG, TK>;
  const size_t smem = gmres_smem_bytes<DIM, DEG, TK>(restart);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "batched gmres smem attribute");
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return cuda_fail(e, "batched gmres occupancy");
  if (per_sm < 1) return fail(DG_ECUDA, "batched GMRES kernel does not fit on an SM");
  const int gtot = ctx->sm_count * (per_sm < 2 ? per_sm : 2);
  for (int first = 0; first < n_items; first += gtot) {
    const int B = std::min(gtot, n_items - first);
    const GmresItem<TK>* it = items + first;
    // CTAs in proportion to node counts, at least one each
    std::vector<int> ctas(B, 1);
    double wsum = 0.0;
    for (int i = 0; i < B; ++i) wsum += (double)it[i].m->Nn;
    int used = 0;
    for (int i = 0; i < B; ++i) {
      const int cap = std::max(1, std::min(512, it[i].npartial / 3));
      ctas[i] = std::min(cap, std::max(1, (int)((double)(gtot - B) * it[i].m->Nn / wsum) + 1));
      used += ctas[i];
    }
    while (used > gtot) {  // rounding overshoot: take from the largest
      int j = (int)(std::max_element(ctas.begin(), ctas.end()) - ctas.begin());
      if (ctas[j] <= 1) break;
      --ctas[j];
      --used;
    }
    std::vector<GmresPArgs<TK>> args(B);
    std::vector<int> cta_member, cta_rank;
    for (int i = 0; i < B; ++i) {
      GmresPArgs<TK>& a = args[i];
      const dg_mesh* m = it[i].m;
      a.mv64 = m->v64;
      a.mvk = view<TK>(m);
      a.h64 = it[i].h64;
      a.hk = it[i].hk;
      a.b = it[i].b;
      a.x = it[i].x;
      a.Q = it[i].Q;
      a.w = it[i].w;
      a.w64 = it[i].w64;
      a.gv = m->d_vec_scratch64;
      a.partial = it[i].partial;
      a.out = it[i].out;
      a.lmax = it[i].lmax;
      a.lmax = it[i].lmax;
      a.phase = nullptr;
      a.alpha = it[i].alpha;
      a.tol = it[i].tol;
      a.inner_tol = it[i].inner_tol;
      a.m = restart;
      a.max_iters = it[i].max_iters;
      a.n = m->Nn;
      a.method = it[i].method;
      for (int r = 0; r < ctas[i]; ++r) {
        cta_member.push_back(i);
        cta_rank.push_back(r);
      }
    }
    const int G = (int)cta_member.size();
    const size_t b_args = ((sizeof(GmresPArgs<TK>) * B) + 255) & ~(size_t)255;
    const size_t b_map = (((size_t)2 * G + B) * sizeof(int) + 255) & ~(size_t)255;
    const size_t b_bar = ((size_t)2 * B) * sizeof(unsigned int);
    const size_t need = b_args + b_map + b_bar + 256;
    unsigned char* dev;
    unsigned char* host;
    std::vector<unsigned char> staging;
    if (ctx->arena) {  // graph capture: tables go to the plan's arena, uploaded after the capture
      const size_t off = ctx->arena->take(need);
      if (off == SIZE_MAX) return fail(DG_EINVAL, "batch plan argument arena is full");
      dev = ctx->arena->dev + off;
      host = ctx->arena->host.data() + off;
    } else {
      if (need > ctx->batch_bytes) {
        if (ctx->d_batch) {
          DG_CUDA(cudaStreamSynchronize(s));
          cudaFree(ctx->d_batch);
        }
        ctx->d_batch = nullptr;
        ctx->batch_bytes = 0;
        DG_CUDA(cudaMalloc(&ctx->d_batch, need * 2));
        ctx->batch_bytes = need * 2;
      }
      dev = (unsigned char*)ctx->d_batch;
      staging.assign(b_args + b_map, 0);
      host = staging.data();
    }
    std::memcpy(host, args.data(), sizeof(GmresPArgs<TK>) * B);
    int* hm = (int*)(host + b_args);
    std::memcpy(hm, cta_member.data(), G * sizeof(int));
    std::memcpy(hm + G, cta_rank.data(), G * sizeof(int));
    std::memcpy(hm + 2 * G, ctas.data(), B * sizeof(int));
    const int miss = ctx->batch_missing_cta_member - first;
    // test hook: declare a CTA that never arrives (kept within the partial-sum buffers' bounds)
    if (miss >= 0 && miss < B && ctas[miss] + 1 <= std::min(512, it[miss].npartial / 3)) hm[2 * G + miss] += 1;
    if (!ctx->arena) DG_CUDA(cudaMemcpyAsync(dev, host, b_args + b_map, cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaMemsetAsync(dev + b_args + b_map, 0, b_bar, s));
    BatchMap map;
    const int* dm = (const int*)(dev + b_args);
    map.cta_member = dm;
    map.cta_rank = dm + G;
    map.member_ctas = dm + 2 * G;
    map.bar_count = (unsigned int*)(dev + b_args + b_map);
    map.bar_gen = map.bar_count + B;
    map.err = err;
    map.timeout_ns = ctx->batch_timeout_ns;
    const GmresPArgs<TK>* dargs = (const GmresPArgs<TK>*)dev;
    count_launches(ctx, 1);
    void* kargs[] = {(void*)&dargs, (void*)&map};
    e = cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(256), kargs, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "batched GMRES launch");
    // the shared argument table is rewritten by the next chunk: keep launches ordered
    if (!ctx->arena && first + B < n_items) DG_CUDA(cudaStreamSynchronize(s));
  }
  return DG_OK;
}


#define DG_INSTANTIATE_DEGREE(DIM, DEG, T)                                                                       \
  template int run_explicit<DIM, DEG, T>(const dg_mesh*, const T*, T*, T*, bool, cudaStream_t, const int*);     \
  template int run_grad<DIM, DEG, T>(const dg_mesh*, const T*, const T*, T*, cudaStream_t, const int*);         \
  template int run_div<DIM, DEG, T, false>(const dg_mesh*, const T*, const T*, T, T*, cudaStream_t, const int*); \
  template int run_div<DIM, DEG, T, true>(const dg_mesh*, const T*, const T*, T, T*, cudaStream_t, const int*);  \
  template int run_gmres<DIM, DEG, T>(const dg_mesh*, const double*, const T*, const double*, double*, double,    \
                                      double, double, int, int, int, T*, T*, double*, double*, int, double*,      \
                                      double*, unsigned long long*, cudaStream_t);                               \
  template int run_gmres_batched<DIM, DEG, T>(dg_ctx*, const GmresItem<T>*, int, int, int*, cudaStream_t);     \
  template int run_explicit_pack<DIM, DEG, T>(dg_ctx*, OpPack<T>&, bool, cudaStream_t);                         \
  template int run_grad_pack<DIM, DEG, T>(dg_ctx*, OpPack<T>&, cudaStream_t);                                   \
  template int run_div_pack<DIM, DEG, T>(dg_ctx*, OpPack<T>&, cudaStream_t);

}  // namespace dg
