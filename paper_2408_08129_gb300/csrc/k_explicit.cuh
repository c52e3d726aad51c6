// Explicit DG operator (Eq. (1) discretised in space, Sec. 2), in two passes:
//
//  1. explicit_face_kernel: one thread per face node.  Reads the two traces
//     (on a 2:1 subface the coarse trace is the coarse polynomial of the
//     perturbation evaluated at the fine face node), evaluates the Rusanov
//     normal flux and writes Fh = |N| F*.n into the face scratch buffer.
//     Every face flux is computed exactly once; no atomics.
//  2. explicit_cell_kernel: one thread per node, CPB cells per CTA.  Volume
//     term by sum factorisation (one 1D weak-derivative contraction per axis
//     through shared memory), then the node gathers the face fluxes of the
//     faces it lies on (minus side -Fh, plus side +Fh, coarse side
//     +It Fh over its subfaces), applies M^-1 = 1/(w J) and adds the source.
//
//  R_i = [ sum_a sum_k Dw[i_a][k] Ft^a(k)  - faces / w_end ] / J_i + S_i
#pragma once

#include "dg_device.cuh"

namespace dg {

// Face node t (< nf * NF) of the face pass: Fh[v][t] = |N| F*.n
template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__device__ __forceinline__ void explicit_face_item(const MeshView<T>& mv, const T* __restrict__ U,
                                                   T* __restrict__ Fh, int64_t t) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, NF = S::NF, V = S::V;
  const int64_t total = (int64_t)mv.nf * NF;
  const int f = (int)(t / NF), k = (int)(t % NF);
  const int64_t Nn = mv.n_nodes;
  const int64_t im = mv.fnode_m[t];
  const T rb = mv.rhob[im], pb = mv.pb[im];
  T um[V], up[V], n[DIM];
  load_pert<V, T, PERT>(U, Nn, im, mv.rhob, mv.pb, um);
#pragma unroll
  for (int b = 0; b < DIM; ++b) n[b] = mv.fn[(int64_t)b * total + t];
  const T sj = mv.fsj[t];
  T out[V];
  if (f < mv.nconf + mv.nsub) {
    const int cp = mv.face_p[f], lfp = mv.face_lfp[f];
    if (f < mv.nconf) {
      const int64_t ip = mv.fnode_p[t];
      load_pert<V, T, PERT>(U, Nn, ip, mv.rhob, mv.pb, up);
    } else {
      // coarse polynomial (perturbation) at this fine face node: tensor of 1D I_s
      const int s = mv.face_s[f];
      const T* I = mv.tab + S::T_I;
#pragma unroll
      for (int v = 0; v < V; ++v) up[v] = T(0);
      if (DIM == 2) {
        const T* Is = I + s * N * N + k * N;
        for (int j = 0; j < N; ++j) {
          T uc[V];
          load_pert<V, T, PERT>(U, Nn, (int64_t)cp * NC + face_node<DIM, DEG>(lfp, j), mv.rhob, mv.pb, uc);
          const T wgt = Is[j];
#pragma unroll
          for (int v = 0; v < V; ++v) up[v] += wgt * uc[v];
        }
      } else {
        const int k1 = k % N, k2 = k / N;
        const T* I1 = I + (s & 1) * N * N + k1 * N;
        const T* I2 = I + ((s >> 1) & 1) * N * N + k2 * N;
        for (int j2 = 0; j2 < N; ++j2) {
          for (int j1 = 0; j1 < N; ++j1) {
            T uc[V];
            load_pert<V, T, PERT>(U, Nn, (int64_t)cp * NC + face_node<DIM, DEG>(lfp, j1 + N * j2), mv.rhob,
                                  mv.pb, uc);
            const T wgt = I1[j1] * I2[j2];
#pragma unroll
            for (int v = 0; v < V; ++v) up[v] += wgt * uc[v];
          }
        }
      }
    }
    T Fm[V], Fp[V], lm, lp;
    normal_flux<DIM, T, FULL>(um, rb, pb, n, Fm, lm);
    normal_flux<DIM, T, FULL>(up, rb, pb, n, Fp, lp);
    const T lam = lm > lp ? lm : lp;
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = T(0.5) * (Fm[v] + Fp[v]) - T(0.5) * lam * (up[v] - um[v]);
  } else {
    // slip wall: Rusanov flux against the mirror state, in closed form
    const T rho = rb + um[0];
    const T irho = T(1) / rho;
    T mn = T(0), m2 = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      mn += um[1 + b] * n[b];
      m2 += um[1 + b] * um[1 + b];
    }
    const T un = mn * irho;
    T lam = fabs(un), pp = T(0);
    if (FULL) {
      pp = gm1<T>() * (um[V - 1] - T(0.5) * m2 * irho);
      lam += sqrt(T(1.4) * (pb + pp) * irho);
    }
    const T mom = mn * un + pp + lam * mn;
    out[0] = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) out[1 + b] = mom * n[b];
    out[V - 1] = T(0);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) Fh[(int64_t)v * total + t] = sj * out[v];
}

template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__global__ void __launch_bounds__(256) explicit_face_kernel(MeshView<T> mv, const T* __restrict__ U,
                                                            T* __restrict__ Fh, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)mv.nf * Shape<DIM, DEG>::NF) return;
  explicit_face_item<DIM, DEG, T, FULL, PERT>(mv, U, Fh, t);
}

// Face codes (face << 2 | side, see MeshView::cell_face) of the faces node idx
// of cell c lies on, one per axis; -1 where the node is interior along that axis.
// Loaded early so that their latency overlaps other work.
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void load_face_codes(const MeshView<T>& mv, int64_t c, const int* idx, int* codes) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    codes[a] = -1;
    if (idx[a] == 0 || idx[a] == DEG) codes[a] = mv.cell_face[c * 2 * DIM + 2 * a + (idx[a] == DEG ? 1 : 0)];
  }
}

// Gather the face contributions of node idx for NV fields stored [v][nf*NF]
// in Fh, given its face codes.  sign_minus / sign_plus multiply the minus-side
// / plus-side (and coarse-side) contributions.  Results are divided by w_end
// by the caller.
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void gather_faces_codes(const MeshView<T>& mv, const T* __restrict__ Fh,
                                                   const int* codes, const int* idx, const T* sIt, T sign_minus,
                                                   T sign_plus, bool skip_walls, T* acc) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NF = S::NF;
  const int64_t total = (int64_t)mv.nf * NF;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int code = codes[a];
    if (code < 0) continue;
    const int f = code >> 2, side = code & 3;
    const int kt = tangential_index<DIM, DEG>(a, idx);
    if (side == 3 && skip_walls) continue;
    if (side != 2) {
      const T sg = (side == 1) ? sign_plus : sign_minus;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sg * Fh[(int64_t)v * total + (int64_t)f * NF + kt];
    } else {
      // coarse side: sum over subfaces s of It_s (weighted transposed interpolation)
      if (DIM == 2) {
        for (int s = 0; s < 2; ++s) {
          const T* It = sIt + s * N * N + kt * N;
          const int64_t base = (int64_t)(f + s) * NF;
          for (int q = 0; q < N; ++q) {
            const T wgt = sign_plus * It[q];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += wgt * Fh[(int64_t)v * total + base + q];
          }
        }
      } else {
        const int i1 = kt % N, i2 = kt / N;
        for (int s = 0; s < 4; ++s) {
          const T* It1 = sIt + (s & 1) * N * N + i1 * N;
          const T* It2 = sIt + ((s >> 1) & 1) * N * N + i2 * N;
          const int64_t base = (int64_t)(f + s) * NF;
          for (int q2 = 0; q2 < N; ++q2) {
            for (int q1 = 0; q1 < N; ++q1) {
              const T wgt = sign_plus * It1[q1] * It2[q2];
#pragma unroll
              for (int v = 0; v < NV; ++v) acc[v] += wgt * Fh[(int64_t)v * total + base + q1 + N * q2];
            }
          }
        }
      }
    }
  }
}

template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void gather_faces(const MeshView<T>& mv, const T* __restrict__ Fh, int64_t c,
                                             const int* idx, const T* sIt, T sign_minus, T sign_plus,
                                             bool skip_walls, T* acc) {
  int codes[DIM];
  load_face_codes<DIM, DEG, T>(mv, c, idx, codes);
  gather_faces_codes<DIM, DEG, T, NV>(mv, Fh, codes, idx, sIt, sign_minus, sign_plus, skip_walls, acc);
}

// Cells [batch*CPB, batch*CPB + CPB) of the cell pass.  Called by a whole
// block; sF holds V * CPB * NC elements, sDw and sIt the tables (loaded by the
// caller; read only after the first block barrier).
template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__device__ __forceinline__ void explicit_cell_batch(const MeshView<T>& mv, const T* __restrict__ U,
                                                    const T* __restrict__ Fh, T* __restrict__ R, int64_t batch,
                                                    T (*sF)[Shape<DIM, DEG>::CPB * Shape<DIM, DEG>::NC],
                                                    const T* sDw, const T* sIt) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, V = S::V, CPB = S::CPB;
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int64_t c = batch * CPB + lc;
  const bool active = (lc < CPB) && (c < mv.n_cells);
  const int64_t Nn = mv.n_nodes;
  const int64_t idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  T u[V], F[V][DIM], src[V], acc[V];
  T rb = T(0), pb = T(0), ij = T(0);
  T Ja[DIM][DIM];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = T(0);
  if (active) {
    rb = mv.rhob[idx];
    pb = mv.pb[idx];
    ij = mv.invJ[idx];
    load_pert<V, T, PERT>(U, Nn, idx, mv.rhob, mv.pb, u);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) Ja[a][b] = mv.Ja[(int64_t)(a * DIM + b) * Nn + idx];
    const T rho = rb + u[0];
    const T irho = T(1) / rho;
    T m2 = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) m2 += u[1 + b] * u[1 + b];
    const T pp = gm1<T>() * (u[V - 1] - T(0.5) * m2 * irho);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      const T ub = u[1 + b] * irho;
      F[0][b] = u[1 + b];
#pragma unroll
      for (int a = 0; a < DIM; ++a) F[1 + a][b] = u[1 + a] * ub;
      if (FULL) {
        F[1 + b][b] += pp;
        F[V - 1][b] = (u[V - 1] + pp + pb * (T(1.4) / gm1<T>())) * ub;
      } else {
        F[V - 1][b] = T(0.5) * m2 * irho * irho * u[1 + b];
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) src[v] = T(0);
    if (FULL) src[DIM] = -u[0] * mv.gravity;  // -(rho - rho_b) g
    src[V - 1] = -mv.gravity * u[DIM];         // -g m_z
  }
  // volume term, one axis at a time through shared memory
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T ft = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) ft += Ja[a][b] * F[v][b];
        sF[v][lc * NC + i] = ft;
      }
    }
    __syncthreads();
    if (active) {
      constexpr int st0 = 1, st1 = N, st2 = N * N;
      const int stride = a == 0 ? st0 : (a == 1 ? st1 : st2);
      const int i0 = lc * NC + i - id[a] * stride;
      const T* Dw = sDw + id[a] * N;
#pragma unroll
      for (int kk = 0; kk < N; ++kk) {
        const T dw = Dw[kk];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += dw * sF[v][i0 + kk * stride];
      }
    }
    __syncthreads();
  }
  if (!active) return;
  T facc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) facc[v] = T(0);
  gather_faces<DIM, DEG, T, V>(mv, Fh, c, id, sIt, T(-1), T(1), false, facc);
  const T iwend = mv.tab[S::T_IWEND];
#pragma unroll
  for (int v = 0; v < V; ++v) R[(int64_t)v * Nn + idx] = (acc[v] + facc[v] * iwend) * ij + src[v];
}

template <int DIM, int DEG, typename T, bool FULL, bool PERT>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) explicit_cell_kernel(MeshView<T> mv,
                                                                                 const T* __restrict__ U,
                                                                                 const T* __restrict__ Fh,
                                                                                 T* __restrict__ R, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sF[S::V][S::CPB * S::NC];
  __shared__ T sDw[N * N];
  __shared__ T sIt[2 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sDw[q] = mv.tab[S::T_DW + q];
  for (int q = threadIdx.x; q < 2 * N * N; q += blockDim.x) sIt[q] = mv.tab[S::T_IT + q];
  explicit_cell_batch<DIM, DEG, T, FULL, PERT>(mv, U, Fh, R, blockIdx.x, sF, sDw, sIt);
}

}  // namespace dg
