// Operators of the implicit pressure stage (Sec. 2 IMEX split; Sec. 3.2
// pressure loop), centred traces, in a one-pass cell form: every cell pass
// computes the face terms of its own nodes (no face pass, no face buffer).
// The persistent solves run the passes between grid barriers; standalone
// calls launch them one kernel per operator:
//
//  gradient (strong form):  g_b = [ sum_a Ja^a_b (D_a p) + Gh_b / w_end ] / J,
//      face value Gh_b = 1/2 |N| n_b (p+ - p-), added with + on both sides
//      and through It on the coarse side; zero on walls (p^ = p-).
//  divergence (weak form):  div = [ -sum_a sum_k Dw[i_a][k] (Ja^a.f)(k) + Dh/w_end ] / J,
//      face value Dh = |N| {f}.n, + on the minus side, - on the plus and
//      coarse sides; zero on walls.
//  Helmholtz:  A p = p/(gamma-1) - alpha div(h grad p), as grad(h-scaled)
//      followed by the divergence with the Helmholtz epilogue.
//
// The per-batch work is written as device functions so that the persistent
// Krylov kernels (k_gmres.cuh) can run it between their grid barriers.
#pragma once

#include "dg_device.cuh"
#include "k_explicit.cuh"

namespace dg {

// Interpolated coarse value of an NV-component field at fine face node k of
// subface position s, from the coarse cell's values on its face lfp:
// X[v * vstride + cbase + face_node(lfp, j)] (global memory or a shared tile).
// (Node indices are below 2^31, so they are 32-bit here; the field offsets
// v * vstride are taken once per field.)
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void coarse_interp(const T* __restrict__ X, int64_t vstride, int cbase, int lfp,
                                              int s, int k, const T* sI, T* out) {
  constexpr int N = DEG + 1;
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = T(0);
  if (DIM == 2) {
    const T* Is = sI + s * N * N + k * N;
    for (int j = 0; j < N; ++j) {
      const int ic = cbase + face_node<DIM, DEG>(lfp, j);
#pragma unroll
      for (int v = 0; v < NV; ++v) out[v] += Is[j] * (X + v * vstride)[ic];
    }
  } else {
    const int k1 = k % N, k2 = k / N;
    const T* I1 = sI + (s & 1) * N * N + k1 * N;
    const T* I2 = sI + ((s >> 1) & 1) * N * N + k2 * N;
#pragma unroll 1
    for (int j2 = 0; j2 < N; ++j2)
      for (int j1 = 0; j1 < N; ++j1) {
        const int ic = cbase + face_node<DIM, DEG>(lfp, j1 + N * j2);
        const T wgt = I1[j1] * I2[j2];
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] += wgt * (X + v * vstride)[ic];
      }
  }
}

// Weight of fine face node q of subface position s in the coarse-side sum at
// coarse face node kt: the weighted transposed interpolation It.
template <int DIM, int DEG, typename T>
__device__ __forceinline__ T coarse_weight(const T* sIt, int s, int kt, int q) {
  constexpr int N = DEG + 1;
  if (DIM == 2) return sIt[s * N * N + kt * N + q];
  return sIt[(s & 1) * N * N + (kt % N) * N + (q % N)] * sIt[((s >> 1) & 1) * N * N + (kt / N) * N + (q / N)];
}

// ---------------------------------------------------------------- gradient
//
// Face terms are computed by the cells themselves (no face pass, no face
// buffer).  A node on a conforming face takes the neighbour's node value; a
// node on a fine subface interpolates the coarse neighbour's face polynomial
// at its point.  Both sides evaluate the same expression on the same values,
// so the face value is the same on both sides.  The coarse side of a 2:1 face
// needs the face values at all fine points of its subfaces: the batch's
// threads compute them once, one fine point each, into shared memory (the
// batch's coarse-side entry list, coarse_fill below), and the sums through It
// at the coarse face nodes follow (coarse_reduce / coarse_sum).

// Number of fine points behind one coarse face, and the shared-memory buffer
// (elements) the coarse sides need per cell batch for NV values per point and
// per coarse face node: kCoarseSlots coarse faces per cell of the batch fit
// one round.
constexpr int kCoarseSlots = 2;
template <int DIM, int DEG>
__host__ __device__ constexpr int coarse_points() {
  return Shape<DIM, DEG>::NSUB * Shape<DIM, DEG>::NF;
}
template <int DIM, int DEG, int NV>
__host__ __device__ constexpr int coarse_buffer() {
  return Shape<DIM, DEG>::CPB * kCoarseSlots * NV * (coarse_points<DIM, DEG>() + Shape<DIM, DEG>::NF);
}

// Whether the pass uses metric entry J d xi^a / d x_b: all of them in
// general; on meshes whose cells are affine in the horizontal coordinates
// (aff: MeshView::aff, or the metric recomputed from the heights) only the
// diagonal and the last row (xi depends on x alone, eta on y alone).  The
// test is warp-uniform, and a compile-time true for those entries.
template <int DIM>
__device__ __forceinline__ bool metric_used(int a, int b, bool aff) {
  return a == b || a == DIM - 1 || !aff;
}

// One cell batch of the mesh's active partition: cells [c0, c1) (at most
// CPB), coarse-side entries [e0, e1) (MeshView::bdesc, one 16-byte load).
struct BatchRange {
  int c0, c1, e0, e1;
};
template <typename T>
__device__ __forceinline__ BatchRange batch_range(const MeshView<T>& mv, int64_t b) {
  const int4 v = mv.bdesc[b];
  return BatchRange{v.x, v.y, v.z, v.w};
}

// Coarse sides of the batch's 2:1 faces, through the batch's entry list
// (MeshView::bdesc, ce_*).  A round takes FPR coarse faces (slots) of the
// batch, EPR = FPR * NP fine points, the threads taking them in turn:
// coarse_fill writes the NV face values of each point to buf[v * EPR + k]
// (k = the point's place in the round), reading global memory only, so that
// round 0 is filled before the batch's first barrier and its loads overlap
// the batch's own; after that barrier, coarse_reduce forms at every node kt
// of every coarse face of the round sum_s sum_q sign * It * value, one
// thread per (face, node) (out[v * OPR + slot * NF + kt], all lanes busy);
// after one more barrier, coarse_sum adds each node's values to acc[0..NV).
// The buffer (coarse_buffer) holds the points' values, then the sums.
template <int DIM, int DEG>
struct CoarseRounds {
  using S = Shape<DIM, DEG>;
  static constexpr int NP = coarse_points<DIM, DEG>();
  static constexpr int FPR = S::CPB * kCoarseSlots;  // slots per round (the buffer's capacity)
  static constexpr int EPR = FPR * NP;               // points per round
  static constexpr int OPR = FPR * S::NF;            // coarse face nodes per round
  __device__ __forceinline__ static int rounds(int e0, int e1) { return ((e1 - e0) / NP + FPR - 1) / FPR; }
};

// A CTA's own cell batch, read once for a whole Krylov cycle of a persistent
// solve when the CTA has exactly one batch: the face links and coarse-face
// word of each thread's node, and the batch's round-0 coarse-side entries.
// The passes then read these from shared memory instead of global memory,
// which takes one dependent global load off each pass's critical path.
template <int DIM, int DEG, typename T>
struct BatchCache {
  using S = Shape<DIM, DEG>;
  static constexpr int EPR = CoarseRounds<DIM, DEG>::EPR;
  int links[DIM * S::THREADS];
  int coarse[S::THREADS];
  int meta[EPR];
  int node[EPR];
  T w[DIM * EPR];
};

// point(cc, lf, s, q, node, w, val): the NV values at fine point q of subface
// s of local face lf of batch cell cc (the fine side's node `node`, w = 1/2 |N| n / w_end there)
template <int DIM, int DEG, typename T, int NV, class Point>
__device__ __forceinline__ void coarse_fill(const MeshView<T>& mv, const BatchRange& br, int r, T* buf,
                                            Point&& point, const BatchCache<DIM, DEG, T>* bc = nullptr) {
  using R = CoarseRounds<DIM, DEG>;
  constexpr int NF = Shape<DIM, DEG>::NF;
  const int base = br.e0 + r * R::EPR;
  const int kend = br.e1 - base < R::EPR ? br.e1 - base : R::EPR;
  const bool cached = bc && r == 0;
  for (int k = threadIdx.x; k < kend; k += blockDim.x) {
    const int e = base + k;
    const int meta = cached ? bc->meta[k] : mv.ce_meta[e];
    const int node = cached ? bc->node[k] : mv.ce_node[e];
    T w[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) w[b] = cached ? bc->w[b * R::EPR + k] : mv.ce_w[(int64_t)b * mv.n_ce + e];
    const int j = meta >> 9;
    T val[NV];
    point(br.c0 + (meta & 63), (meta >> 6) & 7, j / NF, j % NF, node, w, val);
#pragma unroll
    for (int v = 0; v < NV; ++v) buf[v * R::EPR + k] = val[v];
  }
}

// The sums of round r at the coarse face nodes (whole block, after the
// barrier that follows the round's fill; another barrier must follow before
// coarse_sum reads them)
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void coarse_reduce(const BatchRange& br, int r, const T* sIt, T sign, T* buf) {
  using R = CoarseRounds<DIM, DEG>;
  using S = Shape<DIM, DEG>;
  constexpr int NF = S::NF;
  const int left = (br.e1 - br.e0) / R::NP - r * R::FPR;
  const int nsl = left < R::FPR ? left : R::FPR;
  T* out = buf + NV * R::EPR;
  for (int t = threadIdx.x; t < nsl * NF; t += blockDim.x) {
    const int sl = t / NF, kt = t % NF;
    const T* b = buf + sl * R::NP;
    T o[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) o[v] = T(0);
    for (int sp = 0; sp < S::NSUB; ++sp)
      for (int q = 0; q < NF; ++q) {
        const T wgt = sign * coarse_weight<DIM, DEG, T>(sIt, sp, kt, q);
#pragma unroll
        for (int v = 0; v < NV; ++v) o[v] += wgt * b[v * R::EPR + sp * NF + q];
      }
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * R::OPR + t] = o[v];
  }
}

// The same sums formed by each coarse face node's own thread, straight from
// the round's point values (no barrier after the fill's; the lanes of the
// other nodes idle meanwhile): the cheaper form in FP32, where the passes are
// bound by latency rather than by arithmetic.
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void coarse_sum_direct(int coarse, int r, const int* id, const T* sIt, T sign,
                                                  const T* buf, T* acc) {
  using R = CoarseRounds<DIM, DEG>;
  using S = Shape<DIM, DEG>;
  constexpr int NF = S::NF;
  const unsigned cmask = (unsigned)coarse & 0xffu;
  if (!cmask) return;
  const int slot0 = coarse >> 8;
#pragma unroll
  for (int lf = 0; lf < 2 * DIM; ++lf) {
    if (!((cmask >> lf) & 1u)) continue;
    const int a = lf >> 1;
    if (id[a] != ((lf & 1) ? DEG : 0)) continue;
    const int slot = slot0 + __popc(cmask & ((1u << lf) - 1u));
    if (slot / R::FPR != r) continue;
    const int kt = tangential_index<DIM, DEG>(a, id);
    const T* b = buf + (slot % R::FPR) * R::NP;
    for (int sp = 0; sp < S::NSUB; ++sp)
      for (int q = 0; q < NF; ++q) {
        const T wgt = sign * coarse_weight<DIM, DEG, T>(sIt, sp, kt, q);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += wgt * b[v * R::EPR + sp * NF + q];
      }
  }
}

// Which form a pass takes: the dense reduction in FP64 (arithmetic-bound),
// the direct sums in FP32 (latency-bound)
template <typename T>
__host__ __device__ constexpr bool coarse_dense() {
  return sizeof(T) == 8;
}

// coarse = MeshView::cell_coarse of this thread's cell (0 if none or inactive)
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void coarse_sum(int coarse, int r, const int* id, const T* buf, T* acc) {
  using R = CoarseRounds<DIM, DEG>;
  constexpr int NF = Shape<DIM, DEG>::NF;
  const unsigned cmask = (unsigned)coarse & 0xffu;
  if (!cmask) return;
  const int slot0 = coarse >> 8;
  const T* out = buf + NV * R::EPR;
#pragma unroll
  for (int lf = 0; lf < 2 * DIM; ++lf) {
    if (!((cmask >> lf) & 1u)) continue;
    const int a = lf >> 1;
    if (id[a] != ((lf & 1) ? DEG : 0)) continue;
    const int slot = slot0 + __popc(cmask & ((1u << lf) - 1u));
    if (slot / R::FPR != r) continue;
    const int o = (slot % R::FPR) * NF + tangential_index<DIM, DEG>(a, id);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += out[v * R::OPR + o];
  }
}

// The rounds after round 0 (rare: more coarse faces in one batch than a round
// holds), each between block barriers; called by the whole block.
template <int DIM, int DEG, typename T, int NV, class Point>
__device__ __forceinline__ void coarse_more_rounds(const MeshView<T>& mv, const BatchRange& br, int coarse,
                                                   const int* id, const T* sIt, T sign, T* buf, T* acc,
                                                   Point&& point) {
  const int nr = CoarseRounds<DIM, DEG>::rounds(br.e0, br.e1);
  for (int r = 1; r < nr; ++r) {
    __syncthreads();
    coarse_fill<DIM, DEG, T, NV>(mv, br, r, buf, point);
    __syncthreads();
    if (coarse_dense<T>()) {
      coarse_reduce<DIM, DEG, T, NV>(br, r, sIt, sign, buf);
      __syncthreads();
      coarse_sum<DIM, DEG, T, NV>(coarse, r, id, buf, acc);
    } else {
      coarse_sum_direct<DIM, DEG, T, NV>(coarse, r, id, sIt, sign, buf, acc);
    }
  }
}

// A pass's hook between the loads of the batch's own data and the first read
// of data other CTAs wrote in the previous phase: the persistent solves wait
// there for the grid barrier they arrived at (a split barrier), so that the
// own loads' latency overlaps the barrier's; called by the whole block.
struct NoWait {
  __device__ __forceinline__ void operator()() const {}
};

// Face links of node id of cell c, one per axis: the link of the cell face the
// node lies on along that axis (MeshView::cell_link), or kind 3 (no face
// term) where the node is interior along the axis.  Loaded early so that
// their latency overlaps other work.
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void load_face_links(const MeshView<T>& mv, int c, const int* id, int* links) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    links[a] = 3;
    if (id[a] == 0 || id[a] == DEG) links[a] = mv.cell_link[2 * DIM * c + 2 * a + (id[a] == DEG ? 1 : 0)];
  }
}

// The other side's NV values at the face node of node id on its face along
// axis a (X[v * vstride + node]): on a conforming face the neighbour's node,
// on the fine side of a 2:1 face the coarse cell's polynomial at this point.
// link kind must be 0 or 1.
template <int DIM, int DEG, typename T, int NV>
__device__ __forceinline__ void other_trace(const T* __restrict__ X, int64_t vstride, int link, int a, const int* id,
                                            const T* sI, T* out) {
  constexpr int NC = Shape<DIM, DEG>::NC;
  const int nb = (int)((unsigned)link >> 4);
  const int lfo = 2 * a + (id[a] == DEG ? 0 : 1);  // the neighbour's face is the opposite one
  const int kt = tangential_index<DIM, DEG>(a, id);
  if ((link & 3) == 0) {
    const int o = nb * NC + face_node<DIM, DEG>(lfo, kt);
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = (X + v * vstride)[o];
  } else {
    coarse_interp<DIM, DEG, T, NV>(X, vstride, nb * NC, lfo, (link >> 2) & 3, kt, sI, out);
  }
}

// Outward face normal |N| n of node id on its face along axis a, times
// 1/(2 w_end): the node's own metric row +-Ja[a] / 2 (the same face seen from
// either side of a conforming face; on a 2:1 face the fine side's), with the
// lifting factor 1/w_end of the face term folded in (hw = 1/(2 w_end)).
template <int DIM, int DEG, typename T>
__device__ __forceinline__ T half_sign(int a, const int* id, T hw) {
  return id[a] == DEG ? hw : -hw;
}

// Fill bc for batch br (whole block; ends with a block barrier).
template <int DIM, int DEG, typename T>
__device__ __forceinline__ void batch_cache_fill(const MeshView<T>& mv, const BatchRange& br,
                                                 BatchCache<DIM, DEG, T>* bc) {
  using S = Shape<DIM, DEG>;
  using R = CoarseRounds<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC;
  const int t = threadIdx.x;
  if (t < S::THREADS) {
    const int lc = t / NC, i = t % NC;
    const int c = br.c0 + lc;
    int id[3] = {i % N, (i / N) % N, i / (N * N)};
    int links[DIM];
    if (c < br.c1) {
      load_face_links<DIM, DEG, T>(mv, c, id, links);
      bc->coarse[t] = mv.cell_coarse[c];
    } else {
#pragma unroll
      for (int a = 0; a < DIM; ++a) links[a] = 3;
      bc->coarse[t] = 0;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) bc->links[a * S::THREADS + t] = links[a];
  }
  const int kend = br.e1 - br.e0 < R::EPR ? br.e1 - br.e0 : R::EPR;
  for (int k = t; k < kend; k += blockDim.x) {
    const int e = br.e0 + k;
    bc->meta[k] = mv.ce_meta[e];
    bc->node[k] = mv.ce_node[e];
#pragma unroll
    for (int b = 0; b < DIM; ++b) bc->w[b * R::EPR + k] = mv.ce_w[(int64_t)b * mv.n_ce + e];
  }
  __syncthreads();
}

// Cells [br.c0, br.c1): g_b = h [sum_a Ja^a_b (D_a p) + face_b / w_end] / J.
// Called by a whole block with blockDim >= CPB*NC; contains __syncthreads.
// sII holds the interpolation tables I (2 N^2) followed by It (2 N^2); sJ is
// the coarse-pass buffer (coarse_buffer<DIM, DEG, DIM>() elements).
// GZ: metric terms from the heights (metric_from_z), staged in sz (CPB*NC).
// AFF: the mesh is known to be horizontally affine (MeshView::aff) at compile
// time, so the vanishing metric entries drop out of the code; otherwise the
// runtime flag only predicates them off.
template <int DIM, int DEG, typename T, bool GZ = false, bool AFF = false, class Wait = NoWait>
__device__ __forceinline__ void grad_cell_batch(const MeshView<T>& mv, const T* __restrict__ p,
                                                const T* __restrict__ h, T* __restrict__ g, const BatchRange& br,
                                                T* sp, T* sJ, const T* sD, const T* sII, T* sz = nullptr,
                                                const BatchCache<DIM, DEG, T>* bc = nullptr, Wait wait = Wait{}) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC;
  const bool aff = GZ || AFF || mv.aff;
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int c = br.c0 + lc;
  const bool active = c < br.c1;
  const int64_t Nn = mv.n_nodes;
  const int idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  int links[DIM];
  T Jl[DIM][DIM];
  T po[DIM];  // the other side's value at this node's faces
  T scale = T(0), pv = T(0);
  int coarse = 0;
  const bool has_coarse = br.e1 > br.e0;
  if (active) {
    pv = p[idx];
    sp[lc * NC + i] = pv;
    if (bc) {
#pragma unroll
      for (int a = 0; a < DIM; ++a) links[a] = bc->links[a * S::THREADS + threadIdx.x];
      coarse = bc->coarse[threadIdx.x];
    } else {
      load_face_links<DIM, DEG, T>(mv, c, id, links);
      coarse = mv.cell_coarse[c];
    }
    if (GZ) {
      sz[lc * NC + i] = mv.zdev[idx];
      scale = h ? h[idx] : T(1);
    } else {
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) Jl[a][b] = metric_used<DIM>(a, b, aff) ? (mv.Ja + (a * DIM + b) * Nn)[idx] : T(0);
      scale = mv.invJ[idx] * (h ? h[idx] : T(1));
    }
  }
  wait();  // from here on, other CTAs' values of p
  if (active) {
    // neighbour traces: issued before the batch's barrier, their latency overlaps it
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      if ((links[a] & 3) < 2) other_trace<DIM, DEG, T, 1>(p, 0, links[a], a, id, sII, &po[a]);
  }
  // coarse sides, round 0: the jump at each fine point times 1/2 |N| n / w_end, from the fine value and
  // the coarse cell's polynomial
  auto gpoint = [&](int cc, int lf, int s, int q, int node, const T* w, T* val) {
    T pp;
    coarse_interp<DIM, DEG, T, 1>(p, 0, cc * NC, lf, s, q, sII, &pp);
    const T jmp = pp - p[node];
#pragma unroll
    for (int b = 0; b < DIM; ++b) val[b] = jmp * w[b];
  };
  if (has_coarse) coarse_fill<DIM, DEG, T, DIM>(mv, br, 0, sJ, gpoint, bc);
  __syncthreads();
  // FP64: round 0's sums at the coarse face nodes, while the cells' own work follows
  if (coarse_dense<T>() && has_coarse) coarse_reduce<DIM, DEG, T, DIM>(br, 0, sII + 2 * N * N, T(1), sJ);
  T facc[DIM], dp[DIM];  // facc: the face terms, already divided by w_end
#pragma unroll
  for (int b = 0; b < DIM; ++b) facc[b] = dp[b] = T(0);
  if (GZ && active) {
    T ij;
    metric_from_z<DIM, DEG, T>(mv, c, sz + lc * NC, id, sD, Jl, ij);
    scale *= ij;
  }
  if (active) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int i0 = lc * NC + i - id[a] * stride;
      const T* D = sD + id[a] * N;
      T s = T(0);
#pragma unroll
      for (int kk = 0; kk < N; ++kk) s += D[kk] * sp[i0 + kk * stride];
      dp[a] = s;
    }
    // face terms: 1/2 (p_other - p_own) |N| n / w_end on conforming and fine-side faces (zero
    // jump on walls, p^ = p-; coarse sides in the coarse pass)
    const T hw = T(0.5) * mv.tab[S::T_IWEND];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if ((links[a] & 3) >= 2) continue;
      const T jmp = half_sign<DIM, DEG, T>(a, id, hw) * (po[a] - pv);
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        if (metric_used<DIM>(a, b, aff)) facc[b] += jmp * Jl[a][b];
    }
  }
  // coarse sides (FP64: round 0's sums are in sJ after this barrier)
  if (has_coarse) {
    if (coarse_dense<T>()) {
      __syncthreads();
      coarse_sum<DIM, DEG, T, DIM>(coarse, 0, id, sJ, facc);
    } else {
      coarse_sum_direct<DIM, DEG, T, DIM>(coarse, 0, id, sII + 2 * N * N, T(1), sJ, facc);
    }
    coarse_more_rounds<DIM, DEG, T, DIM>(mv, br, coarse, id, sII + 2 * N * N, T(1), sJ, facc, gpoint);
  }
  if (active) {
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T s = facc[b];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        if (metric_used<DIM>(a, b, aff)) s += Jl[a][b] * dp[a];
      (g + b * Nn)[idx] = s * scale;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- divergence

// An epilogue with a pre(i) method has it called for the node before the
// divergence pass's first barrier (to load the operands of its update early)
template <class E>
__device__ __forceinline__ auto epi_pre(E& e, int64_t i, int) -> decltype(e.pre(i), void()) {
  e.pre(i);
}
template <class E>
__device__ __forceinline__ void epi_pre(E&, int64_t, long) {}

// Cells of one batch: epi(idx, v) receives v = HELM ? scale * (ident p/(gamma-1) - alpha div) : div
// at every node of the batch (the caller stores it, or fuses further pointwise work).
// Called by a whole block with blockDim >= CPB*NC; contains __syncthreads.
// sF: DIM * CPB * NC elements; sJ: coarse-pass buffer (coarse_buffer<DIM, DEG, 1>() elements).
// GZ: metric terms from the heights (metric_from_z with sD), staged in sz (CPB*NC).
// AFF: as for the gradient.
template <int DIM, int DEG, typename T, bool HELM, class Epi, bool GZ = false, bool AFF = false,
          class Wait = NoWait>
__device__ __forceinline__ void div_cell_batch(const MeshView<T>& mv, const T* __restrict__ fld,
                                               const T* __restrict__ p, T alpha, T scale, T ident, Epi& epi,
                                               const BatchRange& br, T* sF, T* sJ, const T* sDw, const T* sII,
                                               T* sz = nullptr, const T* sD = nullptr,
                                               const BatchCache<DIM, DEG, T>* bc = nullptr, Wait wait = Wait{}) {
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N, NC = S::NC, CPB = S::CPB;
  const bool aff = GZ || AFF || mv.aff;
  const int lc = threadIdx.x / NC, i = threadIdx.x % NC;
  const int c = br.c0 + lc;
  const bool active = c < br.c1;
  const int64_t Nn = mv.n_nodes;
  const int idx = c * NC + i;
  int id[3] = {i % N, (i / N) % N, i / (N * N)};
  int links[DIM];
  T ft[DIM];  // Ja^a . f for each axis a
  T fv[DIM];
  T ij = T(0), pv = T(0);
  T Jl[DIM][DIM];
  int coarse = 0;
  const bool has_coarse = br.e1 > br.e0;
  if (active) {
#pragma unroll
    for (int b = 0; b < DIM; ++b) fv[b] = (fld + b * Nn)[idx];
    if (bc) {
#pragma unroll
      for (int a = 0; a < DIM; ++a) links[a] = bc->links[a * S::THREADS + threadIdx.x];
      coarse = bc->coarse[threadIdx.x];
    } else {
      load_face_links<DIM, DEG, T>(mv, c, id, links);
      coarse = mv.cell_coarse[c];
    }
    if (HELM) pv = p[idx];
    epi_pre(epi, idx, 0);
    if (GZ) {
      sz[lc * NC + i] = mv.zdev[idx];
    } else {
      ij = mv.invJ[idx];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) Jl[a][b] = metric_used<DIM>(a, b, aff) ? (mv.Ja + (a * DIM + b) * Nn)[idx] : T(0);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b)
          if (metric_used<DIM>(a, b, aff)) s += Jl[a][b] * fv[b];
        ft[a] = s;
      }
    }
  }
  // coarse sides, round 0: |N| {f}.n / (2 w_end) at each fine point from the fine value and the coarse
  // cell's polynomial
  auto dpoint = [&](int cc, int lf, int s, int q, int node, const T* w, T* val) {
    T fc[DIM];
    coarse_interp<DIM, DEG, T, DIM>(fld, Nn, cc * NC, lf, s, q, sII, fc);
    T sum = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) sum += ((fld + b * Nn)[node] + fc[b]) * w[b];
    val[0] = sum;
  };
  wait();  // from here on, other CTAs' values of f
  if (has_coarse) coarse_fill<DIM, DEG, T, 1>(mv, br, 0, sJ, dpoint, bc);
  if (GZ) {
    __syncthreads();
    if (active) {
      metric_from_z<DIM, DEG, T>(mv, c, sz + lc * NC, id, sD, Jl, ij);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b)
          if (metric_used<DIM>(a, b, aff)) s += Jl[a][b] * fv[b];
        ft[a] = s;
      }
    }
  }
  // all DIM contravariant components staged at once (sF holds DIM * CPB * NC)
  if (active) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) sF[(a * CPB + lc) * NC + i] = ft[a];
  }
  __syncthreads();
  // FP64: round 0's sums at the coarse face nodes, while the cells' own work follows
  if (coarse_dense<T>() && has_coarse) coarse_reduce<DIM, DEG, T, 1>(br, 0, sII + 2 * N * N, T(-1), sJ);
  T acc = T(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int i0 = (a * CPB + lc) * NC + i - id[a] * stride;
      const T* Dw = sDw + id[a] * N;
#pragma unroll
      for (int kk = 0; kk < N; ++kk) acc -= Dw[kk] * sF[i0 + kk * stride];
    }
  }
  T facc = T(0);  // the face terms, already divided by w_end
  // face terms: 1/2 (f_own + f_other).|N| n / w_end on conforming and fine-side faces (zero
  // normal flux on walls; coarse sides in the coarse pass); f_own.|N| n is the node's own
  // contravariant component ft[a]
  if (active) {
    const T hw = T(0.5) * mv.tab[S::T_IWEND];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if ((links[a] & 3) >= 2) continue;
      T fo[DIM];
      other_trace<DIM, DEG, T, DIM>(fld, Nn, links[a], a, id, sII, fo);
      T sum = ft[a];
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        if (metric_used<DIM>(a, b, aff)) sum += fo[b] * Jl[a][b];
      facc += half_sign<DIM, DEG, T>(a, id, hw) * sum;
    }
  }
  // coarse sides (FP64: round 0's sums are in sJ after this barrier)
  if (has_coarse) {
    if (coarse_dense<T>()) {
      __syncthreads();
      coarse_sum<DIM, DEG, T, 1>(coarse, 0, id, sJ, &facc);
    } else {
      coarse_sum_direct<DIM, DEG, T, 1>(coarse, 0, id, sII + 2 * N * N, T(-1), sJ, &facc);
    }
    coarse_more_rounds<DIM, DEG, T, 1>(mv, br, coarse, id, sII + 2 * N * N, T(-1), sJ, &facc, dpoint);
  }
  if (active) {
    const T dv = (acc + facc) * ij;
    if (HELM)
      epi(idx, scale * (ident * pv * inv_gm1<T>() - alpha * dv));
    else
      epi(idx, dv);
  }
  __syncthreads();  // sF and sJ are rewritten by the next batch
}

// ---------------------------------------------------------------- standalone one-pass kernels
//
// dg_apply_grad / dg_apply_div / dg_apply_implicit: one CTA per cell batch,
// the face terms computed by the cells themselves (no face buffer: the only
// intermediate of the Helmholtz operator is the h-scaled gradient between
// the two launches).  GZ: the metric terms are recomputed from the nodal
// heights instead of loaded (used in FP32 on meshes affine in x and y, where
// it cuts the geometry read per node from d^2 + 1 values to one).

template <typename T>
struct StoreOut {
  T* out;
  __device__ __forceinline__ void operator()(int64_t i, T v) const { out[i] = v; }
};

template <int DIM, int DEG, typename T, bool GZ, bool AFF>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) grad_cell_kernel(MeshView<T> mv,
                                                                           const T* __restrict__ p,
                                                                           const T* __restrict__ h,
                                                                           T* __restrict__ g,
                                                                           const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sp[S::CPB * S::NC];
  __shared__ T sz[GZ ? S::CPB * S::NC : 1];
  __shared__ T sJ[coarse_buffer<DIM, DEG, DIM>()];
  __shared__ T sD[N * N];
  __shared__ T sII[4 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sD[q] = mv.tab[S::T_D + q];
  for (int q = threadIdx.x; q < 4 * N * N; q += blockDim.x) sII[q] = mv.tab[S::T_I + q];
  __syncthreads();  // the fine-side traces read the interpolation tables before the batch's first barrier
  grad_cell_batch<DIM, DEG, T, GZ, AFF>(mv, p, h, g, batch_range(mv, blockIdx.x), sp, sJ, sD, sII, sz);
}

template <int DIM, int DEG, typename T, bool HELM, bool GZ, bool AFF>
__global__ void __launch_bounds__(Shape<DIM, DEG>::THREADS) div_cell_kernel(MeshView<T> mv,
                                                                          const T* __restrict__ f,
                                                                          const T* __restrict__ p, T alpha,
                                                                          T* __restrict__ out,
                                                                          const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = Shape<DIM, DEG>;
  constexpr int N = S::N;
  __shared__ T sF[DIM * S::CPB * S::NC];
  __shared__ T sz[GZ ? S::CPB * S::NC : 1];
  __shared__ T sJ[coarse_buffer<DIM, DEG, 1>()];
  __shared__ T sDw[N * N];
  __shared__ T sD[GZ ? N * N : 1];
  __shared__ T sII[4 * N * N];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    sDw[q] = mv.tab[S::T_DW + q];
    if (GZ) sD[q] = mv.tab[S::T_D + q];
  }
  for (int q = threadIdx.x; q < 4 * N * N; q += blockDim.x) sII[q] = mv.tab[S::T_I + q];
  __syncthreads();
  StoreOut<T> epi{out};
  div_cell_batch<DIM, DEG, T, HELM, StoreOut<T>, GZ, AFF>(mv, f, p, alpha, T(1), T(1), epi,
                                                          batch_range(mv, blockIdx.x), sF, sJ, sDw, sII, sz, sD);
}

}  // namespace dg
