// Internal declarations shared by the host and device translation units of the
// DG library.  Nothing here is part of the C ABI (include/dg_atmo.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dg_atmo.h"

namespace dg {

constexpr double kGamma = 1.4;   // Sec. 3.1
constexpr double kRgas = 287.0;  // Sec. 2
constexpr int kMaxDegree = 5;
constexpr int kMaxRestart = 64;

// thread-local error message, set by fail()
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define DG_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return ::dg::cuda_fail(e__, #call); \
  } while (0)

// 1D tables of one degree, in the device layout used by every kernel:
//   D  [n*n]  D[i*n+k]  = l_k'(xi_i)                   (nodal derivative)
//   Dw [n*n]  Dw[i*n+k] = w_k l_i'(xi_k) / w_i          (weak derivative / w_i)
//   I  [2*n*n] I[s*n*n + f*n + j] = l_j((xi_f + 2s - 1)/2)  (coarse -> half s)
//   It [2*n*n] It[s*n*n + i*n + f] = (w_f / w_i) I[s][f][i]  (its weighted transpose)
//   w  [n], then 1/w_end (w_end = w_0 = w_r), then the nodes xi [n]
struct Tables1D {
  int degree = 0;
  std::vector<double> xi, w, D, Dw, I, It;
  std::vector<double> packed() const;  // D|Dw|I|It|w|1/w_end
};
Tables1D make_tables(int degree);
inline int table_size(int n) { return 6 * n * n + 2 * n + 1; }
// Lagrange basis on `nodes` at point x: out[j] = l_j(x)
void lagrange_eval(const std::vector<double>& nodes, double x, double* out);

// Device views handed to kernels (by value).
template <typename T>
struct MeshView {
  int64_t n_cells;
  int64_t n_nodes;
  int nconf, nsub, nwall, nf;  // faces: [0,nconf) conforming, then subfaces, then walls
  const T* Ja;      // [dim*dim][n_nodes], Ja[a*dim+b] = J d xi^a / d x_b
  const T* invJ;    // [n_nodes]
  const T* rhob;    // [n_nodes] background density
  const T* pb;      // [n_nodes] background pressure
  const T* wJ;      // [n_nodes] w_i J_i (mass matrix diagonal)
  const int* face_m;    // [nf] minus (fine) cell
  const int* face_lfm;  // [nf] minus local face
  const int* face_p;    // [nf] plus cell / coarse cell (-1 for walls)
  const int* face_lfp;  // [nf] plus / coarse local face
  const int* face_s;    // [nf] packed subface position (subfaces only)
  const T* fn;      // [dim][nf*NF] unit normal out of the minus side
  const T* fsj;     // [nf*NF] |J grad xi^a| (surface Jacobian)
  const int* cell_face;  // [n_cells*2*dim] (face << 2) | side; side 0 minus, 1 plus, 2 coarse, 3 wall
  const int* fnode_m;    // [nf*NF] node index of each face node on the minus side
  const int* fnode_p;    // [nf*NF] node index on the plus side (conforming faces; -1 otherwise)
  const int* cell_cmask; // [n_cells] bit lf set if local face lf is the coarse side of a 2:1 face
  // [n_cells*2*dim] per cell face: (neighbour cell << 4) | (s << 2) | kind, read as unsigned;
  // kind 0 conforming (the neighbour), 1 fine side of a 2:1 face (the coarse cell, s = the
  // subface position), 2 coarse side, 3 wall
  const int* cell_link;
  const T* tab;     // packed Tables1D of the mesh's degree
  T gravity;
  // Geometry in compact form, for kernels that recompute the metric terms:
  // every cell is affine in the horizontal coordinates (x = x0 + hb_a 2^-l
  // (xi + 1), likewise y), so J d xi^a / d x_b and J follow from the nodal
  // heights alone.  zdev is the height of a node above its computational
  // height (z - zeta: the terrain-following displacement, small next to z,
  // which keeps its derivatives accurate in FP32).
  const T* zdev;          // [n_nodes]
  const int* cell_level;  // [n_cells] refinement level
  T hb[3];                // half width of a base cell per axis
  int geo_z;              // 1 if every cell is affine in x (and y)
  int aff;                // 1 if every cell is affine in x (and y) to rounding: the metric entries
                          // outside the diagonal and the last row are stored as zeros and the
                          // implicit passes skip them
  const T* cell_zeta0;    // [n_cells] computational height of the cell's lower face
  // Hydrostatic background as a function of height: cubic Hermite data at
  // bg_m + 1 equally spaced heights from bg_z0 (spacing 1/bg_idz), four values
  // per height: p_bar, dz dp_bar/dz, rho_bar, dz drho_bar/dz (dz = the spacing)
  const T* bg_tab;
  T bg_z0, bg_idz;
  int bg_m;
  // Cell batches of the implicit cell passes (one CTA each; the mesh's active
  // partition): batch b = cells [bdesc[b].x, bdesc[b].y) (at most CPB), its
  // coarse-side entries [bdesc[b].z, bdesc[b].w): per cell in order, per
  // coarse local face in order (a slot), per fine point j = s NF + q of the
  // face's subfaces; ce_meta = lc | lf << 6 | j << 9, ce_node = the fine-side
  // node, ce_w[b * n_ce + e] = 1/2 |N| n_b / w_end at it (w_end the GLL end
  // weight: the face terms enter the cell passes divided by it).  cell_coarse[c] =
  // coarse-face mask | (batch slot of the cell's first one) << 8.
  const int4* bdesc;
  int nbat;
  const int* cell_coarse;
  const int* ce_meta;
  const int* ce_node;
  const T* ce_w;
  int n_ce;
};

}  // namespace dg

namespace dg {
// Argument tables of batched launches recorded into a CUDA graph: the tables
// are written into `host` while the graph is captured and copied to `dev` once
// the capture has ended (before the graph's first launch), so the captured
// launches read tables that stay in place for every replay.
struct BatchArena {
  unsigned char* dev = nullptr;
  std::vector<unsigned char> host;
  size_t used = 0;
  // 256-byte aligned region of `bytes`, or SIZE_MAX if the arena is full
  size_t take(size_t bytes) {
    const size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > host.size()) return SIZE_MAX;
    used = off + bytes;
    return off;
  }
};
}  // namespace dg

struct dg_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t own_stream = nullptr;
  // optional per-operator timing with CUDA events (see dg_profile_*)
  bool prof = false;
  bool prof_clocks = false;  // in-kernel phase and per-CTA clocks of the persistent solves too
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  std::vector<std::pair<int, size_t>> ev_pending;  // (category, index of the start event)
  double prof_ms[8] = {0};
  long long prof_n[8] = {0};
  long long launches = 0;  // kernels launched through this context
  unsigned long long* d_phase = nullptr;  // [16] ns per fused-GMRES phase (profiling on)
  void* d_batch = nullptr;  // workspace of batched solves (argument table, CTA map, barriers)
  size_t batch_bytes = 0;
  int* d_batch_err = nullptr;  // barrier-timeout flag of batched launches
  // bounded barrier of batched launches: the wait limit, and a test hook that
  // declares one CTA more for one member than its launch gives it (-1: off)
  unsigned long long batch_timeout_ns = 2000000000ull;
  int batch_missing_cta_member = -1;
  dg::BatchArena* arena = nullptr;  // set while a batch plan is being captured
};

namespace dg {
inline void count_launches(dg_ctx* c, int n) {
  if (c) c->launches += n;
}
// Record a start event for category `cat` on stream s; returns a token for prof_end
// (or SIZE_MAX when profiling is off).  Events are resolved by prof_resolve().
size_t prof_begin(dg_ctx* c, cudaStream_t s);
void prof_end(dg_ctx* c, int cat, size_t tok, cudaStream_t s);
void prof_resolve(dg_ctx* c);  // synchronises the device first
struct ProfScope {
  dg_ctx* c;
  int cat;
  size_t tok;
  cudaStream_t s;
  ProfScope(dg_ctx* c_, int cat_, cudaStream_t s_) : c(c_), cat(cat_), tok(prof_begin(c_, s_)), s(s_) {}
  ~ProfScope() { prof_end(c, cat, tok, s); }
};
}  // namespace dg

namespace dg {
struct CellPartition {
  void* d_int = nullptr;  // int4 bdesc[nbat], cell_coarse[K], ce_meta[E], ce_node[E]
  void* d_f64 = nullptr;  // ce_w [dim][E]
  void* d_f32 = nullptr;
  int nbat = 0, n_ce = 0;
  double cost_max = 0.0;  // the largest batch's work (nodes + face points)
};
}  // namespace dg

struct dg_mesh {
  dg_ctx* ctx = nullptr;
  dg_mesh_desc desc{};
  int dim = 0, degree = 0, n = 0, nc = 0, nf_nodes = 0, V = 0;
  int64_t K = 0, Nn = 0;
  int max_level = 0;
  double min_edge = 0;
  // host tables
  std::vector<uint8_t> level;
  std::vector<int32_t> ijk;
  std::vector<int32_t> conf;   // [nconf*4]
  std::vector<int32_t> subs;   // [nsub*4] fine, lf_fine, coarse, s (sorted by coarse, lf, s)
  std::vector<int32_t> subs_lfc;
  std::vector<int32_t> walls;  // [nwall*2]
  std::vector<double> X;       // [dim][K][nc]
  int nconf = 0, nsub = 0, nwall = 0, nf = 0;
  size_t device_bytes = 0;
  // device memory: one block each for FP64 and FP32 geometry + int tables + scratch
  void* d_int = nullptr;
  void* d_f64 = nullptr;
  void* d_f32 = nullptr;
  void* d_scratch = nullptr;  // face fluxes + grad intermediate (FP64-sized)
  size_t scratch_bytes = 0;
  dg::MeshView<double> v64{};
  dg::MeshView<float> v32{};
  double* d_face_scratch64 = nullptr;
  double* d_vec_scratch64 = nullptr;  // [dim][Nn]
  double* d_red_scratch = nullptr;    // [2*512] block partials of the conservation sums
  double* d_tau = nullptr;            // [Nn] Rayleigh damping rate per node (NULL: no sponge layer)
  // autotuned Helmholtz solver per precision: the timed first solve of each
  // form (0 = GMRES, one launch per Krylov kernel; 1 = GMRES persistent;
  // 2 = Chebyshev persistent; 0 ms = not timed) and the form chosen last
  mutable int tuned_form[2] = {-1, -1};
  mutable float tuned_ms[2][3] = {{0, 0, 0}, {0, 0, 0}};
  // cell partitions of the implicit passes: [0] CPB consecutive cells per
  // batch, [1] balanced for the persistent solves (small meshes: cost-balanced
  // batches, one per CTA; large meshes: the uniform batches in a cost-balanced
  // order over the CTAs); the autotuner picks one per precision
  dg::CellPartition part[2];
  int n_parts = 0;
  int active_part = 0;
  mutable int tuned_part[2] = {0, 0};
  mutable float tuned_ms_balanced[2][3] = {{0, 0, 0}, {0, 0, 0}};
};

namespace dg {
// Make partition k (0 uniform, 1 cost-balanced) the one the mesh's implicit passes use.
void set_partition(const dg_mesh* m, int k);
}  // namespace dg
