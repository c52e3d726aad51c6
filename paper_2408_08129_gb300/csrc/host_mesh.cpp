// Mesh construction on the host: connectivity of the 2:1 tree forest, the
// terrain-following isoparametric geometry, metric terms, face normals and the
// hydrostatic background, followed by one upload per precision.
//
// Sec. 3.1: flow over orography on a terrain-following mesh refined near the
// ground with neighbours of different resolution both horizontally and
// vertically (no hanging nodes in the DG sense, Sec. 2).  Mesh-map reading:
// z = zeta + h(x,y)(1 - zeta/H), isoparametric of degree r on base cells,
// refined cells sampling their base cell's polynomial (watertight 2:1 faces);
// metric terms J grad(xi^a) by rotated nodal derivatives (2D) or cross
// products of nodal tangents (3D; exact discrete metric identities because x
// and y are affine per cell).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <unordered_map>
#include <unordered_set>

#include "dg_internal.h"
#include "partition.h"

namespace dg {

namespace {

inline uint64_t key_of(int l, const int* c) {
  return ((uint64_t)l << 60) | ((uint64_t)(uint32_t)c[0] << 40) | ((uint64_t)(uint32_t)c[1] << 20) |
         (uint64_t)(uint32_t)c[2];
}

double hill(const dg_mesh_desc& d, double x, double y) {
  const double xc = d.hill_xc, yc = d.hill_yc, a = d.hill_half_width;
  switch (d.hill_kind) {
    case DG_HILL_NONE:
      return 0.0;
    case DG_HILL_GAUSS: {
      double r2 = (x - xc) * (x - xc) + (d.dim == 3 ? (y - yc) * (y - yc) : 0.0);
      return d.hill_hc * std::exp(-std::log(2.0) * r2 / (a * a));
    }
    case DG_HILL_BELL: {
      double q = 1.0 + ((x - xc) / a) * ((x - xc) / a) + (d.dim == 3 ? ((y - yc) / a) * ((y - yc) / a) : 0.0);
      return d.hill_hc / (q * std::sqrt(q));
    }
    case DG_HILL_PARABOLA: {
      double s = 1.0 - ((x - xc) / a) * ((x - xc) / a) - (d.dim == 3 ? ((y - yc) / a) * ((y - yc) / a) : 0.0);
      return d.hill_hc * s;
    }
  }
  return 0.0;
}

// hydrostatic background at height z (Sec. 3.1; stratified p with the factor g restored)
void background(const dg_mesh_desc& d, double z, double* rho, double* p) {
  const double g = 9.81;
  if (d.atm_kind == DG_ATM_NONE) {
    *rho = 0.0;
    *p = 0.0;
  } else if (d.atm_kind == DG_ATM_ISOTHERMAL) {
    *p = d.atm_p_ref * std::exp(-g * z / (kRgas * d.atm_T));
    *rho = *p / (kRgas * d.atm_T);
  } else {
    const double n2 = d.atm_N * d.atm_N;
    const double cg = (kGamma - 1.0) / kGamma;
    const double rho_ref = d.atm_p_ref / (kRgas * d.atm_T);
    const double s = std::exp(-n2 * z / g);
    const double base = 1.0 - (g * g / n2) * cg * (rho_ref / d.atm_p_ref) * (1.0 - s);
    *p = d.atm_p_ref * std::pow(base, 1.0 / cg);
    *rho = rho_ref * std::pow(*p / d.atm_p_ref, 1.0 / kGamma) * s;
  }
}

inline int ipow(int b, int e) {
  int r = 1;
  while (e--) r *= b;
  return r;
}

}  // namespace

// node index of face node k on local face lf (tangential axes ascending, first fastest)
int host_face_node(int dim, int n, int lf, int k) {
  const int a = lf >> 1, side = lf & 1;
  int idx[3] = {0, 0, 0};
  idx[a] = side ? n - 1 : 0;
  int t = 0;
  for (int b = 0; b < dim; ++b) {
    if (b == a) continue;
    idx[b] = (t == 0) ? (k % n) : (k / n);
    ++t;
  }
  return idx[0] + n * idx[1] + n * n * idx[2];
}

// Caller-given conforming faces and walls, checked against the cells' levels
// and integer coordinates (the subfaces are checked here too and copied by the
// caller of this function).
int caller_topology(dg_mesh* m, std::vector<int32_t>& conf, std::vector<int32_t>& walls) {
  const dg_mesh_desc& d = m->desc;
  const int dim = d.dim;
  const int64_t K = d.n_cells;
  if (!d.conforming || !d.subfaces || !d.walls)
    if (!((d.conforming || d.n_conforming == 0) && (d.subfaces || d.n_subfaces == 0) && (d.walls || d.n_walls == 0)))
      return fail(DG_EINVAL, "face table pointer missing for a non-zero count");
  if (d.n_conforming < 0 || d.n_subfaces < 0 || d.n_walls < 0) return fail(DG_EINVAL, "negative face count");
  if (d.n_conforming + d.n_subfaces + d.n_walls > ((int64_t)1 << 29)) return fail(DG_EINVAL, "too many faces");
  auto cell_ok = [&](int64_t c) { return c >= 0 && c < K; };
  auto lf_ok = [&](int lf) { return lf >= 0 && lf < 2 * dim; };
  // same-level neighbour coordinate of cell c across local face lf; false at a wall
  auto neighbour = [&](int64_t c, int lf, int* nb) {
    const int l = m->level[c], a = lf >> 1;
    for (int b = 0; b < 3; ++b) nb[b] = b < dim ? m->ijk[c * dim + b] : 0;
    nb[a] += (lf & 1) ? 1 : -1;
    const int nmax = d.base[a] << l;
    if (nb[a] < 0 || nb[a] >= nmax) {
      if (!d.periodic[a]) return false;
      nb[a] = (nb[a] + nmax) % nmax;
    }
    return true;
  };
  for (int64_t j = 0; j < d.n_conforming; ++j) {
    const int32_t* e = d.conforming + 4 * j;
    if (!cell_ok(e[0]) || !cell_ok(e[2]) || !lf_ok(e[1]) || e[3] != (e[1] ^ 1))
      return fail(DG_EUNBALANCED, "bad conforming face entry");
    int nb[3];
    if (m->level[e[0]] != m->level[e[2]] || !neighbour(e[0], e[1], nb))
      return fail(DG_EUNBALANCED, "conforming face between cells that are not same-level neighbours");
    for (int b = 0; b < dim; ++b)
      if (nb[b] != m->ijk[(int64_t)e[2] * dim + b])
        return fail(DG_EUNBALANCED, "conforming face between cells that are not same-level neighbours");
    conf.insert(conf.end(), e, e + 4);
  }
  for (int64_t j = 0; j < d.n_subfaces; ++j) {
    const int32_t* e = d.subfaces + 4 * j;
    if (!cell_ok(e[0]) || !cell_ok(e[2]) || !lf_ok(e[1]) || e[3] < 0 || e[3] >= (1 << (dim - 1)))
      return fail(DG_EUNBALANCED, "bad subface entry");
    int nb[3];
    if (m->level[e[0]] != m->level[e[2]] + 1 || !neighbour(e[0], e[1], nb))
      return fail(DG_EUNBALANCED, "2:1 face between cells that are not one level apart and adjacent");
    int s = 0, t = 0;
    for (int b = 0; b < dim; ++b) {
      if (nb[b] >> 1 != m->ijk[(int64_t)e[2] * dim + b])
        return fail(DG_EUNBALANCED, "2:1 face between cells that are not one level apart and adjacent");
      if (b == (e[1] >> 1)) continue;
      s |= (m->ijk[(int64_t)e[0] * dim + b] & 1) << t;
      ++t;
    }
    if (s != e[3]) return fail(DG_EUNBALANCED, "subface position does not match the cell coordinates");
  }
  for (int64_t j = 0; j < d.n_walls; ++j) {
    const int32_t* e = d.walls + 2 * j;
    int nb[3];
    if (!cell_ok(e[0]) || !lf_ok(e[1]) || neighbour(e[0], e[1], nb))
      return fail(DG_EUNBALANCED, "wall entry not on a non-periodic domain boundary");
    walls.insert(walls.end(), e, e + 2);
  }
  return DG_OK;
}

// Caller-given node coordinates must close every face: both sides of a
// conforming face at the same points, and each fine face on its coarse face's
// polynomial (evaluated at the fine points with the subinterval
// interpolation), to 1e-9 of the domain size.
int check_watertight(const dg_mesh* m, const Tables1D& tab, const std::vector<int>& face_m,
                     const std::vector<int>& face_lfm, const std::vector<int>& face_p,
                     const std::vector<int>& face_lfp, const std::vector<int>& face_s) {
  const int dim = m->dim, n = m->n, nc = m->nc, NF = m->nf_nodes;
  const int64_t K = m->K;
  double ext = 0.0;
  for (int a = 0; a < dim; ++a) ext = std::max(ext, m->desc.extent[a]);
  const double tol = 1e-9 * ext;
  auto X = [&](int b, int64_t c, int q) { return m->X[((size_t)b * K + c) * nc + q]; };
  for (int f = 0; f < m->nconf + m->nsub; ++f) {
    const bool sub = f >= m->nconf;
    for (int k = 0; k < NF; ++k) {
      const int qm = host_face_node(dim, n, face_lfm[f], k);
      for (int b = 0; b < dim; ++b) {
        double xo;
        if (!sub) {
          xo = X(b, face_p[f], host_face_node(dim, n, face_lfp[f], k));
        } else {
          // coarse face polynomial at fine face node k of subface position s
          const int s = face_s[f], k1 = k % n, k2 = k / n;
          xo = 0.0;
          for (int j2 = 0; j2 < (dim == 3 ? n : 1); ++j2)
            for (int j1 = 0; j1 < n; ++j1) {
              double w = tab.I[(size_t)(s & 1) * n * n + (size_t)k1 * n + j1];
              if (dim == 3) w *= tab.I[(size_t)((s >> 1) & 1) * n * n + (size_t)k2 * n + j2];
              xo += w * X(b, face_p[f], host_face_node(dim, n, face_lfp[f], j1 + n * j2));
            }
        }
        double diff = std::fabs(X(b, face_m[f], qm) - xo);
        // across a periodic boundary the two sides sit one period apart along that axis
        if (m->desc.periodic[b] && std::fabs(diff - m->desc.extent[b]) <= tol) diff = 0.0;
        if (!(diff <= tol)) return fail(DG_EUNBALANCED, "node coordinates are not watertight across a face");
      }
    }
  }
  return DG_OK;
}

namespace {

// Coarse sides of the 2:1 faces per cell (see build_mesh) and the work per cell
struct CoarseLists {
  int dim = 0, np = 0;
  std::vector<int> cmask;   // [K] coarse-face mask
  std::vector<int> off;     // [K+1] first coarse face of each cell (in units of faces)
  std::vector<int> node;    // [faces * np] fine node of each point
  std::vector<double> w;    // [faces * np * dim] 1/2 |N| n of each point
  std::vector<double> cost; // [K] work of the cell's implicit passes (nodes + face points)
};

// One partition of the cells into batches (bstart: K-terminated starts) with
// its coarse-side entry lists, uploaded to a device block of its own; order
// (optional) places batch order[p] at position p.
int build_partition(dg_mesh* m, const CoarseLists& cl, const std::vector<int>& bstart, CellPartition& P,
                    const std::vector<int>* order = nullptr) {
  const int dim = cl.dim, np = cl.np;
  const int nbat = (int)bstart.size() - 1;
  std::vector<int4> bdesc(nbat);
  std::vector<int> cell_coarse(m->K, 0), meta, node;
  std::vector<double> w;
  double cmax = 0.0;
  for (int b = 0; b < nbat; ++b) {
    const int e0 = (int)meta.size();
    int slot = 0;
    double cst = 0.0;
    for (int c = bstart[b]; c < bstart[b + 1]; ++c) {
      const int lc = c - bstart[b];
      cst += cl.cost[c];
      cell_coarse[c] = cl.cmask[c] | (slot << 8);
      for (int k = cl.off[c]; k < cl.off[c + 1]; ++k, ++slot) {
        int lf = 0, seen = -1;  // local face of the cell's (k - off)-th coarse face
        for (; lf < 2 * dim; ++lf)
          if ((cl.cmask[c] >> lf) & 1)
            if (++seen == k - cl.off[c]) break;
        for (int j = 0; j < np; ++j) {
          meta.push_back(lc | (lf << 6) | (j << 9));
          node.push_back(cl.node[(size_t)k * np + j]);
        }
      }
    }
    bdesc[b] = make_int4(bstart[b], bstart[b + 1], e0, (int)meta.size());
    cmax = std::max(cmax, cst);
  }
  const size_t E = meta.size();
  w.assign((size_t)dim * E, 0.0);
  for (int b = 0; b < nbat; ++b)
    for (int e = bdesc[b].z; e < bdesc[b].w; ++e) {
      // the batch's entries follow the per-cell lists in order: entry e is global point
      // off[c0] np + (e - e0)
      const size_t g = (size_t)cl.off[bstart[b]] * np + (size_t)(e - bdesc[b].z);
      for (int d = 0; d < dim; ++d) w[(size_t)d * E + e] = cl.w[g * dim + d];
    }
  if (order) {
    std::vector<int4> placed(nbat);
    for (int p = 0; p < nbat; ++p) placed[p] = bdesc[(*order)[p]];
    bdesc.swap(placed);
  }
  const size_t n_int = 4 * (size_t)nbat + (size_t)m->K + 2 * E;
  DG_CUDA(cudaMalloc(&P.d_int, n_int * sizeof(int) + 64));
  DG_CUDA(cudaMalloc(&P.d_f64, w.size() * sizeof(double) + 64));
  DG_CUDA(cudaMalloc(&P.d_f32, w.size() * sizeof(float) + 64));
  int* ib = (int*)P.d_int;
  DG_CUDA(cudaMemcpy(ib, bdesc.data(), (size_t)nbat * sizeof(int4), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(ib + 4 * (size_t)nbat, cell_coarse.data(), (size_t)m->K * sizeof(int), cudaMemcpyHostToDevice));
  if (E) {
    DG_CUDA(cudaMemcpy(ib + 4 * (size_t)nbat + m->K, meta.data(), E * sizeof(int), cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(ib + 4 * (size_t)nbat + m->K + E, node.data(), E * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<float> wf(w.begin(), w.end());
    DG_CUDA(cudaMemcpy(P.d_f64, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(P.d_f32, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  P.nbat = nbat;
  P.n_ce = (int)E;
  P.cost_max = cmax;
  m->device_bytes += n_int * sizeof(int) + w.size() * (sizeof(double) + sizeof(float));
  return DG_OK;
}

}  // namespace

// Make partition k the one every implicit cell pass of the mesh uses.
void set_partition(const dg_mesh* cm, int k) {
  dg_mesh* m = const_cast<dg_mesh*>(cm);
  if (k < 0 || k >= m->n_parts) k = 0;
  const CellPartition& P = m->part[k];
  if (!P.d_int) return;
  const int* ib = (const int*)P.d_int;
  auto put = [&](auto& v, auto* w) {
    v.bdesc = (const int4*)ib;
    v.nbat = P.nbat;
    v.cell_coarse = ib + 4 * (size_t)P.nbat;
    v.ce_meta = v.cell_coarse + m->K;
    v.ce_node = v.ce_meta + P.n_ce;
    v.ce_w = w;
    v.n_ce = P.n_ce;
  };
  put(m->v64, (const double*)P.d_f64);
  put(m->v32, (const float*)P.d_f32);
  m->active_part = k;
}

int build_mesh(dg_mesh* m) {
  const dg_mesh_desc& d = m->desc;
  const int dim = d.dim, r = d.degree, n = r + 1;
  m->dim = dim;
  m->degree = r;
  m->n = n;
  m->nc = ipow(n, dim);
  m->nf_nodes = ipow(n, dim - 1);
  m->V = dim + 2;
  m->K = d.n_cells;
  m->Nn = m->K * m->nc;
  const int64_t K = m->K;
  const int nc = m->nc, NF = m->nf_nodes;

  // ---------------------------------------------------------------- topology
  std::unordered_map<uint64_t, int> leaf;
  leaf.reserve(K * 2);
  std::unordered_set<uint64_t> internal;
  m->max_level = 0;
  for (int64_t c = 0; c < K; ++c) {
    int l = m->level[c];
    int ijk[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      ijk[a] = m->ijk[c * dim + a];
      if (ijk[a] < 0 || ijk[a] >= (d.base[a] << l)) return fail(DG_EINVAL, "cell coordinate out of range");
    }
    if (!leaf.emplace(key_of(l, ijk), (int)c).second) return fail(DG_EINVAL, "duplicate cell");
    m->max_level = std::max(m->max_level, l);
    for (int ll = l - 1; ll >= 0; --ll) {
      for (int a = 0; a < 3; ++a) ijk[a] >>= 1;
      internal.insert(key_of(ll, ijk));
    }
  }
  for (const auto& kv : leaf)
    if (internal.count(kv.first)) return fail(DG_EINVAL, "a cell overlaps a refined cell");

  std::vector<int32_t> conf, walls;
  struct Sub {
    int fine, lff, coarse, lfc, s;
  };
  std::vector<Sub> subs;
  const bool caller_faces = d.conforming || d.subfaces || d.walls;
  if (caller_faces) {
    int rc = caller_topology(m, conf, walls);
    if (rc != DG_OK) return rc;
    for (int64_t j = 0; j < d.n_subfaces; ++j) {
      const int32_t* e = d.subfaces + 4 * j;
      subs.push_back({e[0], e[1], e[2], e[1] ^ 1, e[3]});
    }
  }
  for (int64_t c = 0; c < (caller_faces ? 0 : K); ++c) {
    const int l = m->level[c];
    int ijk[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) ijk[a] = m->ijk[c * dim + a];
    for (int a = 0; a < dim; ++a) {
      for (int side = 0; side < 2; ++side) {
        const int lf = 2 * a + side;
        const int nmax = d.base[a] << l;
        int nb[3] = {ijk[0], ijk[1], ijk[2]};
        nb[a] += side ? 1 : -1;
        if (nb[a] < 0 || nb[a] >= nmax) {
          if (!d.periodic[a]) {
            walls.push_back((int32_t)c);
            walls.push_back(lf);
            continue;
          }
          nb[a] = (nb[a] + nmax) % nmax;
        }
        auto it = leaf.find(key_of(l, nb));
        if (it != leaf.end()) {
          if (side == 1) {
            conf.push_back((int32_t)c);
            conf.push_back(lf);
            conf.push_back(it->second);
            conf.push_back(lf - 1);
          }
          continue;
        }
        int par[3] = {nb[0] >> 1, nb[1] >> 1, nb[2] >> 1};
        auto ip = (l > 0) ? leaf.find(key_of(l - 1, par)) : leaf.end();
        if (ip != leaf.end()) {
          int s = 0, t = 0;
          for (int b = 0; b < dim; ++b) {
            if (b == a) continue;
            s |= (ijk[b] & 1) << t;
            ++t;
          }
          subs.push_back({(int)c, lf, ip->second, 2 * a + (1 - side), s});
          continue;
        }
        if (internal.count(key_of(l, nb))) {
          // coarse side: the children touching this face must be leaves (2:1)
          for (int o = 0; o < (1 << dim); ++o) {
            int ch[3] = {0, 0, 0};
            for (int b = 0; b < dim; ++b) ch[b] = 2 * nb[b] + ((o >> b) & 1);
            if (((o >> a) & 1) != (side ? 0 : 1)) continue;
            if (!leaf.count(key_of(l + 1, ch))) return fail(DG_EUNBALANCED, "mesh is not 2:1 balanced");
          }
          continue;
        }
        return fail(DG_EUNBALANCED, "mesh is not 2:1 balanced");
      }
    }
  }
  std::sort(subs.begin(), subs.end(), [](const Sub& x, const Sub& y) {
    if (x.coarse != y.coarse) return x.coarse < y.coarse;
    if (x.lfc != y.lfc) return x.lfc < y.lfc;
    return x.s < y.s;
  });
  m->nconf = (int)(conf.size() / 4);
  m->nsub = (int)subs.size();
  m->nwall = (int)(walls.size() / 2);
  m->nf = m->nconf + m->nsub + m->nwall;
  m->conf = conf;
  m->walls = walls;
  m->subs.clear();
  m->subs_lfc.clear();
  for (const Sub& s : subs) {
    m->subs.insert(m->subs.end(), {s.fine, s.lff, s.coarse, s.s});
    m->subs_lfc.push_back(s.lfc);
  }

  const int nf = m->nf;
  std::vector<int> face_m(nf), face_lfm(nf), face_p(nf), face_lfp(nf), face_s(nf, 0);
  std::vector<int> cell_face(K * 2 * dim, -1);
  // every cell face takes exactly one entry (caller tables may list one twice)
  auto claim = [&](int c, int lf, int code) {
    int& slot = cell_face[(size_t)c * 2 * dim + lf];
    if (slot >= 0) return false;
    slot = code;
    return true;
  };
  for (int f = 0; f < m->nconf; ++f) {
    face_m[f] = conf[4 * f];
    face_lfm[f] = conf[4 * f + 1];
    face_p[f] = conf[4 * f + 2];
    face_lfp[f] = conf[4 * f + 3];
    if (!claim(face_m[f], face_lfm[f], (f << 2) | 0) || !claim(face_p[f], face_lfp[f], (f << 2) | 1))
      return fail(DG_EUNBALANCED, "a cell face is listed twice");
  }
  const int nsubface = 1 << (dim - 1);
  for (int j = 0; j < m->nsub; ++j) {
    const int f = m->nconf + j;
    const Sub& s = subs[j];
    face_m[f] = s.fine;
    face_lfm[f] = s.lff;
    face_p[f] = s.coarse;
    face_lfp[f] = s.lfc;
    face_s[f] = s.s;
    if (!claim(s.fine, s.lff, (f << 2) | 0)) return fail(DG_EUNBALANCED, "a cell face is listed twice");
    if (s.s == 0) {
      // the coarse face's subfaces must be the next 2^(d-1) entries, s = 0, 1, ...
      for (int q = 0; q < nsubface; ++q) {
        if (j + q >= m->nsub || subs[j + q].coarse != s.coarse || subs[j + q].lfc != s.lfc || subs[j + q].s != q)
          return fail(DG_EUNBALANCED, "incomplete set of subfaces on a 2:1 face");
      }
      if (!claim(s.coarse, s.lfc, (f << 2) | 2)) return fail(DG_EUNBALANCED, "a cell face is listed twice");
    } else if (j == 0 || subs[j - 1].coarse != s.coarse || subs[j - 1].lfc != s.lfc) {
      return fail(DG_EUNBALANCED, "incomplete set of subfaces on a 2:1 face");
    }
  }
  for (int j = 0; j < m->nwall; ++j) {
    const int f = m->nconf + m->nsub + j;
    face_m[f] = walls[2 * j];
    face_lfm[f] = walls[2 * j + 1];
    face_p[f] = -1;
    face_lfp[f] = -1;
    if (!claim(face_m[f], face_lfm[f], (f << 2) | 3)) return fail(DG_EUNBALANCED, "a cell face is listed twice");
  }
  for (size_t i = 0; i < cell_face.size(); ++i)
    if (cell_face[i] < 0) return fail(DG_EUNBALANCED, "mesh is not watertight");

  // ---------------------------------------------------------------- geometry
  Tables1D tab = make_tables(r);
  const double H = d.extent[dim - 1];
  double hb[3];
  for (int a = 0; a < dim; ++a) hb[a] = d.extent[a] / d.base[a];
  m->min_edge = 1e300;
  for (int a = 0; a < dim; ++a) m->min_edge = std::min(m->min_edge, hb[a] / (1 << m->max_level));

  m->X.assign((size_t)dim * K * nc, 0.0);
  std::vector<double> Xb((size_t)dim * nc), tmp((size_t)dim * nc), tmp2((size_t)dim * nc);
  std::unordered_map<uint64_t, std::vector<double>> interp_cache;  // (level, axis, offset) -> n x n
  std::vector<int> mi((size_t)nc * 3);
  for (int q = 0; q < nc; ++q) {
    mi[3 * q] = q % n;
    mi[3 * q + 1] = (q / n) % n;
    mi[3 * q + 2] = q / (n * n);
  }
  if (d.node_xyz) m->X.assign(d.node_xyz, d.node_xyz + (size_t)dim * K * nc);
  for (int64_t c = 0; c < (d.node_xyz ? 0 : K); ++c) {
    const int l = m->level[c];
    int ijk[3] = {0, 0, 0}, bijk[3] = {0, 0, 0}, off[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      ijk[a] = m->ijk[c * dim + a];
      bijk[a] = ijk[a] >> l;
      off[a] = ijk[a] - (bijk[a] << l);
    }
    // base cell nodes: analytic terrain-following map at the base GLL nodes
    for (int q = 0; q < nc; ++q) {
      double comp[3];
      for (int a = 0; a < dim; ++a) comp[a] = bijk[a] * hb[a] + 0.5 * (tab.xi[mi[3 * q + a]] + 1.0) * hb[a];
      for (int a = 0; a < dim; ++a) Xb[(size_t)a * nc + q] = comp[a];
      const double zeta = comp[dim - 1];
      const double hx = hill(d, comp[0], dim == 3 ? comp[1] : 0.0);
      Xb[(size_t)(dim - 1) * nc + q] = zeta + hx * (1.0 - zeta / H);
    }
    // interpolate axis by axis onto this cell's nodes (sum factorisation)
    const std::vector<double>* src = &Xb;
    std::vector<double>* dst = &tmp;
    for (int a = 0; a < dim; ++a) {
      uint64_t key = ((uint64_t)l << 32) | ((uint64_t)a << 24) | (uint64_t)off[a];
      auto itc = interp_cache.find(key);
      if (itc == interp_cache.end()) {
        std::vector<double> L((size_t)n * n);
        for (int i = 0; i < n; ++i) {
          const double ref = -1.0 + (2.0 * off[a] + tab.xi[i] + 1.0) / (double)(1 << l);
          lagrange_eval(tab.xi, ref, &L[(size_t)i * n]);
        }
        itc = interp_cache.emplace(key, std::move(L)).first;
      }
      const std::vector<double>& L = itc->second;
      const int stride = ipow(n, a);
      for (int b = 0; b < dim; ++b)
        for (int q = 0; q < nc; ++q) {
          const int ia = mi[3 * q + a];
          const int q0 = q - ia * stride;
          double s = 0.0;
          for (int j = 0; j < n; ++j) s += L[(size_t)ia * n + j] * (*src)[(size_t)b * nc + q0 + j * stride];
          (*dst)[(size_t)b * nc + q] = s;
        }
      src = dst;
      dst = (dst == &tmp) ? &tmp2 : &tmp;
    }
    for (int b = 0; b < dim; ++b)
      for (int q = 0; q < nc; ++q) m->X[((size_t)b * K + c) * nc + q] = (*src)[(size_t)b * nc + q];
  }

  if (d.node_xyz) {
    for (double v : m->X)
      if (!std::isfinite(v)) return fail(DG_EINVAL, "non-finite node coordinate");
    int rc = check_watertight(m, tab, face_m, face_lfm, face_p, face_lfp, face_s);
    if (rc != DG_OK) return rc;
  }

  // height of every node above its computational height, and whether every
  // cell is affine in the horizontal coordinates (then the metric terms
  // follow from these heights)
  std::vector<double> zdev(m->Nn);
  bool geo_z = true;
  bool aff = true;  // affine in x (and y) to rounding
  for (int64_t c = 0; c < K; ++c) {
    const int l = m->level[c];
    for (int q = 0; q < nc; ++q) {
      for (int a = 0; a < dim; ++a) {
        const double h = hb[a] / (double)(1 << l);
        const double comp = m->ijk[c * dim + a] * h + 0.5 * (tab.xi[mi[3 * q + a]] + 1.0) * h;
        const double xv = m->X[((size_t)a * K + c) * nc + q];
        if (a < dim - 1) {
          if (std::fabs(xv - comp) > 1e-9 * d.extent[a]) geo_z = false;
          if (std::fabs(xv - comp) > 1e-12 * d.extent[a]) aff = false;
        } else {
          zdev[(size_t)c * nc + q] = xv - comp;
        }
      }
    }
  }

  // metric terms at nodes
  std::vector<double> Ja((size_t)dim * dim * m->Nn), invJ(m->Nn), wJ(m->Nn), rhob(m->Nn), pb(m->Nn);
  for (int64_t c = 0; c < K; ++c) {
    for (int q = 0; q < nc; ++q) {
      double t[3][3] = {{0}};  // t[a][b] = d x_b / d xi^a
      for (int a = 0; a < dim; ++a) {
        const int stride = ipow(n, a);
        const int ia = mi[3 * q + a];
        const int q0 = q - ia * stride;
        for (int b = 0; b < dim; ++b) {
          double s = 0.0;
          for (int k = 0; k < n; ++k) s += tab.D[ia * n + k] * m->X[((size_t)b * K + c) * nc + q0 + k * stride];
          t[a][b] = s;
        }
      }
      double M[3][3] = {{0}}, J;
      if (dim == 2) {
        J = t[0][0] * t[1][1] - t[1][0] * t[0][1];
        M[0][0] = t[1][1];
        M[0][1] = -t[1][0];
        M[1][0] = -t[0][1];
        M[1][1] = t[0][0];
      } else {
        for (int a = 0; a < 3; ++a) {
          const double* u = t[(a + 1) % 3];
          const double* v = t[(a + 2) % 3];
          M[a][0] = u[1] * v[2] - u[2] * v[1];
          M[a][1] = u[2] * v[0] - u[0] * v[2];
          M[a][2] = u[0] * v[1] - u[1] * v[0];
        }
        J = t[0][0] * M[0][0] + t[0][1] * M[0][1] + t[0][2] * M[0][2];
      }
      if (!(J > 0.0)) return fail(DG_EINVAL, "non-positive Jacobian (hill too steep for the mesh)");
      const int64_t idx = c * nc + q;
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) Ja[(size_t)(a * dim + b) * m->Nn + idx] = M[a][b];
      invJ[idx] = 1.0 / J;
      double wq = 1.0;
      for (int a = 0; a < dim; ++a) wq *= tab.w[mi[3 * q + a]];
      wJ[idx] = wq * J;
      background(d, m->X[((size_t)(dim - 1) * K + c) * nc + q], &rhob[idx], &pb[idx]);
    }
  }
  // on cells affine in the horizontal coordinates (node positions within 1e-12 of the domain
  // size of the affine ones) the metric entries outside the diagonal and the last row vanish;
  // what the differentiation leaves there is rounding of the derivative of constant
  // coordinates, set to zero here, and the implicit passes skip those entries
  if (aff)
    for (int64_t i = 0; i < m->Nn; ++i)
      for (int a = 0; a < dim - 1; ++a)
        for (int b = 0; b < dim; ++b)
          if (b != a) Ja[(size_t)(a * dim + b) * m->Nn + i] = 0.0;
  // face-node normals from the minus (fine) side
  std::vector<double> fn((size_t)dim * nf * NF), fsj((size_t)nf * NF);
  for (int f = 0; f < nf; ++f) {
    const int c = face_m[f], lf = face_lfm[f], a = lf >> 1, side = lf & 1;
    for (int k = 0; k < NF; ++k) {
      const int64_t idx = (int64_t)c * nc + host_face_node(dim, n, lf, k);
      double N[3], s = 0.0;
      for (int b = 0; b < dim; ++b) {
        N[b] = (2 * side - 1) * Ja[(size_t)(a * dim + b) * m->Nn + idx];
        s += N[b] * N[b];
      }
      s = std::sqrt(s);
      fsj[(size_t)f * NF + k] = s;
      for (int b = 0; b < dim; ++b) fn[(size_t)b * nf * NF + (size_t)f * NF + k] = N[b] / s;
    }
  }

  // node indices of the face nodes on both sides (saves the face-table look-ups)
  if (m->Nn >= ((int64_t)1 << 31)) return fail(DG_EINVAL, "too many nodes for 32-bit node indices");
  std::vector<int> fnode_m((size_t)nf * NF), fnode_p((size_t)nf * NF, -1);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < NF; ++k) {
      fnode_m[(size_t)f * NF + k] = face_m[f] * nc + host_face_node(dim, n, face_lfm[f], k);
      if (f < m->nconf) fnode_p[(size_t)f * NF + k] = face_p[f] * nc + host_face_node(dim, n, face_lfp[f], k);
    }

  // Rayleigh damping rate per node: sin^2 profile over the top sponge_depth of physical height,
  // and over sponge_lateral_width from the lateral boundaries; the larger of the two
  std::vector<double> tau;
  const bool top_layer = d.sponge_depth > 0.0 && d.sponge_rate > 0.0;
  const bool lat_layer = d.sponge_lateral_width > 0.0 && d.sponge_lateral_rate > 0.0;
  if (top_layer || lat_layer) {
    const double H = d.extent[dim - 1], zd = H - d.sponge_depth;
    const double half_pi = 0.5 * 3.14159265358979323846;
    tau.assign(m->Nn, 0.0);
    for (int64_t i = 0; i < m->Nn; ++i) {
      const int64_t c = i / nc, q = i % nc;
      double t = 0.0;
      const double z = m->X[((size_t)(dim - 1) * K + c) * nc + q];
      if (top_layer && z > zd) {
        const double sv = std::sin(half_pi * std::min(1.0, (z - zd) / d.sponge_depth));
        t = d.sponge_rate * sv * sv;
      }
      if (lat_layer) {
        double dist = 1e300;
        for (int a = 0; a < dim - 1; ++a) {
          const double x = m->X[((size_t)a * K + c) * nc + q];
          dist = std::min(dist, std::min(x, d.extent[a] - x));
        }
        if (dist < d.sponge_lateral_width) {
          const double sv = std::sin(half_pi * (d.sponge_lateral_width - std::max(dist, 0.0)) / d.sponge_lateral_width);
          t = std::max(t, d.sponge_lateral_rate * sv * sv);
        }
      }
      tau[i] = t;
    }
  }

  // the background as a function of height (cubic Hermite data every ~25 m;
  // interpolation error ~ (dz / scale height)^4 / 384, far below FP32 rounding)
  double zlo = 1e300, zhi = -1e300;
  for (int64_t i = 0; i < m->Nn; ++i) {
    const double z = m->X[(size_t)(dim - 1) * K * nc + (size_t)i];
    zlo = std::min(zlo, z);
    zhi = std::max(zhi, z);
  }
  zlo -= 1.0;
  zhi += 1.0;
  const int bg_m = (int)std::min(4096.0, std::max(16.0, std::ceil((zhi - zlo) / 25.0)));
  const double bg_dz = (zhi - zlo) / bg_m;
  std::vector<double> bgtab((size_t)4 * (bg_m + 1));
  for (int k = 0; k <= bg_m; ++k) {
    double rho, p;
    const double z = zlo + k * bg_dz;
    background(d, z, &rho, &p);
    const double g = 9.81;
    double drho = 0.0;
    if (d.atm_kind == DG_ATM_ISOTHERMAL) drho = -rho * g / (kRgas * d.atm_T);
    if (d.atm_kind == DG_ATM_STRATIFIED) drho = rho * (-rho * g / (kGamma * p) - d.atm_N * d.atm_N / g);
    bgtab[4 * k] = p;
    bgtab[4 * k + 1] = -rho * g * bg_dz;  // hydrostatic: dp/dz = -rho g
    bgtab[4 * k + 2] = rho;
    bgtab[4 * k + 3] = drho * bg_dz;
  }
  std::vector<double> zeta0(K);
  for (int64_t c = 0; c < K; ++c)
    zeta0[c] = m->ijk[c * dim + dim - 1] * (hb[dim - 1] / (double)(1 << m->level[c]));

  // ---------------------------------------------------------------- upload
  const std::vector<double> tabp = tab.packed();
  std::vector<int> cell_link((size_t)K * 2 * dim, 3);
  for (int f = 0; f < nf; ++f) {
    const int kind = f < m->nconf ? 0 : (f < m->nconf + m->nsub ? 1 : 3);
    if (kind == 3) continue;
    cell_link[(size_t)face_m[f] * 2 * dim + face_lfm[f]] =
        (int)(((uint32_t)face_p[f] << 4) | ((uint32_t)face_s[f] << 2) | (uint32_t)kind);
    if (kind == 0) cell_link[(size_t)face_p[f] * 2 * dim + face_lfp[f]] = (int)(((uint32_t)face_m[f] << 4) | 0u);
    else cell_link[(size_t)face_p[f] * 2 * dim + face_lfp[f]] = 2;
  }
  std::vector<int> cell_cmask(K, 0);
  for (int64_t c = 0; c < K; ++c)
    for (int lf = 0; lf < 2 * dim; ++lf)
      if ((cell_face[c * 2 * dim + lf] & 3) == 2) cell_cmask[c] |= 1 << lf;
  // Coarse sides of the 2:1 faces per cell, in cell order and local-face order: each coarse
  // face's NSUB NF fine points (j = s NF + q), the fine node and 1/2 |N| n / w_end there
  // (fsj fn / (2 w_end), w_end the GLL end weight);
  // the cell batches (partitions) index these lists.  Work per cell for the balanced partition:
  // its nodes, plus one per coarse-side point and per fine-side face node.
  const int nsubf = 1 << (dim - 1), np_c = nsubf * NF;
  const double iwend = 1.0 / tab.w[0];  // the face terms enter the cell passes divided by the end weight
  CoarseLists cl;
  cl.dim = dim;
  cl.np = np_c;
  cl.cmask = cell_cmask;
  cl.off.assign(K + 1, 0);
  cl.cost.assign(K, (double)nc);
  // work per cell in units of a node's work (about 14 d FP64 operations per node and pass pair):
  // a coarse-side point costs its interpolation (NF (1 + d) operations) and its share of the
  // sums at the coarse face nodes (NF more); a fine-side face node its interpolation
  const double k_coarse = (2.0 + dim) * NF / (14.0 * dim), k_fine = (1.0 + dim) * NF / (14.0 * dim);
  for (int64_t c = 0; c < K; ++c) {
    cl.off[c] = (int)(cl.node.size() / np_c);
    for (int lf = 0; lf < 2 * dim; ++lf) {
      const int link = cell_link[(size_t)c * 2 * dim + lf];
      if ((link & 3) == 1) cl.cost[c] += k_fine * NF;
      if (!((cell_cmask[c] >> lf) & 1)) continue;
      const int f = cell_face[c * 2 * dim + lf] >> 2;
      for (int j = 0; j < np_c; ++j) {
        const size_t t = (size_t)(f + j / NF) * NF + (size_t)(j % NF);
        cl.node.push_back(fnode_m[t]);
        for (int b = 0; b < dim; ++b) cl.w.push_back(0.5 * fsj[t] * fn[(size_t)b * nf * NF + t] * iwend);
      }
      cl.cost[c] += k_coarse * np_c;
    }
  }
  cl.off[K] = (int)(cl.node.size() / np_c);
  const size_t n_int = (size_t)5 * nf + 2 * cell_face.size() + 2 * (size_t)nf * NF + 2 * (size_t)K;
  const size_t n_real = (size_t)dim * dim * m->Nn + 5 * (size_t)m->Nn + (size_t)(dim + 1) * nf * NF + tabp.size() +
                        (size_t)K + bgtab.size();
  auto pad = [](size_t x) { return (x + 31) & ~(size_t)31; };
  DG_CUDA(cudaSetDevice(m->ctx->device));
  DG_CUDA(cudaMalloc(&m->d_int, pad(n_int) * sizeof(int)));
  DG_CUDA(cudaMalloc(&m->d_f64, pad(n_real) * sizeof(double) + 64 * 8));
  DG_CUDA(cudaMalloc(&m->d_f32, pad(n_real) * sizeof(float) + 64 * 8));
  m->scratch_bytes = (pad((size_t)m->V * nf * NF) + pad((size_t)dim * m->Nn) + 2 * 512) * sizeof(double);
  DG_CUDA(cudaMalloc(&m->d_scratch, m->scratch_bytes));
  m->device_bytes = pad(n_int) * 4 + pad(n_real) * 12 + 1024 + m->scratch_bytes;
  if (!tau.empty()) {
    DG_CUDA(cudaMalloc(&m->d_tau, tau.size() * sizeof(double)));
    DG_CUDA(cudaMemcpy(m->d_tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice));
    m->device_bytes += tau.size() * sizeof(double);
  }
  m->d_face_scratch64 = (double*)m->d_scratch;
  m->d_vec_scratch64 = (double*)m->d_scratch + pad((size_t)m->V * nf * NF);
  m->d_red_scratch = m->d_vec_scratch64 + pad((size_t)dim * m->Nn);

  std::vector<int> ibuf;
  ibuf.reserve(n_int);
  for (auto* v : {&face_m, &face_lfm, &face_p, &face_lfp, &face_s}) ibuf.insert(ibuf.end(), v->begin(), v->end());
  ibuf.insert(ibuf.end(), cell_face.begin(), cell_face.end());
  ibuf.insert(ibuf.end(), fnode_m.begin(), fnode_m.end());
  ibuf.insert(ibuf.end(), fnode_p.begin(), fnode_p.end());
  ibuf.insert(ibuf.end(), cell_cmask.begin(), cell_cmask.end());
  for (int64_t c = 0; c < K; ++c) ibuf.push_back((int)m->level[c]);
  ibuf.insert(ibuf.end(), cell_link.begin(), cell_link.end());
  DG_CUDA(cudaMemcpy(m->d_int, ibuf.data(), ibuf.size() * sizeof(int), cudaMemcpyHostToDevice));

  std::vector<double> rbuf;
  rbuf.reserve(n_real);
  size_t o_Ja = rbuf.size();
  rbuf.insert(rbuf.end(), Ja.begin(), Ja.end());
  size_t o_invJ = rbuf.size();
  rbuf.insert(rbuf.end(), invJ.begin(), invJ.end());
  size_t o_rhob = rbuf.size();
  rbuf.insert(rbuf.end(), rhob.begin(), rhob.end());
  size_t o_pb = rbuf.size();
  rbuf.insert(rbuf.end(), pb.begin(), pb.end());
  size_t o_wJ = rbuf.size();
  rbuf.insert(rbuf.end(), wJ.begin(), wJ.end());
  size_t o_fn = rbuf.size();
  rbuf.insert(rbuf.end(), fn.begin(), fn.end());
  size_t o_fsj = rbuf.size();
  rbuf.insert(rbuf.end(), fsj.begin(), fsj.end());
  size_t o_zdev = rbuf.size();
  rbuf.insert(rbuf.end(), zdev.begin(), zdev.end());
  size_t o_tab = rbuf.size();
  rbuf.insert(rbuf.end(), tabp.begin(), tabp.end());
  size_t o_zeta0 = rbuf.size();
  rbuf.insert(rbuf.end(), zeta0.begin(), zeta0.end());
  size_t o_bg = rbuf.size();
  rbuf.insert(rbuf.end(), bgtab.begin(), bgtab.end());
  DG_CUDA(cudaMemcpy(m->d_f64, rbuf.data(), rbuf.size() * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<float> fbuf(rbuf.begin(), rbuf.end());
  DG_CUDA(cudaMemcpy(m->d_f32, fbuf.data(), fbuf.size() * sizeof(float), cudaMemcpyHostToDevice));

  auto fill = [&](auto& v, auto* base) {
    v.n_cells = K;
    v.n_nodes = m->Nn;
    v.nconf = m->nconf;
    v.nsub = m->nsub;
    v.nwall = m->nwall;
    v.nf = nf;
    v.Ja = base + o_Ja;
    v.invJ = base + o_invJ;
    v.rhob = base + o_rhob;
    v.pb = base + o_pb;
    v.wJ = base + o_wJ;
    v.fn = base + o_fn;
    v.fsj = base + o_fsj;
    v.tab = base + o_tab;
    const int* ib = (const int*)m->d_int;
    v.face_m = ib;
    v.face_lfm = ib + nf;
    v.face_p = ib + 2 * (size_t)nf;
    v.face_lfp = ib + 3 * (size_t)nf;
    v.face_s = ib + 4 * (size_t)nf;
    v.cell_face = ib + 5 * (size_t)nf;
    v.fnode_m = v.cell_face + cell_face.size();
    v.fnode_p = v.fnode_m + (size_t)nf * NF;
    v.cell_cmask = v.fnode_p + (size_t)nf * NF;
    v.gravity = (decltype(v.gravity))d.gravity;
    v.zdev = base + o_zdev;
    v.cell_level = v.cell_cmask + K;
    v.cell_link = v.cell_level + K;
    for (int a = 0; a < 3; ++a) v.hb[a] = (decltype(v.gravity))(a < dim ? 0.5 * hb[a] : 0.0);
    v.geo_z = geo_z ? 1 : 0;
    v.aff = aff ? 1 : 0;
    v.cell_zeta0 = base + o_zeta0;
    v.bg_tab = base + o_bg;
    v.bg_z0 = (decltype(v.gravity))zlo;
    v.bg_idz = (decltype(v.gravity))(1.0 / bg_dz);
    v.bg_m = bg_m;
  };
  fill(m->v64, (const double*)m->d_f64);
  fill(m->v32, (const float*)m->d_f32);
  const int cpb = nc >= 256 ? 1 : 256 / nc;
  {
    std::vector<int> bstart;
    for (int64_t c = 0; c < K; c += cpb) bstart.push_back((int)c);
    bstart.push_back((int)K);
    int rc = build_partition(m, cl, bstart, m->part[0]);
    if (rc != DG_OK) return rc;
    m->n_parts = 1;
    // balanced partition for the persistent solves (two CTAs per SM, CTA r taking batches r,
    // r + G, ...): where the uniform batches do not fill the CTAs, cost-balanced batches, one per
    // CTA; where there are more batches than CTAs, the uniform batches ordered so that every
    // CTA's share of the work is about the same (largest first to the least loaded CTA)
    const int target = 2 * m->ctx->sm_count;
    const int64_t nbu = (int64_t)bstart.size() - 1;
    if (nbu <= target && K > nbu) {
      bstart = balanced_batches(cl.cost, cpb, (int)std::min<int64_t>(target, K));
      rc = build_partition(m, cl, bstart, m->part[1]);
      if (rc != DG_OK) return rc;
      m->n_parts = 2;
    } else if (nbu > target) {
      std::vector<double> bcost(nbu, 0.0);
      for (int64_t b = 0; b < nbu; ++b)
        for (int c = bstart[b]; c < bstart[b + 1]; ++c) bcost[b] += cl.cost[c];
      const std::vector<int> order = balanced_order(bcost, target);
      rc = build_partition(m, cl, bstart, m->part[1], &order);
      if (rc != DG_OK) return rc;
      m->n_parts = 2;
    }
  }
  set_partition(m, 0);
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_mesh_create(dg_ctx* ctx, const dg_mesh_desc* desc, dg_mesh** out) {
  if (!ctx || !desc || !out) return fail(DG_EINVAL, "null argument");
  if (desc->dim != 2 && desc->dim != 3) return fail(DG_EINVAL, "dim must be 2 or 3");
  if (desc->degree < 1 || desc->degree > kMaxDegree) return fail(DG_EINVAL, "degree must be in 1..5");
  if (desc->n_cells <= 0 || !desc->level || !desc->ijk) return fail(DG_EINVAL, "empty mesh");
  if (desc->n_cells > (int64_t)1 << 28) return fail(DG_EINVAL, "too many cells");
  for (int a = 0; a < desc->dim; ++a)
    if (desc->base[a] <= 0 || desc->base[a] >= (1 << 12) || !(desc->extent[a] > 0.0))
      return fail(DG_EINVAL, "bad base grid or extent");
  if (desc->atm_kind < 0 || desc->atm_kind > 2 || desc->hill_kind < 0 || desc->hill_kind > 3)
    return fail(DG_EINVAL, "bad hill or atmosphere kind");
  if (desc->atm_kind != DG_ATM_NONE && (!(desc->atm_T > 0) || !(desc->atm_p_ref > 0)))
    return fail(DG_EINVAL, "bad atmosphere parameters");
  if (desc->atm_kind == DG_ATM_STRATIFIED && !(desc->atm_N > 0)) return fail(DG_EINVAL, "bad buoyancy frequency");
  if (!(desc->sponge_depth >= 0.0) || !(desc->sponge_rate >= 0.0) ||
      desc->sponge_depth > desc->extent[desc->dim - 1] || !std::isfinite(desc->sponge_u0))
    return fail(DG_EINVAL, "bad sponge layer parameters");
  for (int a = 0; a < desc->dim - 1; ++a)
    if (!(desc->sponge_lateral_width >= 0.0) || desc->sponge_lateral_width > 0.5 * desc->extent[a] ||
        !(desc->sponge_lateral_rate >= 0.0))
      return fail(DG_EINVAL, "bad lateral sponge layer parameters");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ENOMEM, "host allocation failed");
  m->ctx = ctx;
  m->desc = *desc;
  m->desc.level = nullptr;
  m->desc.ijk = nullptr;
  // the optional caller geometry and face tables are read by build_mesh during this call only
  m->level.assign(desc->level, desc->level + desc->n_cells);
  m->ijk.assign(desc->ijk, desc->ijk + desc->n_cells * desc->dim);
  for (uint8_t l : m->level)
    if (l > 7) {
      delete m;
      return fail(DG_EINVAL, "refinement level above 7");
    }
  int st;
  try {
    st = build_mesh(m);
  } catch (const std::exception& e) {
    st = fail(DG_EINVAL, e.what());
  }
  m->desc.node_xyz = nullptr;
  m->desc.conforming = m->desc.subfaces = m->desc.walls = nullptr;
  if (st != DG_OK) {
    dg_mesh_destroy(m);
    return st;
  }
  *out = m;
  return DG_OK;
}

extern "C" int dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_OK;
  cudaFree(m->d_int);
  cudaFree(m->d_f64);
  cudaFree(m->d_f32);
  cudaFree(m->d_scratch);
  if (m->d_tau) cudaFree(m->d_tau);
  for (auto& P : m->part) {
    if (P.d_int) cudaFree(P.d_int);
    if (P.d_f64) cudaFree(P.d_f64);
    if (P.d_f32) cudaFree(P.d_f32);
  }
  delete m;
  return DG_OK;
}

extern "C" int dg_mesh_get_info(const dg_mesh* m, dg_mesh_info* info) {
  if (!m || !info) return fail(DG_EINVAL, "null argument");
  info->dim = m->dim;
  info->degree = m->degree;
  info->n_vars = m->V;
  info->nodes_per_cell = m->nc;
  info->n_cells = m->K;
  info->n_nodes = m->Nn;
  info->n_dof = m->Nn * m->V;
  info->n_conforming = m->nconf;
  info->n_subfaces = m->nsub;
  info->n_walls = m->nwall;
  info->max_level = m->max_level;
  info->min_edge = m->min_edge;
  info->device_bytes = m->device_bytes;
  for (int p = 0; p < 2; ++p) {
    info->solver_form[p] = m->tuned_form[p];
    info->n_batches[p] = p < m->n_parts ? m->part[p].nbat : 0;
    info->solver_partition[p] = m->tuned_part[p];
    for (int f = 0; f < 3; ++f) {
      info->solver_ms[p][f] = m->tuned_ms[p][f];
      info->solver_ms_balanced[p][f] = m->tuned_ms_balanced[p][f];
    }
  }
  return DG_OK;
}

extern "C" int dg_mesh_set_partition(dg_mesh* m, int k) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (k < 0 || k >= m->n_parts) return fail(DG_EINVAL, "cell partition not built for this mesh");
  set_partition(m, k);
  m->tuned_part[0] = m->tuned_part[1] = k;  // the steps' partition too, until the autotuner next runs
  return DG_OK;
}

extern "C" int dg_mesh_get_faces(const dg_mesh* m, int32_t* conforming, int32_t* subfaces, int32_t* walls) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (conforming) std::memcpy(conforming, m->conf.data(), m->conf.size() * sizeof(int32_t));
  if (subfaces) std::memcpy(subfaces, m->subs.data(), m->subs.size() * sizeof(int32_t));
  if (walls) std::memcpy(walls, m->walls.data(), m->walls.size() * sizeof(int32_t));
  return DG_OK;
}

extern "C" int dg_mesh_get_coords(const dg_mesh* m, double* xyz) {
  if (!m || !xyz) return fail(DG_EINVAL, "null argument");
  std::memcpy(xyz, m->X.data(), m->X.size() * sizeof(double));
  return DG_OK;
}
