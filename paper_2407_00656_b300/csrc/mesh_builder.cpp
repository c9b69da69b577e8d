// mesh_builder.cpp -- host preprocessing for the HGKS GPU path.
//
// From node coordinates and cell-to-node lists this builds, once per mesh:
//   * cell geometry (volume, centroid, central second moments),
//   * a Morton (Z-order) renumbering of cells for locality of the gathers,
//   * faces by sorting sorted-node keys (CellFace / FaceCell of Section 3.1),
//     periodic pairing by translated centroids, tagged physical boundaries,
//   * one ghost slot per physical boundary face: the interior cell mirrored
//     across the face plane (Algorithm 1, "add ghost cell according to
//     boundary condition"),
//   * the two-layer WENO stencil of Algorithm 1 and the sub-stencils of
//     Section 2.3 (tetrahedra: four 7-cell stencils; hexahedra: eight octants),
//   * triangular prisms, given as hexahedra with nodes 2 = 3 and 6 = 7 (the
//     paper defines no prism): the side face 2 3 7 6 collapses to an edge and
//     is dropped (its cell-face entry points at a flux record that stays
//     zero), the two triangles take the 3-point rule padded with a
//     zero-weight fourth point, and the two octants at the collapsed edge
//     take the two side faces that meet there,
//   * least-squares pseudo-inverses for the quadratic P0 and linear Pm of
//     Eq. polys in coordinates centred on the cell and scaled by |cell|^(1/3),
//   * face Gauss points: 3-point degree-2 rule on triangles, 2x2 Gauss on
//     bilinear quads, with per-point unit normals and weights times area.
#include "mesh_builder.h"

#include "hgks_internal.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <climits>
#include <cstdio>
#include <cstring>
#include <numeric>

namespace hgks {
namespace {

struct P3 {
  double x, y, z;
};
inline P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline P3 operator*(double s, P3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dotp(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline P3 crossp(P3 a, P3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double comp(P3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Local faces (node positions within the cell).  Tet face p is opposite node
// p.  Hex faces: bottom, four sides in cyclic order, top.
const int kTetFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int kHexFace[6][4] = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};

// Second moments are kept as the 6 unique entries xx yy zz xy yz zx.
constexpr int kMa[6] = {0, 1, 2, 0, 1, 2};
constexpr int kMb[6] = {0, 1, 2, 1, 2, 0};

// Tetrahedron: volume by the triple product, centroid, central second moments
// by the 4-point degree-2 rule (exact for quadratics).
void tet_geometry(const P3 v[4], double& vol, P3& c, double mo[6]) {
  vol = dotp(crossp(v[1] - v[0], v[2] - v[0]), v[3] - v[0]) / 6.0;
  c = 0.25 * (v[0] + v[1] + v[2] + v[3]);
  const double a = 0.5854101966249685, b = 0.1381966011250105;
  for (int k = 0; k < 6; ++k) mo[k] = 0.0;
  for (int q = 0; q < 4; ++q) {
    P3 x = {0, 0, 0};
    for (int j = 0; j < 4; ++j) x = x + (j == q ? a : b) * v[j];
    P3 d = x - c;
    for (int k = 0; k < 6; ++k) mo[k] += 0.25 * comp(d, kMa[k]) * comp(d, kMb[k]);
  }
}

// Trilinear hexahedron: 3-point Gauss-Legendre per direction.
void hex_geometry(const P3 v[8], double& vol, P3& c, double mo[6]) {
  const double r = std::sqrt(0.6);
  const double gp[3] = {0.5 * (1 - r), 0.5, 0.5 * (1 + r)};
  const double gw[3] = {5.0 / 18, 8.0 / 18, 5.0 / 18};
  double xs[27][3], ws[27];
  int q = 0;
  vol = 0.0;
  c = {0, 0, 0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k, ++q) {
        const double s = gp[i], t = gp[j], u = gp[k];
        const double sm = 1 - s, tm = 1 - t, um = 1 - u;
        // trilinear shape functions in the node order 0..7
        const double N[8] = {sm * tm * um, s * tm * um, s * t * um, sm * t * um,
                             sm * tm * u,  s * tm * u,  s * t * u,  sm * t * u};
        P3 x = {0, 0, 0};
        for (int a = 0; a < 8; ++a) x = x + N[a] * v[a];
        // Jacobian columns d x / d(s,t,u)
        P3 js = tm * um * (v[1] - v[0]) + t * um * (v[2] - v[3]) + tm * u * (v[5] - v[4]) + t * u * (v[6] - v[7]);
        P3 jt = sm * um * (v[3] - v[0]) + s * um * (v[2] - v[1]) + sm * u * (v[7] - v[4]) + s * u * (v[6] - v[5]);
        P3 ju = sm * tm * (v[4] - v[0]) + s * tm * (v[5] - v[1]) + s * t * (v[6] - v[2]) + sm * t * (v[7] - v[3]);
        const double w = gw[i] * gw[j] * gw[k] * dotp(crossp(js, jt), ju);
        xs[q][0] = x.x; xs[q][1] = x.y; xs[q][2] = x.z;
        ws[q] = w;
        vol += w;
        c = c + w * x;
      }
  c = (1.0 / vol) * c;
  for (int k = 0; k < 6; ++k) mo[k] = 0.0;
  for (q = 0; q < 27; ++q) {
    const double d[3] = {xs[q][0] - c.x, xs[q][1] - c.y, xs[q][2] - c.z};
    for (int k = 0; k < 6; ++k) mo[k] += ws[q] * d[kMa[k]] * d[kMb[k]];
  }
  for (int k = 0; k < 6; ++k) mo[k] /= vol;
}

// Gauss points of a face given its nodes in cyclic order.
struct FaceGeo {
  int ng;
  P3 x[4], n[4];
  double w[4];
  P3 centroid, nmean;  // weighted Gauss-point centroid and unit mean normal
};

FaceGeo face_geo(const P3* p, int nn) {
  FaceGeo g;
  if (nn == 3) {
    P3 av = 0.5 * crossp(p[1] - p[0], p[2] - p[0]);
    const double area = std::sqrt(dotp(av, av));
    P3 n = (1.0 / area) * av;
    P3 fc = (1.0 / 3.0) * (p[0] + p[1] + p[2]);
    g.ng = 3;
    for (int k = 0; k < 3; ++k) {
      // barycentric (2/3, 1/6, 1/6): halfway between the centroid and vertex k
      g.x[k] = fc + 0.5 * (p[k] - fc);
      g.n[k] = n;
      g.w[k] = area / 3.0;
    }
    g.centroid = fc;
    g.nmean = n;
    return g;
  }
  const double e = 0.5 / std::sqrt(3.0);
  const double gq[2] = {0.5 - e, 0.5 + e};
  g.ng = 4;
  P3 asum = {0, 0, 0}, csum = {0, 0, 0};
  double wsum = 0.0;
  int k = 0;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j, ++k) {
      const double s = gq[i], t = gq[j];
      P3 x = (1 - s) * (1 - t) * p[0] + s * (1 - t) * p[1] + s * t * p[2] + (1 - s) * t * p[3];
      P3 xs = (1 - t) * (p[1] - p[0]) + t * (p[2] - p[3]);
      P3 xt = (1 - s) * (p[3] - p[0]) + s * (p[2] - p[1]);
      P3 av = 0.25 * crossp(xs, xt);  // weight 1/4 per point on the unit square
      const double a = std::sqrt(dotp(av, av));
      g.x[k] = x;
      g.n[k] = (1.0 / a) * av;
      g.w[k] = a;
      asum = asum + av;
      csum = csum + a * x;
      wsum += a;
    }
  g.centroid = (1.0 / wsum) * csum;
  g.nmean = (1.0 / std::sqrt(dotp(asum, asum))) * asum;
  return g;
}

// Morton key of a point quantised to 21 bits per axis.
uint64_t spread21(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

// Least-squares pseudo-inverse of the m x n matrix A (row-major, m >= n) by
// modified Gram-Schmidt with one re-orthogonalisation pass: A = Q R,
// pinv = R^{-1} Q^T, written to out[i*m + r] (n rows).  Returns false if R is
// numerically singular.
bool mgs2_pinv(const double* A, int m, int n, double* out) {
  std::vector<double> Q(m * n), R(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    std::vector<double> v(m);
    for (int r = 0; r < m; ++r) v[r] = A[r * n + j];
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < j; ++i) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += Q[r * n + i] * v[r];
        R[i * n + j] += s;
        for (int r = 0; r < m; ++r) v[r] -= s * Q[r * n + i];
      }
    }
    double nv = 0.0;
    for (int r = 0; r < m; ++r) nv += v[r] * v[r];
    nv = std::sqrt(nv);
    R[j * n + j] = nv;
    if (nv == 0.0) return false;
    for (int r = 0; r < m; ++r) Q[r * n + j] = v[r] / nv;
  }
  double dmax = 0.0;
  for (int j = 0; j < n; ++j) dmax = std::max(dmax, R[j * n + j]);
  for (int j = 0; j < n; ++j)
    if (R[j * n + j] <= 1e-10 * dmax) return false;
  for (int r = 0; r < m; ++r) {
    // solve R x = (row r of Q)^T, i.e. column r of Q^T
    for (int i = n - 1; i >= 0; --i) {
      double s = Q[r * n + i];
      for (int k = i + 1; k < n; ++k) s -= R[i * n + k] * out[k * m + r];
      out[i * m + r] = s / R[i * n + i];
    }
  }
  return true;
}

struct Member {
  int32_t id;     // cell (< nc) or ghost slot (>= nc)
  int8_t sh[3];   // periodic image, in units of the periods
  bool operator==(const Member& o) const {
    return id == o.id && sh[0] == o.sh[0] && sh[1] == o.sh[1] && sh[2] == o.sh[2];
  }
};

}  // namespace

int build_host_mesh(const hgks_mesh_desc& d, HostMesh& m, std::string& err) {
  char buf[256];
  const int ct = d.cell_type;
  const int nfc = ct == HGKS_TET4 ? 4 : 6;
  const int fnn = ct == HGKS_TET4 ? 3 : 4;
  m.ctype = ct;
  m.nfc = nfc;
  m.G = fnn;
  m.M = ct == HGKS_TET4 ? 4 : 8;
  m.KM = ct == HGKS_TET4 ? 6 : 3;
  const int64_t nc = d.n_cells;
  m.nc = nc;
  if (nc >= (int64_t(1) << 30)) { err = "too many cells"; return HGKS_EINVAL; }
  auto node = [&](int64_t i) { return P3{d.xyz[3 * i], d.xyz[3 * i + 1], d.xyz[3 * i + 2]}; };
  for (int64_t i = 0; i < nc * ct; ++i)
    if (d.cell_nodes[i] < 0 || d.cell_nodes[i] >= d.n_nodes) { err = "cell node index out of range"; return HGKS_EINVAL; }
  // prisms: hexahedra with nodes 2 = 3 and 6 = 7 and six distinct nodes
  std::vector<uint8_t> prism0(nc, 0);
  if (ct == HGKS_HEX8)
    for (int64_t c = 0; c < nc; ++c) {
      const int64_t* v = d.cell_nodes + 8 * c;
      int distinct = 0;
      for (int a = 0; a < 8; ++a) {
        bool seen = false;
        for (int b = 0; b < a; ++b) seen = seen || v[b] == v[a];
        distinct += !seen;
      }
      prism0[c] = v[2] == v[3] && v[6] == v[7];
      if (distinct != (prism0[c] ? 6 : 8)) {
        std::snprintf(buf, sizeof buf, "cell %lld: a hexahedron needs 8 distinct nodes, a prism nodes 2 = 3 and 6 = 7",
                      (long long)c);
        err = buf;
        return HGKS_EINVAL;
      }
    }

  // ---- 1. cell geometry in caller order
  std::vector<double> vol0(nc), cen0(3 * nc), mom0(6 * nc);
  int64_t bad = -1;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    P3 v[8];
    for (int a = 0; a < ct; ++a) v[a] = node(d.cell_nodes[c * ct + a]);
    double vol, mo[6];
    P3 cc;
    if (ct == HGKS_TET4) tet_geometry(v, vol, cc, mo);
    else hex_geometry(v, vol, cc, mo);
    vol0[c] = vol;
    cen0[3 * c] = cc.x; cen0[3 * c + 1] = cc.y; cen0[3 * c + 2] = cc.z;
    for (int k = 0; k < 6; ++k) mom0[6 * c + k] = mo[k];
    if (!(vol > 0.0)) {
#pragma omp critical
      bad = c;
    }
  }
  if (bad >= 0) {
    std::snprintf(buf, sizeof buf, "cell %lld has a non-positive volume", (long long)bad);
    err = buf;
    return HGKS_EMESH;
  }

  // ---- 2. Morton order of the centroids
  std::vector<int64_t>& perm = m.perm;
  perm.resize(nc);
  std::iota(perm.begin(), perm.end(), 0);
  if (d.sfc_reorder && nc > 1) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t c = 0; c < nc; ++c)
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], cen0[3 * c + a]); hi[a] = std::max(hi[a], cen0[3 * c + a]); }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (ext <= 0) ext = 1;
    std::vector<uint64_t> key(nc);
    for (int64_t c = 0; c < nc; ++c) {
      uint64_t q[3];
      for (int a = 0; a < 3; ++a) q[a] = (uint64_t)((cen0[3 * c + a] - lo[a]) / ext * 2097151.0);
      key[c] = spread21(q[0]) | spread21(q[1]) << 1 | spread21(q[2]) << 2;
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  }
  std::vector<int32_t> inv(nc);
  for (int64_t i = 0; i < nc; ++i) inv[perm[i]] = (int32_t)i;
  auto cnode = [&](int64_t cnew, int a) { return d.cell_nodes[perm[cnew] * ct + a]; };
  auto lnode = [&](int64_t cnew, int p, int a) { return cnode(cnew, ct == HGKS_TET4 ? kTetFace[p][a] : kHexFace[p][a]); };
  auto is_prism = [&](int64_t cnew) { return prism0[perm[cnew]] != 0; };
  // distinct nodes of local face p in cyclic order: fnn, 3 for a prism's
  // triangles, 0 for its collapsed side face
  auto face_nodes = [&](int64_t cnew, int p, int64_t out[4]) {
    if (!is_prism(cnew)) {
      for (int a = 0; a < fnn; ++a) out[a] = lnode(cnew, p, a);
      return fnn;
    }
    if (p == 3) return 0;
    if (p == 0 || p == 5) {
      for (int a = 0; a < 3; ++a) out[a] = lnode(cnew, p, a);
      return 3;
    }
    for (int a = 0; a < 4; ++a) out[a] = lnode(cnew, p, a);
    return 4;
  };
  auto ccen = [&](int64_t cnew) { int64_t o = perm[cnew]; return P3{cen0[3 * o], cen0[3 * o + 1], cen0[3 * o + 2]}; };

  // ---- 3. faces: sort (cell, local face) incidences by their sorted node keys
  using Key = std::array<int64_t, 4>;
  const int64_t ninc = nc * nfc;
  std::vector<Key> keys(ninc);
  for (int64_t c = 0; c < nc; ++c)
    for (int p = 0; p < nfc; ++p) {
      Key k = {-2, -2, -2, -2};  // a collapsed face: sorts first, never matched
      int64_t fv[4];
      const int nn = face_nodes(c, p, fv);
      if (nn > 0) {
        k = {-1, -1, -1, -1};
        for (int a = 0; a < nn; ++a) k[a] = fv[a];
        std::sort(k.begin(), k.begin() + nn);
      }
      keys[c * nfc + p] = k;
    }
  std::vector<int64_t> order(ninc);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return keys[a] < keys[b] || (keys[a] == keys[b] && a < b); });
  int64_t first = 0;  // skip the collapsed faces
  while (first < ninc && keys[order[first]][0] == -2) ++first;

  struct FaceT {
    int32_t own, nbr;   // nbr = -1 for physical boundary
    int8_t lown, lnbr;
    int8_t sh[3];       // neighbour image shift seen from the owner (units of periods)
    int32_t tag;
  };
  std::vector<FaceT> faces;
  faces.reserve(ninc / 2 + 16);
  std::vector<int64_t> singles;
  for (int64_t i = first; i < ninc;) {
    int64_t j = i + 1;
    while (j < ninc && keys[order[j]] == keys[order[i]]) ++j;
    if (j - i == 2) {
      int64_t a = order[i], b = order[i + 1];
      FaceT f{};
      f.own = (int32_t)(a / nfc); f.lown = (int8_t)(a % nfc);
      f.nbr = (int32_t)(b / nfc); f.lnbr = (int8_t)(b % nfc);
      faces.push_back(f);
    } else if (j - i == 1) {
      singles.push_back(order[i]);
    } else {
      err = "a face is shared by more than two cells";
      return HGKS_EMESH;
    }
    i = j;
  }

  // ---- 4. boundary faces: tagged ones, then periodic pairing of the rest
  std::vector<std::pair<Key, int32_t>> btags;
  for (int64_t b = 0; b < d.n_bfaces; ++b) {
    Key k = {-1, -1, -1, -1};
    int nn = 0;
    for (int a = 0; a < 4; ++a)
      if (d.bface_nodes[4 * b + a] >= 0) k[nn++] = d.bface_nodes[4 * b + a];
    std::sort(k.begin(), k.begin() + nn);
    btags.push_back({k, d.bface_tag[b]});
  }
  std::sort(btags.begin(), btags.end());
  auto face_centroid = [&](int64_t inc) {
    int64_t c = inc / nfc;
    int p = (int)(inc % nfc);
    int64_t fv[4];
    const int nn = face_nodes(c, p, fv);
    P3 s = {0, 0, 0};
    for (int a = 0; a < nn; ++a) s = s + node(fv[a]);
    return (1.0 / nn) * s;
  };
  double pmax = 0.0;
  if (d.periods)
    for (int a = 0; a < 3; ++a) pmax = std::max(pmax, d.periods[a]);
  const double ptol = 1e-7 * std::max(pmax, 1.0);
  struct PKey {
    int64_t q[3];
    int64_t inc;
    bool operator<(const PKey& o) const {
      for (int a = 0; a < 3; ++a) if (q[a] != o.q[a]) return q[a] < o.q[a];
      return inc < o.inc;
    }
  };
  std::vector<PKey> pcand;
  for (int64_t inc : singles) {
    const Key& k = keys[inc];
    auto it = std::lower_bound(btags.begin(), btags.end(), std::make_pair(k, INT32_MIN));
    int32_t tag = (it != btags.end() && it->first == k) ? it->second : 0;
    if (tag == HGKS_BC_FARFIELD || tag == HGKS_BC_WALL) {
      FaceT f{};
      f.own = (int32_t)(inc / nfc); f.lown = (int8_t)(inc % nfc);
      f.nbr = -1; f.lnbr = -1; f.tag = tag;
      faces.push_back(f);
      continue;
    }
    if (!d.periods || pmax <= 0.0) {
      err = "boundary face without a tag and no periods given";
      return HGKS_EMESH;
    }
    // canonical position: coordinates reduced modulo the periods
    P3 c = face_centroid(inc);
    PKey pk;
    pk.inc = inc;
    for (int a = 0; a < 3; ++a) {
      int64_t q = std::llround(comp(c, a) / ptol);
      if (d.periods[a] > 0) {
        int64_t P = std::llround(d.periods[a] / ptol);
        q %= P;
        if (q < 0) q += P;
        if (q > P - 2) q = 0;  // a point within rounding of the upper plane
      }
      pk.q[a] = q;
    }
    pcand.push_back(pk);
  }
  std::sort(pcand.begin(), pcand.end());
  for (size_t i = 0; i < pcand.size();) {
    size_t j = i + 1;
    while (j < pcand.size() && std::abs(pcand[j].q[0] - pcand[i].q[0]) <= 1 &&
           std::abs(pcand[j].q[1] - pcand[i].q[1]) <= 1 && std::abs(pcand[j].q[2] - pcand[i].q[2]) <= 1)
      ++j;
    if (j - i != 2) {
      err = "periodic boundary faces do not pair up";
      return HGKS_EMESH;
    }
    int64_t a = pcand[i].inc, b = pcand[i + 1].inc;
    if (a / nfc > b / nfc) std::swap(a, b);
    FaceT f{};
    f.own = (int32_t)(a / nfc); f.lown = (int8_t)(a % nfc);
    f.nbr = (int32_t)(b / nfc); f.lnbr = (int8_t)(b % nfc);
    P3 ca = face_centroid(a), cb = face_centroid(b);
    for (int ax = 0; ax < 3; ++ax) {
      double L = d.periods[ax];
      f.sh[ax] = L > 0 ? (int8_t)std::llround((comp(ca, ax) - comp(cb, ax)) / L) : 0;
    }
    faces.push_back(f);
    i = j;
  }
  // owner = lower cell index; faces ordered by owner for coalesced reads
  for (auto& f : faces)
    if (f.nbr >= 0 && f.nbr < f.own) {
      std::swap(f.own, f.nbr);
      std::swap(f.lown, f.lnbr);
      for (int a = 0; a < 3; ++a) f.sh[a] = (int8_t)-f.sh[a];
    }
  std::stable_sort(faces.begin(), faces.end(), [](const FaceT& a, const FaceT& b) {
    return a.own < b.own || (a.own == b.own && a.nbr < b.nbr);
  });
  const int64_t nf = (int64_t)faces.size();
  m.nf = nf;
  if (nf >= (int64_t(1) << 30)) { err = "too many faces"; return HGKS_EINVAL; }
  auto shiftvec = [&](const int8_t* sh) {
    P3 s = {0, 0, 0};
    if (d.periods) s = {sh[0] * d.periods[0], sh[1] * d.periods[1], sh[2] * d.periods[2]};
    return s;
  };

  // ---- 5. face geometry, ghosts, cell-face and neighbour tables
  const int G = fnn;
  m.fown.resize(nf); m.fnbr.resize(nf);
  m.fdl.assign(G * 3 * nf, 0.0); m.fdr.assign(G * 3 * nf, 0.0);
  m.fn.assign(G * 3 * nf, 0.0); m.fw.assign(G * nf, 0.0);
  m.cface.assign(nfc * nc, -1);
  std::vector<Member> nb(nc * nfc, Member{-1, {0, 0, 0}});  // id -1: no face (a prism's collapsed side)
  std::vector<double> area(nc, 0.0);
  std::vector<P3> gpt;  // mirror plane points of the ghosts
  int64_t ng = 0;
  for (const auto& f : faces) if (f.nbr < 0) ++ng;
  m.ng = ng;
  m.gsrc.resize(ng); m.gtag.resize(ng); m.gnrm.resize(3 * ng);
  gpt.resize(ng);
  int64_t gi = 0;
  for (int64_t fi = 0; fi < nf; ++fi) {
    const FaceT& f = faces[fi];
    P3 pts[4];
    int64_t fv[4];
    const int nn = face_nodes(f.own, f.lown, fv);
    for (int a = 0; a < nn; ++a) pts[a] = node(fv[a]);
    FaceGeo g = face_geo(pts, nn);
    for (int k = g.ng; k < G; ++k) {  // a triangle among quads: zero-weight points at the centroid
      g.x[k] = g.centroid;
      g.n[k] = g.nmean;
      g.w[k] = 0.0;
    }
    P3 co = ccen(f.own);
    if (dotp(g.nmean, g.centroid - co) < 0) {
      for (int k = 0; k < g.ng; ++k) g.n[k] = -1.0 * g.n[k];
      g.nmean = -1.0 * g.nmean;
    }
    m.fown[fi] = f.own;
    P3 cn = {0, 0, 0}, sv = shiftvec(f.sh);
    if (f.nbr >= 0) {
      m.fnbr[fi] = f.nbr;
      cn = ccen(f.nbr);
    } else {
      m.fnbr[fi] = -f.tag;
    }
    double asum = 0.0;
    for (int k = 0; k < G; ++k) {
      P3 dl = g.x[k] - co;
      P3 dr = g.x[k] - sv - cn;
      for (int a = 0; a < 3; ++a) {
        m.fdl[(k * 3 + a) * nf + fi] = comp(dl, a);
        m.fdr[(k * 3 + a) * nf + fi] = f.nbr >= 0 ? comp(dr, a) : 0.0;
        m.fn[(k * 3 + a) * nf + fi] = comp(g.n[k], a);
      }
      m.fw[k * nf + fi] = g.w[k];
      asum += g.w[k];
    }
    m.cface[f.lown * nc + f.own] = (int32_t)(2 * fi);
    area[f.own] += asum;
    Member& mo = nb[f.own * nfc + f.lown];
    if (f.nbr >= 0) {
      m.cface[f.lnbr * nc + f.nbr] = (int32_t)(2 * fi + 1);
      area[f.nbr] += asum;
      mo = Member{f.nbr, {f.sh[0], f.sh[1], f.sh[2]}};
      nb[f.nbr * nfc + f.lnbr] = Member{f.own, {(int8_t)-f.sh[0], (int8_t)-f.sh[1], (int8_t)-f.sh[2]}};
    } else {
      m.gsrc[gi] = f.own;
      m.gtag[gi] = f.tag;
      for (int a = 0; a < 3; ++a) m.gnrm[a * ng + gi] = comp(g.nmean, a);
      gpt[gi] = g.centroid;
      mo = Member{(int32_t)(nc + gi), {0, 0, 0}};
      ++gi;
    }
  }
  for (int64_t c = 0; c < nc; ++c)
    if (is_prism(c)) m.cface[3 * nc + c] = (int32_t)(2 * nf);  // the zero flux record past the last face
  for (int64_t i = 0; i < nfc * nc; ++i)
    if (m.cface[i] < 0) { err = "internal error: cell face not assigned"; return HGKS_EMESH; }

  // ---- 6. per-cell arrays
  m.vol.resize(nc); m.hdt.resize(nc); m.hinv.resize(nc);
  m.cen.resize(3 * nc); m.mom.resize(6 * nc);
  for (int64_t c = 0; c < nc; ++c) {
    int64_t o = perm[c];
    const double v = vol0[o], h = std::cbrt(v);
    m.vol[c] = v;
    m.hinv[c] = 1.0 / h;
    m.hdt[c] = 3.0 * v / area[c];
    for (int a = 0; a < 3; ++a) m.cen[a * nc + c] = cen0[3 * o + a];
    for (int k = 0; k < 6; ++k) m.mom[k * nc + c] = mom0[6 * o + k] / (h * h);
  }

  // geometry of a stencil member seen from the target: centroid and raw moments
  auto member_geo = [&](const Member& r, P3& c, double mo[6]) {
    P3 sv = shiftvec(r.sh);
    if (r.id < nc) {
      c = ccen(r.id) + sv;
      int64_t o = perm[r.id];
      for (int k = 0; k < 6; ++k) mo[k] = mom0[6 * o + k];
      return;
    }
    const int64_t g = r.id - nc;
    const int64_t s = m.gsrc[g];
    const P3 n = {m.gnrm[g], m.gnrm[ng + g], m.gnrm[2 * ng + g]};
    const P3 cs = ccen(s);
    c = cs - 2.0 * dotp(cs - gpt[g], n) * n + sv;
    // reflect the moment tensor: (I - 2nn^T) S (I - 2nn^T)
    const int64_t o = perm[s];
    double S[3][3];
    for (int k = 0; k < 6; ++k) { S[kMa[k]][kMb[k]] = mom0[6 * o + k]; S[kMb[k]][kMa[k]] = mom0[6 * o + k]; }
    const double nv[3] = {n.x, n.y, n.z};
    double Rm[3][3], T[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Rm[a][b] = (a == b) - 2.0 * nv[a] * nv[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double t = 0;
        for (int k = 0; k < 3; ++k) t += S[a][k] * Rm[k][b];
        T[a][b] = t;
      }
    for (int k = 0; k < 6; ++k) {
      double t = 0;
      for (int j = 0; j < 3; ++j) t += Rm[kMa[k]][j] * T[j][kMb[k]];
      mo[k] = t;
    }
  };

  // ---- 7. stencils (Algorithm 1) and sub-stencils (Section 2.3)
  const int KCAP = ct == HGKS_TET4 ? 16 : 36;
  auto big_stencil = [&](int64_t c, Member* out) {
    int n = 0;
    auto add = [&](const Member& r) {
      if (r.id < 0) return;
      if (r.id == c && r.sh[0] == 0 && r.sh[1] == 0 && r.sh[2] == 0) return;
      for (int k = 0; k < n; ++k) if (out[k] == r) return;
      out[n++] = r;
    };
    for (int p = 0; p < nfc; ++p) add(nb[c * nfc + p]);
    for (int p = 0; p < nfc; ++p) {
      const Member r = nb[c * nfc + p];
      if (r.id < 0 || r.id >= nc) continue;  // ghosts have no neighbours
      for (int q = 0; q < nfc; ++q) {
        Member r2 = nb[(int64_t)r.id * nfc + q];
        for (int a = 0; a < 3; ++a) r2.sh[a] = (int8_t)(r2.sh[a] + r.sh[a]);
        add(r2);
      }
    }
    return n;
  };
  int K = 0;
  for (int64_t c = 0; c < nc; ++c) {
    Member tmp[36];
    K = std::max(K, big_stencil(c, tmp));
  }
  if (K < 9) { err = "big stencil has fewer than 9 cells"; return HGKS_EMESH; }
  // hexahedral meshes: the kernels are compiled for even stencil sizes from
  // 18 (prisms reach odd ones); shorter stencils are padded with the cell
  // itself and zero weights
  if (ct == HGKS_HEX8) K = K <= 18 ? 18 : (K + 1) / 2 * 2;
  m.K = K;
  const int M = m.M, KM = m.KM;
  m.sten.assign((int64_t)K * nc, 0);
  const int64_t ncp = (nc + 31) / 32 * 32;
  m.ncp = ncp;
  m.pinv0.assign((int64_t)9 * K * ncp, 0.0);
  m.subidx.assign((int64_t)M * KM * ncp, 0);
  m.pinvm.assign((int64_t)M * 3 * KM * ncp, 0.0);
  int64_t fail = -1;
  const char* fail_msg = "";
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t c = 0; c < nc; ++c) {
    Member big[36];
    const int n = big_stencil(c, big);
    (void)KCAP;
    auto pos = [&](const Member& r) {
      if (r.id < 0) return -1;
      for (int k = 0; k < n; ++k) if (big[k] == r) return k;
      return -1;
    };
    // sub-stencil member positions
    int sub[8][6], subn[8];
    if (ct == HGKS_TET4) {
      // S_m: the three face neighbours other than the one opposite the table
      // entry, plus the neighbours of face neighbour m other than the cell
      static const int kSets[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}};
      for (int s = 0; s < 4; ++s) {
        int cnt = 0;
        auto put = [&](int k) {
          if (k < 0) return;
          for (int i = 0; i < cnt; ++i) if (sub[s][i] == k) return;
          sub[s][cnt++] = k;
        };
        for (int a = 0; a < 3; ++a) put(pos(nb[c * nfc + kSets[s][a]]));
        const Member r = nb[c * nfc + s];
        if (r.id < nc)
          for (int q = 0; q < nfc; ++q) {
            Member r2 = nb[(int64_t)r.id * nfc + q];
            for (int a = 0; a < 3; ++a) r2.sh[a] = (int8_t)(r2.sh[a] + r.sh[a]);
            if (r2.id == c && r2.sh[0] == 0 && r2.sh[1] == 0 && r2.sh[2] == 0) continue;
            put(pos(r2));
          }
        subn[s] = cnt;
      }
    } else {
      // octant {bottom|top, side s, side s+1}; a prism's two octants at the
      // collapsed edge (sides 2-3 and 3-4) take the sides 2 and 4 meeting there
      const bool pr = is_prism(c);
      for (int top = 0; top < 2; ++top)
        for (int s = 0; s < 4; ++s) {
          const int o = top * 4 + s;
          const bool edge = pr && (s == 1 || s == 2);
          sub[o][0] = pos(nb[c * nfc + (top ? 5 : 0)]);
          sub[o][1] = pos(nb[c * nfc + (edge ? 2 : 1 + s)]);
          sub[o][2] = pos(nb[c * nfc + (edge ? 4 : 1 + (s + 1) % 4)]);
          subn[o] = 3;
        }
    }
    // least-squares rows: averages over each member of the zero-mean basis
    // x y z xx yy zz xy yz zx (centred on the cell, scaled by h)
    const P3 ci = ccen(c);
    const double hi = m.hinv[c];
    double mi[6];
    for (int k = 0; k < 6; ++k) mi[k] = m.mom[k * nc + c];
    std::vector<double> A(n * 9);
    for (int k = 0; k < n; ++k) {
      P3 ck;
      double mo[6];
      member_geo(big[k], ck, mo);
      const double dv[3] = {(ck.x - ci.x) * hi, (ck.y - ci.y) * hi, (ck.z - ci.z) * hi};
      for (int a = 0; a < 3; ++a) A[k * 9 + a] = dv[a];
      for (int q = 0; q < 6; ++q) A[k * 9 + 3 + q] = mo[q] * hi * hi + dv[kMa[q]] * dv[kMb[q]] - mi[q];
    }
    std::vector<double> P0(9 * n);
    bool ok = mgs2_pinv(A.data(), n, 9, P0.data());
    for (int s = 0; s < M && ok; ++s) {
      if (subn[s] < 3) { ok = false; break; }
      double As[6 * 3], Ps[3 * 6];
      for (int r = 0; r < subn[s]; ++r) {
        if (sub[s][r] < 0) { ok = false; break; }
        for (int a = 0; a < 3; ++a) As[r * 3 + a] = A[sub[s][r] * 9 + a];
      }
      if (!ok || !mgs2_pinv(As, subn[s], 3, Ps)) { ok = false; break; }
      for (int r = 0; r < subn[s]; ++r) {
        m.subidx[((int64_t)s * KM + r) * ncp + c] = (uint8_t)sub[s][r];
        for (int a = 0; a < 3; ++a) m.pinvm[((int64_t)(s * 3 + a) * KM + r) * ncp + c] = Ps[a * subn[s] + r];
      }
    }
    if (!ok) {
#pragma omp critical
      { fail = c; fail_msg = "rank-deficient WENO stencil"; }
      continue;
    }
    for (int k = 0; k < K; ++k) m.sten[(int64_t)k * nc + c] = k < n ? big[k].id : (int32_t)c;
    for (int dd = 0; dd < 9; ++dd)
      for (int k = 0; k < n; ++k) m.pinv0[((int64_t)dd * K + k) * ncp + c] = P0[dd * n + k];
  }
  if (fail >= 0) {
    std::snprintf(buf, sizeof buf, "%s at cell %lld (caller index %lld)", fail_msg, (long long)fail,
                  (long long)perm[fail]);
    err = buf;
    return HGKS_EMESH;
  }
  return HGKS_OK;
}

int build_union(const std::vector<const HostMesh*>& parts, HostMesh& u, std::vector<int32_t>& cmesh,
                std::vector<int64_t>& coff, std::string& err) {
  if (parts.empty()) { err = "empty batch"; return HGKS_EINVAL; }
  const HostMesh& a = *parts[0];
  u = HostMesh();
  u.ctype = a.ctype; u.nfc = a.nfc; u.G = a.G; u.M = a.M; u.KM = a.KM;
  int64_t nc = 0, nf = 0, ng = 0;
  int K = 0;
  std::vector<int64_t> foff, goff;
  coff.clear();
  for (const HostMesh* p : parts) {
    if (p->ctype != a.ctype) { err = "a batch needs one cell type"; return HGKS_EINVAL; }
    coff.push_back(nc); foff.push_back(nf); goff.push_back(ng);
    nc += p->nc; nf += p->nf; ng += p->ng;
    K = std::max(K, p->K);
  }
  if (nc >= (int64_t(1) << 30) || nf >= (int64_t(1) << 30)) { err = "batch too large"; return HGKS_EINVAL; }
  u.nc = nc; u.nf = nf; u.ng = ng; u.K = K;
  const int64_t ncp = (nc + 31) / 32 * 32;
  u.ncp = ncp;
  const int M = u.M, KM = u.KM, G = u.G, nfc = u.nfc;
  cmesh.assign(nc, 0);
  u.vol.resize(nc); u.hdt.resize(nc); u.hinv.resize(nc); u.cen.resize(3 * nc); u.mom.resize(6 * nc);
  u.sten.assign((int64_t)K * nc, 0);
  u.pinv0.assign((int64_t)9 * K * ncp, 0.0);
  u.subidx.assign((int64_t)M * KM * ncp, 0);
  u.pinvm.assign((int64_t)M * 3 * KM * ncp, 0.0);
  u.cface.resize((int64_t)nfc * nc);
  u.gsrc.resize(ng); u.gtag.resize(ng); u.gnrm.resize(3 * ng);
  u.fown.resize(nf); u.fnbr.resize(nf);
  u.fdl.resize((int64_t)G * 3 * nf); u.fdr.resize((int64_t)G * 3 * nf); u.fn.resize((int64_t)G * 3 * nf);
  u.fw.resize((int64_t)G * nf);
  for (size_t i = 0; i < parts.size(); ++i) {
    const HostMesh& p = *parts[i];
    const int64_t co = coff[i], fo = foff[i], go = goff[i];
    for (int64_t c = 0; c < p.nc; ++c) {
      const int64_t uc = co + c;
      cmesh[uc] = (int32_t)i;
      u.vol[uc] = p.vol[c]; u.hdt[uc] = p.hdt[c]; u.hinv[uc] = p.hinv[c];
      for (int a3 = 0; a3 < 3; ++a3) u.cen[a3 * nc + uc] = p.cen[a3 * p.nc + c];
      for (int q = 0; q < 6; ++q) u.mom[q * nc + uc] = p.mom[q * p.nc + c];
      for (int k = 0; k < K; ++k) {
        int64_t j = k < p.K ? p.sten[k * p.nc + c] : c;  // padding: the cell itself
        u.sten[k * nc + uc] = (int32_t)(j < p.nc ? co + j : nc + go + (j - p.nc));
      }
      for (int d = 0; d < 9; ++d)
        for (int k = 0; k < p.K; ++k) u.pinv0[((int64_t)d * K + k) * ncp + uc] = p.pinv0[((int64_t)d * p.K + k) * p.ncp + c];
      for (int r = 0; r < M * KM; ++r) u.subidx[(int64_t)r * ncp + uc] = p.subidx[(int64_t)r * p.ncp + c];
      for (int r = 0; r < M * 3 * KM; ++r) u.pinvm[(int64_t)r * ncp + uc] = p.pinvm[(int64_t)r * p.ncp + c];
      for (int q = 0; q < nfc; ++q) {
        const int32_t e = p.cface[q * p.nc + c];
        // a member's zero record (past its faces) becomes the union's
        u.cface[q * nc + uc] = e == (int32_t)(2 * p.nf) ? (int32_t)(2 * nf) : (int32_t)(e + 2 * fo);
      }
    }
    for (int64_t g = 0; g < p.ng; ++g) {
      u.gsrc[go + g] = (int32_t)(co + p.gsrc[g]);
      u.gtag[go + g] = p.gtag[g];
      for (int a3 = 0; a3 < 3; ++a3) u.gnrm[a3 * ng + go + g] = p.gnrm[a3 * p.ng + g];
    }
    for (int64_t f = 0; f < p.nf; ++f) {
      const int64_t uf = fo + f;
      u.fown[uf] = (int32_t)(co + p.fown[f]);
      u.fnbr[uf] = p.fnbr[f] >= 0 ? (int32_t)(co + p.fnbr[f]) : p.fnbr[f];
      for (int r = 0; r < G * 3; ++r) {
        u.fdl[r * nf + uf] = p.fdl[r * p.nf + f];
        u.fdr[r * nf + uf] = p.fdr[r * p.nf + f];
        u.fn[r * nf + uf] = p.fn[r * p.nf + f];
      }
      for (int r = 0; r < G; ++r) u.fw[r * nf + uf] = p.fw[r * p.nf + f];
    }
  }
  return HGKS_OK;
}

int64_t mesh_static_bytes(const HostMesh& m, int nmesh) {
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t nc = m.nc, nf = m.nf, ng = m.ng, ncp = m.ncp;
  int64_t b = 0;
  b += al(8 * nc) * 4;                         // volinv, hdt, hinv, caller index (int32 in an 8-byte slot)
  b += al(8 * 3 * nc) + al(8 * 6 * nc);        // (centroid slot), mom
  b += al(4 * (int64_t)m.K * nc);              // sten
  b += al(8 * (int64_t)9 * m.K * ncp);         // pinv0
  b += al((int64_t)m.M * m.KM * ncp);          // subidx
  b += al(8 * (int64_t)m.M * 3 * m.KM * ncp);  // pinvm
  b += al(4 * (int64_t)m.nfc * nc);            // cface
  b += al(4 * ng) * 2 + al(8 * 3 * ng);        // ghosts
  b += al(4 * nf) * 2;                         // fown, fnbr
  b += al(8 * (int64_t)m.G * 3 * nf) * 3 + al(8 * (int64_t)m.G * nf);  // fdl fdr fn fw
  b += al(4 * (int64_t)m.G * 3 * nf) * 3 + al(4 * (int64_t)m.G * nf);  // their binary32 roundings
  b += al(rec32_bytes(m.K, m.M, m.KM) * (ncp / 32));  // binary32 reconstruction records
  if (nmesh > 1) b += al(4 * nc);              // member of each cell
  return b + 256;
}

int64_t solver_work_bytes(const HostMesh& m, int precision, int nmesh) {
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t nc = m.nc, nf = m.nf, nce = nc + m.ng;
  const bool f32 = precision == HGKS_FP32_MIXED;
  const int64_t rs = f32 ? 4 : 8;
  int64_t b = 0;
  b += al(8 * 5 * nce) * 2;                    // Q, Q* (with ghost slots)
  b += al(8 * 5 * nc);                         // R (partial S2O4 sum)
  if (f32) b += al(4 * 8 * nce);               // binary32 copy of the stage state, 32 B per cell
  b += al(rs * (f32 ? kCoefRec32 : kCoefRec64) * nc);  // reconstruction coefficients
  b += al(rs * (f32 ? kFluxRec32 : kFluxRec64) * (nf + 1));  // face flux and its time slope, + a zero record
  b += al((int64_t)sizeof(Control) * nmesh);  // control blocks
  b += al((int64_t)sizeof(GridBar));           // barrier of the persistent step kernel
  return b + 256;
}

int64_t device_bytes(const HostMesh& m, int precision) {
  return mesh_static_bytes(m, 1) + solver_work_bytes(m, precision, 1);
}

}  // namespace hgks
