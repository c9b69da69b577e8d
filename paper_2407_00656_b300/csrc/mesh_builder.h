// mesh_builder.h -- host-side mesh preprocessing for the HGKS GPU path.
//
// Produces the structure-of-arrays data that the kernels read: cells ordered
// along a Morton curve, faces ordered by owner, boundary ghost slots, padded
// two-layer WENO stencils with their least-squares pseudo-inverses
// (Section 2.3, Algorithm 1) and face Gauss-point geometry (Section 2.1).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "hgks.h"

namespace hgks {

struct HostMesh {
  int ctype = 0;   // 4 or 8 nodes per cell
  int nfc = 0;     // faces per cell: 4 or 6
  int G = 0;       // Gauss points per face: 3 or 4
  int M = 0;       // sub-stencils per cell: 4 or 8
  int KM = 0;      // padded sub-stencil size: 6 (tet) or 3 (hex)
  int K = 0;       // padded big-stencil size (max over cells)
  int64_t nc = 0, nf = 0, ng = 0;
  int64_t ncp = 0;  // row pitch of pinv0, subidx, pinvm: nc rounded up to 32, so that
                    // 32 consecutive cells of a row start on a 256-byte boundary

  // cell order: new index -> caller index
  std::vector<int64_t> perm;

  // Every array is structure-of-arrays: component j of item i at [j*n + i]
  // (n = nc, ng or nf), so that consecutive threads read consecutive words.

  // per cell, new order
  std::vector<double> vol;       // [nc]
  std::vector<double> hdt;       // [nc] 3|cell|/|surface|
  std::vector<double> cen;       // [3][nc]
  std::vector<double> mom;       // [6][nc] central second moments / h^2 (xx yy zz xy yz zx)
  std::vector<double> hinv;      // [nc] 1/h, h = |cell|^(1/3)
  std::vector<int32_t> sten;     // [K][nc] indices into cells+ghosts (padding: the cell itself)
  std::vector<double> pinv0;     // [9*K][ncp] quadratic least-squares inverse, row d col k at d*K+k
  std::vector<uint8_t> subidx;   // [M*KM][ncp] positions in the big stencil
  std::vector<double> pinvm;     // [M*3*KM][ncp] linear inverses, (m,d,r) at (m*3+d)*KM+r
  std::vector<int32_t> cface;    // [nfc][nc] 2*face + (1 if the cell is the face's neighbour);
                                 // 2*nf for the collapsed side of a prism (a flux record kept zero)

  // per ghost (one per physical boundary face)
  std::vector<int32_t> gsrc;     // [ng] mirrored interior cell
  std::vector<int32_t> gtag;     // [ng] HGKS_BC_FARFIELD or HGKS_BC_WALL
  std::vector<double> gnrm;      // [3][ng] unit outward normal of the mirror plane

  // per face, ordered by owner
  std::vector<int32_t> fown;     // [nf]
  std::vector<int32_t> fnbr;     // [nf] neighbour cell, or -tag for a physical boundary
  std::vector<double> fdl;       // [G*3][nf] Gauss point minus owner centroid
  std::vector<double> fdr;       // [G*3][nf] Gauss point (neighbour image) minus neighbour centroid
  std::vector<double> fn;        // [G*3][nf] unit normal, owner -> neighbour
  std::vector<double> fw;        // [G][nf] quadrature weight times area
};

// Build from a validated description; returns HGKS_OK or an error code with
// a message in err.
int build_host_mesh(const hgks_mesh_desc& d, HostMesh& m, std::string& err);

// Disjoint union of member meshes of one cell type: cells, ghosts and faces
// concatenated member by member (cell offsets in coff), stencils padded to
// the largest K, cmesh[c] = member of union cell c.  perm of the union is left
// empty; each member keeps its own.
int build_union(const std::vector<const HostMesh*>& parts, HostMesh& u, std::vector<int32_t>& cmesh,
                std::vector<int64_t>& coff, std::string& err);

// Device bytes, including alignment padding, of the static mesh arrays (a
// device mesh over nmesh members), of one solver's state and work arrays
// (precision HGKS_FP64 or HGKS_FP32_MIXED), and of both for a single mesh.
int64_t mesh_static_bytes(const HostMesh& m, int nmesh);
int64_t solver_work_bytes(const HostMesh& m, int precision, int nmesh);
int64_t device_bytes(const HostMesh& m, int precision);

}  // namespace hgks
