// Internal declarations shared by the host set-up (C++) and the CUDA
// translation units of libgcmg.  Nothing here is part of the public C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace gcmg {

constexpr int KMAX = 4;
constexpr int NMAX = KMAX + 1;
constexpr int NSLOT = 27;  // vertices, edges, faces, interior of a hexahedron

// ---------------------------------------------------------------------------
// hanging mask of a cell (16 bits)
//   bits 0-2 : position of the cell inside its parent along x, y, z
//   bits 3-5 : outer face with normal x / y / z hangs on a coarser neighbour
//   bits 6-8 : outer edge along x / y / z hangs on a coarser neighbour
// A cell only has hanging faces/edges on the boundary of its parent, i.e. the
// face with normal d lies on side p_d and the edge along d at (p_t1, p_t2).
// ---------------------------------------------------------------------------
constexpr uint16_t MASK_POS = 0x7;
constexpr uint16_t MASK_FACE = 0x38;
constexpr uint16_t MASK_EDGE = 0x1C0;
constexpr uint16_t MASK_HANG = MASK_FACE | MASK_EDGE;
constexpr uint16_t LS_NONE = 0xFFFF;  // slot without DoFs (Dirichlet)

// per-cell operator metadata, 64 bytes
struct CellMeta {
  uint16_t ls[NSLOT];  // tile-local start of each slot's DoFs, LS_NONE = none
  uint16_t mask;
  uint8_t level;
  uint8_t sub;         // sub-colour inside the tile
  uint8_t pad[6];
};
static_assert(sizeof(CellMeta) == 64, "CellMeta must be 64 bytes");

// per-tile metadata of the lane-per-cell fp32 operator (one lane per cell of
// a tile of at most 32 cells, Morton order): the tile-local entity starts as
// byte offsets (4 x tile-local index), transposed (slot s of the cell in lane
// j at ls[s][j]) so that a warp reads them conflict-free; absent slots
// (Dirichlet entities, lanes without a cell) point to LANE_ZERO zero values
// after the tile's DoFs
constexpr int LANE_ZERO = 32;
struct LaneTile {
  uint16_t ls[NSLOT][32];
  uint16_t mask[32];
  uint8_t level[32];
  uint8_t hang;  // 1: a cell of the tile has a hanging face or edge
  uint8_t pad[31];
};
static_assert(sizeof(LaneTile) % 64 == 0, "LaneTile is copied in 16-byte pieces");
// per tile, for the tiles with hanging cells: per lane the lines of its cell
// on a hanging face or edge, one set per direction D (bit u + (k+1) v for the
// line through the other two coordinates (u, v), in increasing axis order),
// and the 27-bit set of its slots on a hanging face or edge
struct LaneHang {
  uint32_t hl[3][32];
  uint32_t hs[32];
};

struct TileInfo {
  int32_t cell_begin;
  int32_t n_cells;
  int32_t dof_begin;     // first DoF owned by this tile (owned DoFs are contiguous)
  int32_t n_owned;
  int32_t foreign_begin; // into the level's foreign-DoF index list
  int32_t n_foreign;
  int32_t sub_begin;     // into the level's sub-colour offset list
  int32_t n_sub;
};

// ---------------------------------------------------------------------------
// 1D tables of one polynomial degree (host-computed in fp64)
// ---------------------------------------------------------------------------
struct Basis1D {
  int k = 0;
  double xi[NMAX];            // Gauss-Lobatto support points on [0,1]
  double gq[NMAX], gw[NMAX];  // Gauss points / weights on [0,1], k+1 points
  double M[NMAX][NMAX];       // 1D mass matrix
  double K[NMAX][NMAX];       // 1D stiffness matrix
  double B[NMAX][NMAX];       // B = S^{-1}, S^T M S = I, S^T K S = diag(lam)
  double lam[NMAX];
  double I[2][NMAX][NMAX];    // I[p][a][b] = L_b((p + xi_a)/2): child-side interpolation
  double Pq[NMAX][NMAX];      // Pq[q][a] = L_a(gq_q): values at Gauss points
  double Ph[2 * KMAX + 1][NMAX];  // h-prolongation onto the 2k+1 child nodes
};

const Basis1D& basis(int k);
// p-prolongation from degree kc to kf on one cell: P[i][a] = L^{kc}_a(xi^{kf}_i)
void p_prolongation(int kf, int kc, double P[NMAX][NMAX]);
double lagrange(const double* nodes, int n, int a, double t);

// ---------------------------------------------------------------------------
// octree meshes
// ---------------------------------------------------------------------------
struct Cell {
  int32_t l, i, j, k;
};

inline uint64_t cell_key(int l, uint32_t i, uint32_t j, uint32_t k) {
  return ((uint64_t)l << 57) | ((uint64_t)i << 38) | ((uint64_t)j << 19) | (uint64_t)k;
}

struct RefineStep {
  int pred;
  double a, b, c, d;
};

struct Octree {
  double lo = 0.0, hi = 1.0;
  std::unordered_set<uint64_t> leaves, internal;
  int max_level() const;
  // level of the leaf that contains block (l,i,j,k); -1 if the block is refined
  int leaf_level(int l, int i, int j, int k) const;
  void refine(const std::vector<Cell>& marked);
  void refine_step(const RefineStep& s);
  std::vector<Cell> leaves_morton() const;  // leaves in Morton (depth-first) order
};

Octree coarsen_global(const Octree& fine);

// ---------------------------------------------------------------------------
// one multigrid level: DoF numbering, tiles, colours (host side)
// ---------------------------------------------------------------------------
struct LevelHost {
  int k = 1;
  int lmax_lattice = 0;  // lattice resolution 2^lmax_lattice for entity keys
  double lo = 0, hi = 1;
  std::vector<Cell> cells;         // Morton order
  std::vector<uint16_t> mask;      // per cell
  std::vector<int32_t> gstart;     // per cell x 27: global DoF start of the slot, -1 = none
  std::vector<uint32_t> own;       // per cell: 27-bit mask, slot entity is owned by this cell (transfer)
  int64_t n_free = 0;
  // tiles
  int tile_cells = 128;
  std::vector<TileInfo> tiles;
  std::vector<CellMeta> meta;      // per cell
  std::vector<int32_t> foreign;    // foreign DoF global indices, per tile contiguous
  std::vector<uint16_t> subptr;    // per tile: n_sub+1 offsets into the tile's permuted cell list
  std::vector<uint8_t> perm;       // per cell (tile order): local cell index in sub-colour order
  std::vector<int32_t> halo_dofs;  // DoFs that receive contributions from other tiles (increasing)
  std::vector<int32_t> halo_ptr;   // per halo DoF: range into halo_src
  std::vector<int32_t> halo_src;   // foreign-slot indices (positions in `foreign`)
  std::vector<int32_t> halo_pos;   // per foreign slot: its position in the DoF-ordered halo buffer
  int max_local = 0;               // max tile-local DoF count
  std::vector<LaneTile> lane;      // per tile (tiles of at most 32 cells): lane-per-cell metadata
  std::vector<int32_t> lane_order; // tiles with hanging cells, then the others (launch order)
  std::vector<LaneHang> lane_hang; // per tile (zero for tiles without hanging cells)
  int n_hang_tiles = 0;            // tiles with hanging cells (the first entries of lane_order)
  int max_sub = 0;
  // dof coordinates (host) for checks
  std::vector<double> dof_xyz_cache;
  void dof_coordinates(std::vector<double>& xyz) const;
};

void build_level(const Octree& mesh, int k, int tile_cells, int lmax_lattice, LevelHost& L);
void validate_level(const LevelHost& L);

// transfer between a fine level and the next coarser one
struct TransferHost {
  int kind = 0;                      // 0 = h (geometric), 1 = p (polynomial)
  std::vector<int32_t> fine_of;      // per coarse cell: fine cell (identity) or first child; -1: none
  std::vector<uint8_t> refined;      // per coarse cell: 1 if refined (8 children)
};
// allow_missing: coarse cells without a counterpart on the fine level take no
// part (the refinement levels of local smoothing)
void build_transfer_h(const LevelHost& fine, const LevelHost& coarse, TransferHost& T, bool allow_missing = false);
void build_transfer_p(const LevelHost& fine, const LevelHost& coarse, TransferHost& T);

// ---------------------------------------------------------------------------
// local smoothing (Sec. 2.1): refinement levels, refinement edges, the copy of
// Algorithm 1
// ---------------------------------------------------------------------------
// every cell of refinement level l of `fine` (active or refined) as a leaf
Octree refinement_level(const Octree& fine, int l);
// DoFs of a refinement level on its refinement edges: support points on the
// boundary of the region its cells cover, inside the domain (increasing)
std::vector<int32_t> refinement_edge_dofs(const LevelHost& L, const Octree& level_mesh);
// Algorithm 1: every free DoF g of the active level goes to the coarsest
// refinement level among its active cells; per level l the pairs
// (g[l][i], idx[l][i]) of active DoF and level DoF
void local_copy_map(const LevelHost& active, const std::vector<const LevelHost*>& levels,
                    std::vector<std::vector<int32_t>>& g, std::vector<std::vector<int32_t>>& idx);

}  // namespace gcmg
