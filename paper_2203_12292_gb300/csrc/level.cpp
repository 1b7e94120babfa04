// DoF numbering and cell/tile metadata of one multigrid level (host set-up).
//
// Sec. 3.1-3.2: constraints (Dirichlet and hanging nodes) are applied while
// the cell values are set up; following the special-purpose algorithm the
// paper uses, the DoF map G_e of a cell with a hanging face or edge points to
// the DoFs of the constraining (coarse) face or edge, and the cell kernel
// interpolates in place (Sec. 3.2, hanging-node application).
//
// Layout chosen for one GPU:
// * DoFs live on the 27 geometric entities of a hexahedron (8 vertices,
//   12 edges, 6 faces, interior; 1, k-1, (k-1)^2, (k-1)^3 DoFs).  The DoFs of
//   one entity are contiguous, so a cell is described by 27 entity starts.
//   Dirichlet entities carry no DoFs (vectors hold free DoFs only).
// * Cells are in Morton order and grouped into tiles of `tile_cells`
//   consecutive cells.  Each entity is owned by the first tile that touches
//   it and the DoFs owned by one tile are numbered contiguously.  A cell
//   kernel writes its owned DoFs with plain stores and its contributions to
//   the other (foreign) DoFs into one halo slot each; a second kernel adds
//   the halo slots of every DoF in a fixed order.  No atomics: results are
//   reproducible bit for bit.
// * Inside a tile, cells that share an entity get different sub-colours; the
//   shared-memory accumulation runs sub-colour by sub-colour, and the cells
//   are permuted so that each sub-colour is contiguous.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace gcmg {

namespace {

constexpr uint64_t NO_ENTITY = ~0ull;

inline uint64_t ekey(int type, int dir, int logs, uint32_t x, uint32_t y, uint32_t z) {
  return ((uint64_t)type << 61) | ((uint64_t)dir << 59) | ((uint64_t)logs << 54) | ((uint64_t)x << 36) |
         ((uint64_t)y << 18) | (uint64_t)z;
}

struct EntityGeom {
  int32_t corner[3];
  int32_t size;
  uint8_t cls[3];
};

int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

}  // namespace

static uint16_t cell_mask(const Octree& mesh, const Cell& c) {
  if (c.l == 0) return 0;
  const int idx[3] = {c.i, c.j, c.k};
  const int p[3] = {c.i & 1, c.j & 1, c.k & 1};
  const int n = 1 << c.l;
  uint16_t m = (uint16_t)(p[0] | (p[1] << 1) | (p[2] << 2));
  auto coarser = [&](const int* q) {
    for (int d = 0; d < 3; ++d)
      if (q[d] < 0 || q[d] >= n) return false;
    int lv = mesh.leaf_level(c.l, q[0], q[1], q[2]);
    return lv >= 0 && lv < c.l;
  };
  for (int d = 0; d < 3; ++d) {
    int q[3] = {idx[0], idx[1], idx[2]};
    q[d] += p[d] ? 1 : -1;
    if (coarser(q)) m |= (uint16_t)(1u << (3 + d));
  }
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int s1 = p[t1] ? 1 : -1, s2 = p[t2] ? 1 : -1;
    int qa[3] = {idx[0], idx[1], idx[2]}, qb[3] = {idx[0], idx[1], idx[2]}, qc[3] = {idx[0], idx[1], idx[2]};
    qa[t1] += s1;
    qb[t2] += s2;
    qc[t1] += s1;
    qc[t2] += s2;
    if (coarser(qa) || coarser(qb) || coarser(qc)) m |= (uint16_t)(1u << (6 + d));
  }
  return m;
}

// is slot (cx,cy,cz) on a hanging face or hanging edge of a cell with mask m?
static bool slot_hanging(uint16_t m, const int* cl) {
  const int p[3] = {m & 1, (m >> 1) & 1, (m >> 2) & 1};
  for (int d = 0; d < 3; ++d)
    if ((m >> (3 + d)) & 1)
      if (cl[d] == 2 * p[d]) return true;
  for (int d = 0; d < 3; ++d)
    if ((m >> (6 + d)) & 1) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      if (cl[t1] == 2 * p[t1] && cl[t2] == 2 * p[t2]) return true;
    }
  return false;
}

void build_level(const Octree& mesh, int k, int tile_cells, int LM, LevelHost& L) {
  if (LM > 17) throw std::runtime_error("mesh too deep (max level 17)");
  L.k = k;
  L.lo = mesh.lo;
  L.hi = mesh.hi;
  L.lmax_lattice = LM;
  L.tile_cells = tile_cells;
  L.cells = mesh.leaves_morton();
  const int nc = (int)L.cells.size();
  const int top = 1 << LM;
  L.mask.assign(nc, 0);

  // entity of every slot
  std::vector<int32_t> eid((size_t)nc * NSLOT, -1);
  std::vector<uint8_t> hang_slot((size_t)nc * NSLOT, 0);
  std::unordered_map<uint64_t, int32_t> emap;
  emap.reserve((size_t)nc * 8);
  std::vector<int32_t> endofs;
  std::vector<EntityGeom> egeom;
  for (int ci = 0; ci < nc; ++ci) {
    const Cell& c = L.cells[ci];
    const uint16_t m = cell_mask(mesh, c);
    L.mask[ci] = m;
    const int idx[3] = {c.i, c.j, c.k};
    for (int s = 0; s < NSLOT; ++s) {
      const int cl[3] = {s % 3, (s / 3) % 3, s / 9};
      const bool hang = slot_hanging(m, cl);
      int X[3], size, logs;
      if (hang) {
        logs = LM - c.l + 1;
        size = 1 << logs;
        for (int d = 0; d < 3; ++d) X[d] = (idx[d] >> 1) << logs;
      } else {
        logs = LM - c.l;
        size = 1 << logs;
        for (int d = 0; d < 3; ++d) X[d] = idx[d] << logs;
      }
      int corner[3], ndim = 0, dir = 0;
      bool bnd = false;
      for (int d = 0; d < 3; ++d) {
        corner[d] = X[d] + (cl[d] == 2 ? size : 0);
        if (cl[d] == 1) ++ndim;
        else if (corner[d] == 0 || corner[d] == top) bnd = true;
      }
      if (ndim == 1) {
        for (int d = 0; d < 3; ++d)
          if (cl[d] == 1) dir = d;
      } else if (ndim == 2) {
        for (int d = 0; d < 3; ++d)
          if (cl[d] != 1) dir = d;
      }
      hang_slot[(size_t)ci * NSLOT + s] = hang;
      const int nd = ipow(k - 1, ndim);
      if (bnd || nd == 0) continue;
      const uint64_t key = ekey(ndim, dir, ndim == 0 ? 0 : logs, corner[0], corner[1], corner[2]);
      auto it = emap.find(key);
      int32_t e;
      if (it == emap.end()) {
        e = (int32_t)endofs.size();
        emap.emplace(key, e);
        endofs.push_back(nd);
        EntityGeom g;
        for (int d = 0; d < 3; ++d) {
          g.corner[d] = corner[d];
          g.cls[d] = (uint8_t)cl[d];
        }
        g.size = size;
        egeom.push_back(g);
      } else {
        e = it->second;
      }
      eid[(size_t)ci * NSLOT + s] = e;
    }
  }
  const int ne = (int)endofs.size();
  // entity type: number of interior axes (3 interior, 2 face, 1 edge, 0 vertex)
  auto etype = [&](int32_t e) {
    return (egeom[e].cls[0] == 1) + (egeom[e].cls[1] == 1) + (egeom[e].cls[2] == 1);
  };

  // Tiles of consecutive cells.  Every entity is owned by the first tile that
  // touches it (Morton order); the DoFs a tile owns are numbered
  // contiguously.  A tile adds its contributions to DoFs owned by other
  // tiles ("foreign" DoFs) into a halo buffer, one slot per (tile, foreign
  // DoF); a second pass adds the halo slots of every DoF in a fixed order.
  const int nt = (nc + tile_cells - 1) / tile_cells;
  std::vector<int32_t> owner(ne, -1);
  for (int t = 0; t < nt; ++t) {
    const int c0 = t * tile_cells, c1 = std::min(nc, c0 + tile_cells);
    for (int ci = c0; ci < c1; ++ci)
      for (int s = 0; s < NSLOT; ++s) {
        int32_t e = eid[(size_t)ci * NSLOT + s];
        if (e >= 0 && owner[e] < 0) owner[e] = t;
      }
  }
  std::vector<int32_t> estart(ne, -1);
  int64_t next = 0;
  L.tiles.assign(nt, TileInfo{});
  L.meta.assign(nc, CellMeta{});
  L.foreign.clear();
  L.subptr.clear();
  L.perm.assign(nc, 0);
  L.max_local = 0;
  L.max_sub = 0;
  std::vector<int32_t> lstart_of(ne, -1);
  for (int t = 0; t < nt; ++t) {
    const int c0 = t * tile_cells, c1 = std::min(nc, c0 + tile_cells);
    TileInfo& T = L.tiles[t];
    T.cell_begin = c0;
    T.n_cells = c1 - c0;
    T.dof_begin = (int32_t)next;
    // owned entities in first-touch order, then grouped by type (interiors, faces, edges,
    // vertices): the same slot of consecutive cells then lies a type's DoF count apart
    // (27, 9, 3 for Q4) instead of about one cell's DoF count (64 for Q4, a multiple of the
    // 32 shared-memory banks), which spreads the lanes of a warp that gather one node of 32
    // cells over the banks
    std::vector<int32_t> ord;
    for (int ci = c0; ci < c1; ++ci)
      for (int s = 0; s < NSLOT; ++s) {
        int32_t e = eid[(size_t)ci * NSLOT + s];
        if (e >= 0 && owner[e] == t && estart[e] == -1) {
          estart[e] = -2;  // listed
          ord.push_back(e);
        }
      }
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return etype(x) > etype(y); });
    for (int32_t e : ord) {
      estart[e] = (int32_t)next;
      next += endofs[e];
    }
    if (next > 0x7FFFFFFF) throw std::runtime_error("too many DoFs for 32-bit indices");
    T.n_owned = (int32_t)(next - T.dof_begin);
    // tile-local numbering: owned entities at their offset, foreign ones after
    T.foreign_begin = (int32_t)L.foreign.size();
    int32_t local_next = T.n_owned;
    std::vector<int32_t> touched, fgn;
    for (int ci = c0; ci < c1; ++ci)
      for (int s = 0; s < NSLOT; ++s) {
        int32_t e = eid[(size_t)ci * NSLOT + s];
        if (e < 0 || lstart_of[e] != -1) continue;
        touched.push_back(e);
        if (owner[e] == t) {
          lstart_of[e] = estart[e] - T.dof_begin;
        } else {
          lstart_of[e] = -2;  // listed
          fgn.push_back(e);
        }
      }
    // foreign entities: grouped by type as the owned ones
    std::stable_sort(fgn.begin(), fgn.end(), [&](int32_t x, int32_t y) { return etype(x) > etype(y); });
    for (int32_t e : fgn) {
      lstart_of[e] = local_next;
      local_next += endofs[e];
      for (int q = 0; q < endofs[e]; ++q) L.foreign.push_back(estart[e] + q);
    }
    T.n_foreign = local_next - T.n_owned;
    if (local_next >= (int)LS_NONE) throw std::runtime_error("tile too large for 16-bit local indices");
    L.max_local = std::max(L.max_local, (int)local_next);
    // sub-colours of the cells inside the tile (greedy, in cell order)
    const int n = c1 - c0;
    std::vector<int> sub(n, -1);
    int nsub = 0;
    {
      std::unordered_map<int32_t, std::vector<int>> ecells;
      std::vector<char> used;
      for (int a2 = 0; a2 < n; ++a2) {
        used.assign(n + 1, 0);
        for (int s = 0; s < NSLOT; ++s) {
          int32_t e = eid[(size_t)(c0 + a2) * NSLOT + s];
          if (e < 0) continue;
          auto it = ecells.find(e);
          if (it != ecells.end())
            for (int b2 : it->second) used[sub[b2]] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        sub[a2] = c;
        nsub = std::max(nsub, c + 1);
        for (int s = 0; s < NSLOT; ++s) {
          int32_t e = eid[(size_t)(c0 + a2) * NSLOT + s];
          if (e < 0) continue;
          auto& v = ecells[e];
          if (v.empty() || v.back() != a2) v.push_back(a2);
        }
      }
    }
    T.sub_begin = (int32_t)L.subptr.size();
    T.n_sub = nsub;
    L.max_sub = std::max(L.max_sub, nsub);
    int pos = 0;
    for (int c = 0; c < nsub; ++c) {
      L.subptr.push_back((uint16_t)pos);
      for (int a2 = 0; a2 < n; ++a2)
        if (sub[a2] == c) L.perm[c0 + pos++] = (uint8_t)a2;
    }
    L.subptr.push_back((uint16_t)pos);
    for (int ci = c0; ci < c1; ++ci) {
      CellMeta& cm = L.meta[ci];
      for (int s = 0; s < NSLOT; ++s) {
        int32_t e = eid[(size_t)ci * NSLOT + s];
        cm.ls[s] = e < 0 ? LS_NONE : (uint16_t)lstart_of[e];
      }
      cm.mask = L.mask[ci];
      cm.level = (uint8_t)L.cells[ci].l;
      cm.sub = (uint8_t)sub[ci - c0];
    }
    for (int32_t e : touched) lstart_of[e] = -1;
  }
  // lane-per-cell metadata of tiles of at most 32 cells
  L.lane.clear();
  L.lane_order.clear();
  L.lane_hang.clear();
  L.n_hang_tiles = 0;
  if (tile_cells <= 32) {
    L.lane.assign(nt, LaneTile{});
    for (int t = 0; t < nt; ++t) {
      const TileInfo& T = L.tiles[t];
      LaneTile& lt = L.lane[t];
      const int nloc = T.n_owned + T.n_foreign;
      if (4 * (nloc + LANE_ZERO) >= (int)LS_NONE) throw std::runtime_error("tile too large for 16-bit byte offsets");
      for (int j = 0; j < 32; ++j) {
        const bool cell = j < T.n_cells;
        const CellMeta* cm = cell ? &L.meta[T.cell_begin + j] : nullptr;
        for (int s = 0; s < NSLOT; ++s)
          lt.ls[s][j] = (uint16_t)(4 * ((cell && cm->ls[s] != LS_NONE) ? cm->ls[s] : nloc));
        lt.mask[j] = cell ? cm->mask : 0;
        lt.level[j] = cell ? cm->level : 0;
        if (cell && (cm->mask & MASK_HANG)) lt.hang = 1;
      }
    }
    L.lane_order.clear();
    for (int pass = 1; pass >= 0; --pass)
      for (int t = 0; t < nt; ++t)
        if (L.lane[t].hang == pass) L.lane_order.push_back(t);
    // hanging lines and slots of every lane of the tiles with hanging cells
    L.lane_hang.assign(nt, LaneHang{});
    L.n_hang_tiles = 0;
    const int n = k + 1;
    for (int t = 0; t < nt; ++t) {
      if (!L.lane[t].hang) continue;
      ++L.n_hang_tiles;
      LaneHang& lh = L.lane_hang[t];
      for (int j = 0; j < L.tiles[t].n_cells; ++j) {
        const uint16_t m = L.mask[L.tiles[t].cell_begin + j];
        if (!(m & MASK_HANG)) continue;
        for (int D = 0; D < 3; ++D) {
          const int A1 = D == 0 ? 1 : 0, A2 = D == 2 ? 1 : 2;  // the other two axes, increasing
          const int p1 = (m >> A1) & 1, p2 = (m >> A2) & 1;
          const bool f1 = (m >> (3 + A1)) & 1, f2 = (m >> (3 + A2)) & 1, ed = (m >> (6 + D)) & 1;
          for (int v = 0; v < n; ++v)
            for (int u = 0; u < n; ++u) {
              const bool on1 = u == p1 * k, on2 = v == p2 * k;
              if ((f1 && on1) || (f2 && on2) || (ed && on1 && on2)) lh.hl[D][j] |= 1u << (u + n * v);
            }
        }
        for (int s2 = 0; s2 < NSLOT; ++s2) {
          const int cl[3] = {s2 % 3, (s2 / 3) % 3, s2 / 9};
          if (slot_hanging(m, cl)) lh.hs[j] |= 1u << s2;
        }
      }
    }
  }
  L.n_free = next;
  for (int e = 0; e < ne; ++e)
    if (estart[e] < 0) throw std::runtime_error("entity without an owner tile");
  // halo: the foreign slots of every DoF, grouped by DoF in slot order
  {
    const int64_t nf = (int64_t)L.foreign.size();
    std::vector<int32_t> order(nf);
    for (int64_t i = 0; i < nf; ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a2, int32_t b2) { return L.foreign[a2] < L.foreign[b2]; });
    L.halo_dofs.clear();
    L.halo_ptr.assign(1, 0);
    L.halo_src.assign(nf, 0);
    for (int64_t i = 0; i < nf; ++i) {
      const int32_t g = L.foreign[order[i]];
      if (L.halo_dofs.empty() || L.halo_dofs.back() != g) {
        if (!L.halo_dofs.empty()) L.halo_ptr.push_back((int32_t)i);
        L.halo_dofs.push_back(g);
      }
      L.halo_src[i] = order[i];
    }
    L.halo_ptr.push_back((int32_t)nf);
    if (L.halo_dofs.empty()) L.halo_ptr.assign(1, 0);
    // tiles write each foreign contribution straight to its DoF-ordered position, so that
    // the halo pass reads every DoF's slots contiguously
    L.halo_pos.assign(nf, 0);
    for (int64_t e = 0; e < nf; ++e) L.halo_pos[L.halo_src[e]] = (int32_t)e;
  }
  // global starts and transfer ownership (first non-hanging reference wins)
  L.gstart.assign((size_t)nc * NSLOT, -1);
  L.own.assign(nc, 0u);
  std::vector<char> owned(ne, 0);
  for (int ci = 0; ci < nc; ++ci)
    for (int s = 0; s < NSLOT; ++s) {
      int32_t e = eid[(size_t)ci * NSLOT + s];
      if (e < 0) continue;
      L.gstart[(size_t)ci * NSLOT + s] = estart[e];
      if (!hang_slot[(size_t)ci * NSLOT + s] && !owned[e]) {
        owned[e] = 1;
        L.own[ci] |= 1u << s;
      }
    }
  for (int e = 0; e < ne; ++e)
    if (!owned[e]) throw std::runtime_error("entity without a non-hanging reference");
  // keep entity geometry for coordinates: store in the cells' order
  L.dof_xyz_cache.clear();
  L.dof_xyz_cache.resize((size_t)L.n_free * 3);
  const Basis1D& b = basis(k);
  const double hl = (L.hi - L.lo) / double(top);
  for (int e = 0; e < ne; ++e) {
    const EntityGeom& g = egeom[e];
    int free_axes[3], nf = 0;
    for (int d = 0; d < 3; ++d)
      if (g.cls[d] == 1) free_axes[nf++] = d;
    for (int q = 0; q < endofs[e]; ++q) {
      double x[3];
      for (int d = 0; d < 3; ++d) x[d] = L.lo + g.corner[d] * hl;
      int r = q;
      for (int a = 0; a < nf; ++a) {
        int ia = r % (k - 1);
        r /= (k - 1);
        x[free_axes[a]] = L.lo + (g.corner[free_axes[a]] + g.size * b.xi[ia + 1]) * hl;
      }
      for (int d = 0; d < 3; ++d) L.dof_xyz_cache[((size_t)estart[e] + q) * 3 + d] = x[d];
    }
  }
}

void LevelHost::dof_coordinates(std::vector<double>& xyz) const { xyz = dof_xyz_cache; }

// Check every invariant the tile kernels rely on; throws with a message.
void validate_level(const LevelHost& L) {
  auto fail = [](const std::string& m) { throw std::runtime_error("level check: " + m); };
  const int nc = (int)L.cells.size();
  const int nt = (int)L.tiles.size();
  const int k = L.k;
  auto ndofs = [k](int s) {
    int nd = 0;
    if (s % 3 == 1) ++nd;
    if ((s / 3) % 3 == 1) ++nd;
    if (s / 9 == 1) ++nd;
    return ipow(k - 1, nd);
  };
  int64_t next = 0;
  int cnext = 0;
  std::vector<int32_t> owner_tile(L.n_free, -1);
  for (int t = 0; t < nt; ++t) {
    const TileInfo& T = L.tiles[t];
    if (T.cell_begin != cnext || T.n_cells < 1 || T.n_cells > L.tile_cells) fail("tiles do not partition the cells");
    cnext += T.n_cells;
    if (T.dof_begin != next || T.n_owned < 0) fail("owned ranges do not partition the DoFs");
    for (int i = 0; i < T.n_owned; ++i) owner_tile[T.dof_begin + i] = t;
    next += T.n_owned;
    if (T.n_owned + T.n_foreign > L.max_local || L.max_local >= (int)LS_NONE) fail("local size");
    if (t + 1 < nt && L.tiles[t + 1].foreign_begin != T.foreign_begin + T.n_foreign) fail("foreign lists not contiguous");
  }
  if (cnext != nc || next != L.n_free) fail("tiles do not cover cells/DoFs");
  for (int t = 0; t < nt; ++t) {
    const TileInfo& T = L.tiles[t];
    const int nloc = T.n_owned + T.n_foreign;
    std::vector<int64_t> l2g(nloc);
    for (int q = 0; q < T.n_owned; ++q) l2g[q] = T.dof_begin + q;
    for (int q = 0; q < T.n_foreign; ++q) {
      const int32_t g = L.foreign[T.foreign_begin + q];
      if (g < 0 || g >= L.n_free) fail("foreign index out of range");
      if (owner_tile[g] == t) fail("foreign DoF owned by its own tile");
      l2g[T.n_owned + q] = g;
    }
    const int n = T.n_cells;
    if (T.n_sub < 1 || L.subptr[T.sub_begin] != 0 || L.subptr[T.sub_begin + T.n_sub] != n) fail("sub-colour offsets");
    std::vector<char> seen(n, 0);
    std::vector<int> local_sub(nloc, -1);
    for (int sc = 0; sc < T.n_sub; ++sc)
      for (int q = L.subptr[T.sub_begin + sc]; q < L.subptr[T.sub_begin + sc + 1]; ++q) {
        const int a = L.perm[T.cell_begin + q];
        if (a >= n || seen[a]) fail("sub-colour permutation");
        seen[a] = 1;
        const int ci = T.cell_begin + a;
        if (L.meta[ci].sub != sc) fail("cell sub-colour disagrees with the permutation");
        for (int s = 0; s < NSLOT; ++s) {
          const uint16_t ls = L.meta[ci].ls[s];
          const int32_t gs = L.gstart[(size_t)ci * NSLOT + s];
          if ((ls == LS_NONE) != (gs < 0)) fail("local and global maps disagree on a slot");
          if (ls == LS_NONE) continue;
          for (int o = 0; o < ndofs(s); ++o) {
            if (ls + o >= nloc) fail("local index out of range");
            if (l2g[ls + o] != gs + o) fail("local index maps to the wrong DoF");
            if (local_sub[ls + o] == sc) fail("two cells of one sub-colour share a DoF");
            local_sub[ls + o] = sc;
          }
        }
      }
  }
  // halo: every foreign slot appears exactly once, grouped under its DoF
  const int64_t nf = (int64_t)L.foreign.size();
  std::vector<char> hit(nf, 0);
  const int64_t nh = (int64_t)L.halo_dofs.size();
  if ((int64_t)L.halo_ptr.size() != nh + 1 || L.halo_ptr[0] != 0 || L.halo_ptr[nh] != nf) fail("halo offsets");
  for (int64_t u = 0; u < nh; ++u) {
    if (u > 0 && L.halo_dofs[u] <= L.halo_dofs[u - 1]) fail("halo DoFs not increasing");
    for (int32_t e = L.halo_ptr[u]; e < L.halo_ptr[u + 1]; ++e) {
      const int32_t src = L.halo_src[e];
      if (src < 0 || src >= nf || hit[src]) fail("halo slot used twice or out of range");
      hit[src] = 1;
      if (L.foreign[src] != L.halo_dofs[u]) fail("halo slot under the wrong DoF");
    }
  }
  // the lane kernels' order of accumulation (tiles of at most 32 cells).  Node (a, b, c) of the
  // cell in lane j adds to tile-local DoF ls[slot][j] / 4 + offset (absent slots: the zero region).
  //  * tiles without hanging cells (fp32 kernel, warp c holds plane c): the planes whose nodes
  //    add to one DoF are one plane or lie in {0, k} (warp k adds after warp 0), and no two cells
  //    add to one DoF through the same node (one instruction of one warp);
  //  * tiles with hanging cells and the double-float kernel (x-lines dealt to warps by class):
  //    the classes (b or boundary, c or boundary) of the x-lines that add to one DoF are one class.
  if (!L.lane.empty()) {
    const int n = k + 1;
    auto cls = [k](int x) { return x == 0 ? 0 : (x == k ? 2 : 1); };
    std::vector<int> nslot(n * n * n), noff(n * n * n);
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          const int ca = cls(a), cb = cls(b), cc = cls(c);
          int o = 0, mul = 1;
          if (ca == 1) {
            o += a - 1;
            mul *= k - 1;
          }
          if (cb == 1) {
            o += (b - 1) * mul;
            mul *= k - 1;
          }
          if (cc == 1) o += (c - 1) * mul;
          nslot[a + n * (b + n * c)] = ca + 3 * cb + 9 * cc;
          noff[a + n * (b + n * c)] = o;
        }
    std::vector<uint32_t> planes;
    std::vector<uint64_t> classes;
    std::vector<int64_t> stamp;
    for (int t = 0; t < nt; ++t) {
      const TileInfo& T = L.tiles[t];
      const LaneTile& lt = L.lane[t];
      const int nloc = T.n_owned + T.n_foreign;
      planes.assign(nloc, 0u);
      classes.assign(nloc, 0u);
      stamp.assign(nloc, -1);
      for (int nd = 0; nd < n * n * n; ++nd) {
        const int a = nd % n, b = (nd / n) % n, c = nd / (n * n);
        // the x-line's class: b and c, each either its interior value or "boundary" (0 or k)
        const int xcls = (cls(b) == 1 ? b : n) + (n + 1) * (cls(c) == 1 ? c : n);
        (void)a;
        for (int j = 0; j < T.n_cells; ++j) {
          const int off = lt.ls[nslot[nd]][j];
          if (off % 4 || off / 4 > nloc) fail("lane offset");
          if (off / 4 == nloc) continue;  // the zero region
          const int dof = off / 4 + noff[nd];
          if (dof >= nloc) fail("lane DoF outside the tile");
          planes[dof] |= 1u << c;
          classes[dof] |= uint64_t(1) << xcls;
          if (!lt.hang) {
            const int64_t key = (int64_t)t * 1024 + nd;
            if (stamp[dof] == key) fail("two cells add to one DoF through one node");
            stamp[dof] = key;
          }
        }
      }
      const uint32_t ends = 1u | (1u << k);
      for (int d = 0; d < nloc; ++d) {
        if (!lt.hang && (planes[d] & (planes[d] - 1u)) && (planes[d] & ~ends))
          fail("a DoF added from two planes other than 0 and k");
        if (classes[d] & (classes[d] - 1)) fail("a DoF added from two x-line classes");
      }
    }
  }
  // transfer ownership: every DoF owned by exactly one (cell, slot)
  std::vector<int8_t> owned(L.n_free, 0);
  for (int ci = 0; ci < nc; ++ci)
    for (int s = 0; s < NSLOT; ++s)
      if ((L.own[ci] >> s) & 1u) {
        const int32_t gs = L.gstart[(size_t)ci * NSLOT + s];
        if (gs < 0) fail("owned slot without DoFs");
        for (int o = 0; o < ndofs(s); ++o)
          if (owned[gs + o]++) fail("DoF owned twice for the transfer");
      }
  for (int64_t g = 0; g < L.n_free; ++g)
    if (!owned[g]) fail("DoF without a transfer owner");
}

void build_transfer_h(const LevelHost& fine, const LevelHost& coarse, TransferHost& T, bool allow_missing) {
  T.kind = 0;
  std::unordered_map<uint64_t, int32_t> fidx;
  fidx.reserve(fine.cells.size() * 2);
  for (size_t i = 0; i < fine.cells.size(); ++i) {
    const Cell& c = fine.cells[i];
    fidx.emplace(cell_key(c.l, c.i, c.j, c.k), (int32_t)i);
  }
  const size_t nc = coarse.cells.size();
  T.fine_of.assign(nc, -1);
  T.refined.assign(nc, 0);
  for (size_t ci = 0; ci < nc; ++ci) {
    const Cell& c = coarse.cells[ci];
    auto it = fidx.find(cell_key(c.l, c.i, c.j, c.k));
    if (it != fidx.end()) {
      T.fine_of[ci] = it->second;
      continue;
    }
    auto ch = fidx.find(cell_key(c.l + 1, 2 * c.i, 2 * c.j, 2 * c.k));
    if (ch == fidx.end()) {
      if (allow_missing) continue;  // fine_of stays -1
      throw std::runtime_error("levels are not nested");
    }
    // the eight children are consecutive in Morton order
    for (int q = 0; q < 8; ++q) {
      const Cell& f = fine.cells[ch->second + q];
      if (f.l != c.l + 1 || (f.i >> 1) != c.i || (f.j >> 1) != c.j || (f.k >> 1) != c.k ||
          (f.i & 1) != (q & 1) || (f.j & 1) != ((q >> 1) & 1) || (f.k & 1) != (q >> 2))
        throw std::runtime_error("children not consecutive in Morton order");
    }
    T.fine_of[ci] = ch->second;
    T.refined[ci] = 1;
  }
}

void build_transfer_p(const LevelHost& fine, const LevelHost& coarse, TransferHost& T) {
  if (fine.cells.size() != coarse.cells.size()) throw std::runtime_error("p-transfer needs one mesh");
  T.kind = 1;
  T.fine_of.resize(coarse.cells.size());
  T.refined.assign(coarse.cells.size(), 0);
  for (size_t i = 0; i < coarse.cells.size(); ++i) T.fine_of[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// local smoothing
// ---------------------------------------------------------------------------
Octree refinement_level(const Octree& fine, int l) {
  Octree m;
  m.lo = fine.lo;
  m.hi = fine.hi;
  for (const auto* set : {&fine.leaves, &fine.internal})
    for (uint64_t key : *set)
      if ((int)(key >> 57) == l) m.leaves.insert(key);
  return m;
}

std::vector<int32_t> refinement_edge_dofs(const LevelHost& L, const Octree& level_mesh) {
  std::vector<int32_t> out;
  if (L.cells.empty()) return out;
  const int l = L.cells[0].l;
  const int n = 1 << l;
  const double h = (L.hi - L.lo) / n;
  std::vector<double> xyz;
  L.dof_coordinates(xyz);
  for (int64_t g = 0; g < L.n_free; ++g) {
    // the grid cells of level l whose closure holds the point: one or two per axis
    int lo_idx[3], hi_idx[3];
    for (int d = 0; d < 3; ++d) {
      const double t = (xyz[3 * g + d] - L.lo) / h;
      const double r = std::nearbyint(t);
      if (std::fabs(t - r) < 1e-9) {
        lo_idx[d] = (int)r - 1;
        hi_idx[d] = (int)r;
      } else {
        lo_idx[d] = hi_idx[d] = (int)std::floor(t);
      }
    }
    bool edge = false;
    for (int i = lo_idx[0]; i <= hi_idx[0] && !edge; ++i)
      for (int j = lo_idx[1]; j <= hi_idx[1] && !edge; ++j)
        for (int k = lo_idx[2]; k <= hi_idx[2] && !edge; ++k)
          if (i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n &&
              !level_mesh.leaves.count(cell_key(l, i, j, k)))
            edge = true;
    if (edge) out.push_back((int32_t)g);
  }
  return out;
}

void local_copy_map(const LevelHost& active, const std::vector<const LevelHost*>& levels,
                    std::vector<std::vector<int32_t>>& g, std::vector<std::vector<int32_t>>& idx) {
  const int nl = (int)levels.size();
  const int k = active.k;
  std::vector<std::unordered_map<uint64_t, int32_t>> cidx(nl);
  for (int l = 0; l < nl; ++l)
    for (size_t c = 0; c < levels[l]->cells.size(); ++c) {
      const Cell& cc = levels[l]->cells[c];
      cidx[l].emplace(cell_key(cc.l, cc.i, cc.j, cc.k), (int32_t)c);
    }
  // active cells by increasing level: the first level to reach a DoF keeps it
  std::vector<int32_t> order(active.cells.size());
  for (size_t c = 0; c < order.size(); ++c) order[c] = (int32_t)c;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return active.cells[a].l < active.cells[b].l; });
  std::vector<int32_t> lvl(active.n_free, -1), at(active.n_free, -1);
  for (int32_t c : order) {
    const Cell& cc = active.cells[c];
    if (cc.l >= nl) throw std::runtime_error("active cell finer than the refinement levels");
    auto it = cidx[cc.l].find(cell_key(cc.l, cc.i, cc.j, cc.k));
    if (it == cidx[cc.l].end()) throw std::runtime_error("active cell missing on its refinement level");
    const LevelHost& Lv = *levels[cc.l];
    const int lc = it->second;
    const uint16_t m = active.mask[c];
    for (int s = 0; s < NSLOT; ++s) {
      const int cl[3] = {s % 3, (s / 3) % 3, s / 9};
      if (slot_hanging(m, cl)) continue;  // constrained values: no active DoF here
      const int32_t ga = active.gstart[(size_t)c * NSLOT + s];
      const int32_t gl = Lv.gstart[(size_t)lc * NSLOT + s];
      if (ga < 0) continue;
      if (gl < 0) throw std::runtime_error("refinement level lacks a DoF of an active cell");
      int nd = 0;
      for (int d = 0; d < 3; ++d) nd += cl[d] == 1;
      const int cnt = ipow(k - 1, nd);
      for (int q = 0; q < cnt; ++q)
        if (lvl[ga + q] < 0) {
          lvl[ga + q] = cc.l;
          at[ga + q] = gl + q;
        }
    }
  }
  g.assign(nl, {});
  idx.assign(nl, {});
  for (int64_t d = 0; d < active.n_free; ++d) {
    if (lvl[d] < 0) throw std::runtime_error("an active DoF without a refinement level");
    g[lvl[d]].push_back((int32_t)d);
    idx[lvl[d]].push_back(at[d]);
  }
}

}  // namespace gcmg
