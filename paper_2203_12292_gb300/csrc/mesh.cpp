// Octree meshes of hexahedra on a cube (host set-up).
//
// Sec. 4 ("Examples"): every refinement step is completed by a closure that
// keeps leaves sharing a vertex within one level of each other.
// Sec. 2.2: global coarsening coarsens all cells at once; the hierarchy is
// built by repeating that step until one cell is left.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace gcmg {

namespace {
constexpr int PRED_ALL = 0, PRED_OCTANT_CENTRE = 1, PRED_SPHERE = 2, PRED_SHELL = 3, PRED_OCTANT_STRICT = 4;

inline uint64_t spread3(uint64_t v) {  // interleave helper: bit b -> bit 3b
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}
}  // namespace

int Octree::max_level() const {
  int m = 0;
  for (uint64_t key : leaves) m = std::max(m, (int)(key >> 57));
  return m;
}

int Octree::leaf_level(int l, int i, int j, int k) const {
  if (internal.count(cell_key(l, i, j, k))) return -1;
  for (int ll = l; ll >= 0; --ll, i >>= 1, j >>= 1, k >>= 1)
    if (leaves.count(cell_key(ll, i, j, k))) return ll;
  return -2;
}

void Octree::refine(const std::vector<Cell>& marked) {
  std::vector<Cell> work(marked.rbegin(), marked.rend());
  while (!work.empty()) {
    Cell c = work.back();
    work.pop_back();
    uint64_t key = cell_key(c.l, c.i, c.j, c.k);
    auto it = leaves.find(key);
    if (it == leaves.end()) continue;
    leaves.erase(it);
    internal.insert(key);
    for (int ch = 0; ch < 8; ++ch)
      leaves.insert(cell_key(c.l + 1, 2 * c.i + (ch & 1), 2 * c.j + ((ch >> 1) & 1), 2 * c.k + (ch >> 2)));
    // leaves of level <= l-1 touching c are now two levels coarser than c's
    // children: refine them as well
    const int n = 1 << c.l;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int ii = c.i + dx, jj = c.j + dy, kk = c.k + dz;
          if (ii < 0 || jj < 0 || kk < 0 || ii >= n || jj >= n || kk >= n) continue;
          int ll = leaf_level(c.l, ii, jj, kk);
          if (ll >= 0 && ll < c.l) {
            int s = c.l - ll;
            work.push_back(Cell{ll, ii >> s, jj >> s, kk >> s});
          }
        }
  }
}

void Octree::refine_step(const RefineStep& s) {
  std::vector<Cell> marked;
  for (const Cell& c : leaves_morton()) {
    const double h = (hi - lo) / double(1 << c.l);
    const double x0[3] = {lo + c.i * h, lo + c.j * h, lo + c.k * h};
    const double x1[3] = {x0[0] + h, x0[1] + h, x0[2] + h};
    bool mark = false;
    switch (s.pred) {
      case PRED_ALL: mark = true; break;
      case PRED_OCTANT_CENTRE: {
        mark = true;
        for (int d = 0; d < 3; ++d) {
          double m = 0.5 * (x0[d] + x1[d]);
          mark = mark && (m >= s.a && m <= s.b);
        }
        break;
      }
      case PRED_OCTANT_STRICT: {
        mark = true;
        for (int d = 0; d < 3; ++d) mark = mark && (x1[d] < s.b) && (x0[d] >= s.a);
        break;
      }
      case PRED_SHELL: {
        double r2 = 0;
        for (int d = 0; d < 3; ++d) {
          double m = 0.5 * (x0[d] + x1[d]);
          r2 += m * m;
        }
        double r = std::sqrt(r2);
        mark = (r >= s.a && r <= s.b);
        break;
      }
      case PRED_SPHERE: {
        double dmin2 = 0, dmax2 = 0;
        for (int d = 0; d < 3; ++d) {
          double lo_d = x0[d] - s.a, hi_d = x1[d] - s.a;
          double mn = (lo_d > 0) ? lo_d : (hi_d < 0 ? -hi_d : 0.0);
          double mx = std::max(std::fabs(lo_d), std::fabs(hi_d));
          dmin2 += mn * mn;
          dmax2 += mx * mx;
        }
        mark = dmin2 <= s.b * s.b && s.b * s.b <= dmax2;
        break;
      }
      default: throw std::runtime_error("unknown refinement predicate");
    }
    if (mark) marked.push_back(c);
  }
  refine(marked);
}

std::vector<Cell> Octree::leaves_morton() const {
  const int L = max_level();
  std::vector<std::pair<uint64_t, Cell>> v;
  v.reserve(leaves.size());
  for (uint64_t key : leaves) {
    Cell c{(int)(key >> 57), (int)((key >> 38) & 0x7FFFF), (int)((key >> 19) & 0x7FFFF), (int)(key & 0x7FFFF)};
    const int s = L - c.l;
    uint64_t code = spread3((uint64_t)c.i << s) | (spread3((uint64_t)c.j << s) << 1) | (spread3((uint64_t)c.k << s) << 2);
    v.push_back({code, c});
  }
  std::sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<Cell> out;
  out.reserve(v.size());
  for (auto& p : v) out.push_back(p.second);
  return out;
}

Octree coarsen_global(const Octree& fine) {
  // candidates: refined cells whose eight children are all leaves
  std::unordered_set<uint64_t> cand;
  for (uint64_t key : fine.internal) {
    int l = (int)(key >> 57), i = (int)((key >> 38) & 0x7FFFF), j = (int)((key >> 19) & 0x7FFFF),
        k = (int)(key & 0x7FFFF);
    bool all = true;
    for (int ch = 0; ch < 8 && all; ++ch)
      all = fine.leaves.count(cell_key(l + 1, 2 * i + (ch & 1), 2 * j + ((ch >> 1) & 1), 2 * k + (ch >> 2))) > 0;
    if (all) cand.insert(key);
  }
  auto refined_after = [&](int l, int i, int j, int k) {
    uint64_t key = cell_key(l, i, j, k);
    return fine.internal.count(key) && !cand.count(key);
  };
  // drop candidates that would touch a leaf two levels finer; repeat
  bool changed = true;
  while (changed) {
    changed = false;
    std::vector<uint64_t> drop;
    for (uint64_t key : cand) {
      int l = (int)(key >> 57), i = (int)((key >> 38) & 0x7FFFF), j = (int)((key >> 19) & 0x7FFFF),
          k = (int)(key & 0x7FFFF);
      const int n = 1 << l;
      bool bad = false;
      for (int dz = -1; dz <= 1 && !bad; ++dz)
        for (int dy = -1; dy <= 1 && !bad; ++dy)
          for (int dx = -1; dx <= 1 && !bad; ++dx) {
            if (!dx && !dy && !dz) continue;
            int ii = i + dx, jj = j + dy, kk = k + dz;
            if (ii < 0 || jj < 0 || kk < 0 || ii >= n || jj >= n || kk >= n) continue;
            if (!refined_after(l, ii, jj, kk)) continue;
            for (int ch = 0; ch < 8 && !bad; ++ch) {
              int a = ch & 1, b = (ch >> 1) & 1, c = ch >> 2;
              // only children of the neighbour that touch the candidate
              if ((dx > 0 && a != 0) || (dx < 0 && a != 1)) continue;
              if ((dy > 0 && b != 0) || (dy < 0 && b != 1)) continue;
              if ((dz > 0 && c != 0) || (dz < 0 && c != 1)) continue;
              if (refined_after(l + 1, 2 * ii + a, 2 * jj + b, 2 * kk + c)) bad = true;
            }
          }
      if (bad) drop.push_back(key);
    }
    for (uint64_t key : drop) cand.erase(key);
    changed = !drop.empty();
  }
  Octree c;
  c.lo = fine.lo;
  c.hi = fine.hi;
  for (uint64_t key : fine.internal)
    if (!cand.count(key)) c.internal.insert(key);
  for (uint64_t key : fine.leaves) {
    int l = (int)(key >> 57);
    if (l == 0) {
      c.leaves.insert(key);
      continue;
    }
    uint64_t pk = cell_key(l - 1, ((key >> 38) & 0x7FFFF) >> 1, ((key >> 19) & 0x7FFFF) >> 1, (key & 0x7FFFF) >> 1);
    if (!cand.count(pk)) c.leaves.insert(key);
  }
  for (uint64_t key : cand) c.leaves.insert(key);
  return c;
}

}  // namespace gcmg
