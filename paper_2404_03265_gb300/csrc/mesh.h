// Host-side quadtree, leaf/level node layouts and constraint tables of libpff.
//
// Sec. 3 of Kolditz & Wick (arXiv 2404.03265): Q_k finite elements on locally
// refined quadrilateral meshes with hanging nodes; Sec. 3.2: geometric multigrid
// with local smoothing on the level meshes (all cells of one refinement level).
//
// Storage ("brick layout").  Every refinement level l has a structured node grid
// (spacing h_l / k).  It is cut into square bricks of NB x NB node slots
// (NB = B * k = 30; B = 30 cells for Q1, 15 for Q2).  A node vector is the
// concatenation of the bricks of all levels, NB*NB slots each; a mesh node
// lives in exactly one slot ("home"), the other slots are holes (kept at zero).
//   * leaf mesh: a node's home is the coarsest level among the leaf cells that
//     have it as a node; bricks exist where a level-l leaf cell has a node;
//   * level mesh l (multigrid): nodes of all level-l cells, one level only.
// A brick whose window (its (B+1)^2 cells and (NB+k+1)^2 nodes) is complete and
// single-level is "regular": kernels compute every address from the 3x3
// neighbour bases and read no index table.  Other bricks carry explicit
// per-slot tables.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace pff {

inline uint64_t cell_key(int64_t i, int64_t j) { return (uint64_t(uint32_t(i)) << 32) | uint64_t(uint32_t(j)); }

struct Tree {
  double x0 = 0, x1 = 1, y0 = 0, y1 = 1;
  int ncx = 1, ncy = 1;
  std::vector<std::unordered_set<uint64_t>> lev;  // all cells (leaf or refined) per level

  double hx(int l) const { return (x1 - x0) / (double(ncx) * double(int64_t(1) << l)); }
  double hy(int l) const { return (y1 - y0) / (double(ncy) * double(int64_t(1) << l)); }
  int64_t nx(int l) const { return int64_t(ncx) << l; }
  int64_t ny(int l) const { return int64_t(ncy) << l; }
  bool has(int l, int64_t i, int64_t j) const {
    if (l < 0 || l >= int(lev.size())) return false;
    return lev[l].count(cell_key(i, j)) != 0;
  }
  bool is_leaf(int l, int64_t i, int64_t j) const { return has(l, i, j) && !has(l + 1, 2 * i, 2 * j); }
  void split(int l, int64_t i, int64_t j);
  void balance();
  int finest() const;
  // leaves in canonical order (level, j, i)
  std::vector<std::array<int64_t, 3>> leaves() const;
};

// Device-side brick descriptor (plain data, copied as is).
struct BrickDesc {
  int32_t level;
  int32_t bx, by;
  int32_t irr;           // -1: regular, else index into the irregular tables
  int32_t nbr_base[9];   // storage base of the 3x3 neighbour bricks (index (dy+1)*3+dx+1), -1 absent
};

// codes in irregular window tables
constexpr int32_t kAbsent = -1;
inline int32_t hanging_code(int32_t h) { return -2 - h; }
// own-slot storage actions
constexpr uint8_t kActNone = 0, kActFinal = 1, kActZero = 2;

struct Layout {
  int k = 1, B = 30, NB = 30, W = 32;
  std::vector<BrickDesc> bricks;
  int64_t n_slots = 0;
  std::vector<int32_t> win;       // per irregular brick W*W codes
  std::vector<int32_t> own_part;  // per irregular brick NB*NB partial-slot ids (-1 none)
  std::vector<uint8_t> own_act;   // per irregular brick NB*NB storage actions
  std::vector<uint32_t> cellmask; // per irregular brick ceil((B+1)^2/32) words
  int cm_words() const { return ((B + 1) * (B + 1) + 31) / 32; }
  int n_irregular() const { return int(own_act.size() / size_t(NB * NB)); }
};

struct HangingEntry {
  int32_t slot;            // storage slot of the hanging node (linearisation is stored resolved)
  int32_t parent[3];       // storage slots of the constraining nodes (k+1 used)
  double weight[3];
};

struct LevelMesh {
  int level = 0;
  Layout lay;
  int64_t n_nodes = 0;
  std::vector<int32_t> slot_X, slot_Y;   // finest-grid integer coordinates, -1 for holes
  std::vector<uint8_t> slot_flags;       // bit0 node, bit1 Dirichlet, bit3 refinement edge, bit4 home level of a leaf DoF
  std::vector<int32_t> slot_leaf;        // leaf storage slot at the same position (-1 holes)
  // prolongation P (this level <- level-1) as CSR over this level's slots
  std::vector<int32_t> P_ptr, P_col;
  std::vector<double> P_val;
  // restriction P^T (level-1 <- this level) as CSR over level-1 slots
  std::vector<int32_t> R_ptr, R_col;
  std::vector<double> R_val;
  // leaf nodes whose coarsest level is this one: (leaf slot, level slot)
  std::vector<int32_t> copy_leaf, copy_level;
  int64_t n_cells = 0;
  // per-cell values (modulus E_K, mean of the four children on refined cells):
  // for every cell of this level, its cell slot in this layout, its source (leaf
  // index >= 0, else -1 - q with children cell_child[4q..4q+3], cell slots of
  // level l+1 in the order (2i,2j), (2i,2j+1), (2i+1,2j), (2i+1,2j+1)); sorted by slot
  std::vector<int32_t> cell_dst, cell_src, cell_child;
};

struct Mesh {
  Tree tree;
  bool finalized = false;
  int k = 1;
  int Lf = 0;
  int64_t Xmax = 0, Ymax = 0;
  // leaf cells, canonical order
  std::vector<std::array<int64_t, 3>> leaves;
  // nodes in sorted key order
  std::vector<uint64_t> nkey;
  std::vector<int32_t> nX, nY;
  std::vector<int8_t> nminlev, nmaxlev;
  std::vector<int32_t> nhang;  // hanging-table index or -1
  std::vector<uint8_t> nparent;
  std::vector<int32_t> nslot;  // home storage slot
  // leaf layout
  Layout lay;
  std::vector<int32_t> slot_node;   // node index or -1 (hole)
  std::vector<uint8_t> slot_flags;  // bit0 node, bit1 Dirichlet, bit2 hanging, bit4 pure
  std::vector<HangingEntry> hang;
  int64_t n_partials = 0;
  std::vector<int32_t> fix_slot;    // storage slot of every non-pure node (incl. hanging)
  std::vector<int32_t> fix_ptr, fix_part;
  std::vector<double> fix_w;
  // per leaf cell (canonical order): its cell slot, the leaf-layout slot of the
  // cell's lower-left node position in the brick of the cell's own level; each
  // leaf cell has its own (the lower-left node of a level-l leaf cell lies in a
  // level-l brick).  Per-cell data (modulus E_K, its gradient) use these slots.
  std::vector<int32_t> cell_slot;
  std::vector<LevelMesh> levels;

  int64_t n_nodes() const { return int64_t(nkey.size()); }
  uint64_t key(int64_t X, int64_t Y) const { return uint64_t(Y) * uint64_t(Xmax + 1) + uint64_t(X); }
  int64_t find_node(int64_t X, int64_t Y) const;
  double hmin_diag() const;
};

// Builds leaves, nodes, hanging constraints, the leaf layout and all level meshes.
// Returns an empty string on success, else an error message.
std::string finalize_mesh(Mesh& m, int k);

}  // namespace pff
