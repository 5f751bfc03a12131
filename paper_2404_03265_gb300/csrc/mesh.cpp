// Host-side quadtree and layout construction for libpff (see mesh.h).
#include "mesh.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <tuple>

namespace pff {

void Tree::split(int l, int64_t i, int64_t j) {
  while (int(lev.size()) <= l + 1) lev.emplace_back();
  auto& s = lev[l + 1];
  s.insert(cell_key(2 * i, 2 * j));
  s.insert(cell_key(2 * i + 1, 2 * j));
  s.insert(cell_key(2 * i, 2 * j + 1));
  s.insert(cell_key(2 * i + 1, 2 * j + 1));
}

int Tree::finest() const {
  int L = int(lev.size()) - 1;
  while (L > 0 && lev[L].empty()) --L;
  return L;
}

// 2:1 face balance: the face neighbour of a level-m cell must exist at level m-1.
// Levels are visited fine to coarse; a missing cell is created by splitting its
// leaf ancestor down to the needed level (only coarser levels gain cells).
void Tree::balance() {
  for (int m = int(lev.size()) - 1; m >= 2; --m) {
    std::vector<uint64_t> cells(lev[m].begin(), lev[m].end());
    const int64_t nxm = nx(m), nym = ny(m);
    for (uint64_t c : cells) {
      const int64_t i = int64_t(c >> 32), j = int64_t(c & 0xffffffffu);
      const int64_t nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
      for (const auto& q : nb) {
        if (q[0] < 0 || q[1] < 0 || q[0] >= nxm || q[1] >= nym) continue;
        int64_t pl = m - 1, pi = q[0] >> 1, pj = q[1] >> 1;
        if (has(pl, pi, pj)) continue;
        std::vector<std::array<int64_t, 3>> chain;
        while (!has(pl, pi, pj)) {
          chain.push_back({pl, pi, pj});
          pl -= 1; pi >>= 1; pj >>= 1;
        }
        for (auto it = chain.rbegin(); it != chain.rend(); ++it)
          split(int((*it)[0]) - 1, (*it)[1] >> 1, (*it)[2] >> 1);
      }
    }
  }
}

std::vector<std::array<int64_t, 3>> Tree::leaves() const {
  std::vector<std::array<int64_t, 3>> out;
  for (int l = 0; l < int(lev.size()); ++l)
    for (uint64_t c : lev[l]) {
      const int64_t i = int64_t(c >> 32), j = int64_t(c & 0xffffffffu);
      if (!has(l + 1, 2 * i, 2 * j)) out.push_back({l, i, j});
    }
  std::sort(out.begin(), out.end(), [](const auto& a, const auto& b) {
    return std::make_tuple(a[0], a[2], a[1]) < std::make_tuple(b[0], b[2], b[1]);
  });
  return out;
}

int64_t Mesh::find_node(int64_t X, int64_t Y) const {
  if (X < 0 || Y < 0 || X > Xmax || Y > Ymax) return -1;
  const uint64_t kk = key(X, Y);
  auto it = std::lower_bound(nkey.begin(), nkey.end(), kk);
  if (it == nkey.end() || *it != kk) return -1;
  return int64_t(it - nkey.begin());
}

double Mesh::hmin_diag() const { return std::hypot(tree.hx(Lf), tree.hy(Lf)); }

// Equispaced 1D Lagrange polynomial b of degree k at t (product formula).
static double lagrange(int k, int b, double t) {
  double v = 1.0;
  for (int c = 0; c <= k; ++c)
    if (c != b) v *= (t - double(c) / k) / (double(b) / k - double(c) / k);
  return v;
}

namespace {

struct BrickIndex {
  std::unordered_map<uint64_t, int32_t> id;  // cell_key(bx, by) -> brick id within the layout
  int32_t find(int64_t bx, int64_t by) const {
    if (bx < 0 || by < 0) return -1;
    auto it = id.find(cell_key(bx, by));
    return it == id.end() ? -1 : it->second;
  }
};

// Window cells c (node range [c*k, c*k+k]) that contain window node w >= 0 (1D);
// the caller clips to the window.
inline void cells_of_node(int w, int k, int& lo, int& hi) {
  lo = (w + k - 1) / k - 1;
  hi = w / k;
}

}  // namespace

std::string finalize_mesh(Mesh& m, int k) {
  if (k != 1 && k != 2) return "fe_degree must be 1 or 2";
  Tree& t = m.tree;
  m.k = k;
  m.Lf = t.finest();
  const int Lf = m.Lf;
  m.Xmax = int64_t(t.ncx) * k << Lf;
  m.Ymax = int64_t(t.ncy) * k << Lf;
  m.leaves = t.leaves();
  const int nb1 = k + 1;

  // ---- nodes: every (node, level) occurrence of the leaf cells
  struct Occ { uint64_t key; int32_t level; };
  std::vector<Occ> occ;
  occ.reserve(m.leaves.size() * nb1 * nb1);
  for (const auto& c : m.leaves) {
    const int64_t s = int64_t(1) << (Lf - c[0]);
    for (int b = 0; b <= k; ++b)
      for (int a = 0; a <= k; ++a)
        occ.push_back({m.key((c[1] * k + a) * s, (c[2] * k + b) * s), int32_t(c[0])});
  }
  std::sort(occ.begin(), occ.end(), [](const Occ& a, const Occ& b) {
    return a.key < b.key || (a.key == b.key && a.level < b.level);
  });
  m.nkey.clear(); m.nminlev.clear(); m.nmaxlev.clear();
  for (size_t q = 0; q < occ.size(); ++q) {
    if (q == 0 || occ[q].key != occ[q - 1].key) {
      m.nkey.push_back(occ[q].key);
      m.nminlev.push_back(int8_t(occ[q].level));
      m.nmaxlev.push_back(int8_t(occ[q].level));
    } else {
      m.nmaxlev.back() = int8_t(occ[q].level);
    }
  }
  const int64_t nn = m.n_nodes();
  if (nn >= (int64_t(1) << 30)) return "mesh too large";
  m.nX.resize(nn); m.nY.resize(nn);
  for (int64_t n = 0; n < nn; ++n) {
    m.nX[n] = int32_t(m.nkey[n] % uint64_t(m.Xmax + 1));
    m.nY[n] = int32_t(m.nkey[n] / uint64_t(m.Xmax + 1));
  }

  // ---- hanging nodes: strictly inside a leaf edge, between its own nodes
  double wh[2][3];
  for (int a = 0; a < k; ++a)
    for (int b = 0; b <= k; ++b) wh[a][b] = lagrange(k, b, (2.0 * a + 1.0) / (2.0 * k));
  m.nhang.assign(nn, -1);
  m.nparent.assign(nn, 0);
  struct HN { int64_t node; int64_t par[3]; double w[3]; };
  std::vector<HN> hn;
  for (const auto& c : m.leaves) {
    if (c[0] >= Lf) continue;
    const int64_t s = int64_t(1) << (Lf - c[0]);
    const int64_t X0 = c[1] * k * s, Y0 = c[2] * k * s, X1 = (c[1] + 1) * k * s, Y1 = (c[2] + 1) * k * s;
    for (int e = 0; e < 4; ++e)
      for (int a = 0; a < k; ++a) {
        const int64_t half = (2 * a + 1) * s / 2;
        int64_t hx, hy;
        int64_t px[3], py[3];
        for (int b = 0; b <= k; ++b) {
          const int64_t along = b * s;
          if (e == 0) { px[b] = X0 + along; py[b] = Y0; }
          else if (e == 1) { px[b] = X0 + along; py[b] = Y1; }
          else if (e == 2) { px[b] = X0; py[b] = Y0 + along; }
          else { px[b] = X1; py[b] = Y0 + along; }
        }
        if (e == 0) { hx = X0 + half; hy = Y0; }
        else if (e == 1) { hx = X0 + half; hy = Y1; }
        else if (e == 2) { hx = X0; hy = Y0 + half; }
        else { hx = X1; hy = Y0 + half; }
        const int64_t n = m.find_node(hx, hy);
        if (n < 0) continue;
        if (m.nhang[n] >= 0) return "hanging node found on two coarse edges";
        HN h{n, {-1, -1, -1}, {0, 0, 0}};
        for (int b = 0; b <= k; ++b) {
          h.par[b] = m.find_node(px[b], py[b]);
          if (h.par[b] < 0) return "missing parent of a hanging node";
          h.w[b] = wh[a][b];
        }
        m.nhang[n] = int32_t(hn.size());
        hn.push_back(h);
      }
  }
  for (const auto& h : hn)
    for (int b = 0; b <= k; ++b) {
      if (m.nhang[h.par[b]] >= 0) return "hanging-node chain (parent is hanging)";
      m.nparent[h.par[b]] = 1;
    }
  auto pure = [&](int64_t n) {
    return m.nhang[n] < 0 && !m.nparent[n] && m.nminlev[n] == m.nmaxlev[n];
  };

  // ---- leaf layout bricks
  Layout& L = m.lay;
  L.k = k;
  L.B = (k == 1) ? 30 : 15;
  L.NB = L.B * k;
  L.W = L.NB + k + 1;
  const int NB = L.NB, W = L.W, B = L.B, NB2 = NB * NB;
  std::vector<std::array<int64_t, 3>> bk;  // (level, by, bx)
  bk.reserve(occ.size() / 4 + 16);
  for (const auto& o : occ) {
    const int l = o.level;
    const int64_t X = int64_t(o.key % uint64_t(m.Xmax + 1)), Y = int64_t(o.key / uint64_t(m.Xmax + 1));
    bk.push_back({l, (Y >> (Lf - l)) / NB, (X >> (Lf - l)) / NB});
  }
  std::sort(bk.begin(), bk.end());
  bk.erase(std::unique(bk.begin(), bk.end()), bk.end());
  if (int64_t(bk.size()) * NB2 >= (int64_t(1) << 31)) return "leaf layout exceeds 2^31 slots";
  std::vector<BrickIndex> bidx(Lf + 1);
  L.bricks.resize(bk.size());
  for (size_t b = 0; b < bk.size(); ++b) {
    bidx[bk[b][0]].id[cell_key(bk[b][2], bk[b][1])] = int32_t(b);
    L.bricks[b].level = int32_t(bk[b][0]);
    L.bricks[b].bx = int32_t(bk[b][2]);
    L.bricks[b].by = int32_t(bk[b][1]);
  }
  L.n_slots = int64_t(bk.size()) * NB2;
  m.slot_node.assign(L.n_slots, -1);
  m.slot_flags.assign(L.n_slots, 0);
  m.nslot.assign(nn, -1);
  for (int64_t n = 0; n < nn; ++n) {
    const int l = m.nminlev[n];
    const int64_t gx = int64_t(m.nX[n]) >> (Lf - l), gy = int64_t(m.nY[n]) >> (Lf - l);
    const int32_t b = bidx[l].find(gx / NB, gy / NB);
    if (b < 0) return "home brick missing";
    const int64_t slot = int64_t(b) * NB2 + (gx % NB) + NB * (gy % NB);
    m.nslot[n] = int32_t(slot);
    m.slot_node[slot] = int32_t(n);
    uint8_t f = 1;
    if (m.nX[n] == 0 || m.nX[n] == m.Xmax || m.nY[n] == 0 || m.nY[n] == m.Ymax) f |= 2;
    if (m.nhang[n] >= 0) f |= 4;
    if (pure(n)) f |= 16;
    m.slot_flags[slot] = f;
  }
  m.hang.resize(hn.size());
  for (size_t h = 0; h < hn.size(); ++h) {
    m.hang[h].slot = m.nslot[hn[h].node];
    for (int b = 0; b < 3; ++b) {
      m.hang[h].parent[b] = (b <= k) ? m.nslot[hn[h].par[b]] : -1;
      m.hang[h].weight[b] = (b <= k) ? hn[h].w[b] : 0.0;
    }
  }

  // ---- brick classification and irregular tables
  struct Part { int64_t node; int32_t level; int32_t id; };
  std::vector<Part> parts;
  L.win.clear(); L.own_part.clear(); L.own_act.clear(); L.cellmask.clear();
  const int CM = L.cm_words();
  std::vector<int64_t> wnode(W * W);
  std::vector<uint8_t> cleaf((B + 1) * (B + 1));
  for (size_t b = 0; b < L.bricks.size(); ++b) {
    BrickDesc& d = L.bricks[b];
    const int l = d.level;
    const int64_t base = int64_t(b) * NB2;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int32_t nbid = bidx[l].find(d.bx + dx, d.by + dy);
        d.nbr_base[(dy + 1) * 3 + dx + 1] = nbid < 0 ? -1 : nbid * NB2;
      }
    bool regular = true;
    for (int cj = 0; cj <= B; ++cj)
      for (int ci = 0; ci <= B; ++ci) {
        const bool lf = t.is_leaf(l, int64_t(d.bx) * B - 1 + ci, int64_t(d.by) * B - 1 + cj);
        cleaf[ci + (B + 1) * cj] = lf;
        if (!lf) regular = false;
      }
    for (int wj = 0; wj < W; ++wj)
      for (int wi = 0; wi < W; ++wi) {
        const int64_t gx = int64_t(d.bx) * NB - k + wi, gy = int64_t(d.by) * NB - k + wj;
        int64_t n = -1;
        if (gx >= 0 && gy >= 0) n = m.find_node(gx << (Lf - l), gy << (Lf - l));
        wnode[wi + W * wj] = n;
        if (n < 0 || m.nminlev[n] != l || m.nhang[n] >= 0) regular = false;
      }
    for (int oj = 0; oj < NB && regular; ++oj)
      for (int oi = 0; oi < NB; ++oi) {
        const int64_t n = wnode[(oi + k) + W * (oj + k)];
        if (n < 0 || !pure(n)) { regular = false; break; }
      }
    if (regular) { d.irr = -1; continue; }
    d.irr = L.n_irregular();
    for (int s = 0; s < W * W; ++s) {
      const int64_t n = wnode[s];
      int32_t code = kAbsent;
      if (n >= 0) code = (m.nhang[n] >= 0) ? hanging_code(m.nhang[n]) : m.nslot[n];
      L.win.push_back(code);
    }
    for (int oj = 0; oj < NB; ++oj)
      for (int oi = 0; oi < NB; ++oi) {
        const int wx = oi + k, wy = oj + k;
        const int64_t n = wnode[wx + W * wy];
        int32_t p = -1;
        if (n >= 0 && !pure(n)) {
          int clo, chi, rlo, rhi;
          cells_of_node(wx, k, clo, chi);
          cells_of_node(wy, k, rlo, rhi);
          bool adj = false;
          for (int cj = rlo; cj <= rhi; ++cj)
            for (int ci = clo; ci <= chi; ++ci)
              if (ci >= 0 && ci <= B && cj >= 0 && cj <= B && cleaf[ci + (B + 1) * cj]) adj = true;
          if (adj) {
            p = int32_t(parts.size());
            parts.push_back({n, l, p});
          }
        }
        L.own_part.push_back(p);
        const int64_t slot = base + oi + NB * oj;
        const int32_t h = m.slot_node[slot];
        L.own_act.push_back(h < 0 ? kActZero : (pure(h) ? kActFinal : kActNone));
      }
    for (int w = 0; w < CM; ++w) {
      uint32_t bits = 0;
      for (int q = 0; q < 32; ++q) {
        const int c = w * 32 + q;
        if (c < (B + 1) * (B + 1) && cleaf[c]) bits |= (1u << q);
      }
      L.cellmask.push_back(bits);
    }
  }
  m.n_partials = int64_t(parts.size());

  // ---- fix-up lists: every non-pure node sums its partials and its hanging children's
  std::vector<std::vector<std::pair<int32_t, double>>> own_parts(nn);
  for (const auto& p : parts) own_parts[p.node].push_back({p.id, 1.0});
  std::vector<std::vector<std::pair<int64_t, double>>> children(nn);
  for (const auto& h : hn)
    for (int b = 0; b <= k; ++b) children[h.par[b]].push_back({h.node, h.w[b]});
  m.fix_slot.clear(); m.fix_ptr.assign(1, 0); m.fix_part.clear(); m.fix_w.clear();
  std::vector<int64_t> fixnodes;
  for (int64_t n = 0; n < nn; ++n)
    if (!pure(n)) fixnodes.push_back(n);
  std::sort(fixnodes.begin(), fixnodes.end(), [&](int64_t a, int64_t b) { return m.nslot[a] < m.nslot[b]; });
  for (int64_t n : fixnodes) {
    m.fix_slot.push_back(m.nslot[n]);
    if (m.nhang[n] < 0) {
      for (const auto& e : own_parts[n]) { m.fix_part.push_back(e.first); m.fix_w.push_back(e.second); }
      for (const auto& ch : children[n])
        for (const auto& e : own_parts[ch.first]) { m.fix_part.push_back(e.first); m.fix_w.push_back(ch.second); }
    }
    m.fix_ptr.push_back(int32_t(m.fix_part.size()));
  }

  // ---- level meshes (all cells of one level), multigrid with local smoothing
  m.levels.clear();
  m.levels.resize(Lf + 1);
  std::vector<BrickIndex> lbidx(Lf + 1);
  std::vector<std::unordered_map<uint64_t, int32_t>> lslot(Lf + 1);  // level-grid key -> slot
  for (int l = 0; l <= Lf; ++l) {
    LevelMesh& lm = m.levels[l];
    lm.level = l;
    Layout& Ll = lm.lay;
    Ll.k = k; Ll.B = B; Ll.NB = NB; Ll.W = W;
    const int64_t gnx = t.nx(l) * k, gny = t.ny(l) * k;  // level node grid max index
    auto gkey = [&](int64_t gx, int64_t gy) { return uint64_t(gy) * uint64_t(gnx + 1) + uint64_t(gx); };
    std::vector<uint64_t> lk;
    lk.reserve(t.lev[l].size() * nb1 * nb1);
    for (uint64_t c : t.lev[l]) {
      const int64_t i = int64_t(c >> 32), j = int64_t(c & 0xffffffffu);
      for (int b = 0; b <= k; ++b)
        for (int a = 0; a <= k; ++a) lk.push_back(gkey(i * k + a, j * k + b));
    }
    std::sort(lk.begin(), lk.end());
    lk.erase(std::unique(lk.begin(), lk.end()), lk.end());
    lm.n_nodes = int64_t(lk.size());
    lm.n_cells = int64_t(t.lev[l].size());
    std::vector<std::array<int64_t, 2>> lbk;
    for (uint64_t q : lk) lbk.push_back({int64_t(q / uint64_t(gnx + 1)) / NB, int64_t(q % uint64_t(gnx + 1)) / NB});
    std::sort(lbk.begin(), lbk.end());
    lbk.erase(std::unique(lbk.begin(), lbk.end()), lbk.end());
    Ll.bricks.resize(lbk.size());
    for (size_t b = 0; b < lbk.size(); ++b) {
      lbidx[l].id[cell_key(lbk[b][1], lbk[b][0])] = int32_t(b);
      Ll.bricks[b].level = l;
      Ll.bricks[b].bx = int32_t(lbk[b][1]);
      Ll.bricks[b].by = int32_t(lbk[b][0]);
    }
    Ll.n_slots = int64_t(lbk.size()) * NB2;
    lm.slot_X.assign(Ll.n_slots, -1);
    lm.slot_Y.assign(Ll.n_slots, -1);
    lm.slot_flags.assign(Ll.n_slots, 0);
    lm.slot_leaf.assign(Ll.n_slots, -1);
    for (uint64_t q : lk) {
      const int64_t gx = int64_t(q % uint64_t(gnx + 1)), gy = int64_t(q / uint64_t(gnx + 1));
      const int32_t b = lbidx[l].find(gx / NB, gy / NB);
      const int64_t slot = int64_t(b) * NB2 + gx % NB + NB * (gy % NB);
      lslot[l][q] = int32_t(slot);
      const int64_t X = gx << (Lf - l), Y = gy << (Lf - l);
      lm.slot_X[slot] = int32_t(X);
      lm.slot_Y[slot] = int32_t(Y);
      uint8_t f = 1;
      if (X == 0 || X == m.Xmax || Y == 0 || Y == m.Ymax) f |= 2;
      // refinement edge: a level-l cell whose closure holds the node is missing
      int clo, chi, rlo, rhi;
      clo = (gx % k == 0) ? gx / k - 1 : gx / k; chi = gx / k;
      rlo = (gy % k == 0) ? gy / k - 1 : gy / k; rhi = gy / k;
      for (int64_t cj = rlo; cj <= rhi; ++cj)
        for (int64_t ci = clo; ci <= chi; ++ci) {
          if (ci < 0 || cj < 0 || ci >= t.nx(l) || cj >= t.ny(l)) continue;
          if (!t.has(l, ci, cj)) f |= 8;
        }
      lm.slot_flags[slot] = f;
      const int64_t ln = m.find_node(X, Y);
      if (ln < 0) return "level node without a leaf node at its position";
      lm.slot_leaf[slot] = m.nslot[ln];
      if (m.nhang[ln] < 0 && m.nminlev[ln] == l) lm.slot_flags[slot] |= 16;  // home level of a leaf DoF
    }
    auto lfind = [&](int64_t gx, int64_t gy) -> int32_t {
      if (gx < 0 || gy < 0 || gx > gnx || gy > gny) return -1;
      auto it = lslot[l].find(gkey(gx, gy));
      return it == lslot[l].end() ? -1 : it->second;
    };
    // window classification
    for (size_t b = 0; b < Ll.bricks.size(); ++b) {
      BrickDesc& d = Ll.bricks[b];
      const int64_t base = int64_t(b) * NB2;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int32_t nbid = lbidx[l].find(d.bx + dx, d.by + dy);
          d.nbr_base[(dy + 1) * 3 + dx + 1] = nbid < 0 ? -1 : nbid * NB2;
        }
      bool regular = true;
      for (int cj = 0; cj <= B; ++cj)
        for (int ci = 0; ci <= B; ++ci) {
          const bool ex = t.has(l, int64_t(d.bx) * B - 1 + ci, int64_t(d.by) * B - 1 + cj);
          cleaf[ci + (B + 1) * cj] = ex;
          if (!ex) regular = false;
        }
      std::vector<int32_t> wsl(W * W);
      for (int wj = 0; wj < W; ++wj)
        for (int wi = 0; wi < W; ++wi) {
          const int32_t s = lfind(int64_t(d.bx) * NB - k + wi, int64_t(d.by) * NB - k + wj);
          wsl[wi + W * wj] = s;
          if (s < 0) regular = false;
        }
      if (regular) { d.irr = -1; continue; }
      d.irr = Ll.n_irregular();
      for (int s = 0; s < W * W; ++s) Ll.win.push_back(wsl[s]);
      for (int oj = 0; oj < NB; ++oj)
        for (int oi = 0; oi < NB; ++oi) {
          Ll.own_part.push_back(-1);
          Ll.own_act.push_back(lm.slot_X[base + oi + NB * oj] >= 0 ? kActFinal : kActZero);
        }
      for (int w = 0; w < CM; ++w) {
        uint32_t bits = 0;
        for (int q = 0; q < 32; ++q) {
          const int c = w * 32 + q;
          if (c < (B + 1) * (B + 1) && cleaf[c]) bits |= (1u << q);
        }
        Ll.cellmask.push_back(bits);
      }
    }
    // transfers from level l-1: nodal interpolation of the coarse Q_k field
    if (l >= 1) {
      const int64_t cnx = t.nx(l - 1), cny = t.ny(l - 1);
      auto& prev = m.levels[l - 1];
      std::vector<std::vector<std::pair<int32_t, double>>> rows(Ll.n_slots);
      std::vector<std::vector<std::pair<int32_t, double>>> cols(prev.lay.n_slots);
      for (uint64_t q : lk) {
        const int64_t gx = int64_t(q % uint64_t(gnx + 1)), gy = int64_t(q / uint64_t(gnx + 1));
        const int32_t fs = lslot[l][q];
        int64_t cx = gx / (2 * k), cy = gy / (2 * k);
        if (cx >= cnx) cx = cnx - 1;
        if (cy >= cny) cy = cny - 1;
        const double tx = double(gx - cx * 2 * k) / (2.0 * k), ty = double(gy - cy * 2 * k) / (2.0 * k);
        for (int b = 0; b <= k; ++b)
          for (int a = 0; a <= k; ++a) {
            const double w = lagrange(k, a, tx) * lagrange(k, b, ty);
            if (w == 0.0) continue;
            const int64_t ccx = cx * k + a, ccy = cy * k + b;
            const uint64_t ckk = uint64_t(ccy) * uint64_t(cnx * k + 1) + uint64_t(ccx);
            auto it = lslot[l - 1].find(ckk);
            if (it == lslot[l - 1].end()) return "prolongation parent missing";
            rows[fs].push_back({it->second, w});
            cols[it->second].push_back({fs, w});
          }
      }
      lm.P_ptr.assign(1, 0); lm.P_col.clear(); lm.P_val.clear();
      for (int64_t s = 0; s < Ll.n_slots; ++s) {
        for (auto& e : rows[s]) { lm.P_col.push_back(e.first); lm.P_val.push_back(e.second); }
        lm.P_ptr.push_back(int32_t(lm.P_col.size()));
      }
      lm.R_ptr.assign(1, 0); lm.R_col.clear(); lm.R_val.clear();
      for (int64_t s = 0; s < prev.lay.n_slots; ++s) {
        std::sort(cols[s].begin(), cols[s].end());
        for (auto& e : cols[s]) { lm.R_col.push_back(e.first); lm.R_val.push_back(e.second); }
        lm.R_ptr.push_back(int32_t(lm.R_col.size()));
      }
    }
  }
  // copy lists: leaf node -> the coarsest level among its leaf cells
  for (int64_t n = 0; n < nn; ++n) {
    if (m.nhang[n] >= 0) continue;
    const int l = m.nminlev[n];
    const int64_t gnx = t.nx(l) * k;
    const int64_t gx = int64_t(m.nX[n]) >> (Lf - l), gy = int64_t(m.nY[n]) >> (Lf - l);
    auto it = lslot[l].find(uint64_t(gy) * uint64_t(gnx + 1) + uint64_t(gx));
    if (it == lslot[l].end()) return "leaf node missing on its coarsest level";
    m.levels[l].copy_leaf.push_back(m.nslot[n]);
    m.levels[l].copy_level.push_back(it->second);
  }
  // cell slots: the slot of a cell's lower-left node position in a brick of its level
  auto cell_slot_in = [&](const std::vector<BrickIndex>& idx, int l, int64_t i, int64_t j) -> int32_t {
    const int64_t gx = i * k, gy = j * k;
    const int32_t b = idx[l].find(gx / NB, gy / NB);
    if (b < 0) return -1;
    return int32_t(int64_t(b) * NB2 + (gx % NB) + NB * (gy % NB));
  };
  std::vector<std::unordered_map<uint64_t, int32_t>> leaf_of(Lf + 1);
  m.cell_slot.resize(m.leaves.size());
  for (size_t c = 0; c < m.leaves.size(); ++c) {
    const auto& lc = m.leaves[c];
    const int32_t sl = cell_slot_in(bidx, int(lc[0]), lc[1], lc[2]);
    if (sl < 0) return "leaf cell without a brick of its level";
    m.cell_slot[c] = sl;
    leaf_of[lc[0]][cell_key(lc[1], lc[2])] = int32_t(c);
  }
  for (int l = 0; l <= Lf; ++l) {
    LevelMesh& lm = m.levels[l];
    std::vector<std::array<int32_t, 6>> rows;  // dst, src, 4 children
    rows.reserve(t.lev[l].size());
    for (uint64_t c : t.lev[l]) {
      const int64_t i = int64_t(c >> 32), j = int64_t(c & 0xffffffffu);
      std::array<int32_t, 6> r{cell_slot_in(lbidx, l, i, j), 0, -1, -1, -1, -1};
      if (r[0] < 0) return "level cell without a brick";
      auto it = leaf_of[l].find(cell_key(i, j));
      if (it != leaf_of[l].end()) {
        r[1] = it->second;
      } else {
        r[1] = -1;
        int q = 2;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            r[q] = cell_slot_in(lbidx, l + 1, 2 * i + a, 2 * j + b);
            if (r[q] < 0) return "child cell without a brick";
            ++q;
          }
      }
      rows.push_back(r);
    }
    std::sort(rows.begin(), rows.end());
    lm.cell_dst.clear(); lm.cell_src.clear(); lm.cell_child.clear();
    for (const auto& r : rows) {
      lm.cell_dst.push_back(r[0]);
      if (r[1] >= 0) {
        lm.cell_src.push_back(r[1]);
      } else {
        lm.cell_src.push_back(-1 - int32_t(lm.cell_child.size() / 4));
        for (int q = 2; q < 6; ++q) lm.cell_child.push_back(r[q]);
      }
    }
  }
  m.finalized = true;
  return "";
}

}  // namespace pff
