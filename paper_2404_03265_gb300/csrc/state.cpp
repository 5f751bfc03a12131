// Device uploads and operator dispatch behind the C-ABI.
#include "state.h"

#include <cstring>

namespace pff {

static DevLayout upload_layout(DevAllocs& mem, const Layout& L) {
  DevLayout d;
  d.bricks = mem.upload(L.bricks);
  d.nbricks = int32_t(L.bricks.size());
  d.win = mem.upload(L.win);
  d.own_part = mem.upload(L.own_part);
  d.own_act = mem.upload(L.own_act);
  std::vector<int32_t> own(L.own_part.size());
  for (size_t i = 0; i < own.size(); ++i)
    own[i] = int32_t(uint32_t(L.own_part[i] + 1) | (uint32_t(L.own_act[i]) << 30));
  d.own = mem.upload(own);
  const std::vector<int32_t> units = sweep_units(L.bricks, d.unit_off);
  d.units = mem.upload(units);
  d.cellmask = mem.upload(L.cellmask);
  return d;
}

std::string upload_mesh(pff_mesh& pm) {
  DevMesh& D = pm.dev;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return std::string("cudaGetDevice: ") + cudaGetErrorString(e);
  if (D.uploaded) {
    if (D.device != dev) return "mesh tables live on another device";
    return "";
  }
  const Mesh& M = pm.m;
  D.leaf = upload_layout(D.mem, M.lay);
  std::vector<DevHanging> hh(M.hang.size());
  for (size_t h = 0; h < M.hang.size(); ++h) {
    hh[h].slot = M.hang[h].slot;
    for (int b = 0; b < 3; ++b) {
      hh[h].parent[b] = M.hang[h].parent[b];
      hh[h].weight[b] = M.hang[h].weight[b];
    }
  }
  D.hang = D.mem.upload(hh);
  D.nhang = int32_t(hh.size());
  D.nfix = int32_t(M.fix_slot.size());
  D.fix_slot = D.mem.upload(M.fix_slot);
  D.fix_ptr = D.mem.upload(M.fix_ptr);
  D.fix_part = D.mem.upload(M.fix_part);
  D.fix_w = D.mem.upload(M.fix_w);
  D.slot_flags = D.mem.upload(M.slot_flags);
  D.n_leaf_cells = int32_t(M.cell_slot.size());
  D.cell_slot = D.mem.upload(M.cell_slot);
  D.levels.resize(M.levels.size());
  int64_t off = 0;
  for (size_t l = 0; l < M.levels.size(); ++l) {
    const LevelMesh& lm = M.levels[l];
    DevMesh::Level& L = D.levels[l];
    L.lay = upload_layout(D.mem, lm.lay);
    L.lv.n_slots = int32_t(lm.lay.n_slots);
    L.lv.off = off;
    off += lm.lay.n_slots;
    L.lv.flags = D.mem.upload(lm.slot_flags);
    L.lv.slot_leaf = D.mem.upload(lm.slot_leaf);
    std::vector<float> pv(lm.P_val.begin(), lm.P_val.end()), rv(lm.R_val.begin(), lm.R_val.end());
    if (l > 0) {
      L.lv.P_ptr = D.mem.upload(lm.P_ptr);
      L.lv.P_col = D.mem.upload(lm.P_col);
      L.lv.P_val = D.mem.upload(pv);
      L.lv.R_ptr = D.mem.upload(lm.R_ptr);
      L.lv.R_col = D.mem.upload(lm.R_col);
      L.lv.R_val = D.mem.upload(rv);
    }
    std::vector<int32_t> gx(lm.slot_X.size()), gy(lm.slot_Y.size());
    for (size_t q = 0; q < gx.size(); ++q) {
      gx[q] = lm.slot_X[q] < 0 ? -1 : (lm.slot_X[q] >> (M.Lf - int(l)));
      gy[q] = lm.slot_Y[q] < 0 ? -1 : (lm.slot_Y[q] >> (M.Lf - int(l)));
    }
    L.gx = D.mem.upload(gx);
    L.gy = D.mem.upload(gy);
    L.n_cells = int32_t(lm.cell_dst.size());
    L.cell_dst = D.mem.upload(lm.cell_dst);
    L.cell_src = D.mem.upload(lm.cell_src);
    L.cell_child = D.mem.upload(lm.cell_child);
  }
  D.lev_total = off;
  {
    // each free leaf node is on the copy list of exactly one level (its home)
    std::vector<int32_t> hoff(size_t(M.lay.n_slots), 0), hslot(size_t(M.lay.n_slots), -1),
        hnsl(size_t(M.lay.n_slots), 0);
    for (size_t l = 0; l < M.levels.size(); ++l) {
      const LevelMesh& lm = M.levels[l];
      for (size_t i = 0; i < lm.copy_leaf.size(); ++i) {
        const int32_t s = lm.copy_leaf[i];
        if (hslot[s] >= 0) {
          D.release();
          return "leaf slot on two copy lists";
        }
        hoff[s] = int32_t(D.levels[l].lv.off);
        hslot[s] = lm.copy_level[i];
        hnsl[s] = D.levels[l].lv.n_slots;
      }
    }
    D.home.off = D.mem.upload(hoff);
    D.home.slot = D.mem.upload(hslot);
    D.home.nsl = D.mem.upload(hnsl);
  }
  if (!D.mem.err.empty()) {
    std::string err = D.mem.err;
    D.release();
    return err;
  }
  D.uploaded = true;
  D.device = dev;
  return "";
}

std::string alloc_problem(pff_problem& pb) {
  const Mesh& M = pb.mesh->m;
  const int64_t ns = M.lay.n_slots;
  pb.lin64 = pb.bufs.alloc<double>(4 * ns);
  pb.lin32 = pb.bufs.alloc<float>(4 * ns);
  pb.cmask = pb.bufs.alloc<uint8_t>(ns);
  pb.cmask_dir = pb.bufs.alloc<uint8_t>(ns);
  pb.ibuf64 = pb.bufs.alloc<double>(3 * M.n_partials);
  pb.ibuf32 = pb.bufs.alloc<float>(3 * M.n_partials);
  const int64_t nh = int64_t(M.hang.size());
  pb.hlin64 = pb.bufs.alloc<double>(4 * nh);
  pb.hlin32 = pb.bufs.alloc<float>(4 * nh);
  pb.hx64 = pb.bufs.alloc<double>(3 * nh);
  pb.hx32 = pb.bufs.alloc<float>(3 * nh);
  if (!pb.bufs.err.empty()) {
    std::string err = pb.bufs.err;
    pb.bufs.release();
    return err;
  }
  cudaMemset(pb.lin64, 0, 4 * ns * sizeof(double));
  cudaMemset(pb.lin32, 0, 4 * ns * sizeof(float));
  cudaError_t e = launch_leaf_cmask(ns, pb.mesh->dev.slot_flags, nullptr, pb.cmask, 0);
  if (e == cudaSuccess) e = launch_leaf_cmask(ns, pb.mesh->dev.slot_flags, nullptr, pb.cmask_dir, 0);
  if (e != cudaSuccess) return std::string("cmask: ") + cudaGetErrorString(e);
  cudaError_t e2 = cudaDeviceSynchronize();
  if (e2 != cudaSuccess) return std::string("sync: ") + cudaGetErrorString(e2);
  return "";
}

void fill_material(const pff_params& prm, ApplyArgs& a, bool unit_E) {
  const double E = unit_E ? 1.0 : prm.E;
  a.mu = E / (2.0 * (1.0 + prm.nu));
  a.lam = E * prm.nu / ((1.0 + prm.nu) * (1.0 - 2.0 * prm.nu));
  a.ell = prm.eps;
  a.kappa = prm.kappa;
  a.p = prm.p;
  a.gc_over_l = prm.Gc / prm.eps;
  a.gc_times_l = prm.Gc * prm.eps;
}

void leaf_modulus(const pff_problem& pb, int precision, ApplyArgs& a) {
  fill_material(pb.prm, a, pb.has_ecell);
  a.ecell = !pb.has_ecell ? nullptr
            : precision == PFF_F64 ? static_cast<const void*>(pb.ecell64) : static_cast<const void*>(pb.ecell32);
}

cudaError_t leaf_apply(pff_problem& pb, int precision, int op, const void* xu, const void* xp, void* yu,
                       void* yp, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  ApplyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lay = D.leaf;
  a.hang = D.hang;
  a.cmask = pb.cmask;
  a.lin = precision == PFF_F64 ? static_cast<const void*>(pb.lin64) : static_cast<const void*>(pb.lin32);
  a.xu = xu; a.xp = xp; a.yu = yu; a.yp = yp;
  a.ibuf = precision == PFF_F64 ? static_cast<void*>(pb.ibuf64) : static_cast<void*>(pb.ibuf32);
  a.hlin = precision == PFF_F64 ? static_cast<const void*>(pb.hlin64) : static_cast<const void*>(pb.hlin32);
  a.hang_x = precision == PFF_F64 ? static_cast<void*>(pb.hx64) : static_cast<void*>(pb.hx32);
  a.nhang = D.nhang;
  a.n_slots = M.lay.n_slots;
  for (int l = 0; l <= M.Lf && l < kMaxLevels; ++l) {
    a.hx[l] = M.tree.hx(l);
    a.hy[l] = M.tree.hy(l);
  }
  leaf_modulus(pb, precision, a);
  fill_cell_constants(a, M.Lf + 1);
  a.fe_degree = M.k;
  a.sweep_sh = pb.sweep_sh;
  int kop = OP_FULL;
  if (op == PFF_OP_JACOBIAN) { kop = OP_FULL; a.mode = MODE_MASK_INPUT | MODE_IDENTITY; }
  else if (op == PFF_OP_TRANSPOSE) { kop = OP_FULL_T; a.mode = MODE_MASK_INPUT | MODE_IDENTITY; }
  else { kop = OP_FULL; a.mode = 0; }
  FixupArgs f;
  f.n = D.nfix; f.n_slots = M.lay.n_slots; f.slot = D.fix_slot; f.ptr = D.fix_ptr; f.part = D.fix_part; f.w = D.fix_w;
  f.cmask = pb.cmask; f.xu = xu; f.xp = xp; f.yu = yu; f.yp = yp; f.ibuf = a.ibuf; f.mode = a.mode;
  cudaError_t e;
  if (precision == PFF_F64) {
    e = launch_apply<double>(a, kop, s);
    if (e == cudaSuccess) e = launch_fixup<double>(f, s);
  } else {
    e = launch_apply<float>(a, kop, s);
    if (e == cudaSuccess) e = launch_fixup<float>(f, s);
  }
  return e;
}

}  // namespace pff
