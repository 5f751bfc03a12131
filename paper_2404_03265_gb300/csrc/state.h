// Library-owned device state behind the opaque handles of include/pff.h.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "mesh.h"
#include "mg.cuh"

namespace pff {

// Owns a list of cudaMalloc'ed blocks.
struct DevAllocs {
  std::vector<void*> ptrs;
  std::string err;
  template <typename T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      if (err.empty()) err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (p && !v.empty()) {
      const cudaError_t e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
      if (e != cudaSuccess && err.empty()) err = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
    }
    return p;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

struct DevMesh {
  DevAllocs mem;
  bool uploaded = false;
  int device = -1;
  DevLayout leaf;
  DevHanging* hang = nullptr;
  int32_t nhang = 0;
  int32_t nfix = 0;
  int32_t* fix_slot = nullptr;
  int32_t* fix_ptr = nullptr;
  int32_t* fix_part = nullptr;
  double* fix_w = nullptr;
  uint8_t* slot_flags = nullptr;
  // multigrid level meshes
  struct Level {
    DevLayout lay;
    DevLevel lv;
    int32_t* gx = nullptr;   // level-grid coordinates (units h_l / k), -1 for holes
    int32_t* gy = nullptr;
  };
  std::vector<Level> levels;
  int64_t lev_total = 0;     // sum of level slot counts
  void release() {
    mem.release();
    levels.clear();
    uploaded = false;
  }
};

}  // namespace pff

struct pff_mesh {
  pff::Mesh m;
  pff::DevMesh dev;
};

struct pff_problem {
  pff_mesh* mesh = nullptr;
  pff_params prm{};
  pff::DevAllocs bufs;
  double* lin64 = nullptr;   // 4 per slot
  float* lin32 = nullptr;
  uint8_t* cmask = nullptr;  // leaf constraint mask: bit0/1 Dirichlet u, bit2 active phi
  double* ibuf64 = nullptr;  // 3 per partial slot
  float* ibuf32 = nullptr;
  bool has_state = false;
};

namespace pff {

struct MGBlock {
  int ncomp = 1;
  int fixbits = 4;                 // constraint-mask bits of the block (3: u_x, u_y; 4: phi)
  double* dinv64 = nullptr;        // ncomp * lev_total
  float* dinv32 = nullptr;
  void* d = nullptr;               // level vectors (T), ncomp * lev_total each
  void* x = nullptr;
  void* r = nullptr;
  void* y = nullptr;
  void* yp = nullptr;
  void* t = nullptr;
  std::vector<double> lam;         // lambda_max estimate per level (level 0 unused)
  int32_t n_coarse = 0;
  int32_t* coarse_idx = nullptr;   // level-0 entries (comp * n_0 + slot) of the coarse interior
  double* coarse_inv = nullptr;    // dense FP64 inverse, n_coarse^2
  double* coarse_tmp = nullptr;
};

}  // namespace pff

struct pff_mg {
  pff_problem* pb = nullptr;
  int precision = PFF_F32;         // arithmetic of the V-cycle
  int degree = 3;                  // Chebyshev degree
  int lanczos_steps = 12;
  double lo = 0.08, hi = 1.2;      // smoothing range [lo, hi] * lambda_max
  pff::DevAllocs mem;
  double* lin64 = nullptr;         // 4 * lev_total (level linearisation)
  float* lin32 = nullptr;
  uint8_t* cmask = nullptr;        // lev_total
  pff::MGBlock blk[2];             // 0: u-u block, 1: phi-phi block
  // FP64 scratch for the eigenvalue estimate and set-up
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *diag = nullptr;
  double *partial = nullptr, *sc = nullptr, *hist = nullptr;
  bool ready = false;
};

namespace pff {

std::string upload_mesh(pff_mesh& m);
std::string alloc_problem(pff_problem& pb);
void fill_material(const pff_params& prm, ApplyArgs& a);
cudaError_t leaf_apply(pff_problem& pb, int precision, int op, const void* xu, const void* xp, void* yu,
                       void* yp, cudaStream_t s);
cudaError_t launch_leaf_cmask(int64_t n, const uint8_t* slot_flags, const uint8_t* active, uint8_t* cmask,
                              cudaStream_t s);
// multigrid (mg_host.cpp)
std::string mg_alloc(pff_mg& mg);
std::string mg_setup(pff_mg& mg, cudaStream_t s);
cudaError_t mg_vcycle(pff_mg& mg, int block, const double* r, double* z, cudaStream_t s);
// level operator y = A_l x of one block (op OP_UU / OP_PP / *_DIAG), precision of T
template <typename T>
cudaError_t level_apply(pff_mg& mg, int level, int op, const T* x, T* y, cudaStream_t s);

}  // namespace pff
