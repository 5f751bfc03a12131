// Library-owned device state behind the opaque handles of include/pff.h.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "mesh.h"

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
  void release() {
    mem.release();
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

std::string upload_mesh(pff_mesh& m);
std::string alloc_problem(pff_problem& pb);
void fill_material(const pff_params& prm, ApplyArgs& a);
cudaError_t leaf_apply(pff_problem& pb, int precision, int op, const void* xu, const void* xp, void* yu,
                       void* yp, cudaStream_t s);
cudaError_t launch_leaf_cmask(int64_t n, const uint8_t* slot_flags, const uint8_t* active, uint8_t* cmask,
                              cudaStream_t s);

}  // namespace pff
