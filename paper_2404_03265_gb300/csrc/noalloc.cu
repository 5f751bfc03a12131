// pff_apply_noalloc: the leaf operator of pff_apply with its interface scratch
// taken from a fixed device array of this file instead of the problem's buffers.
//
// One apply writes one partial sum (3 values) per interface node of an irregular
// brick, and the fix-up kernel that follows it in the same stream condenses them
// (C^T).  pff_apply keeps those partials in buffers made by pff_problem_create.
// This variant keeps them in `g_partials` below, a static device array that is
// part of the library image and is reserved when the CUDA module is loaded.  No
// call here allocates device or pinned memory, directly or through a library.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it per device.
// That first call must be made outside any stream capture.
//
// The array is shared by every problem and every stream on the device, and it
// keeps the previous call's contents.  Nothing in it needs to start at zero:
// the apply kernel writes every partial that the fix-up reads (each interface
// node of an irregular brick is written once per call) before the fix-up runs.
// Calls whose executions overlap on one device (different streams, no ordering
// between them) race on the array; order them on one stream or with events.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "state.h"

namespace {

// 65536 partial sums x 3 components x 8 bytes = 1.5 MiB.  FP32 calls use the
// same array as floats (the first half).
constexpr int64_t kMaxPartials = PFF_NOALLOC_MAX_PARTIALS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[3 * kMaxPartials];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_partials on the current device (set-up on first use).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

pff_status noalloc_fail(pff_status st, const std::string& msg) {
  pff::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" pff_status pff_apply_noalloc(pff_problem* pb, int32_t precision, int32_t op, const void* xu,
                                        const void* xp, void* yu, void* yp, void* stream) {
  using namespace pff;
  try {
    if (!pb || !xu || !xp || !yu || !yp) return noalloc_fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (precision != PFF_F64 && precision != PFF_F32) return noalloc_fail(PFF_ERR_INVALID_ARG, "bad precision");
    if (op < 0 || op > 2) return noalloc_fail(PFF_ERR_INVALID_ARG, "bad operator");
    const Mesh& M = pb->mesh->m;
    const DevMesh& D = pb->mesh->dev;
    if (M.n_partials > kMaxPartials)
      return noalloc_fail(PFF_ERR_INVALID_ARG,
                          "pff_apply_noalloc: the mesh has " + std::to_string(M.n_partials) +
                              " interface partial sums, more than the fixed scratch holds (" +
                              std::to_string(kMaxPartials) + "); use pff_apply");
    if (!pb->has_state) return noalloc_fail(PFF_ERR_STATE, "pff_set_state has not been called");
    if (xu == yu || xp == yp) return noalloc_fail(PFF_ERR_INVALID_ARG, "x and y overlap");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(PFF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(PFF_ERR_INVALID_ARG, "device ordinal out of range");
    if (D.device != dev) return noalloc_fail(PFF_ERR_INVALID_ARG, "the problem lives on another device");
    void* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess)
      return noalloc_fail(PFF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    ApplyArgs a;
    std::memset(&a, 0, sizeof(a));
    a.lay = D.leaf;
    a.hang = D.hang;
    a.cmask = pb->cmask;
    a.lin = precision == PFF_F64 ? static_cast<const void*>(pb->lin64) : static_cast<const void*>(pb->lin32);
    a.xu = xu; a.xp = xp; a.yu = yu; a.yp = yp;
    a.ibuf = scratch;
    a.n_slots = M.lay.n_slots;
    for (int l = 0; l <= M.Lf && l < kMaxLevels; ++l) {
      a.hx[l] = M.tree.hx(l);
      a.hy[l] = M.tree.hy(l);
    }
    leaf_modulus(*pb, precision, a);
    fill_cell_constants(a, M.Lf + 1);
    a.fe_degree = M.k;
    const int kop = op == PFF_OP_TRANSPOSE ? OP_FULL_T : OP_FULL;
    a.mode = op == PFF_OP_CONDENSED ? 0 : (MODE_MASK_INPUT | MODE_IDENTITY);
    FixupArgs f;
    f.n = D.nfix; f.n_slots = M.lay.n_slots; f.slot = D.fix_slot; f.ptr = D.fix_ptr; f.part = D.fix_part;
    f.w = D.fix_w; f.cmask = pb->cmask; f.xu = xu; f.xp = xp; f.yu = yu; f.yp = yp; f.ibuf = scratch;
    f.mode = a.mode;
    const cudaStream_t s = cudaStream_t(stream);
    if (precision == PFF_F64) {
      e = launch_apply<double>(a, kop, s);
      if (e == cudaSuccess) e = launch_fixup<double>(f, s);
    } else {
      e = launch_apply<float>(a, kop, s);
      if (e == cudaSuccess) e = launch_fixup<float>(f, s);
    }
    if (e != cudaSuccess) return noalloc_fail(PFF_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
    return PFF_OK;
  } catch (const std::bad_alloc&) {
    return noalloc_fail(PFF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& ex) {
    return noalloc_fail(PFF_ERR_INVALID_ARG, ex.what());
  }
}
