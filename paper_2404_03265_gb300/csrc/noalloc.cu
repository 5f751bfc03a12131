// pff_apply_noalloc: the leaf operator of pff_apply with its scratch taken from
// a fixed device array of this file instead of the problem's buffers.
//
// One apply of a Q1 mesh first writes the input resolved on each hanging node
// (C x, 3 values per hanging node) and then one partial sum (3 values) per
// interface node of an irregular brick; the fix-up kernel that follows in the
// same stream condenses the partials (C^T).  pff_apply keeps both in buffers
// made by pff_problem_create.  This variant keeps them in `g_partials` below, a
// static device array that is part of the library image: the partials first,
// the hanging inputs after them.  No call here allocates device or pinned
// memory, directly or through a library.
//
// Set-up: pff_problem_create calls noalloc_prepare, which loads this file's
// module on the problem's device and looks up the array's device address with
// cudaGetSymbolAddress (the module may otherwise be loaded lazily, at the first
// use of the array, which would reserve its memory inside the first call).  The
// address is cached per device; a call on a device that was never prepared
// looks it up itself, so make the first call there outside any stream capture.
// The cache does not survive cudaDeviceReset, which also invalidates every
// problem's device buffers.
//
// The array is shared by every problem and every stream on the device, and it
// keeps the previous call's contents.  Nothing in it needs to start at zero:
// every value that is read is written earlier in the same call (each hanging
// input by the first kernel, each partial by the apply kernel before the
// fix-up reads it).  Calls whose executions overlap on one device (different
// streams, no ordering between them) race on the array; order them on one
// stream or with events.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "state.h"

namespace {

// 65536 triples (partial sums and hanging inputs) x 8 bytes = 1.5 MiB.  FP32
// calls use the same array as floats (the first half).
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

}  // namespace

namespace pff {
// Loads the module and caches the array's address on the current device.
cudaError_t noalloc_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaSuccess;   // the call itself reports this
  void* p = nullptr;
  return scratch_address(dev, &p);
}
}  // namespace pff

namespace {

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
    const int64_t nh = M.k == 1 ? int64_t(M.hang.size()) : 0;   // hanging inputs (Q1 only)
    if (M.n_partials + nh > kMaxPartials)
      return noalloc_fail(PFF_ERR_INVALID_ARG,
                          "pff_apply_noalloc: the mesh has " + std::to_string(M.n_partials) +
                              " interface partial sums and " + std::to_string(nh) +
                              " hanging nodes, more triples than the fixed scratch holds (" +
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
    const size_t esz = precision == PFF_F64 ? sizeof(double) : sizeof(float);
    a.hang_x = static_cast<char*>(scratch) + 3 * M.n_partials * esz;
    a.hlin = precision == PFF_F64 ? static_cast<const void*>(pb->hlin64) : static_cast<const void*>(pb->hlin32);
    a.nhang = D.nhang;
    a.n_slots = M.lay.n_slots;
    for (int l = 0; l <= M.Lf && l < kMaxLevels; ++l) {
      a.hx[l] = M.tree.hx(l);
      a.hy[l] = M.tree.hy(l);
    }
    leaf_modulus(*pb, precision, a);
    fill_cell_constants(a, M.Lf + 1);
    a.fe_degree = M.k;
    a.sweep_sh = pb->sweep_sh;
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
