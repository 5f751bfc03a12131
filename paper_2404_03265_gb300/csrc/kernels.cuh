// Device-side argument blocks and launch wrappers of libpff's CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "mesh.h"

namespace pff {

constexpr int kMaxLevels = 32;

// four doubles, 32-byte aligned (linearisation (u_x, u_y, phi, phi_tilde) per slot)
struct __align__(32) dbl4 {
  double x, y, z, w;
};

// Operator selector of the brick kernels.
enum OpKind : int {
  OP_FULL = 0,     // leaf Jacobian A'(U) (Sec. 3.1), 3 components, block lower triangular
  OP_FULL_T = 1,   // its transpose (VJP)
  OP_UU = 2,       // diagonal block uu of a level operator (Sec. 3.2)
  OP_PP = 3,       // diagonal block phi-phi of a level operator
  OP_UU_DIAG = 4,  // diagonal of the uu block (Chebyshev-Jacobi, Sec. 3.2)
  OP_PP_DIAG = 5,  // diagonal of the phi-phi block
  OP_RESID = 6,    // residual R = -A(U)(psi) at the state held in `lin` (Problem 2)
  OP_MASS = 7,     // integral of each basis function (lumped mass, phi component)
  OP_TCV = 8,      // (u . grad phi, psi) per basis function (summed: total crack volume)
  OP_TCV_GRAD = 9, // dJ/dU of J = TCV: (psi_u . grad phi) and (u . grad psi_phi) per basis function
  OP_VJP = 10,     // per cell: x . dR/dtheta for theta = E_K, p, G_c (R = -A, x taken through C)
  OP_PHIT_VJP = 11,// phi rows: (dA/dphi_tilde)^T x = (psi, 2 phi~ [(1-kappa) sigma(u):e(x_u) + p div x_u])
};

// mode bits
constexpr int MODE_MASK_INPUT = 1;   // fixed components of x read as 0
constexpr int MODE_IDENTITY = 2;     // fixed rows: y = x (else y = 0)

struct DevHanging {
  int32_t slot;
  int32_t parent[3];
  double weight[3];
};

struct DevLayout {
  const BrickDesc* bricks = nullptr;
  int32_t nbricks = 0;
  const int32_t* win = nullptr;
  const int32_t* own_part = nullptr;
  const uint8_t* own_act = nullptr;
  const int32_t* own = nullptr;      // both as one word: (own_part + 1) | own_act << 30
  // Q1 cell-loop work units (one warp each): brick << 8 | first owned row << 3 |
  // strip code (strip half-height 15, 5, 3, 1 for codes 0..3); four schedules
  // one after the other (by mesh size; all 15; all 5; all 1), schedule p in
  // units[unit_off[p] .. unit_off[p + 1])
  const int32_t* units = nullptr;
  int32_t unit_off[5] = {0, 0, 0, 0, 0};
  const uint32_t* cellmask = nullptr;
};

// Material constants of the cell kernels (level independent), precomputed on
// the host in the kernel's precision (no double arithmetic in FP32 kernels).
template <typename T>
struct MatConst {
  T c2ml, cl, cm;      // 2 mu + lambda, lambda, mu
  T omk, kap, p, p2;   // 1 - kappa, kappa, p, 2 p
  T gcl, gcL;          // G_c / l, G_c l
  T il, l;             // 1 / l, l
};

// Geometry of a Cartesian hx x hy cell of one refinement level.
template <typename T>
struct LevGeom {
  T ihx, ihy;          // 1/hx, 1/hy
  T jxw;               // hx hy / 4: 2x2 Gauss weight times cell area
  T wx, wy;            // JxW / hx, JxW / hy
  T wpx, wpy;          // 2 G_c l JxW / hx^2, 2 G_c l JxW / hy^2
};

// Q2 tables: 1D Lagrange basis on the nodes 0, 1/2, 1 of [0, 1] at the 3-point
// Gauss points, its derivative, and the Gauss weights (precision of the kernel).
template <typename T>
struct Q2Tab {
  T L[3][3];   // L[a][q] = l_a(g_q)
  T D[3][3];   // D[a][q] = l_a'(g_q)
  T w[3];
};

// Chebyshev step fused into the store of a level apply (OP_UU, OP_PP): instead
// of y = A x the sweep writes, per level entry i (component blocks of n_slots):
//   CHEB_STEP       out[i]  = x + a (x - prev) + b dinv (rhs - A x)
//   CHEB_STEP_ADD   out[i] += the same value
//   CHEB_FIRST_RES  r[i] = rhs - A x, out[i] = c0 dinv r[i] (c0 in a), xprev[i] = 0
// with x the apply's input.  No output may alias the input, prev, dinv or rhs.
enum ChebMode : int { CHEB_OFF = 0, CHEB_STEP = 1, CHEB_STEP_ADD = 2, CHEB_FIRST_RES = 3 };
struct ChebEpi {
  int mode;
  const void* prev;
  const void* dinv;
  const void* rhs;
  void* out;
  void* r;
  void* xprev;
  float af, bf;      // a (or c0) and b in the kernel's precision
  double ad, bd;
};

struct ApplyArgs {
  DevLayout lay;
  const DevHanging* hang;
  const uint8_t* cmask;   // per slot: bit0/bit1 u_x/u_y fixed, bit2 phi fixed
  const void* lin;        // 4 blocks of n_slots T: u_x, u_y, phi, phi_tilde (hanging entries resolved)
  const void* xu;         // 2 blocks of n_slots T: u_x, u_y
  const void* xp;         // n_slots T
  void* yu;
  void* yp;
  void* ibuf;             // 3 T per partial slot
  const void* hlin;       // Q1 leaf: 4 blocks of nhang T, the hanging nodes' linearisation
  void* hang_x;           // Q1 leaf: 3 blocks of nhang T, scratch for the hanging nodes' input (C x)
  int32_t nhang;
  const void* ecell;      // per-cell modulus E_K (T, cell-slot layout) or nullptr: constants carry E
  void* cell_out;         // OP_VJP: 3 blocks of n_slots T (E_K, p, G_c) at cell slots
  int64_t n_slots;
  double hx[kMaxLevels], hy[kMaxLevels];
  double mu, lam;         // Lame constants (E applied, or unit E when ecell is set)
  double ell;             // length scale l
  double kappa, p, gc_over_l, gc_times_l;
  MatConst<float> mf;
  MatConst<double> md;
  LevGeom<float> gf[kMaxLevels];
  LevGeom<double> gd[kMaxLevels];
  Q2Tab<float> q2f;
  Q2Tab<double> q2d;
  int mode;
  int fe_degree;
  int sweep_sh;           // Q1 strip half-height: 0 = by mesh size, else 15, 5 or 1 (schedules of DevLayout::units)
  int pdl_in;             // Q1: launched dependent on the preceding kernel, which wrote x (pdl.cuh)
  ChebEpi ch;             // level applies: fused Chebyshev store (mode CHEB_OFF: plain y = A x)
};

struct FixupArgs {
  int32_t n;
  int64_t n_slots;
  const int32_t* slot;
  const int32_t* ptr;
  const int32_t* part;
  const double* w;
  const uint8_t* cmask;
  const void* xu;
  const void* xp;
  void* yu;
  void* yp;
  const void* ibuf;
  int mode;
};

// fills mf / md / gf / gd from hx, hy and the material
void fill_cell_constants(ApplyArgs& a, int nlevels);

// streaming multiprocessors of the current device (cached)
int sm_count();
// work units of the Q1 cell loop for a layout's bricks (see DevLayout::units)
std::vector<int32_t> sweep_units(const std::vector<BrickDesc>& bricks, int32_t unit_off[5]);

// launchers (return cudaError_t of the launch).  launch_fixup must follow the
// launch_apply whose partial sums it condenses directly on the same stream: it
// is launched programmatically dependent on it.
template <typename T>
cudaError_t launch_apply(const ApplyArgs& a, int op, cudaStream_t s);
template <typename T>
cudaError_t launch_fixup(const FixupArgs& a, cudaStream_t s);

// state conversion: lin64/lin32 blocks (u_x, u_y, phi, phi_t), hanging entries from parents;
// u is the displacement in block layout (u_x block, u_y block)
// hlin64/hlin32: the hanging nodes' linearisation again, 4 blocks of nhang (read by the Q1 sweep)
cudaError_t launch_set_lin(int64_t n_slots, const double* u, const double* phi, const double* phit,
                           const DevHanging* hang, int32_t nhang, int fe_degree,
                           double* lin64, float* lin32, double* hlin64, float* hlin32, cudaStream_t s);

}  // namespace pff
