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
  int32_t n_leaf_cells = 0;
  int32_t* cell_slot = nullptr;   // per leaf cell (canonical order): its cell slot
  // multigrid level meshes
  struct Level {
    DevLayout lay;
    DevLevel lv;
    int32_t* gx = nullptr;   // level-grid coordinates (units h_l / k), -1 for holes
    int32_t* gy = nullptr;
    int32_t n_cells = 0;     // cells of this level and their per-cell value sources
    int32_t* cell_dst = nullptr;
    int32_t* cell_src = nullptr;
    int32_t* cell_child = nullptr;
  };
  std::vector<Level> levels;
  int64_t lev_total = 0;     // sum of level slot counts
  DevHome home;              // per leaf slot: its home level (copy in and out of the V-cycle)
  void release() {
    mem.release();
    levels.clear();
    uploaded = false;
  }
};

// Work space of GMRES and the Newton loop (allocated on first use).
struct SolverWS {
  DevAllocs mem;
  bool ready = false;
  int restart = 0;
  double *V = nullptr, *w = nullptr, *tmp = nullptr, *rhs = nullptr, *R = nullptr, *res = nullptr;
  double* vc = nullptr;   // the newest basis vector in slot layout (zero off the node slots)
  // GMRES keeps its Krylov basis on the node rows only: row i of a basis vector is
  // entry map[i] of the slot-layout vector (3 blocks of n_slots), nc rows
  int32_t* map = nullptr;
  int64_t nc = 0;
  double* wc = nullptr;   // the Arnoldi vector on those rows
  double *dU = nullptr, *du0 = nullptr, *st = nullptr, *ut = nullptr, *B = nullptr;
  uint8_t *act = nullptr, *act_prev = nullptr;
  unsigned long long* stats = nullptr;
  double *partial = nullptr, *h = nullptr, *scal = nullptr;
  double* hh = nullptr;   // one Arnoldi step on the device: both Gram-Schmidt passes and |w|^2 (2 (restart + 1) + 1)
  int* bad = nullptr;
  float *x32 = nullptr, *y32 = nullptr;   // FP32 operator applies inside GMRES (3 blocks each)
};

struct GmresResult {
  int iterations = 0;
  bool converged = false;
  bool breakdown = false;
  double initial = 0.0, estimate = 0.0;
  double t_apply = 0.0, t_vcycle = 0.0, t_orth = 0.0;   // device seconds per phase of the iterations
};

struct NewtonOpts {
  double tol = 1e-8, atol = 1e-13, gmres_rtol = 1e-6, omega = 0.5;
  int restart = 50, gmres_maxiter = 500, max_newton = 100, ls_max = 10;
  int matvec = PFF_F64;   // precision of the Jacobian applies inside GMRES
  const double* phi_tilde = nullptr;   // linearised phase field of the u-equation (phi_old when null)
};

struct NewtonInfo {
  int newton = 0;
  bool converged = false, nonfinite = false, gmres_breakdown = false;
  int linesearch_failures = 0;
  double residual0 = 0.0, margin = 0.0;
  std::vector<double> residual;
  std::vector<int> gmres;
  std::vector<int64_t> active_size, changes;
  std::string error;
  double t_setup = 0.0, t_gmres = 0.0;   // host wall seconds in multigrid set-up and in GMRES
  double t_apply = 0.0, t_vcycle = 0.0, t_orth = 0.0;   // device seconds inside GMRES (GmresResult)
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
  uint8_t* cmask_dir = nullptr;  // Dirichlet bits only (residual evaluation)
  pff::SolverWS ws;
  double* ibuf64 = nullptr;  // 3 per partial slot
  float* ibuf32 = nullptr;
  double* hlin64 = nullptr;  // per hanging node: its resolved linearisation, 4 blocks of n_hang
  float* hlin32 = nullptr;
  double* hx64 = nullptr;    // per hanging node: the input resolved from its parents, 3 blocks of n_hang
  float* hx32 = nullptr;
  bool has_state = false;
  // per-cell modulus E_K (cell-slot layout; levels concatenated like level vectors)
  bool has_ecell = false;
  double* ecell64 = nullptr;      // n_slots
  float* ecell32 = nullptr;
  double* lev_ecell64 = nullptr;  // lev_total
  float* lev_ecell32 = nullptr;
  double* cell_out = nullptr;     // 3 * n_slots: per-cell VJP values
  double* adj_cell = nullptr;     // n_leaf_cells: per-step modulus gradient of the multi-step adjoint
  double* adj_phit = nullptr;     // n_slots: extrapolated phi_tilde of the step the multi-step adjoint is at
  double* adj_pend = nullptr;     // n_slots: phi share of step k's adjoint that reaches step k - 2
  cudaEvent_t gm_ev[4] = {};      // GMRES phase timing (created on first use)
  int sweep_sh = 0;               // Q1 cell-loop strip half-height (pff_set_cell_loop), 0 = by mesh size
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
  std::vector<double> lam;         // lambda_max estimate per level (level 0: only with the Chebyshev coarse solver)
  double c0_a = 0.0, c0_b = 0.0;   // Chebyshev coarse solver: interval [0.9 lambda_min, 1.2 lambda_max] on level 0
  int c0_deg = 0;                  // and its degree
  int32_t n_coarse = 0, coarse_cap = 0;
  int32_t* coarse_idx = nullptr;   // level-0 entries (comp * n_0 + slot) of the coarse interior
  double* coarse_inv = nullptr;    // dense FP64 inverse, n_coarse^2
  double* coarse_tmp = nullptr;
  double* coarse_rc = nullptr;     // scratch of the inversion: panel inverse, old pivot columns and rows
};

}  // namespace pff

struct pff_mg {
  pff_problem* pb = nullptr;
  int precision = PFF_F32;         // arithmetic of the V-cycle
  int degree = 3;                  // Chebyshev degree
  int lanczos_steps = 12;
  int coarse_mode = 0;             // 0: direct FP64 solve on level 0, 1: Chebyshev-Jacobi (Sec. 3.2)
  int fused = 1;                   // Chebyshev steps fused into the level applies' stores
  double lo = 0.08, hi = 1.2;      // smoothing range [lo, hi] * lambda_max
  pff::DevAllocs mem;
  double* lin64 = nullptr;         // 4 * lev_total (level linearisation)
  float* lin32 = nullptr;
  uint8_t* cmask = nullptr;        // lev_total
  pff::MGBlock blk[2];             // 0: u-u block, 1: phi-phi block
  // Set-up: the inverse diagonal and CG eigenvalue estimate of each (block, level)
  // form an independent chain; the chains run on a pool of streams.  FP64 scratch:
  // per block 5 level vectors (diag, r, z, p, q) of ncomp * lev_total, per chain
  // the dot partials, 8 CG scalars and 2 * 64 CG coefficients.
  static constexpr int kSetupStreams = 8;   // the extra stream inverts the second coarse block
  cudaStream_t su_stream[kSetupStreams + 1] = {};
  cudaEvent_t su_done[kSetupStreams + 1] = {};
  cudaEvent_t su_start = nullptr;
  // The chains' launches are captured once as a graph and replayed by later
  // set-ups on su_side while their arguments hold (su_key: the material, the
  // modulus buffers, the cell-loop schedule and the coarse mode they bake in).
  cudaGraphExec_t su_exec = nullptr;
  std::vector<unsigned char> su_key;
  cudaStream_t su_side = nullptr;
  cudaEvent_t su_chains = nullptr;
  int su_setups = 0;               // set-ups run so far (the first one launches directly)
  bool su_graph_ok = true;
  double* su_vec[2] = {nullptr, nullptr};
  double *su_partial = nullptr, *su_sc = nullptr, *su_hist = nullptr;
  // coarse probing: all colours of both blocks at once (in and out, probe_len doubles each)
  double *probe_in = nullptr, *probe_out = nullptr;
  int64_t probe_len = 0;
  bool ready = false;
  // V-cycles replayed as CUDA graphs (one per block, captured after each set-up;
  // inputs and outputs pass through fixed staging vectors of 3 * n_slots doubles)
  bool graphs_ok = true;
  cudaGraphExec_t vc_exec[2] = {nullptr, nullptr};
  // both blocks in one graph: the phi block runs on a forked branch beside the u block
  cudaGraphExec_t vc_both = nullptr;
  cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double *vc_in = nullptr, *vc_out = nullptr;
  int32_t* spd_bad = nullptr;      // per block: set by the coarse inversion when a pivot is not positive
};

namespace pff {

std::string upload_mesh(pff_mesh& m);
std::string alloc_problem(pff_problem& pb);
// message returned by pff_last_error on this thread
void set_last_error(const std::string& msg);
// material constants; unit_E: elastic constants of E = 1 (a per-cell modulus is applied in the kernel)
void fill_material(const pff_params& prm, ApplyArgs& a, bool unit_E = false);
// modulus source of a leaf operator: unit-E constants + the cell array when a modulus field is set
// pff_apply_noalloc's fixed scratch: loads its module and caches its address on
// the current device (noalloc.cu).
cudaError_t noalloc_prepare();
void leaf_modulus(const pff_problem& pb, int precision, ApplyArgs& a);
cudaError_t leaf_apply(pff_problem& pb, int precision, int op, const void* xu, const void* xp, void* yu,
                       void* yp, cudaStream_t s);
cudaError_t launch_leaf_cmask(int64_t n, const uint8_t* slot_flags, const uint8_t* active, uint8_t* cmask,
                              cudaStream_t s);
// solvers (solver.cpp)
cudaError_t leaf_op(pff_problem& pb, int kop, int mode, const double* lin, const uint8_t* cmask, const double* xu,
                    const double* xp, double* yu, double* yp, cudaStream_t s);
std::string ensure_workspace(pff_problem& pb, int restart);
cudaError_t gmres_solve(pff_problem& pb, pff_mg& mg, int transpose, const double* b, double* x, double rtol,
                        int restart, int maxiter, GmresResult& res, cudaStream_t s, int matvec = PFF_F64);
cudaError_t leaf_residual(pff_problem& pb, const double* u, const double* phi, const double* phit, double* R,
                          cudaStream_t s);
cudaError_t lumped_mass(pff_problem& pb, double* B, cudaStream_t s);
cudaError_t total_crack_volume(pff_problem& pb, const double* u, const double* phi, double* out_host, cudaStream_t s);
cudaError_t newton_pdas_step(pff_problem& pb, pff_mg& mg, double* u, double* phi, const double* phi_old,
                             uint8_t* active, const NewtonOpts& o, NewtonInfo& info, cudaStream_t s);
// per-cell modulus and the adjoint TCV gradient (adjoint.cpp)
std::string set_cell_modulus(pff_problem& pb, const double* E_cells, cudaStream_t s);
cudaError_t tcv_gradient(pff_problem& pb, const double* u, const double* phi, double* g, cudaStream_t s,
                         const uint8_t* rows = nullptr);
struct AdjointStats {
  int gmres_total = 0, gmres_max = 0, failed_step = 0;
  GmresResult last;
};
cudaError_t tcv_adjoint_steps(pff_problem& pb, pff_mg& mg, int N, const double* const* u, const double* const* phi,
                              const uint8_t* const* active, const double* p, bool extrapolated, double rtol,
                              int restart, int maxiter, double* gE, double* gp_host, double* ggc_host,
                              AdjointStats& st, std::string& err, cudaStream_t s);
cudaError_t param_vjp(pff_problem& pb, const double* w, double* gE_cells, double* g_host, cudaStream_t s);
cudaError_t tcv_adjoint(pff_problem& pb, pff_mg& mg, const double* u, const double* phi, const double* phi_old,
                        const uint8_t* active, double rtol, int restart, int maxiter, double* gE, double* g_host,
                        GmresResult& gr, std::string& err, cudaStream_t s);
// COD(x) profile (qoi.cu): x host array of nx line positions, result to out_host; synchronises
std::string cod_profile(pff_problem& pb, const double* u, const double* phi, const double* x, int nx, double* out_host,
                        cudaStream_t s);
// cell kernels (cells.cu)
cudaError_t cells_scatter(int32_t n, const double* v, const int32_t* slot, double* out64, float* out32,
                          cudaStream_t s);
cudaError_t cells_level(int32_t n, const int32_t* dst, const int32_t* src, const int32_t* child,
                        const double* leaf_v, const double* finer, double* out64, float* out32, cudaStream_t s);
cudaError_t cells_gather(int32_t n, const double* in, const int32_t* slot, double* out, cudaStream_t s);
// multigrid (mg_host.cpp)
std::string mg_alloc(pff_mg& mg);
void mg_release_graphs(pff_mg& mg);
// the set-up chains' graph (re-captured at the next set-up)
void mg_release_setup_graph(pff_mg& mg);
std::string mg_setup(pff_mg& mg, cudaStream_t s);
cudaError_t mg_vcycle(pff_mg& mg, int block, const double* r, double* z, cudaStream_t s);
// both blocks of the preconditioner on the full vector (u_x | u_y | phi)
cudaError_t mg_precond(pff_mg& mg, const double* v, double* z, cudaStream_t s);
// level operator y = A_l x of one block (op OP_UU / OP_PP / *_DIAG), precision of T
template <typename T>
cudaError_t level_apply(pff_mg& mg, int level, int op, const T* x, T* y, cudaStream_t s, bool pdl = false,
                        const ChebEpi* ch = nullptr);

}  // namespace pff
