// Per-cell modulus, TCV gradient, parameter VJP and the adjoint TCV gradient.
//
// Quantity of interest (Sec. 4): J = TCV = integral of u . grad phi at the
// converged state of a load step (Algorithm 2).  At convergence the free DoFs F
// satisfy [C^T A(U; theta)]_F = 0 while the fixed ones (Dirichlet u, active phi
// = phi_old) and phi_tilde = phi_old do not depend on theta = (p, G_c, E_K).
// With G~ the constrained Jacobian of Sec. 3.1:
//     G~^T lambda = M_f C^T dJ/dU,        dJ/dtheta = (C M_f lambda) . dR/dtheta,  R = -A.
// The transposed solve reuses the block V-cycle (its blocks are symmetric).
#include <cstring>

#include "solve.cuh"
#include "state.h"

namespace pff {

#define RET(call)                             \
  do {                                        \
    const cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

std::string set_cell_modulus(pff_problem& pb, const double* E, cudaStream_t s) {
  if (!E) {
    pb.has_ecell = false;
    return "";
  }
  const DevMesh& D = pb.mesh->dev;
  const int64_t ns = pb.mesh->m.lay.n_slots;
  if (!pb.ecell64) {
    pb.ecell64 = pb.bufs.alloc<double>(ns);
    pb.ecell32 = pb.bufs.alloc<float>(ns);
    pb.lev_ecell64 = pb.bufs.alloc<double>(D.lev_total);
    pb.lev_ecell32 = pb.bufs.alloc<float>(D.lev_total);
    if (!pb.bufs.err.empty()) return pb.bufs.err;
  }
  auto ck = [](cudaError_t e) { return e == cudaSuccess ? std::string() : std::string(cudaGetErrorString(e)); };
  std::string err;
  if ((err = ck(cudaMemsetAsync(pb.ecell64, 0, ns * sizeof(double), s))).size()) return err;
  if ((err = ck(cudaMemsetAsync(pb.ecell32, 0, ns * sizeof(float), s))).size()) return err;
  if ((err = ck(cudaMemsetAsync(pb.lev_ecell64, 0, D.lev_total * sizeof(double), s))).size()) return err;
  if ((err = ck(cudaMemsetAsync(pb.lev_ecell32, 0, D.lev_total * sizeof(float), s))).size()) return err;
  if ((err = ck(cells_scatter(D.n_leaf_cells, E, D.cell_slot, pb.ecell64, pb.ecell32, s))).size()) return err;
  for (int l = int(D.levels.size()) - 1; l >= 0; --l) {
    const DevMesh::Level& L = D.levels[l];
    const double* finer = (l + 1 < int(D.levels.size())) ? pb.lev_ecell64 + D.levels[l + 1].lv.off : nullptr;
    err = ck(cells_level(L.n_cells, L.cell_dst, L.cell_src, L.cell_child, E, finer, pb.lev_ecell64 + L.lv.off,
                         pb.lev_ecell32 + L.lv.off, s));
    if (!err.empty()) return err;
  }
  pb.has_ecell = true;
  return "";
}

cudaError_t tcv_gradient(pff_problem& pb, const double* u, const double* phi, double* g, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  RET(make_state(n, u, phi, phi, D.slot_flags, D.hang, D.nhang, M.k, W.st, s));
  // mode 0: fixed rows (Dirichlet u, active phi) 0, hanging rows 0, C^T applied
  return leaf_op(pb, OP_TCV_GRAD, 0, W.st, pb.cmask, W.tmp, W.tmp + 2 * n, g, g + 2 * n, s);
}

cudaError_t param_vjp(pff_problem& pb, const double* w, double* gE, double* g_host, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  if (!pb.cell_out) {
    pb.cell_out = pb.bufs.alloc<double>(3 * n);
    if (!pb.cell_out) return cudaErrorMemoryAllocation;
  }
  RET(cudaMemsetAsync(pb.cell_out, 0, 3 * n * sizeof(double), s));
  // fixed components of w read as 0 (M_f), hanging ones from their parents (C)
  RET(leaf_op(pb, OP_VJP, MODE_MASK_INPUT, pb.lin64, pb.cmask, w, w + 2 * n, W.tmp, W.tmp + 2 * n, s));
  if (gE) RET(cells_gather(D.n_leaf_cells, pb.cell_out, D.cell_slot, gE, s));
  RET(vsum(n, pb.cell_out + n, W.partial, W.scal, s));
  RET(vsum(n, pb.cell_out + 2 * n, W.partial, W.scal + 1, s));
  RET(cudaMemcpyAsync(g_host, W.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

}  // namespace pff

namespace pff {

cudaError_t tcv_adjoint(pff_problem& pb, pff_mg& mg, const double* u, const double* phi, const double* phi_old,
                        const uint8_t* active, double rtol, int restart, int maxiter, double* gE, double* g_host,
                        GmresResult& gr, std::string& err, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  // the converged state, phi_tilde = phi_old, and its active set
  RET(launch_set_lin(n, u, phi, phi_old, D.hang, D.nhang, M.k, pb.lin64, pb.lin32, s));
  pb.has_state = true;
  RET(launch_leaf_cmask(n, D.slot_flags, active, pb.cmask, s));
  err = mg_setup(mg, s);
  if (!err.empty()) return cudaErrorUnknown;
  RET(tcv_gradient(pb, u, phi, W.rhs, s));
  RET(gmres_solve(pb, mg, 1, W.rhs, W.dU, rtol, restart, maxiter, gr, s));
  if (gr.breakdown || !gr.converged) return cudaSuccess;  // caller reports
  return param_vjp(pb, W.dU, gE, g_host, s);
}

}  // namespace pff
