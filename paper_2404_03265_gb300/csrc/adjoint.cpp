// Per-cell modulus, TCV gradient, parameter VJP and the adjoint TCV gradient.
//
// Quantity of interest (Sec. 4): J = TCV = integral of u . grad phi at the
// converged state of a load step (Algorithm 2).  At convergence the free DoFs F
// satisfy [C^T A(U; theta)]_F = 0 while the fixed ones (Dirichlet u, active phi
// = phi_old) and phi_tilde = phi_old do not depend on theta = (p, G_c, E_K).
// With G~ the constrained Jacobian of Sec. 3.1:
//     G~^T lambda = M_f C^T dJ/dU,        dJ/dtheta = (C M_f lambda) . dR/dtheta,  R = -A.
// The transposed solve reuses the block V-cycle (its blocks are symmetric).
#include <algorithm>
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

cudaError_t tcv_gradient(pff_problem& pb, const double* u, const double* phi, double* g, cudaStream_t s,
                         const uint8_t* rows) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  RET(make_state(n, u, phi, phi, D.slot_flags, D.hang, D.nhang, M.k, W.st, s));
  // mode 0: rows fixed in `rows` (default: Dirichlet u and active phi) 0, hanging rows 0, C^T applied
  return leaf_op(pb, OP_TCV_GRAD, 0, W.st, rows ? rows : pb.cmask, W.tmp, W.tmp + 2 * n, g, g + 2 * n, s);
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
  RET(launch_set_lin(n, u, phi, phi_old, D.hang, D.nhang, M.k, pb.lin64, pb.lin32, pb.hlin64, pb.hlin32, s));
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

namespace pff {

// Checkpointed adjoint over n_steps load steps (see the header of this file):
// step k (1..N) has state (u[k], phi[k]), obstacle phi[k-1], active set
// active[k-1], pressure p[k-1] and phi_tilde = phi[k-1], or, when extrapolated,
// phi_tilde = clip(2 phi[k-1] - phi[k-2], 0, 1) for k >= 2 (Sec. 2).  Backwards
// from gbar^N = C^T dJ/dU^N (Dirichlet rows 0):
//   G~_k^T mu = gbar^k (GMRES; the fixed rows of mu equal gbar there),
//   dJ/dtheta += (C M_f mu) . dR_k/dtheta,
//   v^k = (dA/dphi~)^T C M_f mu,
//   gbar^(k-1) = (0, 0, -v^k + [mu - K^T C M_f mu] on the active rows),
// the bracket being the active-row adjoint of the full step Jacobian, whose free
// rows still see the active values (K = C^T G C).  Extrapolated: d phi~/d phi^(k-1)
// = 2 chi and d phi~/d phi^(k-2) = -chi (chi = 1 strictly inside the clip), so
// -2 chi v^k enters gbar^(k-1) and +chi v^k waits (adj_pend) for gbar^(k-2); the
// share that would reach phi^0 is dropped (the initial state is parameter-free).
cudaError_t tcv_adjoint_steps(pff_problem& pb, pff_mg& mg, int N, const double* const* u, const double* const* phi,
                              const uint8_t* const* active, const double* p, bool extrapolated, double rtol,
                              int restart, int maxiter, double* gE, double* gp_host, double* ggc_host,
                              AdjointStats& st, std::string& err, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  if (gE && !pb.adj_cell) {
    pb.adj_cell = pb.bufs.alloc<double>(D.n_leaf_cells);
    if (!pb.adj_cell) return cudaErrorMemoryAllocation;
  }
  if (extrapolated && N >= 2 && !pb.adj_phit) {
    pb.adj_phit = pb.bufs.alloc<double>(n);
    pb.adj_pend = pb.bufs.alloc<double>(n);
    if (!pb.adj_phit || !pb.adj_pend) return cudaErrorMemoryAllocation;
  }
  const double p_saved = pb.prm.p;
  struct Restore {
    pff_problem& pb; double p;
    ~Restore() { pb.prm.p = p; }
  } restore{pb, p_saved};
  RET(tcv_gradient(pb, u[N], phi[N], W.rhs, s, pb.cmask_dir));
  if (gE) RET(cudaMemsetAsync(gE, 0, D.n_leaf_cells * sizeof(double), s));
  *ggc_host = 0.0;
  bool pend = false;  // adj_pend holds a share for the step being carried into
  for (int k = N; k >= 1; --k) {
    const bool ex = extrapolated && k >= 2;
    const double* phit = phi[k - 1];
    if (ex) {
      RET(extrapolate_phi(n, phi[k - 1], phi[k - 2], pb.adj_phit, s));
      phit = pb.adj_phit;
    }
    RET(launch_set_lin(n, u[k], phi[k], phit, D.hang, D.nhang, M.k, pb.lin64, pb.lin32, pb.hlin64, pb.hlin32, s));
    pb.has_state = true;
    RET(launch_leaf_cmask(n, D.slot_flags, active[k - 1], pb.cmask, s));
    pb.prm.p = p[k - 1];
    err = mg_setup(mg, s);
    if (!err.empty()) return cudaErrorUnknown;
    GmresResult gr;
    RET(gmres_solve(pb, mg, 1, W.rhs, W.dU, rtol, restart, maxiter, gr, s));
    st.gmres_total += gr.iterations;
    st.gmres_max = std::max(st.gmres_max, gr.iterations);
    st.last = gr;
    if (gr.breakdown || !gr.converged) { st.failed_step = k; return cudaSuccess; }
    double g2[2];
    RET(param_vjp(pb, W.dU, gE ? pb.adj_cell : nullptr, g2, s));
    gp_host[k - 1] = g2[0];
    *ggc_host += g2[1];
    if (gE) RET(axpby(D.n_leaf_cells, gE, gE, 1.0, pb.adj_cell, 1.0, s));
    if (k > 1) {
      RET(mask_fixed(n, pb.cmask, W.dU, W.tmp, s));
      // t1 = C^T G^T C (M_f mu) on every row but Dirichlet u; t2 = (dA/dphi~)^T (M_f mu)
      RET(leaf_op(pb, OP_FULL_T, MODE_MASK_INPUT, pb.lin64, pb.cmask_dir, W.tmp, W.tmp + 2 * n, W.R, W.R + 2 * n, s));
      RET(leaf_op(pb, OP_PHIT_VJP, MODE_MASK_INPUT, pb.lin64, pb.cmask_dir, W.tmp, W.tmp + 2 * n, W.du0, W.res, s));
      if (ex) {
        const bool out = k - 2 >= 1;
        RET(adj_carry(n, active[k - 1], W.dU, W.R, W.res, W.rhs, s, phi[k - 1], phi[k - 2],
                      pend ? pb.adj_pend : nullptr, out ? pb.adj_pend : nullptr));
        pend = out;
      } else {
        RET(adj_carry(n, active[k - 1], W.dU, W.R, W.res, W.rhs, s));
      }
    }
  }
  return cudaStreamSynchronize(s);
}

}  // namespace pff
