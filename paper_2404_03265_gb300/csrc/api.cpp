// C-ABI entry points of libpff (declared in include/pff.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "mesh.h"
#include "solve.cuh"
#include "state.h"

using namespace pff;

namespace {
thread_local std::string g_err;

pff_status fail(pff_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define PFF_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? PFF_ERR_OOM : PFF_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

#define PFF_TRY(...)                                               \
  try {                                                            \
    __VA_ARGS__                                                    \
  } catch (const std::bad_alloc&) {                                \
    return fail(PFF_ERR_OOM, "host allocation failed");            \
  } catch (const std::exception& ex) {                             \
    return fail(PFF_ERR_INVALID_ARG, ex.what());                   \
  } catch (...) {                                                  \
    return fail(PFF_ERR_INVALID_ARG, "unknown exception");         \
  }

}  // namespace

namespace pff {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace pff

extern "C" const char* pff_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ mesh
extern "C" pff_status pff_mesh_create(double x0, double x1, double y0, double y1, int32_t ncx, int32_t ncy,
                                      pff_mesh** out) {
  PFF_TRY({
    if (!out) return fail(PFF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(x1 > x0) || !(y1 > y0) || ncx <= 0 || ncy <= 0 || ncx > 4096 || ncy > 4096)
      return fail(PFF_ERR_INVALID_ARG, "invalid domain or coarse grid");
    auto* m = new pff_mesh();
    Tree& t = m->m.tree;
    t.x0 = x0; t.x1 = x1; t.y0 = y0; t.y1 = y1; t.ncx = ncx; t.ncy = ncy;
    t.lev.emplace_back();
    for (int j = 0; j < ncy; ++j)
      for (int i = 0; i < ncx; ++i) t.lev[0].insert(cell_key(i, j));
    *out = m;
    return PFF_OK;
  })
}

static pff_status check_refinable(pff_mesh* m) {
  if (!m) return fail(PFF_ERR_INVALID_ARG, "mesh is NULL");
  if (m->m.finalized) return fail(PFF_ERR_STATE, "mesh already finalized");
  if (m->m.tree.finest() >= 24) return fail(PFF_ERR_INVALID_ARG, "more than 24 refinement levels");
  return PFF_OK;
}

extern "C" pff_status pff_mesh_refine_global(pff_mesh* m, int32_t times) {
  PFF_TRY({
    pff_status st = check_refinable(m);
    if (st) return st;
    if (times < 0) return fail(PFF_ERR_INVALID_ARG, "times < 0");
    for (int r = 0; r < times; ++r) {
      auto lv = m->m.tree.leaves();
      for (auto& c : lv) m->m.tree.split(int(c[0]), c[1], c[2]);
      m->m.tree.balance();
      if (m->m.tree.finest() >= 24) return fail(PFF_ERR_INVALID_ARG, "more than 24 refinement levels");
    }
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_refine_box(pff_mesh* m, int32_t rule, double bx0, double bx1, double by0,
                                          double by1) {
  PFF_TRY({
    pff_status st = check_refinable(m);
    if (st) return st;
    if (rule != 0 && rule != 1) return fail(PFF_ERR_INVALID_ARG, "rule must be 0 or 1");
    Tree& t = m->m.tree;
    auto lv = t.leaves();
    std::vector<std::array<int64_t, 3>> marks;
    for (auto& c : lv) {
      const int l = int(c[0]);
      const double hx = t.hx(l), hy = t.hy(l);
      bool hit;
      if (rule == 0) {
        const double xc = t.x0 + (double(c[1]) + 0.5) * hx, yc = t.y0 + (double(c[2]) + 0.5) * hy;
        hit = bx0 <= xc && xc <= bx1 && by0 <= yc && yc <= by1;
      } else {
        const double xa = t.x0 + double(c[1]) * hx, xb = t.x0 + double(c[1] + 1) * hx;
        const double ya = t.y0 + double(c[2]) * hy, yb = t.y0 + double(c[2] + 1) * hy;
        hit = xa <= bx1 && xb >= bx0 && ya <= by1 && yb >= by0;
      }
      if (hit) marks.push_back(c);
    }
    for (auto& c : marks) t.split(int(c[0]), c[1], c[2]);
    t.balance();
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_refine_marked(pff_mesh* m, const uint8_t* marks, int64_t n_leaves) {
  PFF_TRY({
    pff_status st = check_refinable(m);
    if (st) return st;
    auto lv = m->m.tree.leaves();
    if (!marks || n_leaves != int64_t(lv.size())) return fail(PFF_ERR_INVALID_ARG, "marks length != leaves");
    for (size_t q = 0; q < lv.size(); ++q)
      if (marks[q]) m->m.tree.split(int(lv[q][0]), lv[q][1], lv[q][2]);
    m->m.tree.balance();
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_n_leaves(const pff_mesh* m, int64_t* n) {
  PFF_TRY({
    if (!m || !n) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    *n = m->m.finalized ? int64_t(m->m.leaves.size()) : int64_t(m->m.tree.leaves().size());
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_finalize(pff_mesh* m, int32_t fe_degree) {
  PFF_TRY({
    if (!m) return fail(PFF_ERR_INVALID_ARG, "mesh is NULL");
    if (m->m.finalized) return fail(PFF_ERR_STATE, "mesh already finalized");
    if (fe_degree != 1 && fe_degree != 2) return fail(PFF_ERR_INVALID_ARG, "fe_degree must be 1 or 2");
    std::string e = finalize_mesh(m->m, fe_degree);
    if (!e.empty()) return fail(PFF_ERR_INVALID_ARG, e);
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_info_get(const pff_mesh* m, pff_mesh_info* out) {
  PFF_TRY({
    if (!m || !out) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!m->m.finalized) return fail(PFF_ERR_STATE, "mesh not finalized");
    const Mesh& M = m->m;
    std::memset(out, 0, sizeof(*out));
    out->n_slots = M.lay.n_slots;
    out->n_nodes = M.n_nodes();
    out->n_leaf_cells = int64_t(M.leaves.size());
    out->n_hanging = int64_t(M.hang.size());
    out->n_partials = M.n_partials;
    out->n_bricks = int64_t(M.lay.bricks.size());
    out->n_irregular = M.lay.n_irregular();
    out->x_max = M.Xmax;
    out->y_max = M.Ymax;
    out->h_min = M.hmin_diag();
    out->fe_degree = M.k;
    out->finest_level = M.Lf;
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_slots(const pff_mesh* m, int32_t* X, int32_t* Y, uint8_t* flags) {
  PFF_TRY({
    if (!m) return fail(PFF_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->m.finalized) return fail(PFF_ERR_STATE, "mesh not finalized");
    const Mesh& M = m->m;
    for (int64_t s = 0; s < M.lay.n_slots; ++s) {
      const int32_t n = M.slot_node[s];
      if (X) X[s] = n < 0 ? -1 : M.nX[n];
      if (Y) Y[s] = n < 0 ? -1 : M.nY[n];
      if (flags) flags[s] = M.slot_flags[s] & 7;
    }
    return PFF_OK;
  })
}

extern "C" pff_status pff_mesh_leaf_cells(const pff_mesh* m, int32_t* lij) {
  PFF_TRY({
    if (!m || !lij) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!m->m.finalized) return fail(PFF_ERR_STATE, "mesh not finalized");
    for (size_t q = 0; q < m->m.leaves.size(); ++q)
      for (int r = 0; r < 3; ++r) lij[3 * q + r] = int32_t(m->m.leaves[q][r]);
    return PFF_OK;
  })
}

extern "C" void pff_mesh_destroy(pff_mesh* m) {
  if (!m) return;
  m->dev.release();
  delete m;
}

// ------------------------------------------------------------------ problem
extern "C" pff_status pff_problem_create(pff_mesh* m, const pff_params* prm, pff_problem** out) {
  PFF_TRY({
    if (!m || !prm || !out) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!m->m.finalized) return fail(PFF_ERR_STATE, "mesh not finalized");
    if (!(prm->E > 0) || !(prm->nu > -1.0 && prm->nu < 0.5) || !(prm->Gc > 0) || !(prm->eps > 0) ||
        !(prm->kappa >= 0 && prm->kappa < 1))
      return fail(PFF_ERR_INVALID_ARG, "invalid material parameters");
    std::string e = upload_mesh(*m);
    if (!e.empty()) return fail(PFF_ERR_CUDA, e);
    auto* pb = new pff_problem();
    pb->mesh = m;
    pb->prm = *prm;
    e = alloc_problem(*pb);
    if (!e.empty()) {
      delete pb;
      return fail(PFF_ERR_OOM, e);
    }
    const cudaError_t ce = noalloc_prepare();
    if (ce != cudaSuccess) {
      pb->bufs.release();
      delete pb;
      return fail(PFF_ERR_CUDA, std::string("pff_problem_create: fixed scratch of pff_apply_noalloc: ") +
                                    cudaGetErrorString(ce));
    }
    *out = pb;
    return PFF_OK;
  })
}

extern "C" void pff_problem_destroy(pff_problem* pb) {
  if (!pb) return;
  for (auto& e : pb->gm_ev)
    if (e) cudaEventDestroy(e);
  pb->ws.mem.release();
  pb->bufs.release();
  delete pb;
}

extern "C" pff_status pff_set_state(pff_problem* pb, const double* u, const double* phi, const double* phit,
                                    void* stream) {
  PFF_TRY({
    if (!pb || !u || !phi || !phit) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    const Mesh& M = pb->mesh->m;
    const DevMesh& D = pb->mesh->dev;
    PFF_CUDA(launch_set_lin(M.lay.n_slots, u, phi, phit, D.hang, D.nhang, M.k, pb->lin64, pb->lin32,
                            pb->hlin64, pb->hlin32, cudaStream_t(stream)));
    pb->has_state = true;
    return PFF_OK;
  })
}

extern "C" pff_status pff_set_active(pff_problem* pb, const uint8_t* active, void* stream) {
  PFF_TRY({
    if (!pb || !active) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    PFF_CUDA(launch_leaf_cmask(pb->mesh->m.lay.n_slots, pb->mesh->dev.slot_flags, active, pb->cmask,
                               cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_apply(pff_problem* pb, int32_t precision, int32_t op, const void* xu, const void* xp,
                                void* yu, void* yp, void* stream) {
  PFF_TRY({
    if (!pb || !xu || !xp || !yu || !yp) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (precision != PFF_F64 && precision != PFF_F32) return fail(PFF_ERR_INVALID_ARG, "bad precision");
    if (op < 0 || op > 2) return fail(PFF_ERR_INVALID_ARG, "bad operator");
    if (!pb->has_state) return fail(PFF_ERR_STATE, "pff_set_state has not been called");
    if (xu == yu || xp == yp) return fail(PFF_ERR_INVALID_ARG, "x and y overlap");
    PFF_CUDA(leaf_apply(*pb, precision, op, xu, xp, yu, yp, cudaStream_t(stream)));
    return PFF_OK;
  })
}

// ------------------------------------------------------------------ multigrid
extern "C" pff_status pff_mg_create(pff_problem* pb, int32_t precision, pff_mg** out) {
  PFF_TRY({
    if (!pb || !out) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (precision != PFF_F64 && precision != PFF_F32) return fail(PFF_ERR_INVALID_ARG, "bad precision");
    if (pb->mesh->m.Lf + 1 > kMaxLevels) return fail(PFF_ERR_INVALID_ARG, "too many levels");
    auto* mg = new pff_mg();
    mg->pb = pb;
    mg->precision = precision;
    std::string e = mg_alloc(*mg);
    if (!e.empty()) {
      mg->mem.release();
      delete mg;
      return fail(PFF_ERR_OOM, e);
    }
    *out = mg;
    return PFF_OK;
  })
}

extern "C" pff_status pff_mg_setup(pff_mg* mg, void* stream) {
  PFF_TRY({
    if (!mg) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!mg->pb->has_state) return fail(PFF_ERR_STATE, "pff_set_state has not been called");
    std::string e = mg_setup(*mg, cudaStream_t(stream));
    if (!e.empty()) return fail(PFF_ERR_CUDA, e);
    return PFF_OK;
  })
}

extern "C" pff_status pff_vcycle(pff_mg* mg, int32_t block, const double* r, double* z, void* stream) {
  PFF_TRY({
    if (!mg || !r || !z) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (block != 0 && block != 1) return fail(PFF_ERR_INVALID_ARG, "block must be 0 (u) or 1 (phi)");
    if (!mg->ready) return fail(PFF_ERR_STATE, "pff_mg_setup has not been called");
    if (r == z) return fail(PFF_ERR_INVALID_ARG, "r and z overlap");
    PFF_CUDA(mg_vcycle(*mg, block, r, z, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_mg_lambda(const pff_mg* mg, int32_t block, double* lam, int32_t n) {
  PFF_TRY({
    if (!mg || !lam) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (block != 0 && block != 1) return fail(PFF_ERR_INVALID_ARG, "bad block");
    const auto& v = mg->blk[block].lam;
    if (n < int32_t(v.size())) return fail(PFF_ERR_INVALID_ARG, "lam array too short");
    for (size_t i = 0; i < v.size(); ++i) lam[i] = v[i];
    return PFF_OK;
  })
}

extern "C" void pff_mg_destroy(pff_mg* mg) {
  if (!mg) return;
  mg_release_graphs(*mg);
  mg_release_setup_graph(*mg);
  if (mg->su_side) cudaStreamDestroy(mg->su_side);
  if (mg->su_chains) cudaEventDestroy(mg->su_chains);
  if (mg->cap_stream) cudaStreamDestroy(mg->cap_stream);
  if (mg->cap_stream2) cudaStreamDestroy(mg->cap_stream2);
  if (mg->ev_fork) cudaEventDestroy(mg->ev_fork);
  if (mg->ev_join) cudaEventDestroy(mg->ev_join);
  for (int i = 0; i <= pff_mg::kSetupStreams; ++i) {
    if (mg->su_stream[i]) cudaStreamDestroy(mg->su_stream[i]);
    if (mg->su_done[i]) cudaEventDestroy(mg->su_done[i]);
  }
  if (mg->su_start) cudaEventDestroy(mg->su_start);
  mg->mem.release();
  delete mg;
}

extern "C" pff_status pff_extrapolate_phi(pff_problem* pb, const double* phi_prev, const double* phi_prev2,
                                          double* phi_tilde, void* stream) {
  PFF_TRY({
    if (!pb || !phi_prev || !phi_prev2 || !phi_tilde) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    PFF_CUDA(extrapolate_phi(pb->mesh->m.lay.n_slots, phi_prev, phi_prev2, phi_tilde, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_set_cell_loop(pff_problem* pb, int32_t strip_half_rows) {
  PFF_TRY({
    if (!pb) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (strip_half_rows != 0 && strip_half_rows != 15 && strip_half_rows != 5 && strip_half_rows != 1)
      return fail(PFF_ERR_INVALID_ARG, "strip_half_rows must be 0, 15, 5 or 1");
    pb->sweep_sh = strip_half_rows;
    return PFF_OK;
  })
}

// ------------------------------------------------------------------ solvers
extern "C" pff_status pff_set_pressure(pff_problem* pb, double p) {
  PFF_TRY({
    if (!pb || !std::isfinite(p)) return fail(PFF_ERR_INVALID_ARG, "bad argument");
    pb->prm.p = p;
    return PFF_OK;
  })
}

extern "C" pff_status pff_residual(pff_problem* pb, const double* u, const double* phi, const double* phi_tilde,
                                   double* R, void* stream) {
  PFF_TRY({
    if (!pb || !u || !phi || !phi_tilde || !R) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    PFF_CUDA(leaf_residual(*pb, u, phi, phi_tilde, R, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_lumped_mass(pff_problem* pb, double* B, void* stream) {
  PFF_TRY({
    if (!pb || !B) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    PFF_CUDA(lumped_mass(*pb, B, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_tcv(pff_problem* pb, const double* u, const double* phi, double* out_host, void* stream) {
  PFF_TRY({
    if (!pb || !u || !phi || !out_host) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    PFF_CUDA(total_crack_volume(*pb, u, phi, out_host, cudaStream_t(stream)));
    return PFF_OK;
  })
}

static void fill_info(const NewtonInfo& in, pff_solve_info* out) {
  std::memset(out, 0, sizeof(*out));
  out->newton_iterations = in.newton;
  out->converged = in.converged ? 1 : 0;
  out->linesearch_failures = in.linesearch_failures;
  int tot = 0, mx = 0;
  for (size_t i = 0; i < in.gmres.size(); ++i) {
    tot += in.gmres[i];
    mx = std::max(mx, in.gmres[i]);
    if (i < 128) out->gmres_per_newton[i] = in.gmres[i];
  }
  out->gmres_total = tot;
  out->gmres_max = mx;
  out->active_size = in.active_size.empty() ? 0 : in.active_size.back();
  out->residual0 = in.residual0;
  out->residual = in.residual.empty() ? 0.0 : in.residual.back();
  out->margin = in.margin;
  for (size_t i = 0; i < in.residual.size() && i < 129; ++i) out->residual_history[i] = in.residual[i];
  out->time_mg_setup = in.t_setup;
  out->time_gmres = in.t_gmres;
  out->time_gmres_apply = in.t_apply;
  out->time_gmres_vcycle = in.t_vcycle;
  out->time_gmres_orth = in.t_orth;
}

extern "C" pff_status pff_gmres_solve(pff_problem* pb, pff_mg* mg, int32_t transpose, const double* rhs, double* x,
                                      double rtol, int32_t restart, int32_t maxiter, pff_solve_info* info,
                                      void* stream) {
  PFF_TRY({
    if (!pb || !mg || !rhs || !x) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (restart < 1 || restart > 500 || maxiter < 1 || !(rtol > 0)) return fail(PFF_ERR_INVALID_ARG, "bad options");
    if (!mg->ready) return fail(PFF_ERR_STATE, "pff_mg_setup has not been called");
    std::string e = ensure_workspace(*pb, restart);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    GmresResult gr;
    PFF_CUDA(gmres_solve(*pb, *mg, transpose, rhs, x, rtol, restart, maxiter, gr, cudaStream_t(stream)));
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->gmres_total = gr.iterations;
      info->gmres_max = gr.iterations;
      info->converged = gr.converged ? 1 : 0;
      info->residual0 = gr.initial;
      info->residual = gr.estimate;
      info->time_gmres_apply = gr.t_apply;
      info->time_gmres_vcycle = gr.t_vcycle;
      info->time_gmres_orth = gr.t_orth;
    }
    if (gr.breakdown) return fail(PFF_ERR_GMRES_BREAKDOWN, "GMRES breakdown");
    if (!std::isfinite(gr.estimate)) return fail(PFF_ERR_NONFINITE, "non-finite residual in GMRES");
    if (!gr.converged) return fail(PFF_ERR_NOT_CONVERGED, "GMRES did not reach the tolerance");
    return PFF_OK;
  })
}

extern "C" pff_status pff_newton_pdas_step(pff_problem* pb, pff_mg* mg, double* u, double* phi, const double* phi_old,
                                           uint8_t* active, const pff_newton_opts* opts, pff_solve_info* info,
                                           void* stream) {
  PFF_TRY({
    if (!pb || !mg || !u || !phi || !phi_old || !active) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    NewtonOpts o;
    if (opts) {
      o.tol = opts->tol; o.atol = opts->atol; o.gmres_rtol = opts->gmres_rtol; o.omega = opts->omega;
      o.restart = opts->restart; o.gmres_maxiter = opts->gmres_maxiter; o.max_newton = opts->max_newton;
      o.ls_max = opts->ls_max;
      o.matvec = opts->matvec_precision;
      o.phi_tilde = opts->phi_tilde;
    }
    if (o.matvec != PFF_F64 && o.matvec != PFF_F32) return fail(PFF_ERR_INVALID_ARG, "bad matvec precision");
    if (o.restart < 1 || o.restart > 500 || o.max_newton < 0 || o.ls_max < 1 || !(o.omega > 0 && o.omega <= 1))
      return fail(PFF_ERR_INVALID_ARG, "bad Newton options");
    std::string e = ensure_workspace(*pb, o.restart);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    NewtonInfo ni;
    cudaError_t ce = newton_pdas_step(*pb, *mg, u, phi, phi_old, active, o, ni, cudaStream_t(stream));
    if (info) fill_info(ni, info);
    if (!ni.error.empty()) return fail(PFF_ERR_CUDA, ni.error);
    PFF_CUDA(ce);
    if (ni.nonfinite) return fail(PFF_ERR_NONFINITE, "non-finite Newton residual");
    if (ni.gmres_breakdown) return fail(PFF_ERR_GMRES_BREAKDOWN, "GMRES breakdown inside Newton");
    if (!ni.converged) return fail(PFF_ERR_NOT_CONVERGED, "Newton / active set did not converge");
    return PFF_OK;
  })
}

// ---- per-cell modulus, parameters, TCV gradient, adjoint ---------------------
extern "C" pff_status pff_set_cell_modulus(pff_problem* pb, const double* E_cells, void* stream) {
  PFF_TRY({
    if (!pb) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = set_cell_modulus(*pb, E_cells, cudaStream_t(stream));
    if (!e.empty()) return fail(PFF_ERR_CUDA, "pff_set_cell_modulus: " + e);
    return PFF_OK;
  })
}

extern "C" pff_status pff_set_params(pff_problem* pb, const pff_params* prm) {
  PFF_TRY({
    if (!pb || !prm) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!(prm->E > 0) || !(prm->nu > -1.0 && prm->nu < 0.5) || !(prm->eps > 0) || !(prm->Gc >= 0))
      return fail(PFF_ERR_INVALID_ARG, "bad material parameters");
    pb->prm = *prm;
    return PFF_OK;
  })
}

extern "C" pff_status pff_tcv_gradient(pff_problem* pb, const double* u, const double* phi, double* g,
                                       void* stream) {
  PFF_TRY({
    if (!pb || !u || !phi || !g) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    PFF_CUDA(tcv_gradient(*pb, u, phi, g, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_param_vjp(pff_problem* pb, const double* w, double* gE_cells, double* g_host,
                                    void* stream) {
  PFF_TRY({
    if (!pb || !w || !g_host) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!pb->has_state) return fail(PFF_ERR_STATE, "pff_set_state has not been called");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    PFF_CUDA(param_vjp(*pb, w, gE_cells, g_host, cudaStream_t(stream)));
    return PFF_OK;
  })
}

extern "C" pff_status pff_tcv_adjoint(pff_problem* pb, pff_mg* mg, const double* u, const double* phi,
                                      const double* phi_old, const uint8_t* active, double rtol, int32_t restart,
                                      int32_t maxiter, double* gE_cells, double* g_host, pff_solve_info* info,
                                      void* stream) {
  PFF_TRY({
    if (!pb || !mg || !u || !phi || !phi_old || !active || !g_host) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (mg->pb != pb) return fail(PFF_ERR_INVALID_ARG, "multigrid object of another problem");
    if (restart < 1 || restart > 500 || maxiter < 1 || !(rtol > 0)) return fail(PFF_ERR_INVALID_ARG, "bad options");
    std::string e = ensure_workspace(*pb, restart);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    GmresResult gr;
    std::string err;
    const cudaError_t ce = tcv_adjoint(*pb, *mg, u, phi, phi_old, active, rtol, restart, maxiter, gE_cells, g_host,
                                       gr, err, cudaStream_t(stream));
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->gmres_total = gr.iterations;
      info->gmres_max = gr.iterations;
      info->converged = gr.converged ? 1 : 0;
      info->residual0 = gr.initial;
      info->residual = gr.estimate;
    }
    if (!err.empty()) return fail(PFF_ERR_CUDA, "pff_mg_setup: " + err);
    PFF_CUDA(ce);
    if (gr.breakdown) return fail(PFF_ERR_GMRES_BREAKDOWN, "GMRES breakdown in the adjoint solve");
    if (!std::isfinite(gr.estimate)) return fail(PFF_ERR_NONFINITE, "non-finite residual in the adjoint solve");
    if (!gr.converged) return fail(PFF_ERR_NOT_CONVERGED, "adjoint GMRES did not reach the tolerance");
    return PFF_OK;
  })
}

extern "C" pff_status pff_tcv_adjoint_steps(pff_problem* pb, pff_mg* mg, int32_t n_steps, const double* const* u,
                                            const double* const* phi, const uint8_t* const* active,
                                            const double* p_host, int32_t phi_tilde_mode, double rtol,
                                            int32_t restart, int32_t maxiter, double* gE_cells, double* gp_host,
                                            double* gGc_host, pff_solve_info* info, void* stream) {
  PFF_TRY({
    if (!pb || !mg || !u || !phi || !active || !p_host || !gp_host || !gGc_host)
      return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (n_steps < 1) return fail(PFF_ERR_INVALID_ARG, "n_steps must be >= 1");
    for (int k = 0; k <= n_steps; ++k)
      if (!u[k] || !phi[k]) return fail(PFF_ERR_INVALID_ARG, "NULL state pointer");
    for (int k = 0; k < n_steps; ++k)
      if (!active[k]) return fail(PFF_ERR_INVALID_ARG, "NULL active-set pointer");
    if (mg->pb != pb) return fail(PFF_ERR_INVALID_ARG, "multigrid object of another problem");
    if (restart < 1 || restart > 500 || maxiter < 1 || !(rtol > 0)) return fail(PFF_ERR_INVALID_ARG, "bad options");
    if (phi_tilde_mode != PFF_PHIT_PREVIOUS && phi_tilde_mode != PFF_PHIT_EXTRAPOLATED)
      return fail(PFF_ERR_INVALID_ARG, "phi_tilde_mode must be PFF_PHIT_PREVIOUS or PFF_PHIT_EXTRAPOLATED");
    std::string e = ensure_workspace(*pb, restart);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    AdjointStats st;
    std::string err;
    const cudaError_t ce = tcv_adjoint_steps(*pb, *mg, n_steps, u, phi, active, p_host,
                                             phi_tilde_mode == PFF_PHIT_EXTRAPOLATED, rtol, restart, maxiter,
                                             gE_cells, gp_host, gGc_host, st, err, cudaStream_t(stream));
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->gmres_total = st.gmres_total;
      info->gmres_max = st.gmres_max;
      info->converged = st.failed_step == 0 ? 1 : 0;
      info->residual0 = st.last.initial;
      info->residual = st.last.estimate;
    }
    if (!err.empty()) return fail(PFF_ERR_CUDA, "pff_mg_setup: " + err);
    PFF_CUDA(ce);
    if (st.failed_step) {
      if (st.last.breakdown) return fail(PFF_ERR_GMRES_BREAKDOWN, "GMRES breakdown in the adjoint of a load step");
      return fail(PFF_ERR_NOT_CONVERGED, "adjoint GMRES did not reach the tolerance at load step " +
                                             std::to_string(st.failed_step));
    }
    return PFF_OK;
  })
}

extern "C" pff_status pff_active_set(pff_problem* pb, const double* R, const double* phi, const double* phi_old,
                                     uint8_t* active, int64_t* n_changed, int64_t* n_active, double* margin,
                                     void* stream) {
  PFF_TRY({
    if (!pb || !R || !phi || !phi_old || !active) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    const cudaStream_t s = cudaStream_t(stream);
    SolverWS& W = pb->ws;
    const int64_t n = pb->mesh->m.lay.n_slots;
    PFF_CUDA(lumped_mass(*pb, W.B + 2 * n, s));
    PFF_CUDA(cudaMemcpyAsync(W.act_prev, active, n, cudaMemcpyDeviceToDevice, s));
    PFF_CUDA(cudaMemsetAsync(W.stats, 0, 2 * sizeof(unsigned long long), s));
    const unsigned long long big = 0x7ff0000000000000ull;
    PFF_CUDA(cudaMemcpyAsync(W.stats + 2, &big, sizeof(big), cudaMemcpyHostToDevice, s));
    PFF_CUDA(active_set(n, R, W.B + 2 * n, phi, phi_old, pb->mesh->dev.slot_flags, pb->prm.c, W.act_prev, W.act,
                        W.stats, s));
    PFF_CUDA(cudaMemcpyAsync(active, W.act, n, cudaMemcpyDeviceToDevice, s));
    unsigned long long st[3];
    PFF_CUDA(cudaMemcpyAsync(st, W.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    PFF_CUDA(cudaStreamSynchronize(s));
    if (n_changed) *n_changed = int64_t(st[0]);
    if (n_active) *n_active = int64_t(st[1]);
    if (margin) {
      double m;
      std::memcpy(&m, &st[2], sizeof(m));
      *margin = m;
    }
    return PFF_OK;
  })
}

extern "C" pff_status pff_inverse_diagonal(const pff_mg* mg, int32_t level, int32_t block, double* out,
                                           int32_t* X_host, int32_t* Y_host, int64_t capacity, int64_t* n_out,
                                           void* stream) {
  PFF_TRY({
    if (!mg) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (!mg->ready) return fail(PFF_ERR_STATE, "pff_mg_setup has not been called");
    const Mesh& M = mg->pb->mesh->m;
    const DevMesh& D = mg->pb->mesh->dev;
    if (level < 0 || level >= int32_t(D.levels.size())) return fail(PFF_ERR_INVALID_ARG, "bad level");
    if (block != 0 && block != 1) return fail(PFF_ERR_INVALID_ARG, "bad block");
    const MGBlock& B = mg->blk[block];
    const DevLevel& lv = D.levels[level].lv;
    const int64_t n = int64_t(B.ncomp) * lv.n_slots;
    if (n_out) *n_out = n;
    if (out) {
      if (capacity < n) return fail(PFF_ERR_INVALID_ARG, "output capacity too small");
      PFF_CUDA(cudaMemcpyAsync(out, B.dinv64 + B.ncomp * lv.off, n * sizeof(double), cudaMemcpyDeviceToDevice,
                               cudaStream_t(stream)));
    }
    const LevelMesh& lm = M.levels[level];
    if (X_host) std::memcpy(X_host, lm.slot_X.data(), lm.slot_X.size() * sizeof(int32_t));
    if (Y_host) std::memcpy(Y_host, lm.slot_Y.data(), lm.slot_Y.size() * sizeof(int32_t));
    return PFF_OK;
  })
}

extern "C" pff_status pff_mg_set_coarse(pff_mg* mg, int32_t mode) {
  PFF_TRY({
    if (!mg) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (mode != 0 && mode != 1) return fail(PFF_ERR_INVALID_ARG, "bad coarse mode");
    mg->coarse_mode = mode;
    mg->ready = false;
    mg_release_graphs(*mg);
    return PFF_OK;
  })
}

extern "C" pff_status pff_mg_set_fused_smoother(pff_mg* mg, int32_t on) {
  PFF_TRY({
    if (!mg) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (on != 0 && on != 1) return fail(PFF_ERR_INVALID_ARG, "bad fused-smoother flag");
    mg->fused = on;
    mg_release_graphs(*mg);
    return PFF_OK;
  })
}

extern "C" pff_status pff_cod(pff_problem* pb, const double* u, const double* phi, const double* x_host, int32_t n_x,
                              double* cod_host, void* stream) {
  PFF_TRY({
    if (!pb || !u || !phi || (n_x > 0 && (!x_host || !cod_host))) return fail(PFF_ERR_INVALID_ARG, "NULL argument");
    if (n_x < 0) return fail(PFF_ERR_INVALID_ARG, "n_x < 0");
    std::string e = ensure_workspace(*pb, 50);
    if (!e.empty()) return fail(PFF_ERR_OOM, e);
    e = cod_profile(*pb, u, phi, x_host, n_x, cod_host, cudaStream_t(stream));
    if (!e.empty()) return fail(PFF_ERR_CUDA, "pff_cod: " + e);
    return PFF_OK;
  })
}
