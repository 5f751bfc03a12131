"""Benchmark: matrix-free Jacobian apply throughput (GDoF/s and fraction of the
HBM roofline) on the operator-apply workload of the pressurised-crack test
(16x16 coarse cells on (-10,10)^2, 6 global refinements, 2 refinements of the
box |x|<=2, |y|<=1; Q1 u and phi: 4,096,509 DoFs; Q2: 16,368,207 DoFs).

One step = one application of the constrained Jacobian y = G~ x (Sec. 3.1,
matrix-free cell loop of Sec. 3.3) over the whole mesh in FP32 (headline), with
inputs resident in HBM.  Rotating input sets keep the footprint above L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (one independent problem per GPU, no collective on
the data path); value = DoFs processed by all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobian apply GDoF/s & %HBM peak; solve s/load step, FP32-MG vs FP64 MG"
# FP64 FMA rate of a GB300 (CUDA cores), measured with an independent-chain DFMA
# loop at 2.07 GHz; the FP64 apply is bound by it, not by HBM.
FP64_PEAK_TFLOPS = 1.19
WORKLOAD = "apply"
L2_BYTES = 129 * 2 ** 20


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if os.environ.get("PFF_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cpu" if dist.get_backend() == "gloo" else "cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_rank, t_max):
    """Units processed by all ranks per second (replicas: every rank does the same work)."""
    return ws * units_per_rank / t_max


def build_sets(mesh, n_sets, dtype, seed=0):
    """n_sets independent (problem, x, y) triples with the workload's random inputs."""
    import torch
    from paper_2404_03265_gb300 import Problem
    import synthetic as synth
    X, Y, F = mesh.slots()
    valid = (F & 1) == 1
    info = mesh.info
    Xv, Yv = X[valid], Y[valid]
    u, phi, phit = synth.linearisation(Xv, Yv, info["x_max"], info["y_max"], seed=seed, u_std=1e-3)
    xin = synth.vector(Xv, Yv, seed=seed + 1)
    ns = info["n_slots"]

    def slots(a):
        out = np.zeros((ns,) + a.shape[1:])
        out[valid] = a
        return out

    dev = torch.device("cuda")
    us = torch.tensor(slots(u).T.copy(), device=dev)
    ps, pts = (torch.tensor(slots(a), device=dev) for a in (phi, phit))
    xs = slots(xin)
    sets = []
    eps = 2.0 * info["h_min"]
    for r in range(n_sets):
        pb = Problem(mesh, E=1.0, nu=0.2, Gc=1.0, eps=eps, kappa=1e-10, p=1e-3)
        pb.set_state(us, ps, pts)
        xu = torch.tensor(xs[:, :2].T.copy(), device=dev, dtype=dtype)
        xp = torch.tensor(xs[:, 2], device=dev, dtype=dtype)
        sets.append((pb, xu, xp, torch.empty_like(xu), torch.empty_like(xp)))
    return sets


def time_applies(sets, steps, warmup, ws, per_step=1):
    """Seconds for `steps` timed steps of `per_step` applies each (rotating over
    the input sets), after `warmup` untimed steps; CUDA events on the stream."""
    import torch
    from paper_2404_03265_gb300 import PFF_OP_JACOBIAN
    n = len(sets)
    k = 0
    for i in range(warmup * per_step):
        pb, xu, xp, yu, yp = sets[k % n]
        pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN)
        k += 1
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(steps * per_step):
        pb, xu, xp, yu, yp = sets[k % n]
        pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN)
        k += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def applies_per_step(sets, steps, min_seconds=1.0):
    """Applies per timed step so that `steps` steps take at least min_seconds (at
    least one): the headline's timed region is then long enough for the clock
    sampler whatever --steps is.  From the duration of 50 untimed applies."""
    t = time_applies(sets, 1, 1, 1, per_step=50) / 50
    return max(1, int(np.ceil(min_seconds / (max(steps, 1) * t))))


def time_e2e(mesh, dtype, steps, warmup):
    """Same metric through the C-ABI with HOST buffers.  Every step copies x in
    from pinned host memory, applies, and copies y out to pinned host memory.
    Steps are double-buffered over two device buffer sets and three streams
    (copy in, apply, copy out), so one step's copies overlap its neighbours'
    apply; events order the reuse of each set."""
    import torch
    from paper_2404_03265_gb300 import PFF_OP_JACOBIAN
    sets = build_sets(mesh, 2, dtype, seed=0)
    hxu = sets[0][1].cpu().pin_memory()
    hxp = sets[0][2].cpu().pin_memory()
    hy = [(torch.empty_like(hxu).pin_memory(), torch.empty_like(hxp).pin_memory()) for _ in range(2)]
    s_in, s_ap, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_ap = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    for i in range(2):
        for ev in (ev_in[i], ev_ap[i], ev_out[i]):
            ev.record(s_in)

    def step(k):
        i = k % 2
        pb, xu, xp, yu, yp = sets[i]
        s_in.wait_event(ev_ap[i])            # the apply of step k - 2 has read x_i
        with torch.cuda.stream(s_in):
            xu.copy_(hxu, non_blocking=True)
            xp.copy_(hxp, non_blocking=True)
        ev_in[i].record(s_in)
        s_ap.wait_event(ev_in[i])
        s_ap.wait_event(ev_out[i])           # the copy out of step k - 2 has read y_i
        pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN, stream=s_ap)
        ev_ap[i].record(s_ap)
        s_out.wait_event(ev_ap[i])
        with torch.cuda.stream(s_out):
            hy[i][0].copy_(yu, non_blocking=True)
            hy[i][1].copy_(yp, non_blocking=True)
        ev_out[i].record(s_out)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(steps):
        step(k)
    e1.record(s_out)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    nb = hxu.numel() * hxu.element_size() + hxp.numel() * hxp.element_size()
    nbo = hy[0][0].numel() * hy[0][0].element_size() + hy[0][1].numel() * hy[0][1].element_size()
    # the last step's y, copied out, against a plain apply of the same x on one stream
    pb, xu, xp, yu, yp = sets[0]
    xu.copy_(hxu)
    xp.copy_(hxp)
    yu.zero_()
    yp.zero_()
    pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN)
    torch.cuda.synchronize()
    last = hy[(steps - 1) % 2]
    ref = torch.cat([yu.reshape(-1), yp]).double().cpu()
    got = torch.cat([last[0].reshape(-1), last[1]]).double()
    rel = float((got - ref).norm() / ref.norm())
    if not rel <= 1e-5:
        raise RuntimeError("end-to-end leg: copied-out y differs from a plain apply (relative %.3g)" % rel)
    # reference: the same pinned copies alone, in and out on their own streams
    ci = torch.empty(nb // 4, dtype=torch.float32, device="cuda")
    co = torch.empty(nbo // 4, dtype=torch.float32, device="cuda")
    hi = torch.empty(nb // 4, dtype=torch.float32).pin_memory()
    ho = torch.empty(nbo // 4, dtype=torch.float32).pin_memory()
    rates = {}
    for name, (dst, src, st) in {"h2d": (ci, hi, s_in), "d2h": (ho, co, s_out)}.items():
        for _ in range(3):
            with torch.cuda.stream(st):
                dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(20):
            with torch.cuda.stream(st):
                dst.copy_(src, non_blocking=True)
        z.record(st)
        torch.cuda.synchronize()
        rates[name] = 20 * src.numel() * 4 / (a.elapsed_time(z) / 1e3) / 1e9
    return t, nb, nbo, rel, rates


SOLVE_LOADS = (1e-3, 1.5e-3, 2e-3)


def time_solve(precision, loads=SOLVE_LOADS, matvec=None, coarse="direct"):
    """Load steps of Algorithm 2 on the 1,043,811-DoF band-refined crack mesh
    (16x16 coarse, 5 global, 7 band steps; Q1): line-search Newton / PDAS with
    FP64 GMRES preconditioned by the block V-cycle in the given precision.
    Returns per-step wall time (CUDA events around pff_newton_pdas_step), Newton
    and GMRES counts, TCV, and the final (u, phi) on the host."""
    import torch
    from paper_2404_03265_gb300 import MG, Mesh, Problem, newton_step
    import synthetic as synth
    mesh = Mesh.from_recipe(synth.recipe("solve")).finalize(1)
    info = mesh.info
    ns = info["n_slots"]
    X, Y, F = mesh.slots()
    valid = (F & 1) == 1
    x, y = synth.node_xy(X[valid], Y[valid], info["x_max"], info["y_max"])
    h = info["h_min"]
    po_h = np.ones(ns)
    po_h[valid] = synth.crack_phi_old(x, y, h)
    m = synth.material(h_min=h)
    pb = Problem(mesh, E=m["E"], nu=m["nu"], Gc=m["Gc"], eps=m["eps"], kappa=m["kappa"], p=loads[0], c=m["c"])
    mg = MG(pb, precision, coarse=coarse)
    dev = torch.device("cuda")
    u = torch.zeros((2, ns), dtype=torch.float64, device=dev)
    phi = torch.tensor(po_h, device=dev)
    phi_old = phi.clone()
    act = torch.zeros(ns, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    steps = []
    for p in loads:
        pb.set_pressure(p)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        r = newton_step(pb, mg, u, phi, phi_old, act, check=False, matvec=precision if matvec is None else matvec)
        e1.record(s)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        tcv = pb.tcv(u, phi)
        ph_h = phi.cpu().numpy()[valid]
        half = float(np.abs(x[ph_h < 0.5]).max()) if (ph_h < 0.5).any() else 0.0
        eprime = m["E"] / (1.0 - m["nu"] ** 2)
        tcv_ref = 2.0 * np.pi * p * 1.0 ** 2 / eprime
        k = max(r["newton"], 1)
        steps.append({"p": p, "s": t, "newton": r["newton"], "gmres_mean": r["gmres_total"] / k,
                      "gmres_max": r["gmres_max"], "gmres": r["gmres"], "linesearch_failures": r["linesearch_failures"],
                      "s_mg_setup": r["time_mg_setup"], "s_gmres": r["time_gmres"],
                      "s_gmres_apply": r["time_gmres_apply"], "s_gmres_vcycle": r["time_gmres_vcycle"],
                      "s_gmres_orth": r["time_gmres_orth"],
                      "active": r["active_size"], "converged": bool(r["converged"]), "status": r["status"],
                      "residual": r["residual"], "tcv": tcv, "tcv_rel_err": abs(tcv - tcv_ref) / tcv_ref,
                      "crack_half_length": half})
        phi_old.copy_(phi)
    uh = u.cpu().numpy()[:, valid]
    ph = phi.cpu().numpy()[valid]
    # COD profile of the last step (Sec. 4) beside the closed forms: the paper prints
    # 2 p l0 / E' sqrt(1 - x^2 / l0^2); the one consistent with TCV_ref is twice that
    xs = np.linspace(-0.9, 0.9, 19)
    cod = pb.cod(u, phi, xs)
    p_last = loads[-1]
    base = p_last / (m["E"] / (1.0 - m["nu"] ** 2)) * np.sqrt(1.0 - xs ** 2)
    return {"dofs": 3 * info["n_nodes"], "steps": steps,
            "s_per_load_step": float(np.mean([st["s"] for st in steps])),
            "cod": {"x": [float(v) for v in xs], "cod": [float(v) for v in cod],
                    "rel_err_vs_4pl0_over_Eprime": float(np.max(np.abs(cod - 4.0 * base) / (4.0 * base))),
                    "rel_err_vs_2pl0_over_Eprime": float(np.max(np.abs(cod - 2.0 * base) / (2.0 * base)))}}, uh, ph


LARGE_LOADS = (1e-3, 1.5e-3, 2e-3, 2.5e-3, 3e-3)


def time_large(loads=LARGE_LOADS):
    """The largest workload: Q2 u and phi on the band-refined crack mesh (14x14
    coarse, 6 global, 9 band steps; 16,515,855 DoFs), five load steps of
    Algorithm 2 with the FP32 V-cycle, then the checkpointed adjoint gradient of
    the final TCV with respect to every step's pressure and G_c.  Reports seconds
    per load step, the adjoint's seconds, and the device memory in use."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Mesh, Problem, newton_step, tcv_adjoint_steps
    import synthetic as synth
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    mesh = Mesh.from_recipe(synth.recipe("large")).finalize(2)
    info = mesh.info
    ns = info["n_slots"]
    X, Y, F = mesh.slots()
    valid = (F & 1) == 1
    x, y = synth.node_xy(X[valid], Y[valid], info["x_max"], info["y_max"])
    h = info["h_min"]
    po_h = np.ones(ns)
    po_h[valid] = synth.crack_phi_old(x, y, h)
    m = synth.material(h_min=h)
    pb = Problem(mesh, E=m["E"], nu=m["nu"], Gc=m["Gc"], eps=m["eps"], kappa=m["kappa"], p=loads[0], c=m["c"])
    mg = MG(pb, PFF_F32)
    dev = torch.device("cuda")
    us = [torch.zeros((2, ns), dtype=torch.float64, device=dev)]
    phis = [torch.tensor(po_h, device=dev)]
    acts = []
    act = torch.zeros(ns, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    steps = []
    eprime = m["E"] / (1.0 - m["nu"] ** 2)
    for p in loads:
        pb.set_pressure(p)
        u = us[-1].clone()
        phi = phis[-1].clone()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        r = newton_step(pb, mg, u, phi, phis[-1], act, check=False, matvec=PFF_F32)
        e1.record(s)
        torch.cuda.synchronize()
        tcv = pb.tcv(u, phi)
        k = max(r["newton"], 1)
        steps.append({"p": p, "s": e0.elapsed_time(e1) / 1e3, "newton": r["newton"],
                      "gmres_mean": r["gmres_total"] / k, "gmres_max": r["gmres_max"], "active": r["active_size"],
                      "s_mg_setup": r["time_mg_setup"], "s_gmres": r["time_gmres"],
                      "s_gmres_apply": r["time_gmres_apply"], "s_gmres_vcycle": r["time_gmres_vcycle"],
                      "s_gmres_orth": r["time_gmres_orth"],
                      "converged": bool(r["converged"]), "status": r["status"], "tcv": tcv,
                      "tcv_rel_err": abs(tcv - 2.0 * np.pi * p / eprime) / (2.0 * np.pi * p / eprime)})
        us.append(u)
        phis.append(phi)
        acts.append(act.clone())
        if not r["converged"]:
            break
    out = {"workload": "large: Q2 u and phi, 14x14 coarse on (-10,10)^2, 6 global + 9 band refinements toward "
                       "the crack, %d DoFs, %d levels; Sneddon crack, l = 2 h_min; p = %s; FP32 V-cycle, FP64 "
                       "Newton/GMRES (Jacobian applies inside GMRES in FP32)" % (3 * info["n_nodes"], info["finest_level"] + 1,
                                          ", ".join("%g" % p for p in loads)),
           "dofs": 3 * info["n_nodes"], "steps": steps,
           "s_per_load_step": float(np.mean([st["s"] for st in steps]))}
    if len(acts) == len(loads):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        g = tcv_adjoint_steps(pb, mg, us, phis, acts, list(loads), rtol=1e-8, check=False)
        e1.record(s)
        torch.cuda.synchronize()
        out["adjoint"] = {"s": e0.elapsed_time(e1) / 1e3, "dJ_dp": [float(v) for v in g["p"]], "dJ_dGc": g["Gc"],
                          "gmres_total": g["gmres_total"], "gmres_max": g["gmres_max"],
                          "converged": g["converged"], "status": g["status"]}
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    out["device_bytes_in_use"] = int(free0 - free1)
    out["device_bytes_total"] = int(total)
    return out


def apply_workload_config(dofs):
    """The apply workload's description, shared by both arms."""
    return {"workload": "apply: 16x16 coarse on (-10,10)^2, 6 global + 2 box refinements (|x|<=2,|y|<=1), "
                        "Q1 u and phi, %d DoFs; phi~U[0,1], u~N(0,1e-3), x~N(0,1), seed 0" % dofs,
            "fe_degree": 1, "dofs": dofs, "op": "constrained Jacobian y = G~ x"}


class OracleApplySample:
    """The oracle as it stands, on a bounded sample of the apply workload: its FP64
    cell-by-cell assembly of the Jacobian G (Sec. 3.1) over m leaf cells, then the
    constrained operator G~ = M_f C^T G C M_f + I_fixed applied to the bench's x
    (no active set), restricted to what those cells touch: the rows d of C at the
    cells' vertices, G on d x d, and C^T back onto the DoFs P that the rows d
    constrain to (fixed rows of P: identity).  The cells of step k are the k-th
    run of m cells of one seeded permutation of all leaf cells; m cells stand for
    m / n_cells of one full apply.  The mesh, the linearisation, C and M_f x are
    built once, outside any timing, as the GPU arm's mesh and state are."""

    def __init__(self):
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from oracle import operators as ops
        from oracle.mesh import LeafMesh, build_recipe
        import synthetic as synth
        self.ops = ops
        om = LeafMesh(build_recipe(synth.recipe(WORKLOAD)), 1)
        u, phi, phit = synth.linearisation(om.X, om.Y, om.Xmax, om.Ymax, seed=0, u_std=1e-3)
        x = synth.vector(om.X, om.Y, seed=1)
        self.v = np.concatenate([x[:, 0], x[:, 1], x[:, 2]])
        self.mat = ops.Material(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * om.h_min_diag(), kappa=1e-10, p=1e-3)
        self.st = ops.State(om, u, phi, phit)
        active = np.zeros(om.nn, bool)
        self.fr = ops.free_dofs(om, active).astype(np.float64)
        self.fx = ops.fixed_dofs(om, active).astype(np.float64)
        self.C = ops.C3(om)
        self.om = om
        self.n_cells = len(om.cells)
        self.dofs = 3 * om.nn
        self.frv = self.fr * self.v
        self.xbuf = np.zeros(self.dofs)
        self.perm = np.random.Generator(np.random.PCG64(7)).permutation(self.n_cells)
        self.next = 0

    def step(self, m):
        """One sampled apply of m cells: (P, the contributions of those cells to G~x on P)."""
        if self.next + m > self.n_cells:
            self.next = 0
        cells = np.sort(self.perm[self.next:self.next + m])
        self.next += m
        G = self.ops.assemble_jacobian(self.om, self.mat, self.st, cell_idx=cells)
        nn = self.om.nn
        cn = self.om.cell_nodes[cells].ravel()
        d = np.unique(np.concatenate([cn, cn + nn, cn + 2 * nn]))
        Cd = self.C[d]
        self.xbuf[d] = Cd @ self.frv                      # C M_f x on d
        zd = G[d] @ self.xbuf                             # G is zero outside d x d
        self.xbuf[d] = 0.0
        P, inv = np.unique(Cd.indices, return_inverse=True)
        ctz = np.bincount(inv, weights=Cd.data * np.repeat(zd, np.diff(Cd.indptr)), minlength=len(P))
        return P, self.fr[P] * ctz + self.fx[P] * self.v[P]

    def dofs_per_step(self, m):
        return self.dofs * m / self.n_cells


def oracle_threads():
    cores = 1
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        cores = max([d.get("num_threads", 1) for d in info] + [1])
    except Exception:
        pass
    return cores


def cpu_baseline(budget_s=12.0, cells_per_step=20000):
    """The oracle (OracleApplySample) on host cores: steps of cells_per_step sampled
    leaf cells of the apply workload, repeated for about budget_s seconds."""
    o = OracleApplySample()
    m = min(cells_per_step, o.n_cells)
    o.step(m)   # untimed warm-up
    reps = 0
    t0 = time.perf_counter()
    while True:
        o.step(m)
        reps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": o.dofs_per_step(m) * reps / dt / 1e9, "unit": "GDoF/s", "cores": oracle_threads(),
            "kind": "oracle",
            "sample": "oracle G~x (FP64 cell-by-cell assembly, then M_f C^T G C M_f + I_fixed) on %d sampled leaf "
                      "cells per step of the %d-DoF apply workload (%d cells), each step counted as that fraction "
                      "of one apply; %d steps in %.1f s; os.cpu_count()=%d"
                      % (m, o.dofs, o.n_cells, reps, dt, os.cpu_count() or 0)}


def run_reference(args):
    """The reference arm: the oracle on the apply workload, exactly W untimed and K
    timed steps.  Each step is one OracleApplySample step whose cell count is set
    from two calibration steps so that the W + K steps take about --ref-seconds."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = OracleApplySample()
    o.step(1000)   # first call: one-time costs stay out of the calibration
    probes = []
    for m in (1000, 10000):
        t0 = time.perf_counter()
        o.step(m)
        probes.append((m, time.perf_counter() - t0))
    # t(m) = a + b m; b is kept at least half the mean cost per cell of the larger
    # probe, so that a noisy fit cannot inflate the step size
    b = max((probes[1][1] - probes[0][1]) / (probes[1][0] - probes[0][0]), 0.5 * probes[1][1] / probes[1][0])
    a = max(probes[0][1] - b * probes[0][0], 0.0)
    k, w = max(args.steps, 1), max(args.warmup, 0)
    tau = max(args.ref_seconds, 0.0) / (k + w)
    m = int(min(max((tau - a) / b, 100), o.n_cells))
    for _ in range(w):
        o.step(m)
    t0 = time.perf_counter()
    for _ in range(k):
        o.step(m)
    dt = time.perf_counter() - t0
    value = o.dofs_per_step(m) * k / dt / 1e9
    cb = {"value": value, "unit": "GDoF/s", "cores": oracle_threads(), "kind": "oracle",
          "sample": "oracle G~x (FP64 cell-by-cell assembly, then M_f C^T G C M_f + I_fixed) on %d sampled leaf cells "
                    "per step of the %d-DoF apply workload (%d cells), each step counted as that fraction of one "
                    "apply; %d timed steps in %.1f s after %d warm-up steps; os.cpu_count()=%d"
                    % (m, o.dofs, o.n_cells, k, dt, w, os.cpu_count() or 0)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws,
            "steps": k, "warmup": w, "ms_per_step": 1e3 * dt / k, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(apply_workload_config(o.dofs), l2="host", parallelism="host cores"),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the apply kernels' sources (the key under
    which the committed ncu summaries record their counters)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("apply.cu", "apply_q2.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2404_03265_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled(name, key):
    """Counter `key` ("key: value" line) of the committed ncu summary profiles/<name>,
    or None when the kernel sources have changed since it was captured."""
    import re
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        text = f.read()
    m_hash = re.search(r"first 16 hex\): `([0-9a-f]{16})`", text)
    m_val = re.search(r"^%s: ([0-9.eE+-]+)" % re.escape(key), text, re.M)
    if not m_hash or not m_val or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_val.group(1))


def profiled_traffic():
    """DRAM bytes (read + write) per launch of the FP32 apply kernel from the committed
    ncu summary, or None when the kernel source has changed since it was captured."""
    v = profiled("apply_q1_f32_apply_workload_ncu.md", "bytes_per_launch")
    return None if v is None else int(v)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the load-step timing leg")
    ap.add_argument("--large", action="store_true",
                    help="add the 16.5M-DoF Q2 five-load-step solve and its checkpointed adjoint")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="reference arm: the W + K oracle steps are sized to take about this long")
    ap.add_argument("--profile-apply", action="store_true",
                    help="a small case for ncu: one input set of the apply workload, three FP32 and one FP64 applies "
                         "(Q1), then one FP32 Q2 apply; prints nothing but a short line")
    ap.add_argument("--solve-only", action="store_true",
                    help="run only the first load step of the solve leg (FP32 V-cycle, FP32 GMRES applies) and "
                         "print its record: a small case for profiling the set-up, V-cycle and GMRES kernels")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_apply:
        import torch
        from paper_2404_03265_gb300 import Mesh
        import synthetic as synth
        mesh = Mesh.from_recipe(synth.recipe(WORKLOAD)).finalize(1)
        sets = build_sets(mesh, 1, torch.float32, seed=0)
        time_applies(sets, 3, 0, 1)
        sets = build_sets(mesh, 1, torch.float64, seed=0)
        time_applies(sets, 1, 0, 1)
        del sets
        mesh2 = Mesh.from_recipe(synth.recipe(WORKLOAD)).finalize(2)
        time_applies(build_sets(mesh2, 1, torch.float32, seed=0), 1, 0, 1)
        torch.cuda.synchronize()
        print("profile-apply done")
        return
    if args.solve_only:
        from paper_2404_03265_gb300 import PFF_F32
        r, _, _ = time_solve(PFF_F32, loads=SOLVE_LOADS[:1])
        print(json.dumps({"solve_only": r}))
        return
    args.warmup = max(args.warmup, 3)

    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_2404_03265_gb300 import Mesh
    import synthetic as synth
    from paper_2404_03265_gb300 import _lib

    mesh = Mesh.from_recipe(synth.recipe(WORKLOAD)).finalize(1)
    info = mesh.info
    dofs = 3 * info["n_nodes"]
    n_slots = info["n_slots"]
    per_set_bytes = n_slots * (16 + 12 + 12)
    n_sets = max(2, int(np.ceil(2.2 * L2_BYTES / per_set_bytes)))
    sets = build_sets(mesh, n_sets, torch.float32, seed=0)

    per_step = applies_per_step(sets, args.steps)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    t = time_applies(sets, args.steps, args.warmup, ws, per_step=per_step)
    clocks = sampler.stop() if sampler else None
    t = max_over_ranks(ws, t)
    value = whole_job_rate(ws, dofs * args.steps * per_step, t) / 1e9
    ms = 1e3 * t / args.steps
    t_apply = t / (args.steps * per_step)
    del sets

    # FP64 apply (FP64-ALU bound on GB300), fewer steps
    sets64 = build_sets(mesh, max(2, n_sets // 2), torch.float64, seed=0)
    k64 = max(5, args.steps // 10)
    t64 = time_applies(sets64, k64, 3, 1)
    g64 = dofs * k64 / t64 / 1e9
    del sets64
    # its arithmetic roof: FP64 flops of the cell-loop kernel per launch (ncu DFMA, DADD,
    # DMUL counts of the committed capture) against the measured FP64 FMA rate
    f64_flops = profiled("apply_q1_f64_apply_workload_flops.md", "fp64_flops_per_launch")
    f64 = {"value": g64, "unit": "GDoF/s", "steps": k64, "us_per_apply": 1e6 * t64 / k64,
           "hbm_frac": info["n_nodes"] * 80 / (t64 / k64) / 1e9 / load_peaks()[0],
           "fp64_flops_per_launch": f64_flops,
           "alu_peak_tflops": FP64_PEAK_TFLOPS,
           "alu_frac": None if f64_flops is None else f64_flops / (t64 / k64) / 1e12 / FP64_PEAK_TFLOPS,
           "bound": "alu (FP64 FMA rate)"}

    # Q2 u and phi on the same mesh (16,368,207 DoFs): FP32 and FP64 applies
    mesh2 = Mesh.from_recipe(synth.recipe(WORKLOAD)).finalize(2)
    info2 = mesh2.info
    dofs2 = 3 * info2["n_nodes"]
    per_set2 = info2["n_slots"] * (16 + 12 + 12)
    sets2 = build_sets(mesh2, max(2, int(np.ceil(2.2 * L2_BYTES / per_set2))), torch.float32, seed=0)
    k2 = max(20, args.steps // 10)
    t2 = time_applies(sets2, k2, 3, 1)
    del sets2
    sets2 = build_sets(mesh2, 2, torch.float64, seed=0)
    k2d = max(5, args.steps // 100)
    t2d = time_applies(sets2, k2d, 3, 1)
    del sets2
    q2 = {"dofs": dofs2, "nodes": info2["n_nodes"],
          "f32": {"value": dofs2 * k2 / t2 / 1e9, "unit": "GDoF/s", "steps": k2,
                  "us_per_apply": 1e6 * t2 / k2},
          "f64": {"value": dofs2 * k2d / t2d / 1e9, "unit": "GDoF/s", "steps": k2d,
                  "us_per_apply": 1e6 * t2d / k2d}}

    te, bi, bo, e2e_rel, copy_rates = time_e2e(mesh, torch.float32, max(10, args.steps // 4), 3)
    e2e = whole_job_rate(ws, dofs * max(10, args.steps // 4), max_over_ranks(ws, te)) / 1e9

    if rank != 0:
        return
    hbm, peak_kind = load_peaks()
    alg_bytes = info["n_nodes"] * 10 * 4  # x (3), y (3), linearisation (4) per node, FP32
    achieved = alg_bytes / t_apply / 1e9
    q2["f32"]["hbm_frac"] = info2["n_nodes"] * 40 / (t2 / k2) / 1e9 / hbm
    q2["f64"]["hbm_frac"] = info2["n_nodes"] * 80 / (t2d / k2d) / 1e9 / hbm
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(apply_workload_config(dofs),
                       l2="%d rotating input sets of %.0f MB (> L2 129 MB)" % (n_sets, per_set_bytes / 1e6),
                       step="%d applies of G~x, each on the next of the rotating input sets (the timed region is "
                            "at least 1 s whatever --steps is)" % per_step,
                       applies_per_step=per_step,
                       parallelism="replicas" if ws > 1 else "single GPU"),
        "us_per_apply": 1e6 * t_apply,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "note": "achieved = 40 B/node x nodes per launch / avg pff_apply duration (hanging-node "
                             "pre-pass, cell-loop kernel and interface fix-up kernel, as one call)"},
        "f64_apply": f64,
        "q2_apply": q2,
        "e2e": {"value": e2e, "unit": "GDoF/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "verified_rel_l2": e2e_rel, "pinned_copy_gbs": copy_rates,
                "note": "steps double-buffered over three streams (copy in, apply, copy out); the last step's "
                        "copied-out y equals a plain apply of the same x (verified_rel_l2); pinned_copy_gbs: the "
                        "same copies alone, the bound of this leg"},
        "gpu_launches": 3 * args.steps * per_step,
        "clocks": clocks,
    }
    if not args.no_solve:
        from paper_2404_03265_gb300 import PFF_F32, PFF_F64
        r32, u32, p32 = time_solve(PFF_F32)
        r32d, u32d, p32d = time_solve(PFF_F32, matvec=PFF_F64)
        r32c, u32c, p32c = time_solve(PFF_F32, matvec=PFF_F64, coarse="chebyshev")
        r64, u64, p64 = time_solve(PFF_F64)
        line["solve"] = {
            "workload": "solve: 16x16 coarse on (-10,10)^2, 5 global + 7 band refinements toward the crack "
                        "(|x|<=1+2h_min, |y|<=2h_min), Q1, %d DoFs; Sneddon crack, E=1, nu=0.2, G_c=1, "
                        "l=2h_min, kappa=1e-10, c=1e4; p = %s" % (r32["dofs"], ", ".join("%g" % p for p in SOLVE_LOADS)),
            "unit": "s/load step", "newton_tol": 1e-8, "gmres_rtol": 1e-6,
            "fp32_mg": r32, "fp32_mg_fp64_matvec": r32d, "fp32_mg_chebyshev_coarse": r32c, "fp64_mg": r64,
            "note": "fp32_mg: V-cycle and the Jacobian applies inside GMRES in FP32 (Krylov basis, "
                    "orthogonalisation, Givens, residual, line search, active set and coarse solve in FP64; the "
                    "lambda_max CG in FP64 with FP32 level applies); fp32_mg_fp64_matvec: FP32 V-cycle only; "
                    "fp32_mg_chebyshev_coarse: the same with the "
                    "Chebyshev-Jacobi coarse solver instead of the direct one; fp64_mg: everything in FP64. "
                    "Per step: s_mg_setup and s_gmres are host wall seconds; s_gmres_apply, s_gmres_vcycle and "
                    "s_gmres_orth are device seconds (CUDA events) of the operator applies, block V-cycles and "
                    "Gram-Schmidt inside the GMRES iterations; s - s_mg_setup - s_gmres is residuals, active "
                    "sets and line search",
            "speedup_fp32_mg": r64["s_per_load_step"] / r32["s_per_load_step"],
            "fp32_vs_fp64_rel_l2": {"u": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
                                    "phi": float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))},
            "fp32_fp64_matvec_vs_fp64_rel_l2": {"u": float(np.linalg.norm(u32d - u64) / np.linalg.norm(u64)),
                                                "phi": float(np.linalg.norm(p32d - p64) / np.linalg.norm(p64))},
        }
    if args.large:
        line["large"] = time_large()
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
