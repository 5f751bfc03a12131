"""Pins of the oracle multigrid (oracle/mg.py): Chebyshev polynomial, eigenvalue
estimate bounds, and the local-smoothing V-cycle against an independent
multiplicative subspace correction."""
import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import chebyshev as C

from oracle import mg
from oracle import operators as ops
from oracle.mesh import LeafMesh, build_recipe
import synthetic as synth


def test_chebyshev_error_polynomial():
    """For D^-1 A = diag(lam): x_m = (1 - T_m((theta - lam)/delta) / T_m(sigma)) * x_true."""
    lam = np.linspace(0.01, 1.5, 40)
    lmax = 1.3
    for degree in (1, 2, 3, 5):
        a, b = 0.08 * lmax, 1.2 * lmax
        theta, delta = (a + b) / 2, (b - a) / 2
        xs = np.random.default_rng(1).normal(size=lam.size)
        x = mg.chebyshev(lambda v: lam * v, np.ones_like(lam), lam * xs, lmax, degree)
        Tm = C.Chebyshev.basis(degree)
        factor = Tm((theta - lam) / delta) / Tm(theta / delta)
        assert np.allclose(x, (1 - factor) * xs, rtol=1e-12, atol=1e-13)


def test_splitmix64_known_values():
    # SplitMix64 of 0 and 1 (published reference outputs of the finaliser with seed increment)
    assert mg.splitmix64(0) == 0xE220A8397B1DCDAF
    assert mg.splitmix64(1) == 0x910A2DEC89025CC1


def build(name, k, active_frac=0.0, u_std=0.0, phit_one=True, seed=3):
    leaf = LeafMesh(build_recipe(synth.recipe(name)), k)
    mat = ops.Material(E=1.0, nu=0.2, Gc=1.0, eps=0.5, kappa=1e-10, p=1e-3)
    u, phi, phit = synth.linearisation(leaf.X, leaf.Y, leaf.Xmax, leaf.Ymax, seed=seed, u_std=max(u_std, 1e-300))
    if u_std == 0.0:
        u[:] = 0.0
    if phit_one:
        phit[:] = 1.0
    rng = np.random.default_rng(seed)
    active = (rng.uniform(size=leaf.nn) < active_frac) & ~leaf.is_hanging
    return leaf, mat, u, phi, phit, active


@pytest.mark.parametrize("k", [1, 2])
def test_lambda_estimate_bounds(k):
    leaf, mat, u, phi, phit, active = build("tiny", k, u_std=1e-1, phit_one=False)
    M = mg.MG(leaf, mat, u, phi, phit, active)
    for name in ("uu", "pp"):
        for l, blk in enumerate(M.B[name][1:], start=1):
            I = np.nonzero(blk.interior)[0]
            if len(I) < 2:
                continue
            A = blk.A[I][:, I].toarray()
            D = np.diag(np.diag(A))
            true = sla.eigh(A, D, eigvals_only=True).max()
            assert blk.lam <= true * (1 + 1e-10)
            assert blk.lam >= 0.9 * true


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name,frac", [("tiny", 0.0), ("small", 0.0), ("band4_2_4", 0.0)])
def test_vcycle_equals_subspace_correction(k, name, frac):
    """Constant coefficients (u = 0, phi~ = 1): level operators are Galerkin and the
    local-smoothing V-cycle equals the multiplicative subspace correction computed
    from the leaf matrix and the level-to-leaf interpolations."""
    leaf, mat, u, phi, phit, active = build(name, k, active_frac=frac)
    M = mg.MG(leaf, mat, u, phi, phit, active)
    st = ops.State(leaf, u, phi, phit)
    Gt = ops.constrained_operator(leaf, ops.assemble_jacobian(leaf, mat, st), active)
    nn = leaf.nn
    rng = np.random.default_rng(7)
    for blk, sl, free in (("uu", slice(0, 2 * nn), np.tile(~leaf.dirichlet & ~leaf.is_hanging, 2)),
                          ("pp", slice(2 * nn, 3 * nn), ~active & ~leaf.is_hanging)):
        A = Gt[sl, sl]
        r = rng.normal(size=A.shape[0])
        z = M.vcycle(blk, r)
        e = M.msc(blk, A, r)
        err = np.abs(z[free] - e[free]).max() / np.abs(e[free]).max()
        assert err < 1e-11, (blk, err)


@pytest.mark.parametrize("k", [1, 2])
def test_vcycle_symmetric_and_contracting(k):
    leaf, mat, u, phi, phit, active = build("small", k, active_frac=0.05, u_std=1e-3, phit_one=False)
    M = mg.MG(leaf, mat, u, phi, phit, active)
    st = ops.State(leaf, u, phi, phit)
    Gt = ops.constrained_operator(leaf, ops.assemble_jacobian(leaf, mat, st), active)
    nn = leaf.nn
    rng = np.random.default_rng(2)
    for blk, sl, free in (("uu", slice(0, 2 * nn), np.tile(~leaf.dirichlet & ~leaf.is_hanging, 2)),
                          ("pp", slice(2 * nn, 3 * nn), ~active & ~leaf.is_hanging)):
        A = Gt[sl, sl]
        a = rng.normal(size=A.shape[0]) * free
        b = rng.normal(size=A.shape[0]) * free
        za, zb = M.vcycle(blk, a) * free, M.vcycle(blk, b) * free
        assert abs(a @ zb - b @ za) < 1e-10 * abs(a @ zb)


@pytest.mark.parametrize("k", [1, 2])
def test_vcycle_contracts(k):
    """Stationary iteration x <- x + MG(f - A x) converges fast (no active set: a
    scattered random active set makes coarse levels active by the pessimistic
    level rule, which is the paper's rule, not a defect)."""
    leaf, mat, u, phi, phit, active = build("small", k, active_frac=0.0, u_std=1e-3, phit_one=True)
    M = mg.MG(leaf, mat, u, phi, phit, active)
    st = ops.State(leaf, u, phi, phit)
    Gt = ops.constrained_operator(leaf, ops.assemble_jacobian(leaf, mat, st), active)
    nn = leaf.nn
    rng = np.random.default_rng(2)
    for blk, sl, free in (("uu", slice(0, 2 * nn), np.tile(~leaf.dirichlet & ~leaf.is_hanging, 2)),
                          ("pp", slice(2 * nn, 3 * nn), ~active & ~leaf.is_hanging)):
        A = Gt[sl, sl]
        f = rng.normal(size=A.shape[0]) * free
        x = np.zeros_like(f)
        res0 = np.linalg.norm(f)
        for _ in range(8):
            x = x + M.vcycle(blk, f - A @ x) * free
        assert np.linalg.norm((f - A @ x) * free) < 0.05 * res0


@pytest.mark.parametrize("k", [1, 2])
def test_preconditioner_reaches_every_free_dof(k):
    """With an active set the block V-cycle stays nonsingular on the free DoFs:
    MG(A e) reproduces e's support (no free DoF is left uncorrected)."""
    leaf, mat, u, phi, phit, active = build("band4_2_4", k, active_frac=0.3, u_std=1e-3)
    M = mg.MG(leaf, mat, u, phi, phit, active)
    st = ops.State(leaf, u, phi, phit)
    Gt = ops.constrained_operator(leaf, ops.assemble_jacobian(leaf, mat, st), active)
    nn = leaf.nn
    A = Gt[2 * nn:, 2 * nn:].toarray()
    free = np.nonzero(~active & ~leaf.is_hanging)[0]
    # P^-1 A restricted to free DoFs has no zero rows and is well conditioned
    PA = np.column_stack([M.vcycle("pp", A[:, j]) for j in free])[free]
    sv = np.linalg.svd(PA, compute_uv=False)
    assert sv.min() > 1e-3 * sv.max()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("frac", [0.0, 0.05])
def test_coarse_chebyshev(k, frac):
    """The Chebyshev coarse solver of Sec. 3.2: its level-0 error obeys the exact
    Chebyshev bound over the true spectrum of D^-1 A_0, its interval brackets the
    Ritz values, and the V-cycle with it stays symmetric."""
    leaf, mat, u, phi, phit, active = build("small", k, active_frac=frac, u_std=1e-3, phit_one=False)
    M = mg.MG(leaf, mat, u, phi, phit, active, coarse="chebyshev")
    rng = np.random.default_rng(5)
    for blk in ("uu", "pp"):
        b0 = M.B[blk][0]
        a, b, m = b0.cheb
        if not b0.interior.any():   # every level-0 DoF fixed: nothing to solve
            assert m == 0
            continue
        assert 0 < a < b and m >= 1
        I = np.nonzero(b0.interior)[0]
        A0 = b0.A[I][:, I].toarray()
        Dh = np.sqrt(b0.dinv[I])
        lam = np.linalg.eigvalsh(Dh[:, None] * A0 * Dh[None, :])    # spectrum of D^-1 A_0
        d = np.zeros(b0.A.shape[0])
        d[I] = rng.normal(size=len(I))
        x_direct = np.zeros_like(d)
        x_direct[I] = np.linalg.solve(A0, d[I])
        x_cheb = mg.chebyshev(b0.apply, b0.dinv, d, 1.0, m, a, b)
        e = x_cheb - x_direct
        theta, delta = 0.5 * (b + a), 0.5 * (b - a)
        Tm = lambda t: np.cosh(m * np.arccosh(t)) if t >= 1 else (np.cos(m * np.arccos(t)) if t > -1 else
                                                                   (-1) ** m * np.cosh(m * np.arccosh(-t)))
        factor = max(abs(Tm((theta - l) / delta)) for l in lam) / Tm(theta / delta)
        eA = np.sqrt(e[I] @ A0 @ e[I])
        xA = np.sqrt(x_direct[I] @ A0 @ x_direct[I])
        assert eA <= factor * xA * (1 + 1e-9), (blk, eA / xA, factor)
    nn = leaf.nn
    for blk, n, free in (("uu", 2 * nn, np.tile(~leaf.dirichlet & ~leaf.is_hanging, 2)),
                         ("pp", nn, ~active & ~leaf.is_hanging)):
        x = rng.normal(size=n) * free
        y = rng.normal(size=n) * free
        zx, zy = M.vcycle(blk, x) * free, M.vcycle(blk, y) * free
        assert abs(x @ zy - y @ zx) < 1e-10 * abs(x @ zy)


@pytest.mark.parametrize("k", [1, 2])
def test_global_level_operators_are_uniform_mesh_jacobians(k):
    """On each globally refined level l the level blocks (the cells of level l with
    the linearisation injected from the leaf nodes) equal the u-u and phi-phi
    Jacobian blocks of the uniform mesh with l global refinements, built on its own
    (own node numbering and coordinates) with the same nodal values at the same
    points: variable-coefficient rediscretisation on each level, as the V-cycle of
    Sec. 3.2 uses, and not a Galerkin product."""
    rec = dict(domain=synth.DOMAIN, ncx=2, ncy=2, n_global=2, steps=[("box", -2.0, 2.0, -1.0, 1.0)] * 2)
    leaf = LeafMesh(build_recipe(rec), k)
    u, phi, phit = synth.linearisation(leaf.X, leaf.Y, leaf.Xmax, leaf.Ymax, seed=3, u_std=0.2)
    mat = ops.Material(E=1.0, nu=0.2, Gc=1.3, eps=0.5, kappa=1e-3, p=0.3)
    M = mg.MG(leaf, mat, u, phi, phit, np.zeros(leaf.nn, bool))
    uf = np.stack([leaf.C @ u[:, 0], leaf.C @ u[:, 1]], 1)
    pf, ptf = leaf.C @ phi, leaf.C @ phit
    for l in range(rec["n_global"] + 1):
        uni = LeafMesh(build_recipe(dict(rec, n_global=l, steps=[])), k)
        assert not uni.is_hanging.any()
        s = 1 << (leaf.Lf - l)
        key = (uni.Y * s) * (leaf.Xmax + 1) + uni.X * s
        ln = np.searchsorted(leaf.key, key)
        assert np.array_equal(leaf.key[ln], key)
        G = ops.assemble_jacobian(uni, mat, ops.State(uni, uf[ln], pf[ln], ptf[ln])).toarray()
        lm = M.levels[l]
        li = lm.find(uni.X * s, uni.Y * s)
        assert lm.nn == uni.nn and np.array_equal(np.sort(li), np.arange(lm.nn))
        n = uni.nn
        pu = np.concatenate([li, lm.nn + li])
        Auu = M.B["uu"][l].A.toarray()[np.ix_(pu, pu)]
        App = M.B["pp"][l].A.toarray()[np.ix_(li, li)]
        for got, ref in ((Auu, G[:2 * n, :2 * n]), (App, G[2 * n:, 2 * n:])):
            assert np.abs(ref).max() > 0
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("k", [1, 2])
def test_local_level_operators_are_submesh_jacobians(k):
    """Each locally refined level's blocks equal the Jacobian blocks of a uniform mesh
    built on its own over the level's bounding rectangle (cells of the same size, no
    hanging nodes, own node numbering), assembled over the cells of that level only,
    with the same nodal values: the level operator of local smoothing is the
    rediscretisation on the level's own cells, with the refinement edge left open."""
    rec = dict(domain=synth.DOMAIN, ncx=4, ncy=4, n_global=2, steps=[("box", -2.0, 2.0, -1.0, 1.0)] * 3)
    leaf = LeafMesh(build_recipe(rec), k)
    assert leaf.Lf == 5
    u, phi, phit = synth.linearisation(leaf.X, leaf.Y, leaf.Xmax, leaf.Ymax, seed=4, u_std=0.2)
    mat = ops.Material(E=1.0, nu=0.3, Gc=0.7, eps=0.4, kappa=1e-2, p=0.2)
    M = mg.MG(leaf, mat, u, phi, phit, np.zeros(leaf.nn, bool))
    uf = np.stack([leaf.C @ u[:, 0], leaf.C @ u[:, 1]], 1)
    pf, ptf = leaf.C @ phi, leaf.C @ phit
    x0, x1, y0, y1 = synth.DOMAIN
    not_rect = 0
    for l in range(rec["n_global"] + 1, leaf.Lf + 1):
        lm = M.levels[l]
        i, j = lm.cells[:, 1], lm.cells[:, 2]
        i0, i1, j0, j1 = i.min(), i.max(), j.min(), j.max()
        not_rect += len(lm.cells) < (i1 - i0 + 1) * (j1 - j0 + 1)
        hx = (x1 - x0) / (rec["ncx"] << l)
        hy = (y1 - y0) / (rec["ncy"] << l)
        sub = (x0 + i0 * hx, x0 + (i1 + 1) * hx, y0 + j0 * hy, y0 + (j1 + 1) * hy)
        uni = LeafMesh(build_recipe(dict(domain=sub, ncx=int(i1 - i0 + 1), ncy=int(j1 - j0 + 1), n_global=0,
                                         steps=[])), k)
        assert not uni.is_hanging.any()
        ucell = {(int(a), int(b)): c for c, (_, a, b) in enumerate(uni.cells)}
        idx = np.array(sorted(ucell[(int(a - i0), int(b - j0))] for a, b in zip(i, j)))
        s = 1 << (leaf.Lf - l)
        X, Y = (uni.X + i0 * k) * s, (uni.Y + j0 * k) * s
        key = Y * (leaf.Xmax + 1) + X
        ln = np.minimum(np.searchsorted(leaf.key, key), leaf.nn - 1)
        there = leaf.key[ln] == key              # uniform nodes that are leaf nodes
        li = lm.find(X, Y)                       # uniform nodes that are level nodes
        assert np.all(there[li >= 0])
        assert np.array_equal(np.sort(li[li >= 0]), np.arange(lm.nn))
        z = lambda a: np.where(there.reshape((-1,) + (1,) * (a.ndim - 1)), a[ln], 0.0)
        st = ops.State(uni, z(uf), z(pf), z(ptf))
        G = ops.assemble_jacobian(uni, mat, st, cell_idx=idx).toarray()
        keep = np.nonzero(li >= 0)[0]            # in level order below
        keep = keep[np.argsort(li[keep])]
        n = uni.nn
        gu = np.concatenate([keep, n + keep])
        ref_uu = G[np.ix_(gu, gu)]
        ref_pp = G[np.ix_(2 * n + keep, 2 * n + keep)]
        for got, ref in ((M.B["uu"][l].A.toarray(), ref_uu), (M.B["pp"][l].A.toarray(), ref_pp)):
            assert np.abs(ref).max() > 0
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        # no entries of the uniform assembly outside the level's nodes
        outside = np.setdiff1d(np.arange(3 * n), np.concatenate([gu, 2 * n + keep]))
        assert not np.any(G[outside]) and not np.any(G[:, outside])
    assert not_rect >= 1   # the 2:1 balance closure makes some level non-rectangular


@pytest.mark.parametrize("k", [1, 2])
def test_prolongation_reproduces_qk_polynomials(k):
    """The level prolongation is nodal interpolation of the coarse Q_k field: it maps
    the coarse nodal values of every polynomial x^a y^b with a, b <= k to its fine
    nodal values exactly, on every level of a locally refined mesh; and a monomial
    of degree k + 1 in x is not reproduced (the test would pass a degree-blind P)."""
    rec = dict(domain=synth.DOMAIN, ncx=4, ncy=4, n_global=1, steps=[("box", -2.0, 2.0, -1.0, 1.0)] * 3)
    leaf = LeafMesh(build_recipe(rec), k)
    M = mg.MG(leaf, ops.Material(), np.zeros((leaf.nn, 2)), np.ones(leaf.nn), np.ones(leaf.nn),
              np.zeros(leaf.nn, bool), blocks=("pp",))
    x0, x1, y0, y1 = synth.DOMAIN
    xy = lambda lm: (x0 + lm.X * (x1 - x0) / lm.Xmax, y0 + lm.Y * (y1 - y0) / lm.Ymax)
    missed = 0
    for l in range(1, leaf.Lf + 1):
        fine, coarse, P = M.levels[l], M.levels[l - 1], M.P[l]
        xf, yf = xy(fine)
        xc, yc = xy(coarse)
        for a in range(k + 1):
            for b in range(k + 1):
                got = P @ (xc ** a * yc ** b)
                ref = xf ** a * yf ** b
                assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0), (l, a, b)
        got = P @ xc ** (k + 1)
        missed += np.abs(got - xf ** (k + 1)).max() > 1e-6 * np.abs(xf ** (k + 1)).max()
    assert missed == leaf.Lf
