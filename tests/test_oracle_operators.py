"""Pins of the oracle residual / Jacobian / constrained system (oracle/operators.py)
against closed forms, invariants and finite differences."""
import numpy as np
import pytest

from oracle import operators as ops
from oracle.mesh import LeafMesh, build_recipe
import synthetic as synth


def mesh(name, k):
    return LeafMesh(build_recipe(synth.recipe(name)), k)


def random_state(m, seed=0, u_std=1e-1, E_cells=None):
    xy = m.node_xy()
    u, phi, phit = synth.linearisation(m.X, m.Y, m.Xmax, m.Ymax, seed=seed, u_std=u_std)
    return ops.State(m, u, phi, phit, E_cells)


def const_state(m, ufun=None, phi=1.0, phit=1.0):
    x, y = m.node_xy()
    u = np.zeros((m.nn, 2)) if ufun is None else ufun(x, y)
    return ops.State(m, u, np.full(m.nn, phi), np.full(m.nn, phit))


@pytest.mark.parametrize("k", [1, 2])
def test_elastic_energy_linear_field(k):
    """u = A x: u^T G_uu u = |Omega| (2 mu e:e + lam tr(e)^2), e = sym(A), with g = 1."""
    m = mesh("tiny", k)
    mat = ops.Material(E=1.3, nu=0.2, Gc=1.0, eps=0.5, kappa=0.0, p=0.0)
    A = np.array([[0.3, -0.7], [0.2, 0.5]])
    x, y = m.node_xy()
    u = np.stack([A[0, 0] * x + A[0, 1] * y, A[1, 0] * x + A[1, 1] * y], axis=1)
    st = const_state(m)
    G = ops.assemble_jacobian(m, mat, st)
    nn = m.nn
    v = np.concatenate([m.C @ u[:, 0], m.C @ u[:, 1], np.zeros(nn)])
    e = 0.5 * (A + A.T)
    exact = 400.0 * (2 * mat.mu * np.sum(e * e) + mat.lam * np.trace(e) ** 2)
    assert abs(v @ (G @ v) - exact) < 1e-10 * exact


@pytest.mark.parametrize("k", [1, 2])
def test_rigid_modes_and_patch_test(k):
    """Rigid motions are in the kernel of C^T G_uu C; a linear field leaves zero
    residual on every free interior row (patch test on a mesh with hanging nodes)."""
    m = mesh("small", k)
    mat = ops.Material(E=1.0, nu=0.2, Gc=1.0, eps=0.5, kappa=0.0, p=0.0)
    st = const_state(m)
    G = ops.assemble_jacobian(m, mat, st)
    C = ops.C3(m)
    nn = m.nn
    x, y = m.node_xy()
    for vec in (np.concatenate([np.ones(nn), np.zeros(2 * nn)]),
                np.concatenate([np.zeros(nn), np.ones(nn), np.zeros(nn)]),
                np.concatenate([-y, x, np.zeros(nn)])):
        r = C.T @ (G @ (C @ vec))
        assert np.abs(r[:2 * nn]).max() < 1e-12
    lin = np.concatenate([0.3 * x - 0.1 * y, 0.2 * x + 0.4 * y, np.zeros(nn)])
    r = C.T @ (G @ (C @ lin))
    interior = ~m.dirichlet & ~m.is_hanging
    assert np.abs(r[:nn][interior]).max() < 1e-12
    assert np.abs(r[nn:2 * nn][interior]).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_pure_elasticity_limit(k):
    """phi = phi~ = 1, u = 0: (p, div psi) = 0 for psi in H^1_0 and 1 - phi = 0, so the
    condensed residual vanishes on every free row (U = (0, 1) solves the discrete system)."""
    m = mesh("small", k)
    mat = ops.Material(eps=0.4)
    st = const_state(m)
    A = ops.residual_form(m, mat, st)
    R = ops.condense(m, -A)
    free = ops.free_dofs(m, np.zeros(m.nn, bool))
    assert np.abs(R[free]).max() < 1e-15


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("withE", [False, True])
def test_jacobian_is_derivative_of_residual(k, withE):
    """A(U + t V) is a cubic polynomial in t: the Richardson-extrapolated central
    difference equals G C V up to rounding.  Pins every Jacobian term and the sign
    of the G_c / l term."""
    m = mesh("tiny", k)
    E = None
    if withE:
        E = synth.cell_modulus(m.cells[:, 0], m.cells[:, 1], m.cells[:, 2], seed=4, sigma_log=0.3)
    mat = ops.Material(E=1.0, nu=0.3, Gc=1.7, eps=0.8, kappa=1e-3, p=0.3)
    x, y = m.node_xy()
    u0, phi0, phit = synth.linearisation(m.X, m.Y, m.Xmax, m.Ymax, seed=7, u_std=0.3)
    st = ops.State(m, u0, phi0, phit, E)
    G = ops.assemble_jacobian(m, mat, st)
    rng = np.random.default_rng(11)
    V = rng.normal(size=(m.nn, 3))

    def A_at(t):
        s = ops.State(m, u0 + t * V[:, :2], phi0 + t * V[:, 2], phit, E)
        return ops.residual_form(m, mat, s)

    def D(e):
        return (A_at(e) - A_at(-e)) / (2 * e)

    eps = 1e-2
    fd = (4 * D(eps / 2) - D(eps)) / 3
    v = np.concatenate([V[:, 0], V[:, 1], V[:, 2]])
    gv = G @ (ops.C3(m) @ v)
    assert np.abs(fd - gv).max() < 1e-9 * np.abs(gv).max()


def test_block_structure():
    """Upper-right block (u rows, phi columns) is zero; diagonal blocks symmetric."""
    m = mesh("small", 1)
    mat = ops.Material(eps=0.4, p=1e-2)
    st = random_state(m)
    G = ops.assemble_jacobian(m, mat, st).toarray()
    nn = m.nn
    assert np.abs(G[:2 * nn, 2 * nn:]).max() == 0.0
    Guu = G[:2 * nn, :2 * nn]
    Gpp = G[2 * nn:, 2 * nn:]
    assert np.abs(Guu - Guu.T).max() < 1e-14 * np.abs(Guu).max()
    assert np.abs(Gpp - Gpp.T).max() < 1e-14 * np.abs(Gpp).max()
    assert np.abs(G[2 * nn:, :2 * nn]).max() > 0


def test_constrained_operator_structure():
    m = mesh("small", 1)
    mat = ops.Material(eps=0.4)
    st = random_state(m)
    G = ops.assemble_jacobian(m, mat, st)
    active = np.zeros(m.nn, bool)
    active[::17] = True
    active &= ~m.is_hanging
    Gt = ops.constrained_operator(m, G, active).toarray()
    nn = m.nn
    fixed = ops.fixed_dofs(m, active)
    hang = np.tile(m.is_hanging, 3)
    assert np.allclose(Gt[fixed][:, fixed], np.eye(fixed.sum()))
    assert np.abs(Gt[fixed][:, ~fixed]).max() == 0.0
    assert np.abs(Gt[~fixed][:, fixed]).max() == 0.0
    assert np.abs(Gt[hang]).max() == 0.0 and np.abs(Gt[:, hang]).max() == 0.0


def test_lumped_mass_and_tcv():
    m = mesh("small", 1)
    B = ops.lumped_mass(m)
    assert abs(B.sum() - 400.0) < 1e-10
    assert np.all(B[m.is_hanging] == 0.0) and np.all(B[~m.is_hanging] > 0)
    # u = (x + 10, 0), phi = x: u . grad phi = x + 10, integral 20 * 200 = 4000
    x, y = m.node_xy()
    st = ops.State(m, np.stack([x + 10, 0 * x], 1), x.copy(), np.ones(m.nn))
    assert abs(ops.tcv(m, st) - 4000.0) < 1e-9
    st = ops.State(m, np.stack([0 * x, y], 1), y.copy(), np.ones(m.nn))
    assert abs(ops.tcv(m, st)) < 1e-9


@pytest.mark.parametrize("name,k", [("tiny", 1), ("small", 1), ("small", 2)])
def test_cod_linear_fields_closed_form(name, k):
    """For linear u and phi (exactly represented, also across hanging nodes) u . grad phi is
    linear in y, so COD(x) = int_{-10}^{10} (u_x phi_x + u_y phi_y) dy has a closed form."""
    om = LeafMesh(build_recipe(synth.recipe(name)), k)
    x, y = om.node_xy()
    a, b, c, d, e, f, g, hh, q = 0.3, -0.2, 0.5, 0.1, 0.4, -0.3, 0.7, 0.25, -0.15
    u = np.stack([a + b * x + c * y, d + e * x + f * y], 1)
    phi = g + hh * x + q * y
    st = ops.State(om, u, phi, phi)
    xs = np.array([-9.37, -3.1, -0.4, 0.0, 1.234, 7.77])
    got = ops.cod(om, st, xs)
    # integral over y in (-10, 10) of (a + b x + c y) hh + (d + e x + f y) q
    ref = 20.0 * ((a + b * xs) * hh + (d + e * xs) * q)   # the odd terms in y integrate to 0
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), (got, ref)
    # the same field's TCV, integral of u . grad phi over the domain
    tcv = ops.tcv(om, st)
    assert abs(tcv - 20.0 * 20.0 * (a * hh + d * q)) <= 1e-10 * max(1.0, abs(tcv))


def test_table1_lame_constants():
    """Table 1 lists mu = 0.42 and lambda = 0.28 for E = 1, nu = 0.2 (two digits):
    the plane-strain Lame constants E / (2 (1 + nu)) and E nu / ((1 + nu)(1 - 2 nu))."""
    m = ops.Material(E=1.0, nu=0.2)
    assert round(m.mu, 2) == 0.42 and round(m.lam, 2) == 0.28


@pytest.mark.parametrize("name,k,deg", [("small", 1, 1), ("tiny", 2, 1), ("tiny", 2, 2), ("small", 2, 2)])
def test_residual_sum_rules_closed_form(name, k, deg):
    """Problem 2 for fields linear in x and y, on a mesh with hanging nodes.  Every
    integrand then has degree <= 3 in each variable, so the (k+1)^2 Gauss rule is
    exact, and contracting the assembled form with the nodal values of a linear
    test field w (reproduced exactly on every cell) gives the domain integral of
    the weak form at w, computed here in closed form by exact polynomial
    integration over the square:
        A_u(w)   = (g(phi~) sigma(u), e(w)) + (phi~^2 p, div w),  g = (1 - kappa) phi~^2 + kappa
        A_phi(w) = ((1 - kappa) phi sigma(u):e(u), w) + 2 p (phi div u, w)
                   - G_c / l (1 - phi, w) + G_c l (grad phi, grad w),
    with the plane-strain sigma(u) = 2 mu e(u) + lambda tr e(u) I.  Every term,
    sign and factor enters one of the checked integrals.  For Q2 (3 x 3 Gauss,
    exact to degree 5) the fields may also be quadratic (deg = 2): the integrands
    then have degree <= 5 in each variable, and Q2 reproduces the fields exactly,
    hanging edges included."""
    sp = pytest.importorskip("sympy")
    om = mesh(name, k)
    x0, x1, y0, y1 = synth.DOMAIN
    R = sp.Rational
    E, nu, Gc, ell, kappa, p = R(3, 2), R(1, 5), R(7, 10), R(3, 4), R(1, 20), R(3, 10)
    mu, lam = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    x, y = sp.symbols("x y")
    ux = R(1, 40) + R(3, 200) * x - R(1, 100) * y
    uy = -R(1, 50) + R(1, 80) * x + R(1, 160) * y
    phi = R(1, 2) + R(1, 40) * x + R(1, 60) * y
    phit = R(3, 5) - R(1, 50) * x + R(1, 30) * y
    if deg == 2:
        ux += R(1, 2000) * x * x - R(1, 3000) * x * y
        uy += R(1, 1500) * y * y + R(1, 4000) * x * x
        phi += R(1, 800) * x * y - R(1, 1000) * y * y
        phit += R(1, 900) * x * x + R(1, 700) * x * y
    exx, eyy, exy = sp.diff(ux, x), sp.diff(uy, y), (sp.diff(ux, y) + sp.diff(uy, x)) / 2
    sxx, syy, sxy = 2 * mu * exx + lam * (exx + eyy), 2 * mu * eyy + lam * (exx + eyy), 2 * mu * exy
    g = (1 - kappa) * phit ** 2 + kappa
    integ = lambda f: sp.integrate(sp.integrate(sp.expand(f), (x, x0, x1)), (y, y0, y1))

    def a_u(wx, wy):
        wxx, wyy, wxy = sp.diff(wx, x), sp.diff(wy, y), (sp.diff(wx, y) + sp.diff(wy, x)) / 2
        return integ(g * (sxx * wxx + syy * wyy + 2 * sxy * wxy) + phit ** 2 * p * (wxx + wyy))

    def a_phi(w):
        se = sxx * exx + syy * eyy + 2 * sxy * exy
        return integ((1 - kappa) * phi * se * w + 2 * p * phi * (exx + eyy) * w - Gc / ell * (1 - phi) * w
                     + Gc * ell * (sp.diff(phi, x) * sp.diff(w, x) + sp.diff(phi, y) * sp.diff(w, y)))

    # the oracle on the same fields
    X = x0 + om.X * (x1 - x0) / om.Xmax
    Y = y0 + om.Y * (y1 - y0) / om.Ymax
    ev = lambda f: sp.lambdify((x, y), f, "numpy")(X, Y) * np.ones(om.nn)
    st = ops.State(om, np.stack([ev(ux), ev(uy)], 1), ev(phi), ev(phit))
    mat = ops.Material(E=float(E), nu=float(nu), Gc=float(Gc), eps=float(ell), kappa=float(kappa), p=float(p))
    A = ops.residual_form(om, mat, st)
    nn = om.nn
    Au = (A[:nn], A[nn:2 * nn])
    Ap = A[2 * nn:]
    checks = []
    for wx, wy in ((1, 0), (0, 1), (x, 0), (y, 0), (0, x), (0, y), (x + 2 * y, y - 3 * x)):
        ref = float(a_u(sp.sympify(wx), sp.sympify(wy)))
        got = float(Au[0] @ ev(sp.sympify(wx)) + Au[1] @ ev(sp.sympify(wy)))
        checks.append((got, ref))
    for w in (1, x, y, 2 * x - y):
        ref = float(a_phi(sp.sympify(w)))
        got = float(Ap @ ev(sp.sympify(w)))
        checks.append((got, ref))
    scale = max(abs(r) for _, r in checks)
    for got, ref in checks:
        assert abs(got - ref) <= 1e-12 * scale, (got, ref)
    assert sum(abs(r) > 1e-6 * scale for _, r in checks) >= 8   # the checks are not trivially zero
