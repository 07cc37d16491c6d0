"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
invariants, hand-derived values (tests/golden) or brute force on tiny meshes.
"""

import math
import os

import numpy as np
import pytest

from oracle import average, features, fem, gru, transfer
from oracle.mesh import Mesh, Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def c1_mesh(**kw):
    return Mesh(32, 8, 1, 1, ellipse=(0.2, 0.2, 0.04, 0.06), **kw)


# ---------------------------------------------------------------- mesh / sizes

def test_c1_solid_cells_by_hand():
    # centroid test by hand: cell (2,3) has centroid (0.171875, 0.179375):
    # ((0.171875-0.2)/0.04)^2 + ((0.179375-0.2)/0.06)^2 = 0.494 + 0.118 < 1;
    # cell (2,4): 0.494 + 0.261 < 1; cell (3,3): 1.03 + 0.118 > 1.
    m = c1_mesh()
    assert sorted(map(tuple, np.argwhere(m.solid_coarse)[:, ::-1])) == [(2, 3), (2, 4)]
    assert m.P == 254


def test_feature_and_output_lengths_match_paper():
    # Sec. 5.2: 51 inputs for one-cell patches on level L+1; Sec. 6.2: 18 outputs;
    # Sec. 6.6: 99 inputs and 50 outputs across two levels.
    m1 = Mesh(8, 4, 1, 1)
    assert (m1.n_in, m1.n_out) == (51, 18)
    m2 = Mesh(8, 4, 2, 1)
    assert (m2.n_in, m2.n_out) == (99, 50)


def test_param_counts_match_paper():
    # Sec. 6.2: 3(32*32 + 32*51) = 7968 GRU and 32*18 = 576 output weights.
    assert 3 * 32 * (32 + 51) == 7968
    assert gru.param_count(51, 32, 18) == 7968 + 576
    # Sec. 6.6: N_GRU = 96 with 99 inputs and 50 outputs has 60 960 parameters.
    assert gru.param_count(99, 96, 50) == 60960


def test_node_classes_brute_force():
    m = Mesh(8, 4, 1, 1, ellipse=(0.6, 0.2, 0.3, 0.12))
    assert m.solid_coarse.any()
    xs, ys = m.fine_xy()
    # brute force: every fine cell as a coordinate rectangle with its parent's flag
    cells = []
    for J in range(m.nyf):
        for I in range(m.nxf):
            cx = (I // 2 + 0.5) * m.hxc
            cy = (J // 2 + 0.5) * m.hyc
            solid = ((cx - 0.6) / 0.3) ** 2 + ((cy - 0.2) / 0.12) ** 2 < 1
            cells.append((I * m.hxf, (I + 1) * m.hxf, J * m.hyf, (J + 1) * m.hyf, solid))
    eps = 1e-12
    for j in range(m.nyf + 1):
        for i in range(m.nxf + 1):
            x, y = xs[j, i], ys[j, i]
            touch = [c for c in cells if c[0] - eps <= x <= c[1] + eps and c[2] - eps <= y <= c[3] + eps]
            touch_solid = any(c[4] for c in touch)
            touch_fluid = any(not c[4] for c in touch)
            wall = abs(y) < eps or abs(y - 0.41) < eps
            dirichlet = wall or abs(x) < eps or touch_solid
            assert m.dirichlet[j, i] == dirichlet
            assert m.p_active[j, i] == touch_fluid
            assert m.inflow[j, i] == (abs(x) < eps and not wall and not touch_solid)


def test_multiplicity_brute_force():
    m = Mesh(8, 4, 1, 2, ellipse=(0.6, 0.2, 0.3, 0.12))
    xs, ys = m.fine_xy()
    eps = 1e-12
    W, Hh = m.s * m.hxc, m.s * m.hyc
    rects = [(pi * W, (pi + 1) * W, pj * Hh, (pj + 1) * Hh) for pi, pj in m.patches]
    for j in range(m.nyf + 1):
        for i in range(m.nxf + 1):
            cnt = sum(1 for r in rects if r[0] - eps <= xs[j, i] <= r[1] + eps and r[2] - eps <= ys[j, i] <= r[3] + eps)
            assert m.multiplicity[j, i] == cnt
    assert set(np.unique(m.multiplicity[~m.dirichlet])) <= {1, 2, 4}


# ---------------------------------------------------------------- transfer

def _bilinear(x, y):
    return 0.3 - 1.7 * x + 2.5 * y + 4.25 * x * y


@pytest.mark.parametrize("K", [1, 2, 3])
def test_prolongation_exact_on_bilinear(K):
    m = Mesh(6, 4, K, 1)
    xc, yc = m.coarse_xy()
    xf, yf = m.fine_xy()
    coarse = np.stack([_bilinear(xc, yc).ravel()] * 3)
    fine = transfer.prolongate_raw(m, coarse)
    ref = _bilinear(xf, yf).ravel()
    assert np.abs(fine[0] - ref).max() <= 1e-14 * np.abs(ref).max()


def _p1_single(g):
    """1D linear interpolation to a twice finer grid along both axes."""
    def along(a, axis):
        a = np.moveaxis(a, axis, -1)
        out = np.empty(a.shape[:-1] + (2 * a.shape[-1] - 1,))
        out[..., 0::2] = a
        out[..., 1::2] = 0.5 * (a[..., :-1] + a[..., 1:])
        return np.moveaxis(out, -1, axis)
    return along(along(g, 1), 0)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_prolongation_equals_nested_single_level(K):
    m = Mesh(6, 4, K, 1)
    rng = np.random.default_rng(0)
    xc = rng.normal(size=(1, m.Nc))
    g = xc[0].reshape(m.wyc + 1, m.wxc + 1)
    for _ in range(K):
        g = _p1_single(g)
    fine = transfer.prolongate_raw(m, xc)[0]
    assert np.abs(fine - g.ravel()).max() <= 1e-14
    # coincident nodes are copied exactly
    f2 = fine.reshape(m.wyf + 1, m.wxf + 1)
    assert np.array_equal(f2[::m.r, ::m.r].ravel(), xc[0])


@pytest.mark.parametrize("K", [1, 2])
def test_restriction_is_transpose_of_prolongation(K):
    m = Mesh(8, 4, K, 1)
    rng = np.random.default_rng(1)
    xf = rng.normal(size=(1, m.Nf))
    yc = rng.normal(size=(1, m.Nc))
    lhs = float(transfer.restrict_raw(m, xf)[0] @ yc[0])
    rhs = float(xf[0] @ transfer.prolongate_raw(m, yc)[0])
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    # P 1 = 1 so R preserves the sum
    assert abs(transfer.restrict_raw(m, xf)[0].sum() - xf[0].sum()) <= 1e-12 * np.abs(xf).sum()


def test_ramp_closed_form():
    # omega(t) = 1/2 - cos(2 pi t) / 2 up to t = 1/2, then 1 (Sec. 6.1)
    prm = Params(ramp=True)
    assert [prm.omega(t) for t in (0.0, 0.25, 0.5, 0.75, 3.0)] == pytest.approx([0.0, 0.5, 1.0, 1.0, 1.0],
                                                                                abs=1e-15)
    assert Params().omega(0.0) == 1.0


@pytest.mark.parametrize("t", [0.1, 0.25, 1.0])
def test_dirichlet_overwrite_values(t):
    # S1 overwrites fine Dirichlet velocity nodes: the parabolic inflow at
    # x = 0 (peak u_max at y = H/2, times the ramp), zero on walls and
    # obstacle; every other node keeps the raw prolongation.
    m = Mesh(8, 4, 2, 1, ellipse=(0.6, 0.2, 0.3, 0.12))
    prm = Params(ramp=True)
    rng = np.random.default_rng(8)
    xc = rng.normal(size=(3, m.Nc))
    raw = transfer.prolongate_raw(m, xc)
    xf = transfer.prolongate(m, prm, xc, t)
    d = m.dirichlet.ravel()
    assert np.array_equal(xf[:, ~d], raw[:, ~d]) and np.array_equal(xf[2], raw[2])
    U = xf[0].reshape(m.wyf + 1, m.wxf + 1)
    w = prm.omega(t)
    assert U[m.nyf // 2, 0] == pytest.approx(prm.u_max * w, rel=1e-14)   # y = H/2
    assert U[0, 0] == 0.0 and U[-1, 0] == 0.0
    assert not xf[1, d].any()
    assert not xf[0, d & ~m.inflow.ravel()].any()
    # Simpson's rule is exact for the parabola: mean inflow (2/3) u_max w, so
    # u_max = 1.5 gives a mean of 1 and Re = 100 for an obstacle of size 0.1
    col = U[:, 0]
    simpson = m.hyf / 3 * (col[0] + col[-1] + 4 * col[1:-1:2].sum() + 2 * col[2:-1:2].sum())
    assert simpson / m.ly == pytest.approx(2.0 / 3.0 * prm.u_max * w, rel=1e-13)


def test_restrict_zeroes_coarse_dirichlet_and_pressure():
    m = c1_mesh()
    rng = np.random.default_rng(2)
    bc = transfer.restrict(m, rng.normal(size=(2, m.Nf)))
    assert np.all(bc[:, m.dirichlet_c.ravel()][:2] == 0)
    assert np.all(bc[2] == 0)
    assert np.all(bc[0, ~m.dirichlet_c.ravel()] != 0)


# ---------------------------------------------------------------- residual / rhs

def _poiseuille(m, prm):
    xf, yf = m.fine_xy()
    H = m.ly
    u = prm.u_max * 4 * yf * (H - yf) / H ** 2
    p = 8 * prm.u_max * prm.nu / H ** 2 * (m.lx - xf)
    return np.stack([u.ravel(), np.zeros(m.Nf), p.ravel()])


@pytest.mark.parametrize("K,s", [(1, 1), (2, 1), (2, 2)])
def test_poiseuille_has_zero_residual(K, s):
    # Steady Poiseuille flow solves the Navier-Stokes equations with do-nothing
    # outflow (p(2.2) = 0); the Q1 interpolant of its 1D-quadratic velocity and
    # linear pressure is reproduced exactly by the discretisation, so with
    # v_n = v_{n-1} the Crank-Nicolson residual vanishes on every row.
    m = Mesh(16, 8, K, s)
    prm = Params()
    x = _poiseuille(m, prm)
    b = fem.rhs(m, prm, x[:2])
    r = fem.residual(m, prm, x, b)
    scale = np.abs(b).max()
    assert np.abs(r).max() <= 1e-11 * scale


def test_two_by_two_gauss_equals_three_by_three():
    m = c1_mesh()
    prm = Params()
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3, m.Nf))
    b = rng.normal(size=(2, m.Nf))
    r2 = fem.residual(m, prm, x, b, nq=2)
    r3 = fem.residual(m, prm, x, b, nq=3)
    assert np.abs(r2 - r3).max() <= 1e-12 * np.abs(r3).max()


def _trapz(f, h):
    return h * (f.sum() - 0.5 * (f[0] + f[-1]))


def test_divergence_rows_sum_to_boundary_flux():
    # Divergence theorem: the test functions sum to 1, so the divergence rows
    # sum to the integral of div v, which is the outward flux through the four
    # sides.  v.n is linear along each boundary edge of a bilinear field, so
    # the trapezoidal rule on the nodal values gives the flux exactly.
    m = Mesh(8, 4, 2, 1)
    rng = np.random.default_rng(21)
    u, v = rng.normal(size=(2, m.Nf))
    div = fem.assemble_terms(m, u, v)["div"]
    U, V = u.reshape(m.wyf + 1, m.wxf + 1), v.reshape(m.wyf + 1, m.wxf + 1)
    flux = (_trapz(U[:, -1], m.hyf) - _trapz(U[:, 0], m.hyf)
            + _trapz(V[-1, :], m.hxf) - _trapz(V[0, :], m.hxf))
    assert abs(div.sum() - flux) <= 1e-13 * np.abs(div).sum()


def test_constant_velocity_rhs_is_mass_times_velocity():
    # constant v: convection and diffusion vanish, b = (1/k) (v, phi_i);
    # (1, phi_i) = hx hy at interior nodes
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    v = np.stack([np.full(m.Nf, 0.75), np.full(m.Nf, -0.25)])
    b = fem.rhs(m, prm, v)
    inner = ~m.dirichlet.ravel()
    xs, _ = m.fine_xy()
    interior = inner & (xs.ravel() < m.lx - 1e-12)
    area = m.hxf * m.hyf
    assert np.allclose(b[0, interior], 0.75 * area / prm.k, rtol=1e-13, atol=0)
    assert np.allclose(b[1, interior], -0.25 * area / prm.k, rtol=1e-13, atol=0)
    # outflow nodes carry half the support
    outflow = inner & (xs.ravel() > m.lx - 1e-12)
    assert np.allclose(b[0, outflow], 0.5 * 0.75 * area / prm.k, rtol=1e-13, atol=0)


def test_rhs_sum_identity_with_exact_integrals():
    # partition of unity: sum_i phi_i = 1 and sum_i grad phi_i = 0, so the
    # unconstrained right-hand side sums to (1/k) int v - 1/2 int v.grad v.
    sympy = pytest.importorskip("sympy")
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    X, Y = sympy.symbols("x y")
    uf = 0.4 + 1.5 * X - 0.7 * Y + 2.0 * X * Y
    vf = -0.2 + 0.3 * X + 1.1 * Y - 0.9 * X * Y
    xs, ys = m.fine_xy()
    lam = [sympy.lambdify((X, Y), f, "numpy") for f in (uf, vf)]
    u = lam[0](xs, ys).ravel()
    v = lam[1](xs, ys).ravel()
    terms = fem.assemble_terms(m, u, v)
    bu, bv = fem.rhs_raw(m, prm, terms)
    for comp, f, b in ((0, uf, bu), (1, vf, bv)):
        conv = uf * sympy.diff(f, X) + vf * sympy.diff(f, Y)
        exact = sympy.integrate(f / prm.k - sympy.Rational(1, 2) * conv, (X, 0, m.lx), (Y, 0, m.ly))
        assert abs(b.sum() - float(exact)) <= 1e-11 * abs(float(exact))


def test_pressure_gradient_sign_and_scale():
    # -(p, div phi_i) = (d_x p, phi_i) = c hx hy at interior nodes for p = c x
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    xs, _ = m.fine_xy()
    c = 3.0
    p = (c * xs).ravel()
    zero = np.zeros(m.Nf)
    terms = fem.assemble_terms(m, zero, zero, p)
    Au, Av = fem.velocity_operator(m, prm, terms)
    inner = ~m.dirichlet.ravel() & (xs.ravel() < m.lx - 1e-12)
    assert np.allclose(Au[inner], c * m.hxf * m.hyf, rtol=1e-12)
    assert np.abs(Av[inner]).max() <= 1e-15


def test_divergence_and_lps_of_linear_fields():
    # u = x: (div v, xi_i) = hx hy at interior nodes; a linear pressure has
    # zero fluctuation, so the LPS term vanishes
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    xs, ys = m.fine_xy()
    terms = fem.assemble_terms(m, xs.ravel(), np.zeros(m.Nf))
    inner = (xs > 1e-12) & (xs < m.lx - 1e-12) & (ys > 1e-12) & (ys < m.ly - 1e-12)
    assert np.allclose(terms["div"][inner.ravel()], m.hxf * m.hyf, rtol=1e-12)
    lin = (2.0 * xs - 3.0 * ys + 0.5).ravel()
    assert np.abs(fem.lps_term(m, prm, lin)).max() <= 1e-12


def test_lps_energy_closed_form():
    # p = x^2: on every 2x2 patch p - pi p is a hat of height -hx^2 at the
    # middle column, so (grad f, grad f)_patch = hx^2 * (2hx * 2hy) = 4 hx^3 hy
    # and p^T LPS(p) = alpha * n_patches * 4 hx^3 hy.
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    xs, _ = m.fine_xy()
    p = (xs ** 2).ravel()
    e = float(p @ fem.lps_term(m, prm, p))
    n_patches = (m.nxf // 2) * (m.nyf // 2)
    alpha = prm.alpha0 * (m.hxf ** 2 + m.hyf ** 2) / prm.nu
    exact = alpha * n_patches * 4 * m.hxf ** 3 * m.hyf
    assert abs(e - exact) <= 1e-12 * exact


def test_lps_orthogonal_to_patchwise_bilinear():
    # the LPS test functions are fluctuations xi_i - pi xi_i, so for a vector q
    # that is bilinear on every 2x2 patch, q^T LPS(p) = sum alpha (grad(q - pi q), .) = 0
    m = Mesh(8, 4, 1, 1)
    prm = Params()
    xs, ys = m.fine_xy()
    p = np.random.default_rng(8).normal(size=m.Nf)
    lps = fem.lps_term(m, prm, p)
    q = (1.0 + 2.0 * xs - ys + 3.0 * xs * ys).ravel()
    assert abs(q @ lps) <= 1e-12 * np.abs(q).max() * np.abs(lps).sum()
    assert abs(p @ lps) > 1e-3 * np.abs(p).max() * np.abs(lps).sum()


def test_lps_on_partly_solid_patches():
    # one level with its own mask (K = 0): some projection patches are partly
    # solid and contribute their fluid cells only.  The term is then still a
    # symmetric positive semidefinite form that vanishes on linear pressures,
    # and a patch's centre node, whose fluctuation is symmetric, gets the
    # fluid cells' share (a quarter each) of the all-fluid patch's energy.
    ell = (0.6, 0.2, 0.3, 0.12)
    m = Mesh(16, 8, 0, 1, ellipse=ell)
    blk = m.solid_f.reshape(4, 2, 8, 2)
    part = blk.any(axis=(1, 3)) & ~blk.all(axis=(1, 3))
    assert part.any()
    prm = Params()
    L = np.array([fem.lps_term(m, prm, e) for e in np.eye(m.Nf)]).T
    np.testing.assert_allclose(L, L.T, rtol=0, atol=1e-14 * np.abs(L).max())
    assert np.linalg.eigvalsh(L).min() >= -1e-12 * np.abs(L).max()
    xs, ys = m.fine_xy()
    assert np.abs(L @ (0.3 + 2.0 * xs.ravel() - 5.0 * ys.ravel())).max() <= 1e-12 * np.abs(L).max()
    full = np.array([fem.lps_term(Mesh(16, 8, 0, 1), prm, e) for e in np.eye(m.Nf)]).T
    for n, mm in np.argwhere(part):
        c = (2 * n + 1) * (m.wxf + 1) + 2 * mm + 1
        share = (~blk[n, :, mm, :]).sum() / 4
        assert L[c, c] == pytest.approx(share * full[c, c], rel=1e-13)


def test_residual_zero_rows():
    m = c1_mesh()
    prm = Params()
    rng = np.random.default_rng(4)
    r = fem.residual(m, prm, rng.normal(size=(3, m.Nf)), rng.normal(size=(2, m.Nf)))
    assert np.all(r[:2, m.dirichlet.ravel()] == 0)
    assert np.all(r[2, ~m.p_active.ravel()] == 0)


# ---------------------------------------------------------------- features

def test_features_hand_indexed():
    m = Mesh(8, 4, 1, 1, ellipse=(0.6, 0.2, 0.3, 0.12))
    prm = Params()
    xs, ys = m.fine_xy()
    nxn = m.wxf + 1
    # plant values that encode the node position
    node_id = np.arange(m.Nf, dtype=np.float64)
    r = np.stack([node_id, 1000 + node_id, 2000 + node_id])
    xf = np.stack([0.01 * node_id, -0.02 * node_id, np.zeros(m.Nf)])
    X = features.patch_features(m, prm, xf, r)
    q = max(m.hxc, m.hyc)
    for p, (pi, pj) in enumerate(m.patches):
        row = X[p]
        # fine nodes of patch (pi, pj): (2pi + a, 2pj + b), a, b in 0..2, x fastest
        ids = [(2 * pj + b) * nxn + 2 * pi + a for b in range(3) for a in range(3)]
        assert list(row[0:9]) == ids
        assert list(row[9:18]) == [1000 + i for i in ids]
        assert list(row[18:27]) == [2000 + i for i in ids]
        cids = [(2 * (pj + b)) * nxn + 2 * (pi + a) for b in range(2) for a in range(2)]
        assert np.allclose(row[27:31], [0.01 * i for i in cids])
        assert np.allclose(row[31:35], [-0.02 * i for i in cids])
        assert np.allclose(row[35:39], [q * math.hypot(0.01 * i, 0.02 * i) / prm.nu for i in cids])
    # patch geometry for an axis-aligned cell hx x hy
    hx, hy = m.hxc, m.hyc
    geo = X[0, 39:51]
    assert np.allclose(geo, [hx, hy, hx, hy, hx / hy, hx / hy, 1.0, 1.0] + [math.pi / 2] * 4, rtol=1e-15)
    # patches are numbered lexicographically over fluid patches, x fastest
    order = [tuple(p) for p in m.patches]
    assert order == sorted(order, key=lambda t: (t[1], t[0]))


# ---------------------------------------------------------------- GRU

def _golden_gru():
    rows = {}
    with open(os.path.join(GOLDEN, "gru_hand.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows[parts[0]] = np.array([float(v) for v in parts[1:]])
    return rows


def test_gru_hand_derived():
    l3, l2 = math.log(3.0), math.log(2.0)
    Wx = np.array([[l3, 0, 0], [0, 0, 0], [-l3, 0, 0], [l3, 0, 0], [0, 0, l2], [0, 0, -l2]])
    Uh = np.zeros((6, 2))
    Uh[4] = [0, -8 * l2 / 3]
    Uh[5] = [8 * l2, 0]
    Wfc = np.array([[1.0, 0], [0, 1.0], [1.0, 1.0]])
    X = np.array([[1.0, 0, 0], [0, 0, 1.0]])
    h = np.array([[0.5, -0.5], [0.0, 0.0]])
    hn, d = gru.gru_step(X, h, Wx, Uh, Wfc)
    g = _golden_gru()
    assert np.allclose(hn[0], g["A"][:2], atol=1e-14) and np.allclose(d[0], g["A"][2:], atol=1e-14)
    assert np.allclose(hn[1], g["B"][:2], atol=1e-14) and np.allclose(d[1], g["B"][2:], atol=1e-14)


def test_gru_recurrent_gates_and_zero_weights():
    # zero weights: z = r = 1/2, candidate 0, so h' = h/2 (Eq. gru)
    h = np.array([[0.8, -0.4]])
    hn, d = gru.gru_step(np.ones((1, 3)), h, np.zeros((6, 3)), np.zeros((6, 2)), np.eye(2))
    assert np.allclose(hn, h / 2, atol=1e-15) and np.allclose(d, h / 2, atol=1e-15)
    # U_z only: z = sigma(+-ln 3) = (3/4, 1/4) with h = (1, 0): h' = z*h + (1-z)*0
    l3 = math.log(3.0)
    Uh = np.zeros((6, 2))
    Uh[0] = [l3, 0]
    Uh[1] = [-l3, 0]
    hn, _ = gru.gru_step(np.zeros((1, 3)), np.array([[1.0, 0.0]]), np.zeros((6, 3)), Uh, np.eye(2))
    assert np.allclose(hn, [[0.75, 0.0]], atol=1e-15)


def test_gru_patches_independent():
    rng = np.random.default_rng(5)
    W = (rng.normal(size=(12, 5)), rng.normal(size=(12, 4)), rng.normal(size=(3, 4)))
    X, h = rng.normal(size=(2, 5)), rng.normal(size=(2, 4))
    hn, d = gru.gru_step(X, h, *W)
    for p in range(2):
        h1, d1 = gru.gru_step(X[p:p + 1], h[p:p + 1], *W)
        assert np.allclose(h1, hn[p:p + 1], atol=1e-15) and np.allclose(d1, d[p:p + 1], atol=1e-15)


# ---------------------------------------------------------------- averaging

def test_constant_correction_survives_averaging():
    m = Mesh(8, 4, 2, 2, ellipse=(0.6, 0.2, 0.3, 0.12))
    rng = np.random.default_rng(6)
    xf = rng.normal(size=(3, m.Nf))
    d = np.full((m.P, m.n_out), 0.375)
    v = average.scatter_average(m, d, xf)
    free = ~m.dirichlet.ravel()
    # the mean of equal dyadic predictions is exact, so v = fl(v~ + 0.375)
    assert np.array_equal(v[:, free], xf[:2, free] + 0.375)
    assert np.array_equal(v[:, ~free], xf[:2, ~free])


def test_general_constant_correction_within_one_ulp():
    # a constant c that is not dyadic: the mean of m equal predictions
    # (m = 1, 2 or 4) is c up to the rounding of the sum, one ulp at most
    m = Mesh(8, 4, 2, 2, ellipse=(0.6, 0.2, 0.3, 0.12))
    assert set(np.unique(m.multiplicity[m.multiplicity > 0])) == {1, 2, 4}
    free = ~m.dirichlet.ravel()
    for c in (0.1, -0.7, 1.0 / 3.0, 2.0 ** -30 * 3.1):
        d = np.full((m.P, m.n_out), c)
        v = average.scatter_average(m, d, np.zeros((3, m.Nf)))
        err = np.abs(v[:, free] - c).max()
        assert err <= np.spacing(abs(c)), (c, err)
        assert not v[:, ~free].any()


def test_averaging_of_two_patch_predictions():
    # a node shared by two patches gets the mean of the two predictions
    m = Mesh(4, 2, 1, 1)
    xf = np.zeros((3, m.Nf))
    d = np.zeros((m.P, m.n_out))
    d[0, :] = 1.0     # patch (0,0)
    d[1, :] = 3.0     # patch (1,0)
    v = average.scatter_average(m, d, xf).reshape(2, m.wyf + 1, m.wxf + 1)
    # node (2, 1) (fine) lies on the shared edge of patches (0,0) and (1,0)
    assert v[0, 1, 2] == 2.0 and v[0, 1, 1] == 1.0 and v[0, 1, 3] == 3.0


# ---------------------------------------------------------------- windows

def test_window_matches_full_mesh_in_interior():
    from oracle.step import dnnmg_step
    full = Mesh(16, 8, 1, 2, ellipse=(0.6, 0.2, 0.2, 0.1))
    win = Mesh(16, 8, 1, 2, ellipse=(0.6, 0.2, 0.2, 0.1), window=(4, 0, 12, 8))
    prm = Params()
    rng = np.random.default_rng(7)
    xc = rng.normal(size=(3, full.Nc))
    bf = rng.normal(size=(2, full.Nf))
    H = 4
    W = (rng.normal(size=(3 * H, full.n_in)) * 0.1, rng.normal(size=(3 * H, H)) * 0.1,
         rng.normal(size=(full.n_out, H)) * 0.1)
    h = rng.normal(size=(full.P, H))
    of = dnnmg_step(full, prm, W, xc, h, bf, 0.0)
    xcw = xc.reshape(3, 9, 17)[:, 0:9, 4:13].reshape(3, -1)
    bfw = bf.reshape(2, 17, 33)[:, :, 8:25].reshape(2, -1)
    gidx = full.patch_global_index[win.patches[:, 1], win.patches[:, 0]]
    ow = dnnmg_step(win, prm, W, xcw, h[gidx], bfw, 0.0)
    # coarse nodes far from the two cut edges (x = 4, x = 12 coarse) are exact
    bcf = of["bc"].reshape(3, 9, 17)[:, :, 8:9]
    bcw = ow["bc"].reshape(3, 9, 9)[:, :, 4:5]
    assert np.allclose(bcf, bcw, rtol=1e-13, atol=1e-13 * np.abs(bcf).max())
    # interior patches' hidden states are exact
    inner = (win.patches[:, 0] >= 3) & (win.patches[:, 0] <= 4)
    assert np.allclose(ow["h"][inner], of["h"][gidx[inner]], rtol=1e-13, atol=1e-14)


# ------------------------------------------------------- whole step, d = 0

@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("s", [1, 2])
def test_zero_correction_step_gives_coarse_rhs(K, s):
    # With d = 0 the method falls back to the coarse solver (Sec. 5.1), so the
    # coarse right-hand side it hands on must be the coarse level's own.
    # For nested Q1 spaces a coarse function is exactly a fine function
    # (S1), and R = P^T sums fine tests into coarse tests (S7).  Every term of
    # Eq. 4cranknicholson3 is then integrated exactly on both levels, since
    # 2-point Gauss is exact up to degree 3 per direction and (v.grad v) phi
    # is at most cubic.  So R Rhs_f(P x_c) = Rhs_c(x_c) on every coarse row
    # once x_c holds zero Dirichlet data (ramp at t = 0: zero inflow); fine
    # Dirichlet rows lie where the coarse tests of free nodes vanish.
    from oracle.step import dnnmg_step
    ell = (0.6, 0.2, 0.3, 0.12)
    m = Mesh(8, 4, K, s, ellipse=ell)
    mc = Mesh(8, 4, 0, s, ellipse=ell)          # the coarse level on its own
    assert m.solid_coarse.any()
    prm = Params(ramp=True)
    rng = np.random.default_rng(100 + 10 * K + s)
    xc = rng.normal(size=(3, m.Nc))
    xc[:2, m.dirichlet_c.ravel()] = 0.0
    H = 4
    W = (rng.normal(size=(3 * H, m.n_in)) * 0.1, rng.normal(size=(3 * H, H)) * 0.1,
         np.zeros((m.n_out, H)))
    out = dnnmg_step(m, prm, W, xc, rng.normal(size=(m.P, H)),
                     rng.normal(size=(2, m.Nf)), 0.0)
    assert np.abs(out["d"]).max() == 0.0
    bc_coarse = fem.rhs(mc, prm, xc[:2])
    scale = np.abs(bc_coarse).max()
    assert np.allclose(out["bc"][:2], bc_coarse, rtol=0, atol=1e-13 * scale)
    assert not out["bc"][2].any()
