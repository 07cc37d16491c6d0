"""Brute-force pin of the oracle's finite-element residual and right-hand side.

The oracle assembles S2 and S6 cell by cell with 2x2 Gauss quadrature and a
9x9 local projection per LPS patch.  Here the same operators are built a
different way and compared on random fields:

* every element integral is exact rational arithmetic on polynomials over the
  unit square (no quadrature);
* the matrices are assembled densely over the whole mesh, and the convection
  term is a dense trilinear form;
* the local projection is a global matrix that evaluates each 2h-patch's
  bilinear interpolant at the patch's fine nodes.

The operators follow Sec. 3.1-3.3: the Crank-Nicolson velocity operator of
Eq. nonlinearshort, the divergence and local projection stabilisation of
Eq. disc:ns on pressure rows, and the explicit half of Eq. 4cranknicholson3
for the right-hand side.
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle import fem
from oracle.mesh import Mesh, Params


# ------------------------------------------------- exact polynomials on [0,1]^2

def _pmul(p, q):
    out = {}
    for (a, b), c in p.items():
        for (d, e), f in q.items():
            out[(a + d, b + e)] = out.get((a + d, b + e), Fraction(0)) + c * f
    return out


def _pdiff(p, axis):
    out = {}
    for (a, b), c in p.items():
        k = (a, b)[axis]
        if k:
            key = (a - 1, b) if axis == 0 else (a, b - 1)
            out[key] = out.get(key, Fraction(0)) + c * k
    return out


def _pint(p):
    """Exact integral over the unit square."""
    return sum((c / ((a + 1) * (b + 1)) for (a, b), c in p.items()), Fraction(0))


def _peval(p, x, y):
    return sum(c * x ** a * y ** b for (a, b), c in p.items())


def _corner_basis():
    """Bilinear Lagrange basis of the unit square, keyed by corner (cx, cy)."""
    one = Fraction(1)
    lin = {0: {(0, 0): one, (1, 0): -one}, 1: {(1, 0): one}}       # 1-x, x
    lin_y = {0: {(0, 0): one, (0, 1): -one}, 1: {(0, 1): one}}     # 1-y, y
    return {(cx, cy): _pmul(lin[cx], lin_y[cy]) for cy in (0, 1) for cx in (0, 1)}


CORNERS = [(0, 0), (1, 0), (0, 1), (1, 1)]
_B = _corner_basis()
_DX = {c: _pdiff(_B[c], 0) for c in CORNERS}
_DY = {c: _pdiff(_B[c], 1) for c in CORNERS}


def _tab2(f):
    return np.array([[float(f(a, b)) for b in CORNERS] for a in CORNERS])


# reference-element integrals; first index = test function
M_REF = _tab2(lambda a, b: _pint(_pmul(_B[a], _B[b])))
SXX = _tab2(lambda a, b: _pint(_pmul(_DX[a], _DX[b])))
SYY = _tab2(lambda a, b: _pint(_pmul(_DY[a], _DY[b])))
GX = _tab2(lambda a, b: _pint(_pmul(_B[b], _DX[a])))    # (trial b, d_x test a)
GY = _tab2(lambda a, b: _pint(_pmul(_B[b], _DY[a])))
TX = np.array([[[float(_pint(_pmul(_pmul(_B[b], _DX[c]), _B[a]))) for c in CORNERS]
                for b in CORNERS] for a in CORNERS])      # (test a, carrier b, d_x of c)
TY = np.array([[[float(_pint(_pmul(_pmul(_B[b], _DY[c]), _B[a]))) for c in CORNERS]
                for b in CORNERS] for a in CORNERS])


# ------------------------------------------------------- dense global assembly

def _cells(mesh):
    """(global node ids [4] in CORNERS order) of every fluid fine cell."""
    nxn = mesh.wxf + 1
    out = []
    for j in range(mesh.wyf):
        for i in range(mesh.wxf):
            if not mesh.solid_f[j, i]:
                out.append([(j + cy) * nxn + i + cx for cx, cy in CORNERS])
    return out


def _assemble(mesh, cells=None):
    hx, hy = mesh.hxf, mesh.hyf
    n = mesh.Nf
    M, S, Gx, Gy = (np.zeros((n, n)) for _ in range(4))
    Tx, Ty = np.zeros((n, n, n)), np.zeros((n, n, n))
    for nodes in (_cells(mesh) if cells is None else cells):
        ix = np.ix_(nodes, nodes)
        M[ix] += hx * hy * M_REF
        S[ix] += (hy / hx) * SXX + (hx / hy) * SYY
        Gx[ix] += hy * GX
        Gy[ix] += hx * GY
        ix3 = np.ix_(nodes, nodes, nodes)
        Tx[ix3] += hy * TX
        Ty[ix3] += hx * TY
    return M, S, Gx, Gy, Tx, Ty


def _projection_matrix(mesh, m, n):
    """Global matrix of the bilinear interpolant of the 2h-patch's 4 corners."""
    nxn = mesh.wxf + 1
    Pi = np.zeros((mesh.Nf, mesh.Nf))
    for b in range(3):
        for a in range(3):
            row = (2 * n + b) * nxn + 2 * m + a
            for cx, cy in CORNERS:
                col = (2 * n + 2 * cy) * nxn + 2 * m + 2 * cx
                Pi[row, col] += float(_peval(_B[(cx, cy)], Fraction(a, 2), Fraction(b, 2)))
    return Pi


def _lps_matrix(mesh, prm):
    nxn = mesh.wxf + 1
    alpha = prm.alpha0 * (mesh.hxf ** 2 + mesh.hyf ** 2) / prm.nu
    A = np.zeros((mesh.Nf, mesh.Nf))
    eye = np.eye(mesh.Nf)
    for n in range(mesh.wyf // 2):
        for m in range(mesh.wxf // 2):
            blk = mesh.solid_f[2 * n:2 * n + 2, 2 * m:2 * m + 2]
            if blk.any():
                continue
            cells = [[(2 * n + dj + cy) * nxn + 2 * m + di + cx for cx, cy in CORNERS]
                     for dj in (0, 1) for di in (0, 1)]
            S_patch = _assemble(mesh, cells)[1]
            F = eye - _projection_matrix(mesh, m, n)
            A += alpha * F.T @ S_patch @ F
    return A


def _brute_terms(mesh, prm):
    M, S, Gx, Gy, Tx, Ty = _assemble(mesh)
    return dict(M=M, S=S, Gx=Gx, Gy=Gy, Tx=Tx, Ty=Ty, L=_lps_matrix(mesh, prm))


def _conv(T, u, v, w):
    """(u d_x w + v d_y w, phi_i) from the trilinear tensors."""
    Tx, Ty = T
    return np.einsum("ibc,b,c->i", Tx, u, w) + np.einsum("ibc,b,c->i", Ty, v, w)


def brute_residual(mesh, prm, A, x, b):
    u, v, p = x
    C = (A["Tx"], A["Ty"])
    ru = b[0] - (A["M"] @ u / prm.k + 0.5 * _conv(C, u, v, u)
                 + 0.5 * prm.nu * A["S"] @ u - A["Gx"] @ p)
    rv = b[1] - (A["M"] @ v / prm.k + 0.5 * _conv(C, u, v, v)
                 + 0.5 * prm.nu * A["S"] @ v - A["Gy"] @ p)
    # divergence rows: (d_x u + d_y v, xi_i) = Gx^T u + Gy^T v
    rp = -(A["Gx"].T @ u + A["Gy"].T @ v + A["L"] @ p)
    r = np.array([ru, rv, rp])
    r[:2, mesh.dirichlet.ravel()] = 0.0
    r[2, ~mesh.p_active.ravel()] = 0.0
    return r


def brute_rhs(mesh, prm, A, vel):
    u, v = vel
    C = (A["Tx"], A["Ty"])
    bu = A["M"] @ u / prm.k - 0.5 * _conv(C, u, v, u) - 0.5 * prm.nu * A["S"] @ u
    bv = A["M"] @ v / prm.k - 0.5 * _conv(C, u, v, v) - 0.5 * prm.nu * A["S"] @ v
    out = np.array([bu, bv])
    out[:, mesh.dirichlet.ravel()] = 0.0
    return out


# ----------------------------------------------------------------------- pins

def test_exact_reference_integrals():
    # textbook Q1 values on the unit square: mass diag 1/9, edge 1/18, diagonal
    # 1/36; stiffness diag 2/3, edge -1/6, diagonal -1/3; partition of unity
    # makes each trilinear row sum over the carrier equal the gradient matrix.
    assert np.allclose(M_REF[0], [1 / 9, 1 / 18, 1 / 18, 1 / 36])
    assert np.allclose((SXX + SYY)[0], [2 / 3, -1 / 6, -1 / 6, -1 / 3])
    assert np.allclose(TX.sum(axis=1), GX.T)
    assert np.allclose(TY.sum(axis=1), GY.T)
    assert np.allclose(GX.sum(axis=0), 0.0)


MESHES = {
    "4x2_K1": dict(nxc=4, nyc=2, K=1, s=1),
    "4x2_K2_s2": dict(nxc=4, nyc=2, K=2, s=2),
    "4x4_K1_obstacle": dict(nxc=4, nyc=4, K=1, s=2,
                            solid=np.array([[0, 0, 0, 0], [0, 1, 0, 0],
                                            [0, 1, 1, 0], [0, 0, 0, 0]], bool)),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_residual_equals_dense_assembly(name):
    mesh = Mesh(**MESHES[name])
    prm = Params(nu=0.02, k=0.05, alpha0=0.3)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((3, mesh.Nf))
    b = rng.standard_normal((2, mesh.Nf))
    A = _brute_terms(mesh, prm)
    r_orc = fem.residual(mesh, prm, x, b)
    r_bf = brute_residual(mesh, prm, A, x, b)
    for c in range(3):
        scale = np.abs(r_bf[c]).max()
        assert scale > 0
        np.testing.assert_allclose(r_orc[c], r_bf[c], rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("name", sorted(MESHES))
def test_rhs_equals_dense_assembly(name):
    mesh = Mesh(**MESHES[name])
    prm = Params(nu=0.02, k=0.05)
    rng = np.random.default_rng(12)
    vel = rng.standard_normal((2, mesh.Nf))
    A = _brute_terms(mesh, prm)
    b_orc = fem.rhs(mesh, prm, vel)
    b_bf = brute_rhs(mesh, prm, A, vel)
    scale = np.abs(b_bf).max()
    np.testing.assert_allclose(b_orc, b_bf, rtol=0, atol=1e-12 * scale)


def test_each_term_is_seen():
    # Every operator enters the comparison: switching one off in the brute
    # force moves the residual by far more than the tolerance above.
    mesh = Mesh(**MESHES["4x4_K1_obstacle"])
    prm = Params(nu=0.02, k=0.05, alpha0=0.3)
    rng = np.random.default_rng(13)
    x = rng.standard_normal((3, mesh.Nf))
    b = np.zeros((2, mesh.Nf))
    A = _brute_terms(mesh, prm)
    ref = brute_residual(mesh, prm, A, x, b)
    for key in ("M", "S", "Gx", "Gy", "Tx", "Ty", "L"):
        B = dict(A)
        B[key] = np.zeros_like(A[key])
        moved = np.abs(brute_residual(mesh, prm, B, x, b) - ref).max()
        assert moved > 1e-6 * np.abs(ref).max(), key
