"""The host level solver (the coarse solve of Algorithm 2 and the fine reference solve).

The solver is supporting code outside the correction step; these tests pin
it to the oracle's definition of the discrete system and to what the
mathematics fixes (exact Newton matrix of a quadratic map, quadratic
convergence, the Poiseuille steady state, and the zero-network reduction of
Algorithm 2 to the plain coarse solve).
"""

import numpy as np
import pytest

from oracle import fem, transfer
from oracle.mesh import Mesh, Params
from oracle.step import dnnmg_step
from paper_2008_11520_gb300 import solver

ELL = (0.6, 0.2, 0.3, 0.12)


def pair(nx=16, ny=8, ellipse=ELL, **kw):
    """The same level as a solver Level and as the fine level of an oracle Mesh
    one refinement above (nested masks, as on every level above the coarse one)."""
    prm = Params(**kw)
    solid = solver.refine_mask(solver.ellipse_mask(nx // 2, ny // 2, ellipse), 1)
    lvl = solver.Level(nx, ny, solid, nu=prm.nu, k=prm.k, alpha0=prm.alpha0,
                       u_max=prm.u_max, ramp=prm.ramp)
    mesh = Mesh(nx // 2, ny // 2, 1, 1, ellipse=ellipse)
    return lvl, mesh, prm


def test_geometry_matches_oracle_rules():
    lvl, mesh, _ = pair()
    assert lvl.solid.any()
    assert (lvl.solid == mesh.solid_f).all()
    assert (lvl.dirichlet == mesh.dirichlet.ravel()).all()
    assert (lvl.inflow == mesh.inflow.ravel()).all()
    assert (lvl.p_active == mesh.p_active.ravel()).all()
    fine = solver.refine_mask(lvl.solid, 2)
    assert fine.shape == (32, 64) and fine.sum() == 16 * lvl.solid.sum()


@pytest.mark.parametrize("nu", [1e-3, 0.05])
def test_operator_and_rhs_equal_oracle(nu):
    lvl, mesh, prm = pair(nu=nu, k=0.02, alpha0=0.2)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, lvl.N))
    # oracle residual with b = 0 is -A(x) on free rows
    r = fem.residual(mesh, prm, x, np.zeros((2, lvl.N)))
    A = lvl.operator(x)
    free = [~lvl.dirichlet, ~lvl.dirichlet, lvl.p_active]
    for c in range(3):
        scale = np.abs(A[c][free[c]]).max()
        np.testing.assert_allclose(-A[c][free[c]], r[c][free[c]], rtol=0, atol=1e-12 * scale)
    b_or = fem.rhs(mesh, prm, x[:2])
    np.testing.assert_allclose(lvl.rhs(x[:2]), b_or, rtol=0, atol=1e-12 * np.abs(b_or).max())


def test_newton_matrix_is_exact_derivative():
    # the defect is quadratic in x, so a central difference with any step is exact
    lvl, _, _ = pair(nu=0.01)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, lvl.N))
    e = rng.standard_normal((3, lvl.N))
    b = rng.standard_normal((2, lvl.N))
    Je = (lvl.jacobian(x) @ e.ravel()).reshape(3, lvl.N)
    fd = 0.5 * (lvl.defect(x + e, b, 0.3) - lvl.defect(x - e, b, 0.3))
    np.testing.assert_allclose(Je, fd, rtol=0, atol=1e-11 * np.abs(fd).max())


def test_solution_zeroes_oracle_residual_and_carries_boundary_values():
    lvl, mesh, prm = pair(ramp=True)
    rng = np.random.default_rng(5)
    prev = 0.3 * rng.standard_normal((3, lvl.N))
    b = lvl.rhs(prev[:2])
    hist = []
    t = 0.25
    x = lvl.solve(b, t, x0=prev, history=hist)
    r = fem.residual(mesh, prm, x, b)
    assert np.abs(r).max() <= 1e-10 * np.abs(b).max()
    mask, uD, vD = transfer.dirichlet_velocity(mesh, prm, t)
    assert np.array_equal(x[0, mask], uD[mask]) and np.array_equal(x[1, mask], vD[mask])
    assert not x[2, ~lvl.p_active].any()
    # quadratic convergence: a handful of iterations, each squaring the defect
    assert len(hist) <= 7
    tail = [h for h in hist if h > 1e-9 * hist[0]]
    for a, c in zip(tail[1:], tail[2:]):
        assert c <= 10 * a * a / hist[0] + 1e-13 * hist[0]


def test_poiseuille_is_a_steady_state():
    # without obstacle the nodal Poiseuille profile with its linear pressure drop
    # solves the discrete system exactly (the S2 pin), so a step keeps it
    lvl, _, prm = pair(nx=16, ny=8, ellipse=None)
    X = (np.arange(lvl.N) % (lvl.nx + 1)) * lvl.hx
    y = lvl.y
    x = np.array([prm.u_max * 4 * y * (lvl.ly - y) / lvl.ly ** 2,
                  np.zeros(lvl.N),
                  8 * prm.u_max * prm.nu / lvl.ly ** 2 * (lvl.lx - X)])
    x1 = lvl.advance(x, 0.01)
    np.testing.assert_allclose(x1, x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_zero_network_run_is_the_plain_coarse_solve():
    # Algorithm 2 with d = 0 hands the coarse solver the coarse level's own
    # right-hand side (exact for zero boundary data), so the run equals plain
    # time stepping on the coarse level; the correction is the oracle's step.
    ell = (0.6, 0.2, 0.3, 0.12)
    nxc, nyc, K = 16, 8, 1
    prm = Params(u_max=0.0)
    coarse = solver.Level(nxc, nyc, solver.ellipse_mask(nxc, nyc, ell), u_max=0.0)
    m = Mesh(nxc, nyc, K, 1, ellipse=ell)
    rng = np.random.default_rng(6)
    x0 = np.zeros((3, coarse.N))
    x0[:2] = rng.standard_normal((2, coarse.N))
    x0[:2, coarse.dirichlet] = 0.0
    H = 4
    W = (0.1 * rng.standard_normal((3 * H, m.n_in)), 0.1 * rng.standard_normal((3 * H, H)),
         np.zeros((m.n_out, H)))
    state = {"h": np.zeros((m.P, H)), "bf": np.zeros((2, m.Nf))}

    def correct(xc, t):
        o = dnnmg_step(m, prm, W, xc, state["h"], state["bf"], t)
        state["h"], state["bf"] = o["h"], o["bf"]
        return o["bc"]

    run = solver.dnnmg_run(coarse, correct, 4, x0=x0)
    plain = solver.simulate(coarse, 4, x0=x0)
    for a, b in zip(run, plain):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())
    assert np.abs(plain[-1][:2]).max() > 0.1


def test_level_rejects_odd_cells():
    with pytest.raises(ValueError):
        solver.Level(15, 8)


def test_projection_term_on_partly_solid_patches():
    # a coarse-level mask is not nested: some 2x2-cell patches are partly solid.
    # Each patch then contributes its fluid cells' integrals, so the term stays
    # symmetric, positive semidefinite and zero on linear pressures (pi
    # reproduces them), and it equals the sum of the per-cell forms.
    lvl = solver.Level(16, 8, solver.ellipse_mask(16, 8, ELL))
    blk = lvl.solid.reshape(4, 2, 8, 2).transpose(0, 2, 1, 3).reshape(4, 8, 4)
    assert (blk.any(axis=2) & ~blk.all(axis=2)).any()
    L = lvl.L.toarray()
    np.testing.assert_allclose(L, L.T, rtol=0, atol=1e-14 * np.abs(L).max())
    X = (np.arange(lvl.N) % (lvl.nx + 1)) * lvl.hx
    assert np.abs(L @ (0.3 + 2.0 * X - 5.0 * lvl.y)).max() <= 1e-12 * np.abs(L).max()
    assert np.linalg.eigvalsh(L).min() >= -1e-12 * np.abs(L).max()
    # a pressure living on the nodes of one fully solid patch costs nothing
    n, m = np.argwhere(blk.all(axis=2))[0]
    nodes = [(2 * n + b) * (lvl.nx + 1) + 2 * m + a for b in range(3) for a in range(3)]
    centre = np.zeros(lvl.N)
    centre[nodes[4]] = 1.0
    assert centre @ L @ centre == 0.0
    # a patch with fluid and solid cells: its centre node's energy is the
    # fluid cells' share of the full patch's (each cell holds a quarter)
    n, m = np.argwhere(blk.any(axis=2) & ~blk.all(axis=2))[0]
    c = (2 * n + 1) * (lvl.nx + 1) + 2 * m + 1
    e = np.zeros(lvl.N)
    e[c] = 1.0
    full = solver.Level(16, 8)
    assert e @ L @ e == pytest.approx((~blk[n, m]).sum() / 4 * (e @ full.L @ e), rel=1e-13)


@pytest.fixture(scope="module")
def tl():
    import os
    from paper_2008_11520_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2008_11520_gb300 import dnnmg, timeloop
    return dnnmg, timeloop


@pytest.mark.parametrize("K", [1, 2])
def test_levels_from_mesh_descriptor(tl, K):
    # host-only: the Levels the time loop builds from a library mesh
    # descriptor have the oracle's geometry on both levels and its parameters
    dn, timeloop = tl
    ell = (0.6, 0.2, 0.3, 0.12)
    d = dn.make_desc(16, 8, K, 1, ellipse=ell, precision="f32", ramp=True, nu=0.01, u_max=1.2)
    c, f = timeloop.coarse_level(d), timeloop.fine_level(d)
    om = Mesh(16, 8, K, 1, ellipse=ell)
    assert (c.solid == om.solid_coarse).all() and (f.solid == om.solid_f).all()
    assert (f.dirichlet == om.dirichlet.ravel()).all() and (f.p_active == om.p_active.ravel()).all()
    assert (c.dirichlet == om.dirichlet_c.ravel()).all()
    assert (c.nu, c.k, c.alpha0, c.u_max, c.ramp) == (0.01, 0.01, 0.1, 1.2, True)
    assert (f.nx, f.ny, f.u_max) == (16 * 2 ** K, 8 * 2 ** K, 1.2)
    solid = np.zeros((8, 16), dtype=np.uint8)
    solid[2:6, 6:8] = 1
    c2 = timeloop.coarse_level(dn.make_desc(16, 8, K, 2, solid=solid))
    assert (c2.solid == solid.astype(bool)).all()


def test_chord_iterations_reach_the_newton_solution():
    # reusing a factorisation changes the path, not the solution
    lvl, mesh, prm = pair(ramp=True)
    ref = solver.Level(lvl.nx, lvl.ny, lvl.solid, ramp=True)
    xa = xb = np.zeros((3, lvl.N))
    for n in range(1, 9):
        t = n * lvl.k
        b = lvl.rhs(xa[:2])
        xa = lvl.solve(b, t, x0=xa, newton="chord")
        xb = ref.solve(ref.rhs(xb[:2]), t, x0=xb, newton="exact")
        np.testing.assert_allclose(xa, xb, rtol=0, atol=1e-10 * np.abs(xb).max())
        scale = max(np.abs(b).max(), np.abs(lvl.operator(xa)).max())
        assert np.abs(fem.residual(mesh, prm, xa, b)).max() <= 1e-10 * scale
    assert lvl.factorisations < ref.factorisations / 2


@pytest.mark.parametrize("geometry", ["ellipse", "none", "two", "L"])
def test_solution_conserves_mass(geometry):
    # The pressure rows make (div v, xi_i) + projection term vanish; summed
    # over all nodes the projection terms cancel (pi reproduces constants) and
    # the divergence terms give the net flux out of the fluid, which is the
    # outflow at x = lx minus the inflow at x = 0 (walls and obstacles are
    # no-slip; solid nodes on the outflow column carry zero).  v.n is linear
    # along boundary edges: the trapezoidal rule on nodal values is exact.
    if geometry == "ellipse":
        lvl, _, _ = pair(ramp=True)
    else:
        lvl = solver.Level(32, 8, solver.geometry_mask(32, 8, geometry), ramp=True)
    x = solver.simulate(lvl, 12)[-1]
    U = x[0].reshape(lvl.ny + 1, lvl.nx + 1)
    trapz = lambda f: lvl.hy * (f.sum() - 0.5 * (f[0] + f[-1]))
    q_in, q_out = trapz(U[:, 0]), trapz(U[:, -1])
    assert q_in > 0.05
    assert abs(q_out - q_in) <= 1e-10 * q_in


def test_generated_flows_are_the_level_solutions(tmp_path):
    out = tmp_path / "flows.npz"
    solver.main(["--nxc", "16", "--nyc", "8", "--K", "1", "--steps", "3", "--ratios", "0.6,1.0",
                 "--out", str(out)])
    z = np.load(out)
    assert z["fine"].shape == (2, 4, 2, 33 * 17) and z["coarse"].shape == (2, 3, 3, 17 * 9)
    assert not z["fine"][:, 0].any()
    for i, q in enumerate((0.6, 1.0)):
        ell = tuple(z["ellipses"][i])
        assert ell == (0.2, 0.2, 0.05, 0.05 * q)
        solid = solver.ellipse_mask(16, 8, ell)
        c = solver.Level(16, 8, solid, ramp=True)
        f = solver.Level(32, 16, solver.refine_mask(solid, 1), ramp=True)
        for a, b in zip(z["coarse"][i], solver.simulate(c, 3)):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())
        for a, b in zip(z["fine"][i][1:], solver.simulate(f, 3)):
            np.testing.assert_allclose(a, b[:2], rtol=0, atol=1e-6 * np.abs(b[:2]).max())


def test_operator_equals_oracle_on_a_single_level_mask():
    # the coarse level's own mask leaves projection patches partly solid:
    # both the solver and the oracle then sum over the fluid cells only
    ell = (0.6, 0.2, 0.3, 0.12)
    lvl = solver.Level(16, 8, solver.ellipse_mask(16, 8, ell))
    mesh, prm = Mesh(16, 8, 0, 1, ellipse=ell), Params()
    rng = np.random.default_rng(9)
    x = rng.standard_normal((3, lvl.N))
    r = fem.residual(mesh, prm, x, np.zeros((2, lvl.N)))
    A = lvl.operator(x)
    free = [~lvl.dirichlet, ~lvl.dirichlet, lvl.p_active]
    for c in range(3):
        scale = np.abs(A[c][free[c]]).max()
        np.testing.assert_allclose(-A[c][free[c]], r[c][free[c]], rtol=0, atol=1e-12 * scale)


def test_geometry_flow_is_the_level_solution(tmp_path):
    # Sec. 6.7 geometries: the stored mask is the named one and the stored
    # solutions are the two levels' runs on it
    out = tmp_path / "two.npz"
    solver.main(["--nxc", "32", "--nyc", "8", "--K", "1", "--steps", "3", "--geometry", "two", "--out", str(out)])
    z = np.load(out)
    solid = solver.geometry_mask(32, 8, "two")
    assert solid.sum() > 0 and (z["solid"] == solid).all()
    assert z["fine"].shape == (1, 4, 2, 65 * 17) and z["coarse"].shape == (1, 3, 3, 33 * 9)
    c = solver.Level(32, 8, solid, ramp=True)
    f = solver.Level(64, 16, solver.refine_mask(solid, 1), ramp=True)
    for a, b in zip(z["coarse"][0], solver.simulate(c, 3)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())
    for a, b in zip(z["fine"][0][1:], solver.simulate(f, 3)):
        np.testing.assert_allclose(a, b[:2], rtol=0, atol=1e-6 * np.abs(b[:2]).max())


def test_geometry_masks():
    nx, ny = 64, 16
    xc = (np.arange(nx) + 0.5) * (2.2 / nx)
    yc = (np.arange(ny) + 0.5) * (0.41 / ny)
    assert not solver.geometry_mask(nx, ny, "none").any()
    L = solver.geometry_mask(nx, ny, "L")
    # the upper half of the right half, every cell of it, nothing else
    assert L.sum() == (nx // 2) * (ny // 2) and L[ny // 2:, nx // 2:].all()
    two = solver.geometry_mask(nx, ny, "two")
    j, i = np.nonzero(two)
    # two separate obstacles, each around its centre and inside its bounding box
    left = xc[i] < 0.4
    for sel, (cx, cy) in ((left, (0.2, 0.18)), (~left, (0.6, 0.24))):
        assert sel.any()
        assert (np.abs(xc[i[sel]] - cx) < 0.055).all() and (np.abs(yc[j[sel]] - cy) < 0.045).all()
    with pytest.raises(ValueError):
        solver.geometry_mask(nx, ny, "circle")
    # the parity suite's own masks of the same geometries (written separately for the oracle meshes)
    from helpers import geometry_mask as parity_mask
    for g in ("two", "L"):
        for nxc, nyc in ((64, 12), (40, 10), (128, 32)):
            assert (parity_mask({"nxc": nxc, "nyc": nyc, "geometry": g}) == solver.geometry_mask(nxc, nyc, g)).all()


def test_channel_without_obstacle_is_mirror_symmetric():
    # the empty channel and its parabolic inflow are symmetric about y = H/2, so
    # u is even and v odd under the mirror, on both levels and at every step
    z = solver.generate_flow(16, 8, 1, 4, solver.geometry_mask(16, 8, "none"))
    for sol, (nx, ny) in ((z["coarse"][0][1:], (16, 8)), (z["fine"][0][1:], (32, 16))):
        for x in sol:
            u = np.asarray(x[0], dtype=np.float64).reshape(ny + 1, nx + 1)
            v = np.asarray(x[1], dtype=np.float64).reshape(ny + 1, nx + 1)
            scale = np.abs(u).max()
            assert scale > 1e-3
            np.testing.assert_allclose(u, u[::-1], rtol=0, atol=1e-5 * scale)
            np.testing.assert_allclose(v, -v[::-1], rtol=0, atol=1e-5 * scale)
