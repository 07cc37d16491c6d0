"""The plain multigrid fine solve on the GPU (the method DNN-MG is compared
with, Sec. 3.3-3.4), pinned against the host FP64 solver and the oracle:

* the Newton defect, right-hand side and Jacobian-vector product equal the
  host solver's assembled operator and Newton matrix (FP64, 1e-12);
* the restriction is the transpose of the prolongation and equals the
  oracle's single-level restriction on the velocity components;
* one Vanka sweep (16 cell colours, block Gauss-Seidel) equals a NumPy
  sweep built from the host Newton matrix's dense 12 x 12 cell blocks;
* a V-cycle contracts the defect of the Newton system;
* a whole Newton-GMRES-multigrid time step equals the host solver's
  sparse-LU Newton step (FP64 to 1e-8; FP32 to 5e-4), also on a mask with
  partly solid projection patches.
"""

import numpy as np
import pytest
import torch

from helpers import rel_l2
from oracle import transfer
from oracle.mesh import Mesh as OMesh
from paper_2008_11520_gb300 import solver, synth
from parity import check

pytestmark = pytest.mark.gpu

NXC, NYC, LEVELS = 32, 8, 3          # fine level 64 x 16 (K = 1 refinement of a 32 x 8 mask)
ELL = (0.4, 0.2, 0.12, 0.07)


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def fine_mask():
    return solver.refine_mask(solver.ellipse_mask(NXC, NYC, ELL), 1)


def host_level(nx, ny, solid):
    return solver.Level(nx, ny, solid)


def flow(lev, seed=3, t=0.0):
    """A synthetic velocity/pressure field on the level's nodes with its Dirichlet values."""
    spec = synth.FlowSpec.from_seed(seed, ELL)
    x = synth.coarse_state(spec, lev.nx, lev.ny, t)
    g = lev.boundary_values(t)
    x[0, lev.dirichlet], x[1, lev.dirichlet] = g[0, lev.dirichlet], g[1, lev.dirichlet]
    x[2, ~lev.p_active] = 0.0
    return x


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


def test_mg_operators_match_host(dn):
    solid = fine_mask()
    nx, ny = solid.shape[1], solid.shape[0]
    mg = dn.MG(nx, ny, LEVELS, solid, "f64")
    lev = host_level(nx, ny, solid)
    rng = np.random.default_rng(5)
    x = flow(lev) + 0.05 * rng.standard_normal((3, lev.N))
    b = rng.standard_normal((3, lev.N)) * lev.hx * lev.hy / lev.k
    dx = rng.standard_normal((3, lev.N))
    t = 0.3
    F = mg.field(0)
    mg.defect(0, dev(x), dev(b), t, F)
    check("mg defect", rel_l2(F.cpu().numpy(), lev.defect(x, b, t)), 1e-12, "f64")
    B = mg.field(0)
    mg.rhs(0, dev(x), B)
    ref = np.zeros((3, lev.N))
    ref[:2] = lev.rhs(x[:2])
    check("mg rhs", rel_l2(B.cpu().numpy(), ref), 1e-12, "f64")
    y = mg.field(0)
    mg.jvp(0, dev(x), dev(dx), y)
    Jd = (lev.jacobian(x) @ dx.ravel()).reshape(3, -1)
    check("mg J dx", rel_l2(y.cpu().numpy(), Jd), 1e-12, "f64")
    # the coarser levels' masks: patches all fluid or all solid, nested in the finer ones
    for l in range(1, LEVELS):
        cnx, cny, cs = mg.level(l)
        fnx, fny, fs = mg.level(l - 1)
        assert (cnx, cny) == (fnx // 2, fny // 2)
        blk = cs.reshape(cny // 2, 2, cnx // 2, 2)
        assert np.all(blk.all(axis=(1, 3)) == blk.any(axis=(1, 3)))
        assert not np.any(cs & ~fs.reshape(cny, 2, cnx, 2).all(axis=(1, 3)))


def test_mg_operators_partly_solid_patches(dn):
    # a single level's own centroid mask leaves 2x2-cell projection patches
    # partly solid; the host solver reads the projection sum over the fluid
    # cells of such a patch, and the kernels take the same patch matrices
    solid = solver.ellipse_mask(64, 16, ELL)
    blk = solid.reshape(8, 2, 32, 2)
    assert np.any(blk.any(axis=(1, 3)) & ~blk.all(axis=(1, 3)))
    mg = dn.MG(64, 16, 2, solid, "f64")
    lev = host_level(64, 16, solid)
    rng = np.random.default_rng(6)
    x = flow(lev) + 0.05 * rng.standard_normal((3, lev.N))
    b = rng.standard_normal((3, lev.N)) * lev.hx * lev.hy / lev.k
    dx = rng.standard_normal((3, lev.N))
    F = mg.field(0)
    mg.defect(0, dev(x), dev(b), 0.1, F)
    check("mg defect (partly solid patches)", rel_l2(F.cpu().numpy(), lev.defect(x, b, 0.1)), 1e-12, "f64")
    y = mg.field(0)
    mg.jvp(0, dev(x), dev(dx), y)
    Jd = (lev.jacobian(x) @ dx.ravel()).reshape(3, -1)
    check("mg J dx (partly solid patches)", rel_l2(y.cpu().numpy(), Jd), 1e-12, "f64")
    d0 = 0.1 * rng.standard_normal((3, lev.N))
    d = dev(d0)
    mg.vanka(0, dev(x), dev(b), d, 0.9)
    check("mg Vanka sweep (partly solid patches)", rel_l2(d.cpu().numpy(), vanka_reference(lev, x, b, d0, 0.9)),
          1e-11, "f64")


def test_mg_transfers(dn):
    solid = fine_mask()
    nx, ny = solid.shape[1], solid.shape[0]
    mg = dn.MG(nx, ny, LEVELS, solid, "f64")
    fine = host_level(nx, ny, solid)
    cnx, cny, cs = mg.level(1)
    coarse = host_level(cnx, cny, cs)
    rng = np.random.default_rng(7)
    rf = rng.standard_normal((3, fine.N))
    dc = rng.standard_normal((3, coarse.N))
    # fixed rows hold no residual and no correction
    rf[:2, fine.dirichlet] = 0.0
    rf[2, ~fine.p_active] = 0.0
    dc[:2, coarse.dirichlet] = 0.0
    dc[2, ~coarse.p_active] = 0.0
    rc, df = mg.field(1), mg.field(0)
    mg.restrict(0, dev(rf), rc)
    mg.prolong_add(0, dev(dc), df)
    lhs = float(np.sum(rc.cpu().numpy() * dc))
    rhs = float(np.sum(rf * df.cpu().numpy()))
    check("mg <R r, d> - <r, P d>", abs(lhs - rhs) / abs(rhs), 1e-13, "f64")
    # the velocity components equal the oracle's single-level R = P^T
    om = OMesh(cnx, cny, 1, 1, solid=np.zeros((cny, cnx), dtype=bool))
    ref = transfer.restrict_raw(om, rf[:2])
    got = rc.cpu().numpy()[:2]
    free = ~coarse.dirichlet
    check("mg R vs oracle", rel_l2(got[:, free], ref[:, free]), 1e-14, "f64")
    # injection
    xc = mg.field(1)
    mg.inject(0, dev(rf), xc)
    assert np.array_equal(xc.cpu().numpy(), rf.reshape(3, ny + 1, nx + 1)[:, ::2, ::2].reshape(3, -1))


def vanka_reference(lev, x, r, d0, omega):
    """One Vanka sweep in 16 cell colours from the host Newton matrix: each
    fluid cell of a colour solves its dense 12 x 12 block against the defect
    r - J d on its unknowns and adds omega times the solution."""
    J = lev.jacobian(x).tocsr()
    N, nxn = lev.N, lev.nx + 1
    fixed = np.concatenate([lev.dirichlet, lev.dirichlet, ~lev.p_active])
    d = d0.ravel().copy()
    for cy in range(4):
        for cx in range(4):
            res = r.ravel() - J @ d                       # cells of one colour are independent
            for j in range(cy, lev.ny, 4):
                for i in range(cx, lev.nx, 4):
                    if lev.solid[j, i]:
                        continue
                    nodes = [(j + a // 2) * nxn + i + a % 2 for a in range(4)]
                    dofs = [c * N + n for n in nodes for c in range(3)]
                    A = J[dofs][:, dofs].toarray()
                    z_rhs = res[dofs].copy()
                    for k, q in enumerate(dofs):
                        if fixed[q]:                      # identity row of the Newton matrix
                            A[k, :] = 0.0
                            A[k, k] = 1.0
                    d[dofs] += omega * np.linalg.solve(A, z_rhs)
    # fixed unknowns (identity rows), also those in no fluid cell: correction = their defect
    d[fixed] = r.ravel()[fixed]
    return d.reshape(3, N)


def test_vanka_sweep_matches_reference(dn):
    solid = solver.refine_mask(solver.ellipse_mask(16, 4, (0.4, 0.2, 0.2, 0.1)), 1)   # 32 x 8 fine cells
    nx, ny = solid.shape[1], solid.shape[0]
    mg = dn.MG(nx, ny, 2, solid, "f64")
    lev = host_level(nx, ny, solid)
    rng = np.random.default_rng(9)
    x = flow(lev) + 0.05 * rng.standard_normal((3, lev.N))
    r = rng.standard_normal((3, lev.N))
    d0 = 0.1 * rng.standard_normal((3, lev.N))
    d = dev(d0)
    mg.vanka(0, dev(x), dev(r), d, 0.7)
    check("mg Vanka sweep", rel_l2(d.cpu().numpy(), vanka_reference(lev, x, r, d0, 0.7)), 1e-11, "f64")


def test_vcycle_contracts(dn):
    from paper_2008_11520_gb300.mg import PlainMG
    solid = fine_mask()
    nx, ny = solid.shape[1], solid.shape[0]
    pm = PlainMG(nx, ny, LEVELS, solid, "f64")
    lev = host_level(nx, ny, solid)
    x = dev(flow(lev))
    pm.linearize(x)
    rng = np.random.default_rng(11)
    r = rng.standard_normal((3, lev.N))          # fixed rows included: the cycle must set them
    b = dev(r)
    d = pm.mg.field(0)
    res = b.clone()
    norms = [pm.norm(res)]
    z = pm.mg.field(0)
    for _ in range(6):
        pm.vcycle(0, res, z)
        pm.mg.axpby(1.0, z, 1.0, d)
        pm.mg.jvp(0, x, d, res)
        pm.mg.axpby(1.0, b, -1.0, res)
        norms.append(pm.norm(res))
    rates = [norms[i + 1] / norms[i] for i in range(len(norms) - 1)]
    # The coarse levels are rediscretised, not Galerkin products.  The fine
    # projection term vanishes on a prolongated pressure (P p_c is bilinear on
    # every fine patch), while a coarse level keeps its own, so pressure
    # corrections on coarse scales are damped: the cycle contracts, but not
    # by the textbook factor.  GMRES takes up the rest.
    check("mg V-cycle contraction (worst of 6)", max(rates), 0.75, "f64")


# FP32: the defect of a converged iterate is the rounding of its O(hx hy / k)
# terms (relative 6e-8), and the Newton matrix's condition on this mesh
# (about 1e3 to 1e4, the pressure block) scales that into the solution.
@pytest.mark.parametrize("prec,tol,single", [("f64", 1e-8, False), ("f32", 5e-4, False), ("f64", 1e-8, True)])
def test_newton_mg_step_matches_host(dn, prec, tol, single):
    from paper_2008_11520_gb300.mg import PlainMG
    # single: the level's own centroid mask (partly solid projection patches)
    solid = solver.ellipse_mask(64, 16, ELL) if single else fine_mask()
    nx, ny = solid.shape[1], solid.shape[0]
    pm = PlainMG(nx, ny, LEVELS, solid, prec)
    lev = host_level(nx, ny, solid)
    x0 = flow(lev)
    x0[:2, lev.dirichlet] *= 0.9                   # the step must restore the boundary values
    t1 = 0.01
    ref = lev.solve(lev.rhs(x0[:2]), t1, x0=x0)
    x = dev(x0, pm.mg.real)
    pm.step(x, t1, tol=1e-10 if prec == "f64" else 1e-5, lin_rtol=1e-6 if prec == "f64" else 1e-4)
    got = x.double().cpu().numpy()
    check("plain MG step (u, v)", rel_l2(got[:2], ref[:2]), tol, prec)
    check("plain MG step (p)", rel_l2(got[2], ref[2]), 100 * tol, prec)
    assert pm.stats["newton_iterations"] >= 1 and pm.stats["vcycles"] >= 1
