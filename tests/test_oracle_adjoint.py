"""Pins of the oracle's gradient (oracle.Problem.adjoint, the hand-written FP64
reverse pass) and of its own GMRES, on the CPU.

* The point-charge field E = q x/|x|^3 (the continuum field of a unit sphere at
  potential q): dK/dq per line equals the closed form 0.0720913901, whose event part
  d / (2 sqrt(q E0)) = 0.0707107 comes entirely from the located |E| = E0 crossing.
* Central differences (step 1e-5) of the oracle's forward -- dense assembly, LU
  solve, tracer -- on small meshes with every row kind: a conductor sphere, a
  dielectric body, a closed floating body, an open floating sheet with different
  permittivities on its two sides.  Seeded vertex coordinates, V0 and the
  permittivities.  Tolerance as in the GPU adjoint tests:
  |g - g_FD| <= 1e-4 max(|g_FD|, 1e-3 max|g_FD|) + 50 ulp(|J|)/step.
* The complex-step derivatives of the closed-form pair integrals against central
  differences, including a target whose projection lies exactly on an edge's line
  (d = 0: the case where a guard on d must not drop the derivative f d').
* dJ/deps = 0 where no row depends on a permittivity (Q17 of the design notes).
* GMRES(m) against LU.
"""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

H = 0.02
STEP = 1e-5


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    return oracle


def _combine(bodies, regions):
    Xs, Ts, Rs, off = [], [], [], 0
    for (X, tri), r in bodies:
        Xs.append(X)
        Ts.append(tri + off)
        Rs.append(np.full(len(tri), r, np.int32))
        off += len(X)
    return mg.Mesh(np.concatenate(Xs), np.concatenate(Ts).astype(np.int32), np.concatenate(Rs), regions)


def _with(mesh, X=None, regions=None):
    return mg.Mesh(mesh.X if X is None else X, mesh.tri, mesh.region,
                   mesh.regions if regions is None else regions)


def _J(O, mesh, seeds, w):
    P = O.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    K, st, _, _ = P.trace(u, seeds, O.TraceParams(h=H))
    assert np.all(st == 1)
    return float((K * w).sum())


def _close(g, gfd, J, scale):
    floor = 50 * np.finfo(float).eps * abs(J) / STEP
    tol = 1e-4 * np.maximum(np.abs(gfd), 1e-3 * scale) + floor
    return np.abs(g - gfd) <= tol


def test_point_charge_dK_dq_closed_form(O):
    """K and dK/dq along radial lines of the point charge: -0.858317220 and
    0.0720913901 per line (h = 1e-3; RK4 error far below 1e-8)."""
    seeds = mg.fibonacci_seeds(6)
    w = np.array([1.0, 2.0, 0.5, 1.5, 1.0, 3.0])
    K, st, gq = O.adjoint_point_charge(seeds, w=w, q=1.0)
    assert np.all(st == 1)
    assert np.allclose(K, -0.858317220, atol=1e-8)
    assert abs(gq / w.sum() - 0.0720913901) < 1e-8
    # q = 2: the same lines, K(q) and dK/dq from the closed form's q-dependence
    K2, _, gq2 = O.adjoint_point_charge(seeds, w=1.0, q=2.0)
    Kp = O.trace_point_charge(seeds, q=2.0 + 1e-6)[0].sum()
    Km = O.trace_point_charge(seeds, q=2.0 - 1e-6)[0].sum()
    assert abs(gq2 - (Kp - Km) / 2e-6) < 1e-6 * abs(gq2)


CASES = {
    "sphere": (lambda: mg.sphere_mesh(1), lambda s: s[::4], [(0, "V0", 0)]),
    "dielectric": (lambda: _combine([(mg.icosphere(1, 1.0), 0), (mg.icosphere(1, 0.7, (0.0, 0.0, -2.5)), 1)],
                                    [{"kind": "conductor", "V0": 1.0},
                                     {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}]),
                   lambda s: s[s[:, 2] > 0.3][::2],
                   [(0, "V0", 0), (1, "eps_plus", 0), (1, "eps_minus", 1)]),
    "floating": (lambda: _combine([(mg.icosphere(1, 1.0), 0), (mg.icosphere(1, 0.5, (2.5, 0.3, 0.0)), 1)],
                                  [{"kind": "conductor", "V0": 1.0},
                                   {"kind": "floating", "floating_id": 0, "eps_plus": 1.0}]),
                 lambda s: s[2::5][s[2::5][:, 0] < 0.5],
                 [(0, "V0", 0), (1, "eps_plus", 0)]),
    "sheet": (lambda: _combine([(mg.icosphere(1, 1.0), 0),
                                ((mg.open_cylinder(0.4, -0.5, 0.5, 8, 3)[0] + np.array([2.5, 0.0, 0.0]),
                                  mg.open_cylinder(0.4, -0.5, 0.5, 8, 3)[1]), 1)],
                               [{"kind": "conductor", "V0": 1.0},
                                {"kind": "sheet", "floating_id": 0, "eps_plus": 1.0, "eps_minus": 3.0}]),
              lambda s: s[s[:, 0] < -0.2][::2],
              [(0, "V0", 0), (1, "eps_plus", 0), (1, "eps_minus", 1)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_against_differences(O, name):
    make, pick, params = CASES[name]
    mesh = make()
    seeds = pick(mg.fibonacci_seeds(16))
    w = np.random.default_rng(3).uniform(0.5, 1.5, len(seeds))
    P = O.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    K, gX, gV0, geps = P.adjoint(u, seeds, w, O.TraceParams(h=H))
    J = float((K * w).sum())
    assert abs(J - _J(O, mesh, seeds, w)) <= 1e-13 * abs(J)
    rng = np.random.default_rng(1)
    # coordinates of every body: a few of the first body's, a few of the second's
    n1 = int(mesh.tri[mesh.region == 0].max()) + 1
    flat = np.concatenate([rng.choice(3 * n1, 4, replace=False),
                           rng.choice(np.arange(3 * n1, mesh.X.size), 4, replace=False)
                           if mesh.X.size > 3 * n1 else np.array([], int)])
    g_fd = []
    for f in flat:
        Xp, Xm = mesh.X.copy(), mesh.X.copy()
        Xp.flat[f] += STEP
        Xm.flat[f] -= STEP
        g_fd.append((_J(O, _with(mesh, Xp), seeds, w) - _J(O, _with(mesh, Xm), seeds, w)) / (2 * STEP))
    g_fd = np.array(g_fd)
    scale = np.abs(g_fd).max()
    ok = _close(gX.reshape(-1)[flat], g_fd, J, scale)
    assert ok.all(), (flat[~ok], gX.reshape(-1)[flat][~ok], g_fd[~ok])
    for r, key, col in params:
        rp = [dict(x) for x in mesh.regions]
        rm = [dict(x) for x in mesh.regions]
        rp[r][key] += STEP
        rm[r][key] -= STEP
        gfd = (_J(O, _with(mesh, regions=rp), seeds, w) - _J(O, _with(mesh, regions=rm), seeds, w)) / (2 * STEP)
        g = gV0[r] if key == "V0" else geps[r, col]
        assert _close(np.array([g]), np.array([gfd]), J, abs(gfd)).all(), (name, key, g, gfd)
    if name == "sphere":
        assert np.all(geps == 0.0)


def test_pair_derivatives_complex_step(O):
    """Complex-step derivatives of S and G against central differences of the
    closed form, for targets above, below and in the plane of a triangle, one whose
    projection lies exactly on an edge's line outside the edge, and the own centroid
    moving with the vertices."""
    a, b, c = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.2, 0.9, 0.1])
    c_flat = np.array([0.2, 0.9, 0.0])
    targets = [(np.array([0.4, 0.3, 0.2]), c), (np.array([3.0, 1.0, -0.5]), c),
               (np.array([1.2, 0.8, 0.0]), c_flat),
               # on the line of edge a-b (y = 0, z = 0 plane of a, b), beyond b, above the plane
               (np.array([1.7, 0.0, 0.6]), c_flat)]
    for x, cc in targets:
        dS, dG = O.tri_exact_derivs(x, a, b, cc)
        base = np.concatenate([x, a, b, cc])
        for q in range(12):
            vp, vm = base.copy(), base.copy()
            vp[q] += 1e-6
            vm[q] -= 1e-6
            Sp, Gp = O.tri_exact(vp[:3], vp[3:6], vp[6:9], vp[9:])
            Sm, Gm = O.tri_exact(vm[:3], vm[3:6], vm[6:9], vm[9:])
            assert abs(dS[q] - (Sp - Sm) / 2e-6) < 1e-8
            assert np.abs(dG[q] - (Gp - Gm) / 2e-6).max() < 1e-8
    # own centroid: S_ii(c(X), X) with the principal value
    dS, dG = O.tri_exact_derivs((a + b + c) / 3, a, b, c, self_pair=True, centroid=True)
    base = np.concatenate([a, b, c])
    for q in range(9):
        vp, vm = base.copy(), base.copy()
        vp[q] += 1e-6
        vm[q] -= 1e-6
        Sp, _ = O.tri_exact((vp[:3] + vp[3:6] + vp[6:]) / 3, vp[:3], vp[3:6], vp[6:], self_pair=True)
        Sm, _ = O.tri_exact((vm[:3] + vm[3:6] + vm[6:]) / 3, vm[:3], vm[3:6], vm[6:], self_pair=True)
        assert abs(dS[3 + q] - (Sp - Sm) / 2e-6) < 1e-8


@pytest.mark.parametrize("mesh_name", ["sphere", "device", "sheet"])
def test_gmres_matches_lu(O, mesh_name):
    mesh = {"sphere": lambda: mg.sphere_mesh(2), "device": lambda: mg.device_mesh(scale=0.3),
            "sheet": lambda: mg.sphere_in_sheet_mesh(2)}[mesh_name]()
    P = O.Problem(mesh, eta=4.0, g=3)
    A = P.assemble()
    b = P.rhs()
    u_lu = np.linalg.solve(A, b)
    u, its, rel = P.gmres(b, tol=1e-12, matvec=lambda x: A @ x)
    assert rel <= 1e-12 and its > 0
    assert np.linalg.norm(u - u_lu) / np.linalg.norm(u_lu) < 1e-9
    # and matrix-free (the oracle's own product), to the method's tolerance
    u2, its2, rel2 = P.gmres(b, tol=1e-10, m=30)
    assert rel2 <= 1e-10
    assert np.linalg.norm(u2 - u_lu) / np.linalg.norm(u_lu) < 1e-8
