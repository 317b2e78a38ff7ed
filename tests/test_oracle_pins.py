"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each one compares it
with an independent fact -- the Stokes equations the Oseen tensor must solve,
the Faxen construction T = (1 + a^2/3 Lap) G of Sec. 2.2, textbook contact
values, positive definiteness for r >= 2a (Sec. 2.2), the invariances of Stokes
flow (Sec. 4), finite differences for every derivative, and the period of the
four-sphere orbit printed in Sec. 4.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _column_tensor(orc, r, tensor, a=1.0, eta=1.0):
    """T(r) read off the oracle's *mobility sum* (two particles, unit forces on particle 2)."""
    x = np.array([[0.0, 0.0, 0.0], -np.asarray(r, float)])  # r_1 - r_2 = r
    T = np.zeros((3, 3))
    for b in range(3):
        F = np.zeros((2, 3))
        F[1, b] = 1.0
        T[:, b] = orc.mobility_apply(x, F, tensor, a, eta)[0]
    return T


# ---------------------------------------------------------------- Stokes law / self term

def test_single_sphere_stokes_law(orc):
    g = _golden("two_sphere_mobility.json")
    assert orc.mu0(1.0, 1.0) == pytest.approx(g["stokes_mobility_a1_eta1"], rel=1e-15)
    rng = np.random.default_rng(1)
    for a, eta in [(1.0, 1.0), (0.5, 2.0), (3.0, 0.1)]:
        F = rng.standard_normal((1, 3))
        v = orc.mobility_apply(np.zeros((1, 3)), F, "rpy", a, eta)
        # drag force 6 pi eta a v balances F
        np.testing.assert_allclose(6 * math.pi * eta * a * v, F, rtol=1e-14)


# ---------------------------------------------------------------- Oseen tensor solves Stokes

def test_oseen_solves_stokes_equations(orc):
    """u = G F must be divergence free, satisfy eta Lap u = grad p with the Stokeslet
    pressure p = F.r/(4 pi r^3), and carry the force F through any sphere about the
    origin (Sec. 2.2, Eq. oseenTensor with Eq. stokes).  Checked on the oracle's
    numbers by finite differences and quadrature."""
    eta = 0.7
    F = np.array([0.3, -1.1, 0.8])

    def u(p):
        return orc.pair_tensor(p, "oseen", 1.0, eta) @ F

    def pressure(p):
        return F @ p / (4 * math.pi * np.linalg.norm(p) ** 3)

    h = 1e-3
    rng = np.random.default_rng(2)
    for _ in range(5):
        p0 = rng.standard_normal(3)
        p0 *= rng.uniform(1.0, 3.0) / np.linalg.norm(p0)
        E = np.eye(3) * h
        div = sum((u(p0 + E[d])[d] - u(p0 - E[d])[d]) / (2 * h) for d in range(3))
        lap = sum((u(p0 + E[d]) - 2 * u(p0) + u(p0 - E[d])) / h ** 2 for d in range(3))
        gradp = np.array([(pressure(p0 + E[d]) - pressure(p0 - E[d])) / (2 * h) for d in range(3)])
        scale = np.linalg.norm(gradp)
        assert abs(div) < 1e-6 * scale
        np.testing.assert_allclose(eta * lap, gradp, atol=1e-5 * scale)

    # total force transmitted through a sphere of radius R equals F
    R = 1.7
    nth, nph = 48, 96
    th = (np.arange(nth) + 0.5) * math.pi / nth
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    total = np.zeros(3)
    for t in th:
        for q in ph:
            n = np.array([math.sin(t) * math.cos(q), math.sin(t) * math.sin(q), math.cos(t)])
            p0 = R * n
            J = np.zeros((3, 3))  # J[a, b] = d u_a / d x_b
            for d in range(3):
                e = np.zeros(3)
                e[d] = h
                J[:, d] = (u(p0 + e) - u(p0 - e)) / (2 * h)
            sigma = -pressure(p0) * np.eye(3) + eta * (J + J.T)
            total += sigma @ n * R ** 2 * math.sin(t) * (math.pi / nth) * (2 * math.pi / nph)
    np.testing.assert_allclose(-total, F, rtol=2e-3, atol=2e-3 * np.linalg.norm(F))


# ---------------------------------------------------------------- Rotne-Prager from Faxen

@pytest.fixture(scope="module")
def faxen_tensor():
    """T = (1 + a^2/3 Lap) G, built symbolically from the Oseen tensor (Sec. 2.2)."""
    sp = pytest.importorskip("sympy")
    x, y, z, a, eta = sp.symbols("x y z a eta", positive=True)
    X = [x, y, z]
    r = sp.sqrt(x ** 2 + y ** 2 + z ** 2)
    T = sp.zeros(3, 3)
    for i in range(3):
        for j in range(3):
            G = (sp.KroneckerDelta(i, j) + X[i] * X[j] / r ** 2) / (8 * sp.pi * eta * r)
            lap = sum(sp.diff(G, v, 2) for v in X)
            T[i, j] = sp.simplify(G + a ** 2 / 3 * lap)
    return sp.lambdify((x, y, z, a, eta), T, "numpy")


@pytest.mark.parametrize("tensor", ["rp", "rpy"])
def test_rotne_prager_is_faxen_corrected_oseen(orc, faxen_tensor, tensor):
    rng = np.random.default_rng(3)
    for _ in range(12):
        a = rng.uniform(0.5, 2.0)
        eta = rng.uniform(0.3, 3.0)
        d = rng.standard_normal(3)
        r = d / np.linalg.norm(d) * a * rng.uniform(2.0, 40.0)
        want = np.array(faxen_tensor(*r, a, eta), dtype=float)
        got = _column_tensor(orc, r, tensor, a, eta)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_rotne_prager_tends_to_oseen(orc):
    """Dropping the a^2 Lap terms (a/r -> 0) turns T into G (Sec. 2.2)."""
    e = np.array([0.6, 0.0, 0.8])
    prev = None
    for rr in [10.0, 100.0, 1000.0]:
        Trp = _column_tensor(orc, rr * e, "rp")
        G = _column_tensor(orc, rr * e, "oseen")
        rel = np.abs(Trp - G).max() / np.abs(G).max()
        assert rel < 2.0 / rr ** 2
        if prev is not None:
            assert rel < prev / 50  # the difference decays like (a/r)^2
        prev = rel


# ---------------------------------------------------------------- contact values

def test_two_sphere_contact_values(orc):
    g = _golden("two_sphere_mobility.json")
    m0 = orc.mu0()
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    par = orc.mobility_apply(x, [[1, 0, 0], [1, 0, 0]], "rp") / m0
    per = orc.mobility_apply(x, [[0, 1, 0], [0, 1, 0]], "rp") / m0
    opp_par = orc.mobility_apply(x, [[1, 0, 0], [-1, 0, 0]], "rp") / m0
    opp_per = orc.mobility_apply(x, [[0, 0, 1], [0, 0, -1]], "rp") / m0
    c = g["rp_contact"]
    assert par[0, 0] == pytest.approx(c["equal_forces_parallel"], rel=1e-14)
    assert per[0, 1] == pytest.approx(c["equal_forces_perpendicular"], rel=1e-14)
    assert opp_par[0, 0] == pytest.approx(c["opposite_forces_parallel"], rel=1e-14)
    assert opp_per[0, 2] == pytest.approx(c["opposite_forces_perpendicular"], rel=1e-14)
    for tensor, key in [("rp", "rp_contact"), ("oseen", "oseen_contact")]:
        ev = np.linalg.eigvalsh(orc.assemble(x, tensor)) / m0
        np.testing.assert_allclose(ev, g[key]["eigenvalues_6x6"], rtol=1e-13)
    # Yamakawa continuation at r = a
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    y = g["rpy_overlap_r_eq_a"]
    assert (orc.mobility_apply(x, [[1, 0, 0], [1, 0, 0]], "rpy") / m0)[0, 0] == pytest.approx(
        y["equal_forces_parallel"], rel=1e-14)
    assert (orc.mobility_apply(x, [[0, 1, 0], [0, 1, 0]], "rpy") / m0)[0, 1] == pytest.approx(
        y["equal_forces_perpendicular"], rel=1e-14)


def test_rpy_continuation_is_c1_and_tends_to_self(orc):
    """The overlap form joins RP with matching value and slope at r = 2a, and two
    coincident spheres move like one (T(0) = mu0 I)."""
    e = np.array([0.0, 0.6, 0.8])
    h = 1e-6
    for s in [1.0, 1.0]:
        lo = _column_tensor(orc, (2.0 - h) * e, "rpy")
        hi = _column_tensor(orc, (2.0 + h) * e, "rpy")
        np.testing.assert_allclose(lo, hi, atol=1e-7 * s)
        slope_lo = (_column_tensor(orc, (2.0 - h) * e, "rpy") - _column_tensor(orc, (2.0 - 3 * h) * e, "rpy")) / (2 * h)
        slope_hi = (_column_tensor(orc, (2.0 + 3 * h) * e, "rpy") - _column_tensor(orc, (2.0 + h) * e, "rpy")) / (2 * h)
        np.testing.assert_allclose(slope_lo, slope_hi, atol=1e-5)
    T0 = orc.pair_tensor([0.0, 0.0, 0.0], "rpy")
    np.testing.assert_allclose(T0, orc.mu0() * np.eye(3), rtol=1e-15)


# ---------------------------------------------------------------- matrix structure

def _nonoverlap(rng, n, L, dmin=2.0):
    pts = []
    while len(pts) < n:
        c = rng.uniform(0, L, 3)
        if all(np.linalg.norm(c - p) >= dmin for p in pts):
            pts.append(c)
    return np.array(pts)


def test_mobility_symmetric_positive_definite(orc):
    """mu is symmetric and positive definite when no pair is closer than 2a (Sec. 2.2)."""
    rng = np.random.default_rng(4)
    for n in range(2, 9):
        for L in [4.5, 8.0]:
            x = _nonoverlap(rng, n, L)
            for tensor in ["rpy", "rp"]:
                M = orc.assemble(x, tensor)
                np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-15)
                assert np.linalg.eigvalsh(M).min() > 0.0


def test_oseen_loses_positive_definiteness_when_close(orc):
    """Contrast case: the Oseen tensor is not positive definite for close pairs,
    so the structure test above can tell the two tensors apart."""
    x = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    assert np.linalg.eigvalsh(orc.assemble(x, "oseen")).min() < 0.0


def test_apply_matches_assembled_matrix(orc):
    """The ascending-j loop equals the dense matrix-vector product (second formulation),
    and a vectorised restatement in scalar form A(r) I + B(r) r r^T."""
    rng = np.random.default_rng(5)
    n = 37
    x = rng.uniform(0, 9.0, (n, 3))  # includes overlapping pairs
    F = rng.standard_normal((n, 3))
    for tensor in ["rpy", "rp", "oseen"]:
        v = orc.mobility_apply(x, F, tensor, 1.3, 0.8)
        M = orc.assemble(x, tensor, 1.3, 0.8)
        np.testing.assert_allclose(v, (M @ F.reshape(-1)).reshape(n, 3), rtol=1e-12, atol=1e-14)
    # scalar form, RP, r >= 2a everywhere
    x = _nonoverlap(rng, 20, 12.0)
    F = rng.standard_normal((20, 3))
    a, eta = 1.0, 1.0
    m0 = 1 / (6 * math.pi * eta * a)
    d = x[:, None, :] - x[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    np.fill_diagonal(r, 1.0)
    A = 0.75 * a / r + 0.5 * a ** 3 / r ** 3
    B = (0.75 * a / r - 1.5 * a ** 3 / r ** 3) / r ** 2
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(B, 0.0)
    want = m0 * (F + (A[..., None] * F[None, :, :]).sum(1)
                 + (B[..., None] * (d * F[None, :, :]).sum(-1, keepdims=True) * d).sum(1))
    np.testing.assert_allclose(orc.mobility_apply(x, F, "rp"), want, rtol=1e-12)


def test_rows_match_full_apply(orc):
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 20, (60, 3))
    F = rng.standard_normal((60, 3))
    rows = np.array([0, 59, 17, 17, 3])
    np.testing.assert_array_equal(orc.mobility_rows(x, F, rows, "rpy"), orc.mobility_apply(x, F, "rpy")[rows])


def test_coincident_particles_raise_in_rp_and_oseen(orc):
    x = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0]])
    F = np.ones((2, 3))
    for tensor in ["rp", "oseen"]:
        with pytest.raises(orc.OracleError):
            orc.mobility_apply(x, F, tensor)
    v = orc.mobility_apply(x, F, "rpy")
    np.testing.assert_allclose(v, 2 * orc.mu0() * F, rtol=1e-15)  # two coincident spheres: 2 mu0 F


# ---------------------------------------------------------------- invariances of Stokes flow

def test_invariances(orc):
    """Linearity, time reversal r -> -r, F -> -F => v -> -v (Sec. 4), translation,
    rotation and permutation equivariance."""
    rng = np.random.default_rng(7)
    n = 25
    x = rng.uniform(0, 10, (n, 3))
    F = rng.standard_normal((n, 3))
    G = rng.standard_normal((n, 3))
    for tensor in ["rpy", "rp", "oseen"]:
        v = orc.mobility_apply(x, F, tensor)
        vg = orc.mobility_apply(x, G, tensor)
        np.testing.assert_allclose(orc.mobility_apply(x, 2 * F - 3 * G, tensor), 2 * v - 3 * vg, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(orc.mobility_apply(-x, -F, tensor), -v, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(orc.mobility_apply(x + np.array([3.0, -7.0, 11.0]), F, tensor), v,
                                   rtol=1e-10, atol=1e-13)
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        np.testing.assert_allclose(orc.mobility_apply(x @ Q.T, F @ Q.T, tensor), v @ Q.T, rtol=1e-10, atol=1e-13)
        p = rng.permutation(n)
        np.testing.assert_allclose(orc.mobility_apply(x[p], F[p], tensor), v[p], rtol=1e-13, atol=1e-15)


def test_nearest_image(orc):
    """Nearest-image periodic mode: shifting a particle by a box vector changes nothing,
    and mu stays symmetric (Sec. 3.1, footnote)."""
    rng = np.random.default_rng(8)
    box = np.array([10.0, 12.0, 9.0])
    x = rng.uniform(0, 1, (12, 3)) * box
    F = rng.standard_normal((12, 3))
    v = orc.mobility_apply(x, F, "rpy", box=box)
    y = x.copy()
    y[3] += box * np.array([1, -2, 3])
    np.testing.assert_allclose(orc.mobility_apply(y, F, "rpy", box=box), v, rtol=1e-11, atol=1e-14)
    M = orc.assemble(x, "rpy", box=box)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    # far pairs interact through the closer image
    x2 = np.array([[0.5, 0.5, 0.5], [9.5, 0.5, 0.5]])
    T = orc.assemble(x2, "rp", box=box)[0:3, 3:6]
    np.testing.assert_allclose(T, orc.pair_tensor([1.0, 0, 0], "rp"), rtol=1e-12)


# ---------------------------------------------------------------- forces and Euler

def test_repulsion_is_minus_gradient_of_energy(orc):
    rng = np.random.default_rng(9)
    n = 10
    x = rng.uniform(0, 5.0, (n, 3))
    eps, rc, a = 1.3, 2.5, 1.0

    def energy(y):
        U = 0.0
        for i in range(n):
            for j in range(i + 1, n):
                r = np.linalg.norm(y[i] - y[j])
                if r < rc:
                    U += eps * (2 * a / r) ** 12
        return U

    F = orc.forces(x, gravity=(0, 0, 0), rep_eps=eps, rep_rc=rc, a=a)
    h = 1e-6
    for i in range(n):
        for d in range(3):
            e = np.zeros((n, 3))
            e[i, d] = h
            fd = -(energy(x + e) - energy(x - e)) / (2 * h)
            assert F[i, d] == pytest.approx(fd, rel=1e-5, abs=1e-6 * (1 + np.abs(F).max()))
    g = np.array([0.1, -0.2, -1.0])
    fe = rng.standard_normal((n, 3))
    np.testing.assert_allclose(orc.forces(x, fe, g, 0.0), fe + g, rtol=1e-15)
    # the potential is truncated at r_c: a pair just inside feels -dU/dr of its own
    # energy (Newton's third law holds), a pair just outside feels nothing
    for r, inside in [(0.99 * rc, True), (1.01 * rc, False)]:
        y = np.array([[0.3, -0.2, 0.1], [0.3 + r, -0.2, 0.1]])
        F2 = orc.forces(y, gravity=(0, 0, 0), rep_eps=eps, rep_rc=rc, a=a)
        if inside:
            h = 1e-7
            fd = -(eps * (2 * a / (r + h)) ** 12 - eps * (2 * a / (r - h)) ** 12) / (2 * h)
            assert F2[1, 0] == pytest.approx(fd, rel=1e-6)
            np.testing.assert_allclose(F2[0], -F2[1], rtol=1e-15)
            assert F2[1, 1] == 0.0 and F2[1, 2] == 0.0
        else:
            np.testing.assert_array_equal(F2, 0.0)


def test_euler_step_is_forward_euler(orc):
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 8, (9, 3))
    fe = rng.standard_normal((9, 3))
    g = np.array([0, 0, -1.0])
    dt = 0.05
    x1 = orc.euler(x, 1, dt, fe, g, rep_eps=0.5, rep_rc=2.5)
    F = orc.forces(x, fe, g, 0.5, 2.5)
    np.testing.assert_allclose(x1, x + dt * orc.mobility_apply(x, F, "rpy"), rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------- four-sphere orbit (Sec. 4)

@pytest.fixture(scope="module")
def orbit(orc):
    g = _golden("four_sphere_orbit.json")
    tau = 1.0 / orc.mu0(g["a"], g["eta"])
    dt = g["dt_tau_s"] * tau
    nsteps = int(round(1000.0 / g["dt_tau_s"]))
    x0 = np.array(g["start"])
    _, traj = orc.euler(x0, nsteps, dt, gravity=g["force"], tensor="rp", every=1)
    return g, traj


def _maxima_times(sig, dt):
    k = np.nonzero((sig[1:-1] > sig[:-2]) & (sig[1:-1] >= sig[2:]))[0] + 1
    y0, y1, y2 = sig[k - 1], sig[k], sig[k + 1]
    return (k + 1 + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)) * dt


def test_four_sphere_orbit_period(orbit):
    g, traj = orbit
    t = _maxima_times(traj[:, 0, 0], g["dt_tau_s"])
    assert len(t) >= 2
    period = np.diff(t)
    assert period == pytest.approx(np.full_like(period, g["period_tau_s"]), rel=0.01)


def test_four_sphere_orbit_symmetries(orbit):
    g, traj = orbit
    x1, y1, z1 = traj[:, 0, 0], traj[:, 0, 1], traj[:, 0, 2]
    x2, y2, z2 = traj[:, 1, 0], traj[:, 1, 1], traj[:, 1, 2]
    x3, y3, z3 = traj[:, 2, 0], traj[:, 2, 1], traj[:, 2, 2]
    x4, y4, z4 = traj[:, 3, 0], traj[:, 3, 1], traj[:, 3, 2]
    scale = np.abs(traj).max()
    tol = 1e-12 * scale
    for lhs, rhs in [(x3, -x1), (z3, z1), (z4, z2), (y4, -y2)]:
        assert np.abs(lhs - rhs).max() < tol
    for zero in [y1, y3, x2, x4]:
        assert np.abs(zero).max() < tol
    zcm = 0.5 * (z1 + z2)
    assert np.all(np.diff(zcm) < 0)
    # y2 is x1 shifted by half a period
    half = int(round(0.5 * g["period_tau_s"] / g["dt_tau_s"]))
    i1 = np.argmax(x1[: 2 * half])
    i2 = np.argmax(y2[: 2 * half + i1])
    assert min(abs(i2 - i1 - half), abs(i1 - i2 - half)) < 0.02 * 2 * half


# ---------------------------------------------------------------- derivatives

@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
def test_vjp_matches_central_differences(orc, tensor):
    rng = np.random.default_rng(11)
    n = 7
    x = rng.uniform(0, 4.5, (n, 3))  # overlapping pairs included
    F = rng.standard_normal((n, 3))
    w = rng.standard_normal((n, 3))
    box = np.array([6.0, 0.0, 0.0]) if tensor == "rpy" else None
    gx, gF = orc.vjp(x, F, w, tensor, box=box)
    h = 1e-5

    def L(y, f):
        return (w * orc.mobility_apply(y, f, tensor, box=box)).sum()

    for i in range(n):
        for d in range(3):
            e = np.zeros((n, 3))
            e[i, d] = h
            fdx = (L(x + e, F) - L(x - e, F)) / (2 * h)
            fdF = (L(x, F + e) - L(x, F - e)) / (2 * h)
            assert gx[i, d] == pytest.approx(fdx, rel=1e-6, abs=1e-9)
            assert gF[i, d] == pytest.approx(fdF, rel=1e-8, abs=1e-12)


def test_adjoint_matches_central_differences(orc):
    rng = np.random.default_rng(12)
    n, nsteps, dt = 5, 25, 0.3
    x0 = _nonoverlap(rng, n, 7.0)
    fe = rng.standard_normal((n, 3))
    g = np.array([0.0, 0.0, -1.0])
    target = x0 + rng.standard_normal((n, 3))

    def loss(x, f):
        xT = orc.euler(x, nsteps, dt, f, g)
        return ((xT - target) ** 2).sum()

    xT = orc.euler(x0, nsteps, dt, fe, g)
    gx0, gF = orc.adjoint(x0, fe, 2 * (xT - target), nsteps, dt, g)
    h = 1e-5
    for i in range(n):
        for d in range(3):
            e = np.zeros((n, 3))
            e[i, d] = h
            assert gx0[i, d] == pytest.approx((loss(x0 + e, fe) - loss(x0 - e, fe)) / (2 * h), rel=1e-6, abs=1e-9)
            assert gF[i, d] == pytest.approx((loss(x0, fe + e) - loss(x0, fe - e)) / (2 * h), rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- lubrication (Sec. 2.3)

def _pair_along(e, r):
    e = np.asarray(e, float) / np.linalg.norm(e)
    return np.array([[0.2, -0.4, 0.3], [0.2, -0.4, 0.3] + r * e]), e


def test_lubrication_squeeze_film_limit(orc):
    """Head-on approach of two equal spheres: as the gap h -> 0 the friction force
    tends to Reynolds' squeeze-film result 6 pi eta a*^2 U / h with the reduced radius
    a* = a/2, independent of the expansion the oracle evaluates; the next term is
    O(s log s) relative."""
    a, eta, U = 1.3, 0.7, 0.37
    for s in [1e-3, 1e-4, 1e-5]:
        x, e = _pair_along([0.3, 1.0, -0.5], (2.0 + s) * a)
        v = np.array([0.5 * U * e, -0.5 * U * e])      # closing speed U
        F = orc.lubrication(x, v, a, eta)
        reynolds = 6 * math.pi * eta * (a / 2) ** 2 * U / (s * a)
        assert F[0] @ e == pytest.approx(-reynolds, rel=1.0 * s * abs(math.log(s)) + 1e-12)
        np.testing.assert_allclose(F[0] - (F[0] @ e) * e, 0.0, atol=1e-12 * reynolds)   # no sideways force


def test_lubrication_matches_jeffrey_onishi_coefficients(orc):
    """The two singular resistance functions of equal spheres as Jeffrey & Onishi (1984)
    tabulate them (the source the paper cites): X11A = 1/(4 xi) + (9/40) ln(1/xi) for
    motion along the line of centres and Y11A = (1/6) ln(1/xi) across it, in units of
    6 pi eta a, xi = the gap over a."""
    a, eta = 1.0, 1.0
    mu0 = orc.mu0(a, eta)
    for s in [0.02, 0.3, 0.9]:
        x, e = _pair_along([1.0, 0.2, 0.1], (2.0 + s) * a)
        t = np.cross(e, [0.0, 0.0, 1.0])
        t /= np.linalg.norm(t)
        Fn = orc.lubrication(x, np.array([e, 0 * e]), a, eta)[0]
        Ft = orc.lubrication(x, np.array([t, 0 * t]), a, eta)[0]
        assert -mu0 * (Fn @ e) == pytest.approx(1 / (4 * s) + 9 / 40 * math.log(1 / s), rel=1e-13)
        assert -mu0 * (Ft @ t) == pytest.approx(1 / 6 * math.log(1 / s), rel=1e-13)
        assert abs(Ft @ e) < 1e-13 and abs(Fn @ t) < 1e-13


def test_lubrication_invariants(orc):
    """Galilean invariance, momentum conservation, dissipation, rotation covariance and
    the truncation window 0 < s < 1 (2a < r < 3a)."""
    rng = np.random.default_rng(21)
    n = 40
    x = _nonoverlap(rng, n, 9.0)                       # many pairs inside 3a
    v = rng.standard_normal((n, 3))
    F = orc.lubrication(x, v)
    assert np.abs(F).max() > 0
    np.testing.assert_allclose(orc.lubrication(x, np.tile(v[0], (n, 1))), 0.0, atol=1e-12)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-10 * np.abs(F).max())
    assert float((v * F).sum()) < 0.0
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    np.testing.assert_allclose(orc.lubrication(x @ Q.T, v @ Q.T), F @ Q.T, atol=1e-10 * np.abs(F).max())
    for r, inside in [(2.0, False), (1.5, False), (2.0 + 1e-9, True), (3.0 - 1e-9, True), (3.0, False), (3.5, False)]:
        xx, e = _pair_along([0.0, 0.0, 1.0], r)
        Fp = orc.lubrication(xx, np.array([e, -e]))
        if inside:
            assert np.all(np.isfinite(Fp)) and np.abs(Fp).max() > 0, r
        else:
            np.testing.assert_array_equal(Fp, 0.0)


def test_euler_lubrication_uses_previous_velocities(orc):
    """Sec. 3.1: the first step has no friction (no previous velocity); step n adds the
    friction of the velocities of step n-1 to the forces."""
    rng = np.random.default_rng(22)
    n, dt = 12, 0.05
    x0 = _nonoverlap(rng, n, 6.0)
    fe = rng.standard_normal((n, 3))
    g = np.array([0.0, 0.0, -1.0])
    x1 = orc.euler(x0, 1, dt, fe, g, lubrication=True)
    np.testing.assert_array_equal(x1, orc.euler(x0, 1, dt, fe, g))
    v0 = orc.mobility_apply(x0, fe + g)
    F1 = fe + g + orc.lubrication(x1, v0)
    x2 = x1 + dt * orc.mobility_apply(x1, F1)
    np.testing.assert_allclose(orc.euler(x0, 2, dt, fe, g, lubrication=True), x2, rtol=1e-14, atol=1e-14)
    assert np.abs(x2 - orc.euler(x0, 2, dt, fe, g)).max() > 1e-6   # the friction acted
