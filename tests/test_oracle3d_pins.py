"""Pins of the D3Q19 oracle (oracle/oracle3d.py) against what the mathematics
and the paper fix, independent of the oracle's own formulas: isotropy of
the derived interaction weights (and that the same conditions give the
paper's printed 2D weights), the moment basis, equilibrium and forcing
moments, the BGK reduction of the collision, exact conservation on periodic
boxes, permutation symmetry, slit Poiseuille flow, the inlet momentum the
alpha correction restores, and a uniform stream the open faces keep."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle3d as O3
from paper_2512_12934_gb300 import workloads as W


def _pairings(idx):
    """Sum over perfect matchings of prod delta: the isotropic tensor."""
    if not idx:
        return 1
    a, rest = idx[0], idx[1:]
    tot = 0
    for j in range(len(rest)):
        if a == rest[j]:
            tot += _pairings(rest[:j] + rest[j + 1:])
    return tot


def _shells(dim, rmax2=8):
    out = {}
    for v in itertools.product(range(-2, 3), repeat=dim):
        r2 = sum(c * c for c in v)
        if 0 < r2 <= rmax2:
            out.setdefault(r2, []).append(v)
    return out


def test_3d_weights_are_8th_order_isotropic():
    dx, dy, dz, w = O3.stencil()
    E = np.stack([dx, dy, dz], axis=1)
    assert len(w) == 92 and (w > 0).all()
    e2n = {}
    for order in (2, 4, 6, 8):
        for idx in itertools.product(range(3), repeat=order):
            m = float(np.sum(w * np.prod(E[:, list(idx)], axis=1)))
            p = _pairings(list(idx))
            if p == 0:
                assert abs(m) < 1e-14, (order, idx, m)
            else:
                e2n.setdefault(order, m / p)
                assert abs(m - p * e2n[order]) < 1e-14, (order, idx, m)
    assert abs(e2n[2] - 1.0) < 1e-15  # second moment 1, as the printed 2D weights
    # exact rationals of the unique solution
    want = {1: Fraction(4, 45), 2: Fraction(1, 21), 3: Fraction(2, 105), 4: Fraction(5, 504),
            5: Fraction(1, 315), 6: Fraction(1, 630), 8: Fraction(1, 5040)}
    r2 = dx * dx + dy * dy + dz * dz
    for k, v in want.items():
        assert np.allclose(w[r2 == k], float(v), rtol=0, atol=1e-16)


def test_isotropy_conditions_reproduce_the_printed_2d_weights():
    """The conditions used for 3D, applied to the 2D shells {1,2,4,5,8},
    have the paper's printed weights (Eq. 10) as their unique solution."""
    sh = _shells(2)
    keys = [1, 2, 4, 5, 8]

    def M(r, a, b):
        return sum(Fraction(v[0] ** a * v[1] ** b) for v in sh[r])
    rows = [[M(r, 2, 0) for r in keys], [M(r, 4, 0) - 3 * M(r, 2, 2) for r in keys],
            [M(r, 6, 0) - 5 * M(r, 4, 2) for r in keys], [M(r, 8, 0) - 7 * M(r, 6, 2) for r in keys],
            [9 * M(r, 6, 2) - 15 * M(r, 4, 4) for r in keys]]
    rhs = [Fraction(1), 0, 0, 0, 0]
    # Gauss-Jordan over the rationals
    A = [row[:] + [b] for row, b in zip(rows, rhs)]
    n = len(keys)
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    sol = [A[i][n] / A[i][i] for i in range(n)]
    printed = [Fraction(4, 21), Fraction(4, 45), Fraction(1, 60), Fraction(2, 315), Fraction(1, 5040)]
    assert sol == printed


def test_moment_basis_and_lattice():
    ex, ey, ez, w, opp = O3.lattice()
    T, Ti = O3.moment_matrix()
    assert abs(w.sum() - 1.0) < 1e-15
    for a, ea in enumerate((ex, ey, ez)):
        for b, eb in enumerate((ex, ey, ez)):
            assert abs((w * ea * eb).sum() - (1.0 / 3.0 if a == b else 0.0)) < 1e-15
    G = T @ T.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    assert np.abs(Ti @ T - np.eye(19)).max() < 1e-14
    assert np.array_equal(T[0], np.ones(19))
    assert np.array_equal(T[3], ex) and np.array_equal(T[5], ey) and np.array_equal(T[7], ez)
    for i in range(19):
        assert ex[opp[i]] == -ex[i] and ey[opp[i]] == -ey[i] and ez[opp[i]] == -ez[i]
    # inlet unknown set of an x face: e_x = +1; cross sums vanish (3D alpha is diagonal)
    U = ex > 0
    assert U.sum() == 5
    for a, b in ((ex, ey), (ex, ez), (ey, ez)):
        assert (w[U] * a[U] * b[U]).sum() == 0.0


def test_equilibrium_and_forcing_moments():
    ex, ey, ez, w, _ = O3.lattice()
    E = np.stack([ex, ey, ez], axis=1).astype(float)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = rng.uniform(0.1, 2.0)
        u = rng.uniform(-0.1, 0.1, size=3)
        F = rng.uniform(-1e-3, 1e-3, size=3)
        f = O3.feq(rho, u)
        assert abs(f.sum() - rho) < 1e-15
        assert np.allclose(E.T @ f, rho * u, atol=1e-16)
        P = (E.T * f) @ E
        assert np.allclose(P, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-15)
        g = O3.fbar(u, F)
        assert abs(g.sum()) < 1e-17
        assert np.allclose(E.T @ g, F, atol=1e-18)
        assert np.allclose((E.T * g) @ E, np.outer(u, F) + np.outer(F, u), atol=1e-18)


def test_collision_reduces_to_bgk_with_equal_rates():
    rng = np.random.default_rng(2)
    s_val = 1.3
    s = np.full(19, s_val)
    s[[0, 3, 5, 7]] = 1.0  # conserved moments
    for _ in range(3):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.05, 0.05, size=3)
        F = rng.uniform(-1e-3, 1e-3, size=3)
        # populations whose momentum is consistent with u: sum e f = rho u - F/2
        f = O3.feq(rho, u) + rng.uniform(-1e-3, 1e-3, size=19)
        ex, ey, ez, w, _ = O3.lattice()
        E = np.stack([ex, ey, ez], axis=1).astype(float)
        # project the perturbation so that rho and j match rho, rho u - F/2
        dm = np.array([f.sum() - rho, *(E.T @ f - (rho * u - 0.5 * F))])
        B = np.vstack([np.ones(19), E.T])
        f = f - B.T @ np.linalg.solve(B @ B.T, dm)
        got = O3.collide(f, rho, u, F, s)
        bgk = f - s_val * (f - O3.feq(rho, u)) + (1.0 - 0.5 * s_val) * O3.fbar(u, F)
        assert np.abs(got - bgk).max() < 1e-15


def _momentum(o):
    f = o.f()
    ex, ey, ez, _, _ = O3.lattice()
    return np.array([(f * e[None, :, None, None, None]).sum() for e in (ex, ey, ez)])


def test_periodic_box_conserves_mass_and_momentum():
    w = W.random_box3(7, 6, 5, seed=3, G12=1.2, nu=(0.1, 0.25))
    o = O3.Oracle3D(w.cfg, w.solid, w.rho, w.u)
    m0 = o.scalars()["mass"]
    o.step(1)
    p1 = _momentum(o)
    o.step(10)
    sc = o.scalars()
    assert np.allclose(sc["mass"], m0, rtol=1e-13, atol=0)
    assert np.abs(_momentum(o) - p1).max() < 1e-13


def test_droplet_keeps_the_cube_symmetry():
    w = W.laplace3(n=12, R=3.5, G12=1.6, noise=0.0, width=2.0)
    o = O3.Oracle3D(w.cfg, None, w.rho, w.u)
    o.step(15)
    rho, u, F = o.macros()
    r = rho[0]
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.abs(r - np.transpose(r, perm)).max() < 1e-13
    # x -> -x about the centre (n even, centre at n/2): index i -> n - i
    assert np.abs(r[:, :, 1:] - r[:, :, 1:][:, :, ::-1]).max() < 1e-13
    assert np.abs(u).max() > 0  # spurious currents exist but respect the symmetry


def test_slit_poiseuille_profile():
    w = W.slit3(nx=5, half=8, nz=5, Fb=1e-6, nu=1.0 / 6)
    o = O3.Oracle3D(w.cfg, w.solid, w.rho, w.u)
    o.step(6000)
    rho, u, F = o.macros()
    H = w.meta["H"]
    y = np.arange(1, H + 1) - 0.5
    g = w.meta["Fb"] / (rho[0] + rho[1])[1, 1:-1, 1].mean()
    exact = g / (2.0 * w.meta["nu"]) * y * (H - y)
    got = u[0, 1, 1:-1, 1]
    assert np.abs(got - exact).max() < 0.01 * exact.max()
    assert np.abs(u[1:]).max() < 1e-12


def test_alpha_correction_restores_the_inlet_momentum():
    w = W.duct3(nx=14, ny=8, nz=7, R=2.0, xc=6.0, u_max=0.02, G12=1.2)
    o = O3.Oracle3D(w.cfg, w.solid, w.rho, w.u)
    o.step(3)
    fp = o.fpost()
    Fp = o.force_prev()
    ex, ey, ez, _, _ = O3.lattice()
    prof = w.cfg["faces"][0]["profile"]
    rin = w.cfg["faces"][0]["rho_in"]
    for z in range(1, 6):
        for y in range(1, 7):
            for k in range(2):
                f = fp[k, :, z, y, 0]
                mom = np.array([(ex * f).sum(), (ey * f).sum(), (ez * f).sum()]) + 0.5 * Fp[k, :, z, y, 0]
                want = rin[k] * np.array([prof[z, y], 0.0, 0.0])
                assert np.abs(mom - want).max() < 1e-15


def test_uniform_stream_is_kept_by_the_open_faces():
    """A uniform single-phase stream through a duct periodic in y and z is
    a fixed point of the inlet (Eq. 13 + alpha) and outlet (Eqs. 20-23)."""
    nx, ny, nz, U = 10, 5, 5, 0.03
    cfg = W._base_cfg3(nx, ny, nz, (0, 1, 1), 0.0, (0.0, 0.0), (1.0 / 6, 1.0 / 6))
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": (0, 0), "hi": (ny - 1, nz - 1), "rho_in": (1.0, 0.5),
         "profile": np.full((nz, ny), U)},
        {"kind": "outlet", "side": "xmax", "lo": (0, 0), "hi": (ny - 1, nz - 1), "chi": 1},
    ]
    rho = np.empty((2, nz, ny, nx))
    rho[0], rho[1] = 1.0, 0.5
    u = np.zeros((3, nz, ny, nx))
    u[0] = U
    o = O3.Oracle3D(cfg, None, rho, u)
    o.step(20)
    r, uu, F = o.macros()
    assert np.abs(r[0] - 1.0).max() < 1e-13 and np.abs(r[1] - 0.5).max() < 1e-13
    assert np.abs(uu[0] - U).max() < 1e-13 and np.abs(uu[1:]).max() < 1e-13
    sc = o.scalars()
    assert abs(sc["chi"] - 1.0) < 1e-12 and abs(sc["lambda"] - U) < 1e-13
