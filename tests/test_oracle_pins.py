"""Pins of the FP64 oracle against closed forms, invariants, special cases and brute force.

Each test fixes a part of the oracle by something other than the oracle itself,
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in that part fails it.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import wpccc_inputs as wi
from oracle import wpccc_oracle as O
import brute_force as BF


def _centre(Z, nl, grid, eps=None):
    f = [wi.hydrogenic_radial(n, l, Z, grid.r) for n, l in nl]
    e = np.zeros(len(nl)) if eps is None else np.asarray(eps, float)
    return wi.centre_from_functions(Z, [l for n, l in nl], [n for n, l in nl], f, e)


@pytest.fixture(scope="module")
def grid():
    return wi.radial_grid(2000)


@pytest.fixture(scope="module")
def tiny2c(grid):
    T = _centre(1.0, [(1, 0), (2, 0), (2, 1)], grid)
    P = _centre(2.0, [(1, 0), (2, 1)], grid)
    return wi.Basis(grid=grid, T=T, P=P, quad=wi.make_quadrature(48, 48, 0.5), Z_T=1.0, Z_P=2.0)


# ---------------------------------------------------------------- angular algebra
def test_clebsch_gordan_known_values_and_orthogonality():
    CG = O.clebsch_gordan
    assert CG(1, 0, 1, 0, 0, 0) == pytest.approx(-1 / math.sqrt(3), abs=1e-15)
    assert CG(1, 1, 1, -1, 0, 0) == pytest.approx(1 / math.sqrt(3), abs=1e-15)
    assert CG(1, 0, 1, 0, 2, 0) == pytest.approx(math.sqrt(2 / 3), abs=1e-15)
    assert CG(1, 1, 1, 0, 1, 1) == pytest.approx(1 / math.sqrt(2), abs=1e-15)
    assert CG(2, 0, 1, 0, 1, 0) == pytest.approx(-math.sqrt(2 / 5), abs=1e-15)
    assert CG(1, 0, 1, 0, 1, 0) == 0.0
    # sum_{m1 m2} <j1 m1 j2 m2|J M><j1 m1 j2 m2|J' M'> = delta
    for j1, j2 in [(2, 3), (1, 4), (3, 3)]:
        for J in range(abs(j1 - j2), j1 + j2 + 1):
            for Jp in range(abs(j1 - j2), j1 + j2 + 1):
                for M in range(-min(J, Jp), min(J, Jp) + 1):
                    s = sum(CG(j1, m1, j2, M - m1, J, M) * CG(j1, m1, j2, M - m1, Jp, M)
                            for m1 in range(-j1, j1 + 1) if abs(M - m1) <= j2)
                    assert s == pytest.approx(1.0 if J == Jp else 0.0, abs=1e-13)


def test_wigner_d_closed_form_identity_and_group_law():
    b = 0.73
    c, s = math.cos(b), math.sin(b)
    d1 = {(1, 1): (1 + c) / 2, (1, 0): -s / math.sqrt(2), (1, -1): (1 - c) / 2,
          (0, 1): s / math.sqrt(2), (0, 0): c, (0, -1): -s / math.sqrt(2),
          (-1, 1): (1 - c) / 2, (-1, 0): s / math.sqrt(2), (-1, -1): (1 + c) / 2}
    for (mp, m), val in d1.items():
        assert O.wigner_d(1, mp, m, b) == pytest.approx(val, abs=1e-15)
    for l in range(5):
        ms = range(-l, l + 1)
        assert np.allclose([[O.wigner_d(l, a, c_, 0.0) for c_ in ms] for a in ms], np.eye(2 * l + 1), atol=1e-15)
        A = np.array([[O.wigner_d(l, a, c_, 0.4) for c_ in ms] for a in ms])
        B = np.array([[O.wigner_d(l, a, c_, 0.9) for c_ in ms] for a in ms])
        C = np.array([[O.wigner_d(l, a, c_, 1.3) for c_ in ms] for a in ms])
        assert np.allclose(A @ B, C, atol=1e-13)
        assert np.allclose(A @ A.T, np.eye(2 * l + 1), atol=1e-13)


def test_legendre_closed_forms_and_phase():
    x = np.linspace(-0.95, 0.95, 7)
    sq = np.sqrt(1 - x * x)
    assert np.allclose(O.assoc_legendre(1, 1, x), -sq, atol=1e-15)
    assert np.allclose(O.assoc_legendre(2, 1, x), -3 * x * sq, atol=1e-14)
    assert np.allclose(O.assoc_legendre(2, 2, x), 3 * (1 - x * x), atol=1e-14)
    assert np.allclose(O.assoc_legendre(2, -1, x), 0.5 * x * sq, atol=1e-14)
    # normalisation: int Theta_lq^2 dx = 1
    xg, wg = np.polynomial.legendre.leggauss(40)
    for l in range(5):
        for q in range(-l, l + 1):
            assert np.sum(wg * O.norm_legendre(l, q, xg) ** 2) == pytest.approx(1.0, abs=1e-13)


# ---------------------------------------------------------------- interpolation and Eq. 7
def test_interp5_exact_on_quartics_and_zero_outside(grid):
    r = grid.r
    poly = 0.3 - 1.1 * r + 0.07 * r ** 2 - 2e-3 * r ** 3 + 1e-5 * r ** 4
    x = np.array([r[0] * 0.5, r[0], 0.0371, 1.234567, 17.0, 63.2, r[-3] + 1e-3, r[-1]])
    want = 0.3 - 1.1 * x + 0.07 * x ** 2 - 2e-3 * x ** 3 + 1e-5 * x ** 4
    got = O.interp5(r, poly[None, :], x)[0]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12)
    assert O.interp5(r, poly[None, :], np.array([r[-1] * 1.0001]))[0, 0] == 0.0


def test_radial_integral_1s1s_closed_form_converges():
    # F_0(R) for 1s-1s = 1/R - (1 + 1/R) e^{-2R}; the grid rule is O(h^2) accurate
    errs = []
    for Nr in (1000, 2000, 4000):
        g = wi.radial_grid(Nr)
        f = wi.hydrogenic_radial(1, 0, 1.0, g.r)[None, :]
        e = []
        for R in (0.3, 1.04, 3.7, 12.0):
            ex = 1 / R - (1 + 1 / R) * math.exp(-2 * R)
            e.append(abs(O.radial_F(g, f, f, 0, R)[0] - ex))
        errs.append(max(e))
    assert errs[1] < 5e-5
    assert 3.0 < errs[1] / errs[2] < 5.0          # second-order convergence


def test_direct_1s1s_matches_closed_form(grid):
    c = _centre(1.0, [(1, 0)], grid)
    for b, z in [(0.5, 0.0), (1.0, -2.0), (3.0, 4.0)]:
        R = math.hypot(b, z)
        D = O.direct_block(grid, c, 1.0, R, z / R, other_at_minus_R=False)
        assert D[0, 0] == pytest.approx(-(1 / R - (1 + 1 / R) * math.exp(-2 * R)), abs=5e-5)


# ---------------------------------------------------------------- Eq. 6 structure
def test_direct_hermitian_and_m_reflection(grid):
    c = _centre(1.0, [(1, 0), (2, 1), (3, 2)], grid)
    D = O.direct_block(grid, c, 1.0, 2.3, 0.4, other_at_minus_R=False)
    assert np.allclose(D, D.T, atol=1e-14)
    for i in range(c.N):
        for j in range(c.N):
            ii = [k for k in range(c.N) if c.st_rad[k] == c.st_rad[i] and c.st_m[k] == -c.st_m[i]][0]
            jj = [k for k in range(c.N) if c.st_rad[k] == c.st_rad[j] and c.st_m[k] == -c.st_m[j]][0]
            assert D[ii, jj] == pytest.approx((-1) ** int(c.st_m[i] - c.st_m[j]) * D[i, j], abs=1e-14)


def test_direct_elements_brute_force(tiny2c):
    T, P = tiny2c.T, tiny2c.P
    for b, z in [(1.3, -0.7), (0.6, 2.2)]:
        S, H = O.assemble(tiny2c, b, 1.0, z)
        Ts = [(int(T.rad_n[T.st_rad[i]]), int(T.st_l[i]), int(T.st_m[i]), 1.0) for i in range(T.N)]
        Ps = [(int(P.rad_n[P.st_rad[i]]), int(P.st_l[i]), int(P.st_m[i]), 2.0) for i in range(P.N)]
        DT = BF.direct_elements(Ts, 2.0, b, z)
        DP = BF.direct_elements(Ps, 1.0, b, z, centre_is_projectile=True)
        assert np.abs(H[:T.N, :T.N] - DT).max() < 2e-5
        assert np.abs(H[T.N:, T.N:] - DP).max() < 2e-5


# ---------------------------------------------------------------- Eq. 8/9
def test_two_centre_closed_forms_at_rest(grid):
    # v = 0, 1s on both hydrogen centres: overlap e^{-R}(1+R+R^2/3), <1s_A|-1/r_A|1s_B> = -e^{-R}(1+R)
    T = _centre(1.0, [(1, 0)], grid)
    P = _centre(1.0, [(1, 0)], grid)
    basis = wi.Basis(grid=grid, T=T, P=P, quad=wi.make_quadrature(48, 48, 0.5), Z_T=1.0, Z_P=1.0)
    for b, z in [(0.4, 0.0), (1.5, 1.0), (2.0, -5.0)]:
        R = math.hypot(b, z)
        Smol, Qmol, Qtmol = O.molecular_integrals(basis, b, 0.0, z, reverse=True)
        assert Smol[0, 0].real == pytest.approx(math.exp(-R) * (1 + R + R * R / 3), abs=1e-7)
        assert Qmol[0, 0].real == pytest.approx(-math.exp(-R) * (1 + R), abs=1e-7)
        assert Qtmol[0, 0].real == pytest.approx(-math.exp(-R) * (1 + R), abs=1e-7)
        assert abs(Smol[0, 0].imag) < 1e-15


@pytest.mark.parametrize("b,z,v", [(1.3, -0.7, 0.9), (0.5, 1.8, 2.0), (2.5, 0.3, 1.5)])
def test_two_centre_brute_force(tiny2c, b, z, v):
    T, P = tiny2c.T, tiny2c.P
    S, H = O.assemble(tiny2c, b, v, z)
    Ts = [(int(T.rad_n[T.st_rad[i]]), int(T.st_l[i]), int(T.st_m[i]), 1.0) for i in range(T.N)]
    Ps = [(int(P.rad_n[P.st_rad[i]]), int(P.st_l[i]), int(P.st_m[i]), 2.0) for i in range(P.N)]
    Sb, Qb, Qtb = BF.two_centre_elements(Ts, Ps, 1.0, 2.0, b, z, v)
    NT = T.N
    assert np.abs(S[:NT, NT:] - Sb).max() < 1e-8
    assert np.abs(H[:NT, NT:] - Qb).max() < 1e-8
    assert np.array_equal(H[NT:, :NT], H[:NT, NT:].conj().T)          # Eq. 1's Q^+
    assert np.allclose(S[NT:, :NT], S[:NT, NT:].conj().T, atol=0)
    # the reverse-transfer integral through the same machinery (not used by the path) also matches
    Smol, Qmol, Qtmol = O.molecular_integrals(tiny2c, b, v, z, reverse=True)
    Qt = (O.rotate(T, P, Qtmol, math.acos(z / math.hypot(b, z)))).conj().T
    assert np.abs(Qt - Qtb).max() < 1e-8


def test_far_limit_S_to_identity(tiny2c):
    # radial functions vanish beyond r_max = 100: for R > 2 r_max every two-centre element is exactly 0
    S, H = O.assemble(tiny2c, 1.0, 1.0, 250.0)
    NT = tiny2c.T.N
    assert np.array_equal(S, np.eye(tiny2c.N))
    assert np.all(H[:NT, NT:] == 0) and np.all(H[NT:, :NT] == 0)
    # and they decay like the slowest orbital (2p on Z=1: e^{-r/2}): small at R = 40, negligible at R = 80
    S2, _ = O.assemble(tiny2c, 1.0, 1.0, 40.0)
    S3, _ = O.assemble(tiny2c, 1.0, 1.0, 80.0)
    assert np.abs(S2 - np.eye(tiny2c.N)).max() < 1e-6
    assert np.abs(S3 - np.eye(tiny2c.N)).max() < 1e-13


def test_energy_phases(grid):
    T = _centre(1.0, [(1, 0), (2, 1)], grid, eps=[-0.5, -0.125])
    basis = wi.Basis(grid=grid, T=T, P=None, quad=None, Z_T=1.0, Z_P=1.0)
    T0 = _centre(1.0, [(1, 0), (2, 1)], grid)
    b0 = wi.Basis(grid=grid, T=T0, P=None, quad=None, Z_T=1.0, Z_P=1.0)
    z, v = 1.7, 0.8
    _, H = O.assemble(basis, 1.0, v, z)
    _, H0 = O.assemble(b0, 1.0, v, z)
    # element (1s, 2p m) carries exp(i (eps_1s - eps_2p) z / v)
    assert H[0, 2] == pytest.approx(H0[0, 2] * np.exp(1j * (-0.5 + 0.125) * z / v), abs=1e-15)


# ---------------------------------------------------------------- solve and Algorithm 1
def test_solve_residual(tiny2c):
    S, H = O.assemble(tiny2c, 0.5, 1.2, 0.1)
    X = O.solve(S, H)
    assert np.abs(S @ X - H).max() < 1e-13 * max(1.0, np.abs(H).max())


def test_rk4_one_step_is_taylor_polynomial():
    rng = np.random.default_rng(0)
    M = (rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))) * 0.3
    c0 = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    h = 0.37
    got = O.rk4_path(lambda z: M, np.array([0.0, h]), c0)
    want = sum(np.linalg.matrix_power(h * M, k) @ c0 / math.factorial(k) for k in range(5))
    assert np.abs(got - want).max() < 1e-14


def test_rk4_converges_to_matrix_exponential_propagation(tiny2c):
    # tiny two-centre basis; reference: product of exp(h' M(z_mid)) with h' = h/64 (scipy expm)
    b, v = 1.0, 1.5
    Mf = lambda z: O.coupling_M(tiny2c, b, v, z)
    z0, z1 = -3.0, 3.0
    c0 = O.initial_state(tiny2c)
    zf = np.linspace(z0, z1, 12 * 64 + 1)
    ref = c0.copy()
    for a, bb in zip(zf[:-1], zf[1:]):
        ref = expm((bb - a) * Mf(0.5 * (a + bb))) @ ref
    e = []
    for n in (12, 24, 48):
        c = O.rk4_path(Mf, np.linspace(z0, z1, n + 1), c0)
        e.append(np.abs(c - ref).max())
    # exp-midpoint reference itself carries an O(h'^2) error: compare the RK4 sequence's convergence
    assert e[2] < 1e-4
    assert e[0] > e[1] > e[2]


def test_one_centre_unitarity():
    # S = I and D Hermitian: |c|^2 is conserved up to RK4's (h w)^6/72 per step
    g = wi.radial_grid(1000)
    T = _centre(1.0, [(1, 0), (2, 0), (2, 1)], g, eps=[-0.5, -0.125, -0.125])
    basis = wi.Basis(grid=g, T=T, P=None, quad=None, Z_T=1.0, Z_P=1.0)
    zg = wi.uniform_zgrid(-6.0, 6.0, 0.01)
    c = O.propagate(basis, 0.8, 1.0, zg)
    assert abs(np.vdot(c, c).real - 1.0) < 1e-10
    P = O.probabilities(c)
    # m <-> -m reflection: P(2p, m=+1) == P(2p, m=-1)
    assert P[2] == pytest.approx(P[4], abs=1e-14)
    assert P[1] > 1e-6 and P[3] > 1e-6  # the collision does excite


def test_two_centre_m_reflection_of_probabilities(tiny2c):
    c = O.propagate(tiny2c, 1.0, 1.5, wi.uniform_zgrid(-4.0, 4.0, 0.2))
    P = O.probabilities(c)
    T, Pc = tiny2c.T, tiny2c.P
    idx = lambda cen, off, rad, m: off + [k for k in range(cen.N) if cen.st_rad[k] == rad and cen.st_m[k] == m][0]
    assert P[idx(T, 0, 2, 1)] == pytest.approx(P[idx(T, 0, 2, -1)], rel=1e-10, abs=1e-15)
    assert P[idx(Pc, T.N, 1, 1)] == pytest.approx(P[idx(Pc, T.N, 1, -1)], rel=1e-10, abs=1e-15)


def test_radial_integral_beyond_grid_is_multipole_tail():
    # beyond r_max the 1s-1s multipole integral is 1/R (unit charge inside), up to the e^{-2 r_max} tail
    g = wi.radial_grid(2000)
    f = wi.hydrogenic_radial(1, 0, 1.0, g.r)[None, :]
    for R in (120.0, 300.0):
        assert O.radial_F(g, f, f, 0, R)[0] == pytest.approx(1.0 / R, rel=1e-8)
    # and continuous across the last grid point
    a = O.radial_F(g, f, f, 0, g.r[-1])[0]
    b = O.radial_F(g, f, f, 0, g.r[-1] * (1 + 1e-12))[0]
    assert a == pytest.approx(b, rel=1e-10)


def test_paper_lower_left_block_keeps_the_spectrum_real(grid):
    # Eq. 1 with Q^+ below the diagonal: H Hermitian and S positive definite, so M = -(i/v) S^-1 H has a
    # purely imaginary spectrum; the exact reverse-transfer integral instead gives growing modes when the
    # two centres differ (here C6+ on H with pseudostates).
    basis = wi.make_basis(1.0, 6.0, 2, 1, 3, 4.0, True, Nr=1000, Geta=32, Gtau=32)
    S, H = O.assemble(basis, 0.5, 2.0, 0.0)
    ev = np.linalg.eigvals((-1j / 2.0) * np.linalg.solve(S, H))
    assert np.abs(ev.real).max() < 1e-10
    NT = basis.T.N
    Smol, Qmol, Qtmol = O.molecular_integrals(basis, 0.5, 2.0, 0.0, reverse=True)
    ph = O.phases(basis.T.st_eps, basis.P.st_eps, 0.0, 2.0)
    Qt = (O.rotate(basis.T, basis.P, Qtmol, math.pi / 2) * ph).conj().T
    H2 = H.copy()
    H2[NT:, :NT] = Qt
    ev2 = np.linalg.eigvals((-1j / 2.0) * np.linalg.solve(S, H2))
    assert ev2.real.max() > 1e-3


def test_schur_complement_solve_of_the_overlap():
    """The Schur-complement reading of S k = t used by the Schur solve mode: S = [[I, K], [K^+, I]] is a
    Gram matrix, I - K^+ K = L L^+ (Cholesky, positive pivots), and k_P = (L L^+)^-1 (t_P - K^+ t_T),
    k_T = t_T - K k_P reproduce the direct solve; on the oracle's own two-centre S at close approach."""
    basis = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=20, Gtau=14)
    S, H = O.assemble(basis, 0.4, 1.3, 0.1)
    NT = basis.T.N
    K = S[:NT, NT:]
    assert np.allclose(S[:NT, :NT], np.eye(NT)) and np.allclose(S[NT:, NT:], np.eye(S.shape[0] - NT))
    Lc = np.linalg.cholesky(np.eye(S.shape[0] - NT) - K.conj().T @ K)
    assert np.all(np.diag(Lc).real > 0)
    t = H @ (np.arange(S.shape[0]) + 1j * np.cos(np.arange(S.shape[0])))
    uP = t[NT:] - K.conj().T @ t[:NT]
    kP = np.linalg.solve(Lc.conj().T, np.linalg.solve(Lc, uP))
    kT = t[:NT] - K @ kP
    k = np.concatenate([kT, kP])
    assert np.abs(k - np.linalg.solve(S, t)).max() < 1e-12 * np.abs(k).max()



@pytest.fixture(scope="module")
def schroedinger_case():
    # One-centre hydrogen n <= 3 subset, projectile charge 1, v = 0.8. Reference: the Schroedinger
    # picture i v da/dz = (diag(eps) + D(z)) a, with no energy phases at all, as a product of
    # exp-midpoint steps (scipy expm), Richardson-extrapolated from two step sizes.
    g = wi.radial_grid(1000)
    nl = [(1, 0), (2, 0), (2, 1), (3, 2)]
    eps = np.array([-0.5, -0.125, -0.125, -1.0 / 18.0])
    f = [wi.hydrogenic_radial(n, l, 1.0, g.r) for n, l in nl]
    T = wi.centre_from_functions(1.0, [l for _, l in nl], [n for n, _ in nl], f, eps)
    basis = wi.Basis(grid=g, T=T, P=None, quad=None, Z_T=1.0, Z_P=1.0)
    b, v, z0, z1 = 1.0, 0.8, -10.0, 10.0
    E = np.diag(T.st_eps).astype(np.complex128)
    D = {}

    def schroedinger(n):
        zs = np.linspace(z0, z1, n + 1)
        a = np.zeros(T.N, dtype=np.complex128)
        a[0] = 1.0
        for za, zb in zip(zs[:-1], zs[1:]):
            zm = 0.5 * (za + zb)
            if zm not in D:
                R = math.hypot(b, zm)
                D[zm] = O.direct_block(g, T, 1.0, R, zm / R, other_at_minus_R=False)
            a = expm((-1j / v) * (zb - za) * (E + D[zm])) @ a
        return np.abs(a) ** 2

    P1, P2 = schroedinger(1000), schroedinger(2000)
    return basis, b, v, wi.uniform_zgrid(z0, z1, 0.02), (4.0 * P2 - P1) / 3.0


def test_interaction_picture_matches_schroedinger_picture(schroedinger_case):
    # The oracle propagates interaction-picture amplitudes (Eq. 5 with the energy phases of H);
    # |a|^2 = |c|^2, so the probabilities must agree with the Schroedinger-picture reference. This
    # fixes the -(i/v) factor, the sign and the 1/v of the phases and Algorithm 1's use of M.
    basis, b, v, zg, ref = schroedinger_case
    P = O.probabilities(O.propagate(basis, b, v, zg))
    assert P[1] > 0.05 and P[3] > 0.005 and P[7] > 0.005    # a strong collision: far from first order
    assert np.abs(P - ref).max() < 1e-8


_PHASES, _COUPLING = O.phases, O.coupling_M


@pytest.mark.parametrize("mistake", ["phase sign", "phase z*v", "M without 1/v", "M with +i"])
def test_interaction_picture_mistakes_fail(schroedinger_case, mistake, monkeypatch):
    # each planted mistake in the oracle moves the probabilities far outside the pin's tolerance
    basis, b, v, zg, ref = schroedinger_case
    if mistake == "phase sign":
        monkeypatch.setattr(O, "phases", lambda er, ec, z, v: _PHASES(er, ec, -z, v))
    elif mistake == "phase z*v":
        monkeypatch.setattr(O, "phases", lambda er, ec, z, v: _PHASES(er, ec, z * v * v, v))
    elif mistake == "M without 1/v":
        monkeypatch.setattr(O, "coupling_M", lambda bs, b, v, z: v * _COUPLING(bs, b, v, z))
    else:
        monkeypatch.setattr(O, "coupling_M", lambda bs, b, v, z: -_COUPLING(bs, b, v, z))
    P = O.probabilities(O.propagate(basis, b, v, zg))
    assert np.abs(P - ref).max() > 1e-4


@pytest.fixture(scope="module")
def schroedinger_two_centre():
    # Two-centre p + H, tiny basis (target 1s, 2s, 2p; projectile 1s, 2p), v = 1.2. Without the energy
    # phases the oracle's system reads i v S0 da/dz = (S0 diag(eps) + V0) a, with S0 and V0 the blocks of
    # Eq. 1 at phase zero (K, Q rotated from the molecular frame; D_T, D_P; lower-left Q^+). Reference: that
    # ODE in the form da/dz = -(i/v)(diag(eps) + S0^-1 V0) a, integrated by scipy's DOP853 at rtol 1e-11.
    from scipy.integrate import solve_ivp
    g = wi.radial_grid(1000)
    T = _centre(1.0, [(1, 0), (2, 0), (2, 1)], g, eps=[-0.5, -0.125, -0.125])
    P = _centre(1.0, [(1, 0), (2, 1)], g, eps=[-0.5, -0.125])
    basis = wi.Basis(grid=g, T=T, P=P, quad=wi.make_quadrature(24, 24, 0.5), Z_T=1.0, Z_P=1.0)
    b, v, z0, z1 = 1.0, 1.2, -6.0, 6.0
    NT, N = T.N, basis.N
    eps = np.concatenate([T.st_eps, P.st_eps])

    def generator(z):
        R = math.hypot(b, z)
        th = math.acos(z / R)
        Smol, Qmol = O.molecular_integrals(basis, b, v, z)
        K, Q = O.rotate(T, P, Smol, th), O.rotate(T, P, Qmol, th)
        S0 = np.eye(N, dtype=np.complex128)
        S0[:NT, NT:] = K
        S0[NT:, :NT] = K.conj().T
        V0 = np.zeros((N, N), dtype=np.complex128)
        V0[:NT, :NT] = O.direct_block(g, T, 1.0, R, z / R, other_at_minus_R=False)
        V0[NT:, NT:] = O.direct_block(g, P, 1.0, R, z / R, other_at_minus_R=True)
        V0[:NT, NT:] = Q
        V0[NT:, :NT] = Q.conj().T
        return (-1j / v) * (np.diag(eps) + np.linalg.solve(S0, V0))

    a0 = np.zeros(N, dtype=np.complex128)
    a0[0] = 1.0
    sol = solve_ivp(lambda z, a: generator(z) @ a, (z0, z1), a0, method="DOP853", rtol=1e-11, atol=1e-13)
    assert sol.status == 0
    return basis, b, v, wi.uniform_zgrid(z0, z1, 0.04), np.abs(sol.y[:, -1]) ** 2


def test_two_centre_interaction_picture_matches_schroedinger_picture(schroedinger_two_centre):
    # |a|^2 = |c|^2: fixes the energy phases of K and Q (target-minus-projectile energies), the solve
    # M = -(i/v) S^-1 H of Eq. 4 with phased S, and Algorithm 1 in the two-centre form
    basis, b, v, zg, ref = schroedinger_two_centre
    P = O.probabilities(O.propagate(basis, b, v, zg))
    assert P[basis.T.N] > 0.1                    # capture into the projectile 1s is strong
    assert np.abs(P - ref).max() < 1e-8


def test_two_centre_phase_mistake_fails(schroedinger_two_centre, monkeypatch):
    # the phases of the target-projectile blocks with the opposite sign (diagonal blocks unchanged)
    basis, b, v, zg, ref = schroedinger_two_centre
    monkeypatch.setattr(O, "phases", lambda er, ec, z, v: _PHASES(er, ec, z if er is ec else -z, v))
    P = O.probabilities(O.propagate(basis, b, v, zg))
    assert np.abs(P - ref).max() > 1e-2


def test_parallel_oracle_driver_equals_the_serial_oracle():
    # the pool only reorders independent M(z) evaluations: the amplitudes are bit-identical
    import oracle_parallel as OP
    basis = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=16, Gtau=12)
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.25)
    c1 = OP.propagate(basis, 0.7, 1.2, zg, workers=3, block=7)
    c0 = O.propagate(basis, 0.7, 1.2, zg)
    assert np.array_equal(c1, c0)


def _overlap_balance(basis, b, v, zg, Mfun):
    """(change of c^+ S c over the path, Simpson integral of c^+ (dS/dz) c) for the amplitudes that
    oracle.rk4_path produces step by step with the given M(z)."""
    c = O.initial_state(basis)
    cs, norms = [c], [np.real(c.conj() @ O.assemble(basis, b, v, zg[0])[0] @ c)]
    for k in range(1, zg.size):
        c = O.rk4_path(Mfun, zg[k - 1:k + 1], c)
        cs.append(c)
        norms.append(np.real(c.conj() @ O.assemble(basis, b, v, zg[k])[0] @ c))
    dz = 1e-4
    f = np.array([np.real(ck.conj() @ ((O.assemble(basis, b, v, z + dz)[0] - O.assemble(basis, b, v, z - dz)[0])
                                       / (2 * dz)) @ ck) for ck, z in zip(cs, zg)])
    h = zg[1] - zg[0]
    simpson = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    return norms[-1] - norms[0], simpson


def test_overlap_norm_obeys_its_balance_law():
    # i v S dc/dz = H c with Hermitian H and S (Eq. 1 with the lower-left block Q^+) gives
    # d(c^+ S c)/dz = c^+ (dS/dz) c: the two-centre propagation moves c^+ S c exactly by that integral
    # (it is not conserved: dS/dz != 0).  Planted mistake: the lower-left block Q^T (H not Hermitian)
    basis = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=16, Gtau=12)
    b, v = 0.7, 1.2
    zg = wi.uniform_zgrid(-2.0, 2.0, 0.02)
    drift, integral = _overlap_balance(basis, b, v, zg, lambda z: O.coupling_M(basis, b, v, z))
    assert abs(drift) > 1e-3
    assert abs(drift - integral) < 1e-8

    def M_transposed(z):
        S, H = O.assemble(basis, b, v, z)
        NT = basis.T.N
        H = H.copy()
        H[NT:, :NT] = H[:NT, NT:].T
        return (-1j / v) * np.linalg.solve(S, H)
    drift_m, integral_m = _overlap_balance(basis, b, v, zg, M_transposed)
    assert abs(drift_m - integral_m) > 1e-4
