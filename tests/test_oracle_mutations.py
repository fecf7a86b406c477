"""Plausible mistakes planted in the oracle (on the CPU) must fail the brute-force pins.

Each test swaps one ingredient of the oracle for a wrong-but-plausible variant and
checks that the lab-frame brute-force comparison then fails, so the pins really
constrain that ingredient.
"""
import math

import numpy as np
import pytest
from scipy import special

import wpccc_inputs as wi
from oracle import wpccc_oracle as O
import brute_force as BF


def _centre(Z, nl, grid):
    f = [wi.hydrogenic_radial(n, l, Z, grid.r) for n, l in nl]
    return wi.centre_from_functions(Z, [l for n, l in nl], [n for n, l in nl], f, np.zeros(len(nl)))


@pytest.fixture(scope="module")
def setup():
    g = wi.radial_grid(1500)
    T = _centre(1.0, [(1, 0), (2, 1)], g)
    P = _centre(2.0, [(1, 0), (2, 1)], g)
    basis = wi.Basis(grid=g, T=T, P=P, quad=wi.make_quadrature(40, 40, 0.5), Z_T=1.0, Z_P=2.0)
    b, z, v = 1.3, -0.7, 0.9
    Ts = [(int(T.rad_n[T.st_rad[i]]), int(T.st_l[i]), int(T.st_m[i]), 1.0) for i in range(T.N)]
    Ps = [(int(P.rad_n[P.st_rad[i]]), int(P.st_l[i]), int(P.st_m[i]), 2.0) for i in range(P.N)]
    Sb, Qb, Qtb = BF.two_centre_elements(Ts, Ps, 1.0, 2.0, b, z, v)
    DPb = BF.direct_elements(Ps, 1.0, b, z, centre_is_projectile=True)
    return basis, (b, z, v), (Sb, Qb, Qtb, DPb)


def _errors(basis, bzv, ref):
    # K, Q and the lower-left block (Q^+, Eq. 1) against the brute-force integrals
    b, z, v = bzv
    S, H = O.assemble(basis, b, v, z)
    NT = basis.T.N
    Sb, Qb, Qtb, DPb = ref
    return (np.abs(S[:NT, NT:] - Sb).max(), np.abs(H[:NT, NT:] - Qb).max(),
            np.abs(H[NT:, :NT] - Qb.conj().T).max(), np.abs(H[NT:, NT:] - DPb).max())


def test_unmutated_oracle_passes(setup):
    basis, bzv, ref = setup
    eK, eQ, eQt, eDP = _errors(basis, bzv, ref)
    assert max(eK, eQ, eQt) < 1e-8 and eDP < 2e-5


def test_phase_i_power_instead_of_minus_i_fails(setup, monkeypatch):
    # the paper's printed i^{q-q'}: equivalent to J_d(-x) = (-1)^d J_d(x)
    basis, bzv, ref = setup
    jv = special.jv
    monkeypatch.setattr(O.special, "jv", lambda d, x: (-1.0) ** d * jv(d, x))
    eK, eQ, eQt, _ = _errors(basis, bzv, ref)
    assert min(eK, eQ, eQt) > 1e-4


def test_transposed_wigner_d_fails(setup, monkeypatch):
    basis, bzv, ref = setup
    real = O.wigner_d
    monkeypatch.setattr(O, "wigner_d", lambda j, mp, m, beta: real(j, m, mp, beta))
    eK, eQ, eQt, _ = _errors(basis, bzv, ref)
    assert max(eK, eQ, eQt) > 1e-4


def test_projectile_direct_without_parity_sign_fails(setup, monkeypatch):
    basis, bzv, ref = setup
    real = O.direct_block

    def no_sign(grid, centre, Z, R, cth, other_at_minus_R):
        return real(grid, centre, Z, R, cth, other_at_minus_R=False)
    monkeypatch.setattr(O, "direct_block", no_sign)
    _, _, _, eDP = _errors(basis, bzv, ref)
    assert eDP > 1e-3


def test_legendre_without_condon_shortley_phase_fails(setup, monkeypatch):
    basis, bzv, ref = setup
    real = O.assoc_legendre
    monkeypatch.setattr(O, "assoc_legendre", lambda l, m, x: (-1.0) ** abs(m) * real(l, m, x))
    eK, eQ, eQt, eDP = _errors(basis, bzv, ref)
    assert max(eK, eQ, eQt, eDP) > 1e-4


def test_swapped_charges_in_transfer_integrals_fails(setup, monkeypatch):
    # Q with -Z_P/r_T and Q~ with -Z_T/r_P (the two nuclear charges exchanged)
    basis, bzv, ref = setup
    real = O.molecular_integrals

    def swapped(bs, b, v, z, reverse=False):
        other = wi.Basis(grid=bs.grid, T=bs.T, P=bs.P, quad=bs.quad, Z_T=bs.Z_P, Z_P=bs.Z_T)
        return real(other, b, v, z, reverse)
    monkeypatch.setattr(O, "molecular_integrals", swapped)
    eK, eQ, eQt, _ = _errors(basis, bzv, ref)
    assert eK < 1e-8 and eQ > 1e-3
