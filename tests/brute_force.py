"""Brute-force lab-frame integrals used to pin the oracle's two-centre and direct elements.

Independent of the oracle's Eq. 8/9 machinery: each element is a direct 3-D
quadrature over prolate spheroidal coordinates (eta, tau, phi) with foci at the
two nuclei, in an arbitrary frame around the internuclear axis.  The wave
functions are evaluated in the laboratory frame from closed-form hydrogenic
radial functions and scipy's spherical harmonics, and the electron-translation
phase exp(i v.r) is applied explicitly; no Wigner rotation, no Bessel function
and no molecular-frame factorisation is used.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from wpccc_inputs import hydrogenic_radial


def _psi(n, l, m, Z, vec):
    """Hydrogenic orbital at lab-frame displacement vec[..., 3] from its nucleus."""
    r = np.linalg.norm(vec, axis=-1)
    th = np.arccos(np.clip(vec[..., 2] / np.where(r > 0, r, 1.0), -1.0, 1.0))
    ph = np.arctan2(vec[..., 1], vec[..., 0])
    return hydrogenic_radial(n, l, Z, r) * special.sph_harm_y(l, m, th, ph)


def prolate_grid(b, z, n_u=160, n_tau=96, n_phi=64, u_max=None):
    """Points (relative to T at the origin), weights and the frame of a prolate spheroidal rule."""
    Rv = np.array([b, 0.0, z])
    R = float(np.linalg.norm(Rv))
    ez = Rv / R
    # any perpendicular pair; deliberately not the rotation-about-y frame
    t = np.array([0.3, 0.8, 0.1])
    ex = t - ez * (t @ ez)
    ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    if u_max is None:
        u_max = math.acosh(1.0 + 160.0 / R)
    xu, wu = np.polynomial.legendre.leggauss(n_u)
    u = 0.5 * u_max * (xu + 1.0)
    wu = 0.5 * u_max * wu
    eta = np.cosh(u)
    weta = wu * np.sinh(u)
    tau, wtau = np.polynomial.legendre.leggauss(n_tau)
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    wphi = np.full(n_phi, 2.0 * np.pi / n_phi)
    E, Tt, Ph = np.meshgrid(eta, tau, phi, indexing="ij")
    W = np.einsum("i,j,k->ijk", weta, wtau, wphi)
    rho = 0.5 * R * np.sqrt((E * E - 1.0) * (1.0 - Tt * Tt))
    zp = 0.5 * R * E * Tt
    W = W * (R / 2.0) ** 3 * (E * E - Tt * Tt)
    # position relative to the midpoint, then relative to T (origin) and P (at Rv)
    rmid = (rho * np.cos(Ph))[..., None] * ex + (rho * np.sin(Ph))[..., None] * ey + zp[..., None] * ez
    return rmid, W.ravel(), Rv


def two_centre_elements(T_states, P_states, Z_T, Z_P, b, z, v, VT=None, **kw):
    """Return (S_TP, Q, Qtilde) with S_TP[i,j] = <T_i e^{-iv.r/2}|P_j e^{iv.r/2}>,
    Q[i,j] = <T_i ..| V_T(r_T) |P_j ..> (V_T = -Z_T/r_T unless the callable VT is given),
    Qtilde[j,i] = <P_j ..| -Z_P/r_P |T_i ..>.  States are (n, l, m, Z) tuples; energies are not applied."""
    rmid, W, Rv = prolate_grid(b, z, **kw)
    rT = rmid + 0.5 * Rv
    rP = rmid - 0.5 * Rv
    etf = np.exp(1j * v * rmid[..., 2]).ravel()
    dT = np.linalg.norm(rT, axis=-1).ravel()
    dP = np.linalg.norm(rP, axis=-1).ravel()
    PT = [(_psi(n, l, m, Zs, rT)).ravel() for (n, l, m, Zs) in T_states]
    PP = [(_psi(n, l, m, Zs, rP)).ravel() for (n, l, m, Zs) in P_states]
    S = np.zeros((len(PT), len(PP)), complex)
    Q = np.zeros_like(S)
    Qt = np.zeros((len(PP), len(PT)), complex)
    for i, a in enumerate(PT):
        for j, c in enumerate(PP):
            base = W * np.conj(a) * c * etf
            S[i, j] = base.sum()
            Q[i, j] = (base * ((-Z_T / dT) if VT is None else VT(dT))).sum()
            Qt[j, i] = (W * np.conj(c) * a * np.conj(etf) * (-Z_P / dP)).sum()
    return S, Q, Qt


def direct_elements(states, Z_other, b, z, centre_is_projectile=False, **kw):
    """D[i,j] = <i| -Z_other/|r - R_other| |j> for states on one centre, by the same 3-D rule."""
    rmid, W, Rv = prolate_grid(b, z, **kw)
    rT = rmid + 0.5 * Rv
    rP = rmid - 0.5 * Rv
    own, other = (rP, rT) if centre_is_projectile else (rT, rP)
    dO = np.linalg.norm(other, axis=-1).ravel()
    F = [(_psi(n, l, m, Zs, own)).ravel() for (n, l, m, Zs) in states]
    D = np.zeros((len(F), len(F)), complex)
    for i, a in enumerate(F):
        for j, c in enumerate(F):
            D[i, j] = (W * np.conj(a) * c * (-Z_other / dO)).sum()
    return D


def potential_elements(states, V, b, z, centre_is_projectile=False, **kw):
    """D[i,j] = <i| V(|r - R_other|) |j> for states on one centre and any central potential V of the
    distance to the other nucleus, by the same 3-D rule."""
    rmid, W, Rv = prolate_grid(b, z, **kw)
    rT = rmid + 0.5 * Rv
    rP = rmid - 0.5 * Rv
    own, other = (rP, rT) if centre_is_projectile else (rT, rP)
    Vo = V(np.linalg.norm(other, axis=-1).ravel())
    F = [(_psi(n, l, m, Zs, own)).ravel() for (n, l, m, Zs) in states]
    D = np.zeros((len(F), len(F)), complex)
    for i, a in enumerate(F):
        for j, c in enumerate(F):
            D[i, j] = (W * np.conj(a) * c * Vo).sum()
    return D
