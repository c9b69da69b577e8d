"""Brute-force velocity-space quadrature of the gas-kinetic flux (test helper).

Every moment is a plain weighted sum over a tensor grid in (u, v, w, s = xi^2)
for K = 2 internal degrees of freedom (gamma = 1.4): Gauss-Legendre in u on
each half-line (split at u = 0 for the Heaviside factors), Gauss-Hermite in
v and w, and Gauss-Laguerre in s (d^2 xi = pi ds).  Micro-slopes are solved
with numpy from brute-force Gram matrices, the time integrals of Eq. (flux)
use Gauss-Legendre in t, and F^n, dF/dt come from the 2x2 system of
Section 2.2 solved by numpy.  Nothing here shares code with the oracle.
"""
from __future__ import annotations

import numpy as np

K_INT = 2.0


class Grid:
    def __init__(self, nu=40, nv=28, ns=40, L=9.0, s_scale=0.8, lam_ref=0.5):
        xu, wu = np.polynomial.legendre.leggauss(nu)
        up = 0.5 * L * (xu + 1.0)
        wp = 0.5 * L * wu
        u = np.concatenate([-up[::-1], up])
        wuu = np.concatenate([wp[::-1], wp])
        xv, wv = np.polynomial.hermite.hermgauss(nv)
        v = xv / np.sqrt(lam_ref)
        wvv = wv * np.exp(xv * xv) / np.sqrt(lam_ref)
        xs, ws = np.polynomial.laguerre.laggauss(ns)
        s = xs / s_scale
        wss = ws * np.exp(xs) / s_scale * np.pi
        U, V, W, S = np.meshgrid(u, v, v, s, indexing="ij")
        self.u, self.v, self.w, self.s = U, V, W, S
        self.wt = (wuu[:, None, None, None] * wvv[None, :, None, None] * wvv[None, None, :, None]
                   * wss[None, None, None, :])
        self.pos = (U > 0).astype(np.float64)
        self.neg = 1.0 - self.pos
        self.psi = [np.ones_like(U), U, V, W, 0.5 * (U * U + V * V + W * W + S)]

    def maxwellian(self, rho, Uv, lam):
        c2 = (self.u - Uv[0]) ** 2 + (self.v - Uv[1]) ** 2 + (self.w - Uv[2]) ** 2 + self.s
        return rho * (lam / np.pi) ** ((K_INT + 3) / 2) * np.exp(-lam * c2)

    def integ(self, f):
        return float(np.sum(f * self.wt))

    def mom(self, f):
        """int psi f dXi (5-vector)."""
        return np.array([self.integ(p * f) for p in self.psi])

    def slope_field(self, a):
        return sum(a[i] * self.psi[i] for i in range(5))


def prim(q, gamma=1.4):
    K = (5 - 3 * gamma) / (gamma - 1)
    rho = q[0]
    U = q[1:4] / rho
    lam = (K + 3) * rho / (4 * (q[4] - 0.5 * rho * U @ U))
    return rho, U, lam


def bgk_flux(G: Grid, ql, dql, qr, dqr, dt, mu=0.0, Pr=1.0, tau_c=0.0, nt=20):
    """F^n and dF/dt through the normal e_x.  dql[j], dqr[j]: dQ/dx_j (j = x, y, z)."""
    rl, Ul, ll = prim(ql)
    rr, Ur, lr = prim(qr)
    gl = G.maxwellian(rl, Ul, ll)
    gr = G.maxwellian(rr, Ur, lr)
    q0 = G.mom(gl * G.pos) + G.mom(gr * G.neg)
    r0, U0, l0 = prim(q0)
    g0 = G.maxwellian(r0, U0, l0)

    def gram(g):
        return np.array([[G.integ(G.psi[i] * G.psi[k] * g) for k in range(5)] for i in range(5)])

    Gl, Gr, G0 = gram(gl), gram(gr), gram(g0)
    al = [np.linalg.solve(Gl, dql[j]) for j in range(3)]
    ar = [np.linalg.solve(Gr, dqr[j]) for j in range(3)]
    vel = [G.u, G.v, G.w]
    dq0 = [G.mom(G.slope_field(al[j]) * gl * G.pos) + G.mom(G.slope_field(ar[j]) * gr * G.neg) for j in range(3)]
    ab = [np.linalg.solve(G0, dq0[j]) for j in range(3)]

    def adotu(a):
        return sum(vel[j] * G.slope_field(a[j]) for j in range(3))

    Ab = np.linalg.solve(G0, -G.mom(adotu(ab) * g0))
    Al = np.linalg.solve(Gl, -G.mom(adotu(al) * gl))
    Ar = np.linalg.solve(Gr, -G.mom(adotu(ar) * gr))
    p0, pl, pr = r0 / (2 * l0), rl / (2 * ll), rr / (2 * lr)
    tau = mu / p0 + tau_c * dt * abs(pl - pr) / (pl + pr)

    AU0, AUl, AUr = adotu(ab), adotu(al), adotu(ar)
    A0f, Alf, Arf = G.slope_field(Ab), G.slope_field(Al), G.slope_field(Ar)
    uF = [G.u * p for p in G.psi]

    # flux moments of the pieces of Eq. (flux) that multiply each time weight
    E0 = np.array([G.integ(x * g0) for x in uF])
    E2 = np.array([G.integ(x * AU0 * g0) for x in uF])
    E3 = np.array([G.integ(x * A0f * g0) for x in uF])
    nl = np.array([G.integ(x * gl * G.pos) for x in uF]) + np.array([G.integ(x * gr * G.neg) for x in uF])
    nla = np.array([G.integ(x * AUl * gl * G.pos) for x in uF]) + np.array([G.integ(x * AUr * gr * G.neg) for x in uF])
    nlA = np.array([G.integ(x * Alf * gl * G.pos) for x in uF]) + np.array([G.integ(x * Arf * gr * G.neg) for x in uF])
    # heat flux of the first-order equilibrium part (Prandtl fix reading)
    cu = G.u - U0[0]
    ce = 0.5 * ((G.u - U0[0]) ** 2 + (G.v - U0[1]) ** 2 + (G.w - U0[2]) ** 2 + G.s)
    qrate = G.integ(cu * ce * (-(AU0 + A0f)) * g0)

    def I(T):
        xt, wt = np.polynomial.legendre.leggauss(nt)
        t = 0.5 * T * (xt + 1)
        wt = 0.5 * T * wt
        out = np.zeros(5)
        for ti, wi in zip(t, wt):
            if tau > 0:
                e = np.exp(-ti / tau)
                w1, w2, w3 = 1 - e, (ti + tau) * e - tau, ti - tau + tau * e
                w4, w5 = e, (tau + ti) * e
            else:
                w1, w2, w3, w4, w5 = 1.0, 0.0, ti, 0.0, 0.0
            out += wi * (w1 * E0 + w2 * E2 + w3 * E3 + w4 * nl - w5 * nla - tau * w4 * nlA)
        if tau > 0 and Pr != 1.0:
            out[4] += (1.0 / Pr - 1.0) * tau * T * qrate
        return out

    I1, Ih = I(dt), I(0.5 * dt)
    A = np.array([[dt, 0.5 * dt * dt], [0.5 * dt, dt * dt / 8]])
    F = np.zeros(5)
    dF = np.zeros(5)
    for i in range(5):
        F[i], dF[i] = np.linalg.solve(A, [I1[i], Ih[i]])
    return F, dF
