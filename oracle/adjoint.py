"""Reverse-mode derivative of the RK4 LLG trajectory (FP64), written by hand.

Forward (one step, unit vectors m, per-cell B = mu0 H_eff in tesla):
    k1 = f(s1), s1 = m
    k2 = f(s2), s2 = m + dt/2 k1
    k3 = f(s3), s3 = m + dt/2 k2
    k4 = f(s4), s4 = m + dt k3
    u  = m + dt/6 (k1 + 2 k2 + 2 k3 + k4),   m' = u / |u|
    f(s) = g1 s x B(s) + g2 s x (s x B(s)),   g1 = -gamma/(1+a^2), g2 = a g1   (eq. 2)
    B(s) = L s + c(r) s_x x^ + b_ext + h(r)
with L the linear exchange + demag operator (eq. 5/7 and eq. 13 times mu0),
which is symmetric, and c(r) = 2 Ku(r)/Ms the anisotropy coefficient (eq. 8).

Reverse, for a cotangent lam of m':
    lam_u = (I - m' m'^T) lam / |u|
    lam_m = lam_u, lam_k1 = lam_k4 = dt/6 lam_u, lam_k2 = lam_k3 = dt/3 lam_u
    for stages 4, 3, 2, 1 (vector-Jacobian product of f at s with cotangent lk):
        lam_B   = g1 (lk x s) + g2 ((lk x s) x s)
        lam_loc = g1 (B x lk) + g2 ((s x B) x lk) + g2 (B x (lk x s))
        lam_s   = lam_loc + L lam_B + c (lam_B)_x x^
        dL/dh  += lam_B,  dL/dKu += (2/Ms) s_x (lam_B)_x
        lam_m  += lam_s, and lam_k3 += dt lam_s (stage 4), lam_k2 += dt/2 lam_s
        (stage 3), lam_k1 += dt/2 lam_s (stage 2)
    the cotangent of m is lam_m.
The terms follow from <lam, a x b> = <b x lam, a> = <lam x a, b>.

The whole trajectory is kept in memory (the oracle is for small films).
"""
import numpy as np

from . import MU0


def _cross(a, b):
    return np.cross(a, b, axis=0)


class AdjointFilm:
    """Wraps an oracle ``Film`` (see llg.py) with B(s), L(v) and the reverse sweep."""

    def __init__(self, film):
        self.film = film
        ku = film.Ku if film.ku_map is None else film.ku_map
        self.c_an = 2.0 * np.asarray(ku, dtype=np.float64) / film.Ms
        g = film.gamma / (1.0 + film.alpha * film.alpha)
        self.g1 = -g
        self.g2 = -film.alpha * g

    def B(self, s):
        return MU0 * self.film.h_eff(s)

    def L(self, v):
        """mu0 (H_exch + H_demag) of an arbitrary vector field v (linear, symmetric)."""
        return MU0 * (self.film.h_exchange(v) + self.film.h_demag(v))

    def f(self, s, B):
        sxB = _cross(s, B)
        return self.g1 * sxB + self.g2 * _cross(s, sxB)

    def step_record(self, m, dt):
        s = [m]
        Bs, ks = [], []
        for i, c in enumerate((0.5, 0.5, 1.0, None)):
            B = self.B(s[i])
            k = self.f(s[i], B)
            Bs.append(B)
            ks.append(k)
            if c is not None:
                s.append(m + c * dt * k)
        u = m + dt / 6.0 * (ks[0] + 2.0 * ks[1] + 2.0 * ks[2] + ks[3])
        nu = np.sqrt((u * u).sum(axis=0, keepdims=True))
        return {"s": s, "B": Bs, "nu": nu, "m_next": u / nu}

    def vjp_f(self, s, B, lk):
        lxs = _cross(lk, s)
        lam_B = self.g1 * lxs + self.g2 * _cross(lxs, s)
        lam_loc = (self.g1 * _cross(B, lk) + self.g2 * _cross(_cross(s, B), lk)
                   + self.g2 * _cross(B, lxs))
        return lam_B, lam_loc

    def forward(self, m0, dt, nsteps):
        m = np.asarray(m0, dtype=np.float64)
        rec = []
        for _ in range(nsteps):
            r = self.step_record(m, dt)
            rec.append(r)
            m = r["m_next"]
        return m, rec

    def backward(self, rec, dt, lam_final):
        """Returns (dL/dm0, dL/dh, dL/dKu) for the recorded trajectory and dL/dm_final = lam_final."""
        lam = np.asarray(lam_final, dtype=np.float64)
        gh = np.zeros_like(lam)
        gku = np.zeros(lam.shape[1:])
        Ms = self.film.Ms
        for r in reversed(rec):
            mn, nu = r["m_next"], r["nu"]
            lam_u = (lam - mn * (mn * lam).sum(axis=0, keepdims=True)) / nu
            lam_m = lam_u.copy()
            lk = [dt / 6.0 * lam_u, dt / 3.0 * lam_u, dt / 3.0 * lam_u, dt / 6.0 * lam_u]
            for i in (3, 2, 1, 0):
                s, B = r["s"][i], r["B"][i]
                lam_B, lam_loc = self.vjp_f(s, B, lk[i])
                gh += lam_B
                gku += (2.0 / Ms) * s[0] * lam_B[0]
                lam_s = lam_loc + self.L(lam_B)
                lam_s[0] += self.c_an * lam_B[0]
                lam_m += lam_s
                if i == 3:
                    lk[2] = lk[2] + dt * lam_s
                elif i == 2:
                    lk[1] = lk[1] + 0.5 * dt * lam_s
                elif i == 1:
                    lk[0] = lk[0] + 0.5 * dt * lam_s
            lam = lam_m
        return lam, gh, gku


def tangent_project(m, g):
    """(I - m m^T) g: the gradient with respect to the direction of m (input normalisation)."""
    return g - m * (m * g).sum(axis=0, keepdims=True)
