"""Exact rational DUGKS stepper in three dimensions (a pin for the FP64 3-D
oracle), D3Q15 (Eq. 2.28) or D3Q19 (Eq. 2.6).

Written independently of ``oracle/dugks3d_oracle.c`` from the basic
definitions: it carries the original distribution f and moves between f,
ftilde, fbar and fbar^+ with Eqs. 2.11, 2.13, 2.15 (f_i restored) and 2.17,
where the oracle uses the shortcut Eqs. 2.21 and 2.22; the equilibrium is the
contraction form of Eq. 2.3 with C built by exact polynomial algebra.  Cells
are addressed by integer triples and ghosts are produced on demand (periodic
image or mirrored Dirichlet ghost with non-equilibrium extrapolation), so no
halo arrays exist.  Everything is ``fractions.Fraction``.

Shared readings with the oracle: each tangential slope at a face is
interpolated between the two cells' central differences (the interior cell's
alone at a Dirichlet wall).
"""
from fractions import Fraction as Fr

D3Q15 = ([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 1), (1, 1, -1),
          (1, -1, 1), (-1, 1, 1), (-1, -1, -1), (-1, -1, 1), (-1, 1, -1), (1, -1, -1)],
         [Fr(2, 9)] + [Fr(1, 9)] * 6 + [Fr(1, 72)] * 8)
D3Q19 = ([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
          (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (-1, 0, 1), (1, 0, -1), (0, 1, 1), (0, -1, -1),
          (0, 1, -1), (0, -1, 1)],
         [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12)


def _peval(a, x):
    acc = Fr(0)
    for v in reversed(a):
        acc = acc * x + v
    return acc


def _pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _pder(a):
    return [k * a[k] for k in range(1, len(a))] or [Fr(0)]


def _pint(a):
    return [Fr(0)] + [a[k] / (k + 1) for k in range(len(a))]


class RationalDUGKS3D:
    def __init__(self, faces, bc, bc_value, lattice, c, u, b, alpha, d, dt):
        self.f = [[Fr(v) for v in ax] for ax in faces]  # face coordinates per axis
        self.n = [len(ax) - 1 for ax in self.f]
        self.per = [bc[2 * a] == 0 for a in range(3)]
        self.bcv = [Fr(v) for v in bc_value]
        self.cvec, self.w = D3Q15 if lattice == 15 else D3Q19
        self.c = Fr(c)
        self.u = [Fr(v) for v in u]
        self.b = [Fr(v) for v in b]
        self.d = [Fr(v) for v in d]
        db = _pder(self.b)
        self.cint = _pint(_pmul(db, db))
        self.cs2 = self.c * self.c / 3
        self.lam = Fr(alpha) / self.cs2
        self.dt = Fr(dt)
        self.h = self.dt / 2

    def feq(self, phi):
        cs2, c = self.cs2, self.c
        bv, dv, cv = _peval(self.b, phi), _peval(self.d, phi), _peval(self.cint, phi)
        out = []
        for e, w in zip(self.cvec, self.w):
            ci = [c * x for x in e]
            cb = sum(ci[a] * self.u[a] for a in range(3)) * bv
            contr = Fr(0)
            for a in range(3):
                for g in range(3):
                    delta = 1 if a == g else 0
                    T = cs2 * dv * delta + self.u[a] * self.u[g] * cv - cs2 * phi * delta
                    contr += T * (ci[a] * ci[g] - cs2 * delta)
            out.append(w * (phi + cb / cs2 + contr / (2 * cs2 * cs2)))
        return out

    def centre(self, a, i):
        """centre coordinate of extended cell index i (-1..n) along axis a"""
        n, f = self.n[a], self.f[a]
        if 0 <= i < n:
            return (f[i] + f[i + 1]) / 2
        if self.per[a]:
            L = f[-1] - f[0]
            return self.centre(a, i % n) + (L if i >= n else -L)
        wall = f[0] if i < 0 else f[-1]
        return 2 * wall - self.centre(a, 0 if i < 0 else n - 1)

    def init(self, phi0):
        """phi0[z][y][x] -> ftilde as a dict (x, y, z) -> list"""
        return {(j, k, l): self.feq(Fr(phi0[l][k][j]))
                for l in range(self.n[2]) for k in range(self.n[1]) for j in range(self.n[0])}

    def step(self, ft):
        lam, dt, h, c = self.lam, self.dt, self.h, self.c
        fbp, ftp, phi, feq = {}, {}, {}, {}
        for cell, fv in ft.items():
            p = sum(fv)
            e = self.feq(p)
            f = [(2 * lam * a + dt * q) / (2 * lam + dt) for a, q in zip(fv, e)]              # Eq. 2.11 inverted
            fbar = [(2 * lam + h) / (2 * lam) * a - h / (2 * lam) * q for a, q in zip(f, e)]  # Eq. 2.15
            fbp[cell] = [(2 * lam - h) / (2 * lam + h) * a + 2 * h / (2 * lam + h) * q for a, q in zip(fbar, e)]
            ftp[cell] = [(2 * lam - dt) / (2 * lam + dt) * a + 2 * dt / (2 * lam + dt) * q for a, q in zip(fv, e)]
            phi[cell], feq[cell] = p, e

        def P(cell):
            cell = list(cell)
            for a in range(3):
                if self.per[a]:
                    cell[a] %= self.n[a]
            cell = tuple(cell)
            if cell in fbp:
                return fbp[cell]
            outside = [a for a in range(3) if not 0 <= cell[a] < self.n[a]]
            if len(outside) != 1:
                raise AssertionError("edge or corner ghost requested")
            a = outside[0]
            inner = list(cell)
            inner[a] = 0 if cell[a] < 0 else self.n[a] - 1
            inner = tuple(inner)
            wall = self.bcv[2 * a] if cell[a] < 0 else self.bcv[2 * a + 1]
            eg = self.feq(2 * wall - phi[inner])
            return [g + (x - q) for g, x, q in zip(eg, fbp[inner], feq[inner])]

        def shift(cell, a, s):
            out = list(cell)
            out[a] += s
            return tuple(out)

        def grad(cell, t):
            i = cell[t]
            dx = self.centre(t, i + 1) - self.centre(t, i - 1)
            return [(x - y) / dx for x, y in zip(P(shift(cell, t, 1)), P(shift(cell, t, -1)))]

        flux = {}
        for a in range(3):
            tang = [t for t in range(3) if t != a]
            ranges = [range(self.n[0] + (a == 0)), range(self.n[1] + (a == 1)), range(self.n[2] + (a == 2))]
            for l in ranges[2]:
                for k in ranges[1]:
                    for j in ranges[0]:
                        R = (j, k, l)
                        L = shift(R, a, -1)
                        fi = R[a]
                        xl, xr, xb = self.centre(a, fi - 1), self.centre(a, fi), self.f[a][fi]
                        wgt = (xb - xl) / (xr - xl)
                        PL, PR = P(L), P(R)
                        gts = {}
                        for t in tang:
                            if not self.per[a] and fi == 0:
                                gts[t] = grad(R, t)
                            elif not self.per[a] and fi == self.n[a]:
                                gts[t] = grad(L, t)
                            else:
                                gl, gr = grad(L, t), grad(R, t)
                                gts[t] = [(1 - wgt) * x + wgt * y for x, y in zip(gl, gr)]
                        fb = []
                        for i, e in enumerate(self.cvec):
                            gn = (PR[i] - PL[i]) / (xr - xl)
                            val = (1 - wgt) * PL[i] + wgt * PR[i]
                            cg = e[a] * c * gn + sum(e[t] * c * gts[t][i] for t in tang)
                            fb.append(val - h * cg)                                       # Eqs. 2.19, 2.26
                        pb = sum(fb)
                        eb = self.feq(pb)
                        fo = [(2 * lam * x + h * q) / (2 * lam + h) for x, q in zip(fb, eb)]  # Eq. 2.15 inverted
                        flux[(a, R)] = [e[a] * c * x for e, x in zip(self.cvec, fo)]
        out = {}
        for cell in ft:
            widths = [self.f[a][cell[a] + 1] - self.f[a][cell[a]] for a in range(3)]
            vol = widths[0] * widths[1] * widths[2]
            new = []
            for i in range(len(self.cvec)):
                J = Fr(0)
                for a in range(3):
                    area = vol / widths[a]
                    J += (flux[(a, shift(cell, a, 1))][i] - flux[(a, cell)][i]) * area
                new.append(ftp[cell][i] - dt / vol * J)                                   # Eq. 2.12
            out[cell] = new
        return out

    def to_array(self, ft):
        import numpy as np

        Q = len(self.cvec)
        a = np.zeros((Q, self.n[2], self.n[1], self.n[0]))
        for (j, k, l), v in ft.items():
            for i in range(Q):
                a[i, l, k, j] = float(v[i])
        return a
