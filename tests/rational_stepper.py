"""Exact rational DUGKS stepper for tiny grids (a pin for the FP64 oracle).

Written independently of ``oracle/dugks_oracle.c`` from the paper's basic
definitions rather than its composite formulas: it carries the original
distribution f explicitly and moves between f, ftilde, fbar and fbar^+ with
Eqs. 2.11, 2.13, 2.15 (read with its missing f_i restored) and 2.17, where
the oracle uses the shortcuts Eqs. 2.21 and 2.22.  The equilibrium is written
in the expanded contraction form of Eq. 2.3, and the auxiliary moment C is
built by exact polynomial algebra.  Everything is ``fractions.Fraction``,
so the result is exact; the oracle must agree to FP64 rounding.

Shared readings (the same as the oracle's, since the paper is silent):
2-D reconstruction with a tangential slope interpolated between the two
cells' central differences, and the mirrored ghost with non-equilibrium
extrapolation at Dirichlet walls (interior cell's tangential slope at a wall
face).
"""
from fractions import Fraction as Fr

CVEC = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WEIGHT = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4


def _poly_eval(coef, x):
    acc = Fr(0)
    for a in reversed(coef):
        acc = acc * x + a
    return acc


def _poly_mul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_deriv(a):
    return [k * a[k] for k in range(1, len(a))] or [Fr(0)]


def _poly_integral(a):
    return [Fr(0)] + [a[k] / (k + 1) for k in range(len(a))]


class RationalDUGKS:
    def __init__(self, xf, yf, bc, bc_value, c, u, b, alpha, d, c_zero, dt):
        self.xf = [Fr(v) for v in xf]
        self.yf = [Fr(v) for v in yf]
        self.nx, self.ny = len(xf) - 1, len(yf) - 1
        self.bc = tuple(bc)
        self.bcv = [Fr(v) for v in bc_value]
        self.c = Fr(c)
        self.u = (Fr(u[0]), Fr(u[1]))
        self.b = [Fr(v) for v in b]
        self.d = [Fr(v) for v in d]
        db = _poly_deriv(self.b)
        self.cint = [Fr(0)] if c_zero else _poly_integral(_poly_mul(db, db))
        self.alpha = Fr(alpha)
        self.dt = Fr(dt)
        self.cs2 = self.c * self.c / 3
        self.lam = self.alpha / self.cs2
        self.h = self.dt / 2
        self.xper = bc[0] == 0
        self.yper = bc[2] == 0

    # Eq. 2.3 in expanded form: contraction of (cs2 d - cs2 phi) I + C uu with (c c - cs2 I)
    def feq(self, phi):
        cs2, c = self.cs2, self.c
        bv, dv, cv = _poly_eval(self.b, phi), _poly_eval(self.d, phi), _poly_eval(self.cint, phi)
        uu = self.u[0] ** 2 + self.u[1] ** 2
        out = []
        for (ex, ey), w in zip(CVEC, WEIGHT):
            cu = c * (ex * self.u[0] + ey * self.u[1])
            cc = c * c * (ex * ex + ey * ey)
            contraction = cs2 * (dv - phi) * (cc - 2 * cs2) + cv * (cu * cu - cs2 * uu)
            out.append(w * (phi + cu * bv / cs2 + contraction / (2 * cs2 * cs2)))
        return out

    def init(self, phi0):
        return [[self.feq(Fr(phi0[k][j])) for j in range(self.nx)] for k in range(self.ny)]

    def _centre_x(self, j):
        """Centre coordinate of extended column j (-1..nx)."""
        if 0 <= j < self.nx:
            return (self.xf[j] + self.xf[j + 1]) / 2
        L = self.xf[-1] - self.xf[0]
        if self.xper:
            return self._centre_x(j % self.nx) + (L if j >= self.nx else -L)
        wall = self.xf[0] if j < 0 else self.xf[-1]
        inner = self._centre_x(0 if j < 0 else self.nx - 1)
        return 2 * wall - inner

    def _centre_y(self, k):
        if 0 <= k < self.ny:
            return (self.yf[k] + self.yf[k + 1]) / 2
        L = self.yf[-1] - self.yf[0]
        if self.yper:
            return self._centre_y(k % self.ny) + (L if k >= self.ny else -L)
        wall = self.yf[0] if k < 0 else self.yf[-1]
        inner = self._centre_y(0 if k < 0 else self.ny - 1)
        return 2 * wall - inner

    def step(self, ft):
        nx, ny, lam, dt, h = self.nx, self.ny, self.lam, self.dt, self.h
        phi, feq, fbp, ftp = {}, {}, {}, {}
        for k in range(ny):
            for j in range(nx):
                p = sum(ft[k][j])
                e = self.feq(p)
                # Eq. 2.11 inverted: f = (2 lam ft + dt feq) / (2 lam + dt)
                f = [(2 * lam * a + dt * q) / (2 * lam + dt) for a, q in zip(ft[k][j], e)]
                # Eq. 2.15 (restored): fbar = (2lam+h)/(2lam) f - h/(2lam) feq ; Eq. 2.17: fbar^+
                fbar = [(2 * lam + h) / (2 * lam) * a - h / (2 * lam) * q for a, q in zip(f, e)]
                fbp[(j, k)] = [(2 * lam - h) / (2 * lam + h) * a + 2 * h / (2 * lam + h) * q
                               for a, q in zip(fbar, e)]
                # Eq. 2.13
                ftp[(j, k)] = [(2 * lam - dt) / (2 * lam + dt) * a + 2 * dt / (2 * lam + dt) * q
                               for a, q in zip(ft[k][j], e)]
                phi[(j, k)], feq[(j, k)] = p, e

        def P(j, k):
            """fbar^+ at extended cell (j, k): interior, periodic image or NEE ghost."""
            if self.xper:
                j %= nx
            if self.yper:
                k %= ny
            if (j, k) in fbp:
                return fbp[(j, k)]
            if j < 0 or j >= nx:
                ji, wall = (0, self.bcv[0]) if j < 0 else (nx - 1, self.bcv[1])
                ki = k
            else:
                ki, wall = (0, self.bcv[2]) if k < 0 else (ny - 1, self.bcv[3])
                ji = j
            if not (0 <= ki < ny and 0 <= ji < nx):
                raise AssertionError("corner ghost requested")
            pg = 2 * wall - phi[(ji, ki)]
            eg = self.feq(pg)
            return [g + (a - q) for g, a, q in zip(eg, fbp[(ji, ki)], feq[(ji, ki)])]

        def face_f(fbar_b):
            pb = sum(fbar_b)
            eb = self.feq(pb)
            # Eq. 2.15 inverted at the face: f = (2 lam fbar + h feq) / (2 lam + h)
            return [(2 * lam * a + h * q) / (2 * lam + h) for a, q in zip(fbar_b, eb)]

        def gy(j, k):
            return [(a - b) / (self._centre_y(k + 1) - self._centre_y(k - 1))
                    for a, b in zip(P(j, k + 1), P(j, k - 1))]

        def gx(j, k):
            return [(a - b) / (self._centre_x(j + 1) - self._centre_x(j - 1))
                    for a, b in zip(P(j + 1, k), P(j - 1, k))]

        fluxx, fluxy = {}, {}
        for k in range(ny):
            for jf in range(nx + 1):          # face between columns jf-1 and jf
                jl, jr = jf - 1, jf
                xl, xr, xb = self._centre_x(jl), self._centre_x(jr), self.xf[jf]
                Pl, Pr = P(jl, k), P(jr, k)
                w = (xb - xl) / (xr - xl)
                if not self.xper and jf == 0:
                    gt = gy(jr, k)
                elif not self.xper and jf == nx:
                    gt = gy(jl, k)
                else:
                    gl, gr = gy(jl, k), gy(jr, k)
                    gt = [(1 - w) * a + w * b for a, b in zip(gl, gr)]
                fb = []
                for i, (ex, ey) in enumerate(CVEC):
                    # linear interpolation of value and normal slope at x_b, then the
                    # characteristic foot x_b - c_i h (Eq. 2.19, Eq. 2.26)
                    gn = (Pr[i] - Pl[i]) / (xr - xl)
                    val = (1 - w) * Pl[i] + w * Pr[i]
                    fb.append(val - h * self.c * (ex * gn + ey * gt[i]))
                fluxx[(jf, k)] = face_f(fb)
        for kf in range(ny + 1):
            for j in range(nx):
                kl, kr = kf - 1, kf
                yl, yr, yb = self._centre_y(kl), self._centre_y(kr), self.yf[kf]
                Pl, Pr = P(j, kl), P(j, kr)
                w = (yb - yl) / (yr - yl)
                if not self.yper and kf == 0:
                    gt = gx(j, kr)
                elif not self.yper and kf == ny:
                    gt = gx(j, kl)
                else:
                    gl, gr = gx(j, kl), gx(j, kr)
                    gt = [(1 - w) * a + w * b for a, b in zip(gl, gr)]
                fb = []
                for i, (ex, ey) in enumerate(CVEC):
                    gn = (Pr[i] - Pl[i]) / (yr - yl)
                    val = (1 - w) * Pl[i] + w * Pr[i]
                    fb.append(val - h * self.c * (ex * gt[i] + ey * gn))
                fluxy[(j, kf)] = face_f(fb)
        out = []
        for k in range(ny):
            row = []
            for j in range(nx):
                dx = self.xf[j + 1] - self.xf[j]
                dy = self.yf[k + 1] - self.yf[k]
                cell = []
                for i, (ex, ey) in enumerate(CVEC):
                    # Eq. 2.12: flux through the four faces, outward normals
                    J = (ex * self.c * (fluxx[(j + 1, k)][i] - fluxx[(j, k)][i]) * dy
                         + ey * self.c * (fluxy[(j, k + 1)][i] - fluxy[(j, k)][i]) * dx)
                    cell.append(ftp[(j, k)][i] - dt / (dx * dy) * J)
                row.append(cell)
            out.append(row)
        return out

    @staticmethod
    def to_array(ft):
        import numpy as np
        ny, nx = len(ft), len(ft[0])
        a = np.zeros((9, ny, nx))
        for k in range(ny):
            for j in range(nx):
                for i in range(9):
                    a[i, k, j] = float(ft[k][j][i])
        return a
