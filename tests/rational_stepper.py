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

Optional extensions: a symmetric tensor D with polynomial entries (Eq. 2.3
contracted entry by entry), and a time-independent source F(x, phi) =
sum_k phi^p_k S_k(x) (rate 0 keeps the arithmetic rational), with
R_i = w_i c_i.B'(phi) F / c_s^2 (Remark 3), the interface evolution of
Eq. 2.18 (each of fbar^+, R, F reconstructed at the characteristic foot) and
the update of Eq. 2.12; the time derivatives are backward differences over
the previous step (none on the first step), and a ghost cell carries the
source distributions of the interior cell it mirrors.
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
    def __init__(self, xf, yf, bc, bc_value, c, u, b, alpha, d, c_zero, dt, d_tensor=None, source=()):
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
        self.dt3 = None if d_tensor is None else [[Fr(v) for v in e] for e in d_tensor]
        # source terms (power, field[k][j] as Fractions)
        self.src = [(int(pw), [[Fr(v) for v in row] for row in fld]) for pw, fld in source]
        self.hist = None  # R_i, F_i of the previous step per cell

    # Eq. 2.3 in expanded form: contraction of (cs2 d - cs2 phi) I + C uu with (c c - cs2 I)
    def feq(self, phi):
        cs2, c = self.cs2, self.c
        bv, dv, cv = _poly_eval(self.b, phi), _poly_eval(self.d, phi), _poly_eval(self.cint, phi)
        uu = self.u[0] ** 2 + self.u[1] ** 2
        out = []
        for (ex, ey), w in zip(CVEC, WEIGHT):
            cu = c * (ex * self.u[0] + ey * self.u[1])
            cc = c * c * (ex * ex + ey * ey)
            if self.dt3 is None:
                contraction = cs2 * (dv - phi) * (cc - 2 * cs2) + cv * (cu * cu - cs2 * uu)
            else:  # cs2 D:(c c - cs2 I) with D = [[xx, xy], [xy, yy]], then the -cs2 phi I part
                xx, xy, yy = (_poly_eval(e, phi) for e in self.dt3)
                cx, cy = c * ex, c * ey
                dd = xx * cx * cx + 2 * xy * cx * cy + yy * cy * cy - cs2 * (xx + yy)
                contraction = cs2 * dd - cs2 * phi * (cc - 2 * cs2) + cv * (cu * cu - cs2 * uu)
            out.append(w * (phi + cu * bv / cs2 + contraction / (2 * cs2 * cs2)))
        return out

    def sources(self, j, k, phi):
        """(R_i, F_i) at interior cell (j, k) (Eq. 2.3; R by Remark 3)."""
        F = sum(fld[k][j] * phi ** pw for pw, fld in self.src)
        dbv = _poly_eval(_poly_deriv(self.b), phi)
        R = [w * self.c * (ex * self.u[0] + ey * self.u[1]) * dbv * F / self.cs2 for (ex, ey), w in zip(CVEC, WEIGHT)]
        return R, [w * F for w in WEIGHT]

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

        # sources at t_n and their values S + h/2 dS/dt for Eq. 2.18, dS/dt = (S^n - S^{n-1}) / dt
        cur, sr, sf = {}, {}, {}
        if self.src:
            for k in range(ny):
                for j in range(nx):
                    R, F = self.sources(j, k, phi[(j, k)])
                    Rp, Fp = self.hist[(j, k)] if self.hist is not None else (R, F)
                    cur[(j, k)] = (R, F)
                    sr[(j, k)] = [a + h / 2 * (a - b) / dt for a, b in zip(R, Rp)]
                    sf[(j, k)] = [a + h / 2 * (a - b) / dt for a, b in zip(F, Fp)]

        def interior(j, k):
            """(ji, ki) of the interior cell behind extended cell (j, k), and whether (j, k) is a ghost."""
            if self.xper:
                j %= nx
            if self.yper:
                k %= ny
            if 0 <= j < nx and 0 <= k < ny:
                return j, k, False
            ji = min(max(j, 0), nx - 1)
            ki = min(max(k, 0), ny - 1)
            if (ji != j) and (ki != k):
                raise AssertionError("corner ghost requested")
            return ji, ki, True

        def SR(j, k):
            ji, ki, _ = interior(j, k)
            return sr[(ji, ki)]

        def SF(j, k):
            ji, ki, _ = interior(j, k)
            return sf[(ji, ki)]

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

        def gy(j, k, G=P):
            return [(a - b) / (self._centre_y(k + 1) - self._centre_y(k - 1))
                    for a, b in zip(G(j, k + 1), G(j, k - 1))]

        def gx(j, k, G=P):
            return [(a - b) / (self._centre_x(j + 1) - self._centre_x(j - 1))
                    for a, b in zip(G(j + 1, k), G(j - 1, k))]

        def xface_foot(G, jf, k):
            """G at the characteristic foot x_b - c_i h of x-face jf (Eqs. 2.19, 2.20), per velocity."""
            jl, jr = jf - 1, jf
            xl, xr, xb = self._centre_x(jl), self._centre_x(jr), self.xf[jf]
            Gl, Gr = G(jl, k), G(jr, k)
            w = (xb - xl) / (xr - xl)
            if not self.xper and jf == 0:
                gt = gy(jr, k, G)
            elif not self.xper and jf == nx:
                gt = gy(jl, k, G)
            else:
                gl, gr = gy(jl, k, G), gy(jr, k, G)
                gt = [(1 - w) * a + w * b for a, b in zip(gl, gr)]
            out = []
            for i, (ex, ey) in enumerate(CVEC):
                gn = (Gr[i] - Gl[i]) / (xr - xl)
                out.append((1 - w) * Gl[i] + w * Gr[i] - h * self.c * (ex * gn + ey * gt[i]))
            return out

        def yface_foot(G, j, kf):
            kl, kr = kf - 1, kf
            yl, yr, yb = self._centre_y(kl), self._centre_y(kr), self.yf[kf]
            Gl, Gr = G(j, kl), G(j, kr)
            w = (yb - yl) / (yr - yl)
            if not self.yper and kf == 0:
                gt = gx(j, kr, G)
            elif not self.yper and kf == ny:
                gt = gx(j, kl, G)
            else:
                gl, gr = gx(j, kl, G), gx(j, kr, G)
                gt = [(1 - w) * a + w * b for a, b in zip(gl, gr)]
            out = []
            for i, (ex, ey) in enumerate(CVEC):
                gn = (Gr[i] - Gl[i]) / (yr - yl)
                out.append((1 - w) * Gl[i] + w * Gr[i] - h * self.c * (ex * gt[i] + ey * gn))
            return out

        wr = 2 * lam * h / (2 * lam + h)  # weight of R in Eq. 2.18

        def add_sources(fb, foot, *where):
            if not self.src:
                return fb
            r, f = foot(SR, *where), foot(SF, *where)
            return [a + wr * b + h * q for a, b, q in zip(fb, r, f)]

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
                fluxx[(jf, k)] = face_f(add_sources(fb, xface_foot, jf, k))
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
                fluxy[(j, kf)] = face_f(add_sources(fb, yface_foot, j, kf))
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
                    v = ftp[(j, k)][i] - dt / (dx * dy) * J
                    if self.src:  # Eq. 2.12: dt (S + dt/2 dS/dt) for S = R_i, F_i
                        (R, F), (Rp, Fp) = cur[(j, k)], (self.hist[(j, k)] if self.hist is not None else cur[(j, k)])
                        v += dt * (R[i] + dt / 2 * (R[i] - Rp[i]) / dt) + dt * (F[i] + dt / 2 * (F[i] - Fp[i]) / dt)
                    cell.append(v)
                row.append(cell)
            out.append(row)
        if self.src:
            self.hist = cur
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
