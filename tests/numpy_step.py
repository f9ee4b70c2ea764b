"""A second, independent FP64 statement of one time step of the STG
wall-modelled MRT-LES lattice Boltzmann channel, in plain NumPy with explicit
loops over the cells, for brute-force comparison with the C oracle on tiny
lattices.  It is written from the paper's equations and the readings of its
silent or garbled passages, and shares nothing with the oracle or the CUDA
library: the matrix M is typed from Appendix A.1 row by row, its inverse is
numpy.linalg.inv(M), and every boundary rule is a separate pass in the order
of Algorithm 1 (stream, outlet copy, inlet, wall model, collide).

TEST INFRASTRUCTURE ONLY.
"""
import math

import numpy as np

Q = 19
# Sec. 2.1, eq:vel-set
C = np.array([(0, -1, -1), (-1, 0, -1), (0, 0, -1), (1, 0, -1), (0, 1, -1), (-1, -1, 0),
              (0, -1, 0), (1, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (-1, 1, 0), (0, 1, 0),
              (1, 1, 0), (0, -1, 1), (-1, 0, 1), (0, 0, 1), (1, 0, 1), (0, 1, 1)], dtype=np.int64)
# Sec. 2.1: w_9 = 1/3; 2, 6, 8, 10, 12, 16: 1/18; the rest 1/36
W = np.full(Q, 1.0 / 36.0)
W[9] = 1.0 / 3.0
W[[2, 6, 8, 10, 12, 16]] = 1.0 / 18.0
# Appendix A.1
M = np.array([
    [1] * 19,
    [8, 8, -11, 8, 8, 8, -11, 8, -11, -30, -11, 8, -11, 8, 8, 8, -11, 8, 8],
    [1, 1, -4, 1, 1, 1, -4, 1, -4, 12, -4, 1, -4, 1, 1, 1, -4, 1, 1],
    [0, -1, 0, 1, 0, -1, 0, 1, -1, 0, 1, -1, 0, 1, 0, -1, 0, 1, 0],
    [0, -1, 0, 1, 0, -1, 0, 1, 4, 0, -4, -1, 0, 1, 0, -1, 0, 1, 0],
    [-1, 0, 0, 0, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1, -1, 0, 0, 0, 1],
    [-1, 0, 0, 0, 1, -1, 4, -1, 0, 0, 0, 1, -4, 1, -1, 0, 0, 0, 1],
    [-1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1],
    [-1, -1, 4, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -4, 1, 1],
    [-2, 1, -1, 1, -2, 1, -1, 1, 2, 0, 2, 1, -1, 1, -2, 1, -1, 1, -2],
    [-2, 1, 2, 1, -2, 1, 2, 1, -4, 0, -4, 1, 2, 1, -2, 1, 2, 1, -2],
    [0, -1, -1, -1, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1, 0, -1, -1, -1, 0],
    [0, -1, 2, -1, 0, 1, -2, 1, 0, 0, 0, 1, -2, 1, 0, -1, 2, -1, 0],
    [0, 0, 0, 0, 0, 1, 0, -1, 0, 0, 0, -1, 0, 1, 0, 0, 0, 0, 0],
    [1, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 0, 0, 1],
    [0, 1, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 1, 0],
    [0, 1, 0, -1, 0, -1, 0, 1, 0, 0, 0, -1, 0, 1, 0, 1, 0, -1, 0],
    [-1, 0, 0, 0, 1, 1, 0, 1, 0, 0, 0, -1, 0, -1, -1, 0, 0, 0, 1],
    [1, -1, 0, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 1, 0, 1, -1]], dtype=np.float64)
MINV = np.linalg.inv(M)
CS2 = 1.0 / 3.0
# eq:freeparams (reading: moments 0, 3, 5, 7 at 1.0, omega_1 = 1.19); the
# viscous moments 9, 11, 13, 14, 15 relax with 1 / tau_eff (NaN placeholders)
RATES = np.array([1.0, 1.19, 1.6, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, np.nan,
                  1.6, np.nan, 1.6, np.nan, np.nan, np.nan, 1.98, 1.98, 1.98])
VISCOUS = [9, 11, 13, 14, 15]
OPP = [int(np.flatnonzero((C == -C[q]).all(axis=1))[0]) for q in range(Q)]
MIRROR_Y = [int(np.flatnonzero((C == C[q] * np.array([1, -1, 1])).all(axis=1))[0]) for q in range(Q)]


def f_eq(rho, u):
    """eq:bc_eq."""
    cu = C @ u
    return W * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - (u @ u) / (2 * CS2))


def u_plus(yp, kappa, B):
    """Sec. 2.3 eq:reichard with the textbook coefficients (1/kappa, kappa, B)."""
    return math.log(1.0 + kappa * yp) / kappa + B * (1.0 - math.exp(-yp / 11.0) - yp / 11.0 * math.exp(-yp / 3.0))


class Channel:
    """nx x ny x nz channel; state f[q, k, j, i] post-collision."""

    def __init__(self, nx, ny, nz, re_tau, uniforms, u_b=0.05, c_smag=0.01, kappa=0.4, B=7.8, ell_e=0.4,
                 amp=1.0, k_ratio=1.01, beta=0.5):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.c_smag, self.kappa, self.B = c_smag, kappa, B
        self.u_b = u_b
        delta = ny / 2.0
        self.delta = delta
        d = np.array([min(j + 0.5, ny - j - 0.5) for j in range(ny)])   # first cell centre at 1/2
        self.d = d
        # flow constants: U_b+ the mean of u+ over the cell centres
        ubp = np.mean([u_plus(dj * re_tau / delta, kappa, B) for dj in d])
        self.u_tau = u_b / ubp
        self.nu = self.u_tau * delta / re_tau
        self.tau0 = 3.0 * self.nu + 0.5          # eq:nu
        ut, nu = self.u_tau, self.nu
        # inlet mean profile and prescribed Reynolds stress, a = amp chol(R) (eq:cholesky)
        self.U = np.array([ut * u_plus(dj * ut / nu, kappa, B) for dj in d])
        self.a = np.zeros((ny, 3, 3))
        for j in range(ny):
            dp = d[j] * ut / nu
            s = (1.0 - d[j] / delta) * (1.0 - math.exp(-dp / 26.0)) ** 2
            R = np.diag([3 * s + 0.1, s + 0.1, 2 * s + 0.1]) * ut * ut
            R[0, 1] = R[1, 0] = (-s if j + 0.5 < delta else s) * ut * ut
            self.a[j] = amp * np.linalg.cholesky(R)
        # STG modes
        ell = ell_e * delta * np.tanh(2.0 * d / (ell_e * delta))
        self.maxl = ell.max()
        N = len(uniforms)
        kmin = beta * 2 * math.pi / self.maxl
        self.k = kmin * k_ratio ** np.arange(N)
        self.dn = np.zeros((N, 3))
        self.sn = np.zeros((N, 3))
        self.phi = np.zeros(N)
        for n, (u0, u1, u2, u3) in enumerate(uniforms):
            ct = 1.0 - 2.0 * u0
            st = math.sqrt(max(0.0, 1.0 - ct * ct))
            az, ang = 2 * math.pi * u1, 2 * math.pi * u2
            self.dn[n] = (st * math.cos(az), st * math.sin(az), ct)
            e1 = np.array([ct * math.cos(az), ct * math.sin(az), -st])
            e2 = np.array([-math.sin(az), math.cos(az), 0.0])
            self.sn[n] = math.cos(ang) * e1 + math.sin(ang) * e2
            self.phi[n] = 2 * math.pi * u3
        # modified von Karman spectrum per row, q_n = E(k_n) dk_n normalized
        self.sq = np.zeros((ny, N))
        kcut = 2 * math.pi / 2.0
        for j in range(ny):
            ke = 2 * math.pi / ell[j]
            eps = ut ** 3 / (0.4 * d[j])
            keta = 2 * math.pi * (eps / nu ** 3) ** 0.25
            E = np.zeros(N)
            for n in range(N):
                kk = self.k[n]
                r = kk / ke
                fcut = math.exp(-(4.0 * max(kk - 0.9 * kcut, 0.0) / kcut) ** 3)
                E[n] = r ** 4 / (1 + 2.4 * r * r) ** (17.0 / 6.0) * math.exp(-(12 * kk / keta) ** 2) * fcut \
                    * kk * (k_ratio - 1.0)
            self.sq[j] = np.sqrt(E / E.sum())
        self.t = 0
        self.f = np.zeros((Q, nz, ny, nx))
        for j in range(ny):
            self.f[:, :, j, :] = f_eq(1.0, np.array([self.U[j], 0.0, 0.0]))[:, None, None]
        self.utau = np.full((2, nz, nx), ut)
        self.F = np.zeros((nz, ny, nx, 3))

    def inlet_velocity(self, j, k, t):
        """eq:u_couple, eq:v_fluc, eq:aux_vec at the inlet cell (0, j, k)."""
        y, z = j + 0.5, k + 0.5
        v = np.zeros(3)
        for n in range(len(self.k)):
            # x' = (x - U_b t) 2 pi / (k_n max l_e) at x = 0
            xp = -self.u_b * t * 2 * math.pi / (self.k[n] * self.maxl)
            arg = self.k[n] * (self.dn[n, 0] * xp + self.dn[n, 1] * y + self.dn[n, 2] * z) + self.phi[n]
            v += self.sq[j, n] * self.sn[n] * math.cos(arg)
        return np.array([self.U[j], 0.0, 0.0]) + self.a[j] @ (math.sqrt(6.0) * v)

    def step(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        f = self.f
        p = np.zeros_like(f)
        # 1. pull streaming: z periodic, specular slip walls, x faces unknown
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    for q in range(Q):
                        si, sj, sk, sq = i - C[q, 0], j - C[q, 1], (k - C[q, 2]) % nz, q
                        if sj < 0 or sj >= ny:
                            sj, sq = j, MIRROR_Y[q]
                        if 0 <= si < nx:
                            p[q, k, j, i] = f[sq, sk, sj, si]
        # 2. zero-gradient outlet: unknown populations of x = nx-1 from x = nx-2
        for q in range(Q):
            if C[q, 0] < 0:
                p[q, :, :, nx - 1] = p[q, :, :, nx - 2]
        # 3. inlet (Algorithm 1 steps 4-7)
        for k in range(nz):
            for j in range(ny):
                pc = p[:, k, j, 0].copy()
                uin = self.inlet_velocity(j, k, self.t)
                rho = (sum(pc[q] for q in range(Q) if C[q, 0] == 0)
                       + 2 * sum(pc[q] for q in range(Q) if C[q, 0] < 0)) / (1.0 - uin[0])
                feq = f_eq(rho, uin)
                fneq = np.zeros(Q)
                for q in range(Q):
                    if C[q, 0] <= 0:
                        fneq[q] = pc[q] - feq[q]
                for q in range(Q):
                    if C[q, 0] > 0:
                        fneq[q] = fneq[OPP[q]]
                Pi = np.zeros((3, 3))
                for q in range(Q):
                    Pi += (np.outer(C[q], C[q]) - CS2 * np.eye(3)) * fneq[q]
                for q in range(Q):
                    Qq = np.outer(C[q], C[q]) - CS2 * np.eye(3)
                    p[q, k, j, 0] = feq[q] + W[q] / (2 * CS2 * CS2) * np.sum(Qq * Pi)
        # 4. wall model on the first off-wall cells (steps 9-14)
        F = np.zeros((nz, ny, nx, 3))
        for w, (jw, j2, n) in enumerate(((0, 1, np.array([0.0, 1.0, 0.0])),
                                          (ny - 1, ny - 2, np.array([0.0, -1.0, 0.0])))):
            for k in range(nz):
                for i in range(nx):
                    pw, p2 = p[:, k, jw, i], p[:, k, j2, i]
                    rw, r2 = pw.sum(), p2.sum()
                    uw, u2 = (pw @ C) / rw, (p2 @ C) / r2
                    tv = u2 - (u2 @ n) * n
                    tn = math.sqrt(tv @ tv)
                    if tn < 1e-12:
                        continue
                    ex = tv / tn
                    uh = uw @ ex
                    target = abs(uh)
                    u = self.utau[w, k, i]
                    for _ in range(100):
                        yp = 0.5 * u / self.nu
                        r = u * u_plus(yp, self.kappa, self.B) - target
                        h = 1e-7 * u
                        r2_ = (u + h) * u_plus(0.5 * (u + h) / self.nu, self.kappa, self.B) - target
                        r1_ = (u - h) * u_plus(0.5 * (u - h) / self.nu, self.kappa, self.B) - target
                        du = r / ((r2_ - r1_) / (2 * h))
                        u = u - du
                        if abs(du) < 1e-15 * u:
                            break
                    self.utau[w, k, i] = u
                    F[k, jw, i] = -rw * u * u * ex * (1.0 if uh >= 0 else -1.0)
        # 5. MRT-LES collision with the moment-space Guo force (step 15)
        out = np.zeros_like(f)
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    pc = p[:, k, j, i]
                    Fc = F[k, j, i]
                    rho = pc.sum()
                    u = (pc @ C + 0.5 * Fc) / rho
                    feq = f_eq(rho, u)
                    Pi = np.einsum("q,qa,qb->ab", pc - feq, C, C)
                    Qh = math.sqrt(np.sum(Pi * Pi))
                    tau_eff = 0.5 * (self.tau0 + math.sqrt(self.tau0 ** 2
                                                           + 18 * math.sqrt(2) * self.c_smag * Qh / rho))
                    S = RATES.copy()
                    S[VISCOUS] = 1.0 / tau_eff
                    Ft = np.array([W[q] * ((C[q] - u) / CS2 + (C[q] @ u) * C[q] / CS2 ** 2) @ Fc
                                   for q in range(Q)])
                    m, meq = M @ pc, M @ feq
                    mstar = m - S * (m - meq) + (1.0 - S / 2.0) * (M @ Ft)
                    out[:, k, j, i] = MINV @ mstar
        self.f = out
        self.F = F
        self.t += 1
