"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each check reaches the oracle's result by a route other than the oracle's own
formula: textbook polynomial definitions of the moments, lattice isotropy,
closed-form limits, algebraic identities, values printed in the paper, a
population-space restatement of the special case the paper names, and
closed-form flows.  A plausible slip in the oracle (a dropped term, a wrong
sign or index, a transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, cell_api, default_config
from paper_2304_04214_gb300.inputs import noise, stg_uniforms

Q = 19
CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lattice():
    M, w, c = cell_api.matrix()
    return M, w, c


# --------------------------------------------------------------------------
# Velocity set, weights and moment matrix (Sec. 2.1, Appendix A.1)
# --------------------------------------------------------------------------
def test_velocity_set_and_weight_isotropy(lattice):
    M, w, c = lattice
    # closed under inversion: c_{18-i} = -c_i
    assert np.array_equal(c[::-1], -c)
    assert abs(w.sum() - 1.0) < 1e-15
    # second and fourth isotropic moments of a D3Q19 lattice
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, CS2 * np.eye(3), atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(fourth, iso, atol=1e-15)
    # odd moments vanish
    assert np.allclose(np.einsum("i,ia->a", w, c), 0)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0)


def test_moment_matrix_rows_are_the_textbook_polynomials(lattice):
    """Each row of M equals its d'Humieres (2002) polynomial of c_i."""
    M, w, c = lattice
    cx, cy, cz = c[:, 0].astype(float), c[:, 1].astype(float), c[:, 2].astype(float)
    c2 = cx * cx + cy * cy + cz * cz
    rows = [
        np.ones(Q),
        19 * c2 - 30,
        (21 * c2 * c2 - 53 * c2 + 24) / 2,
        cx, (5 * c2 - 9) * cx,
        cy, (5 * c2 - 9) * cy,
        cz, (5 * c2 - 9) * cz,
        3 * cx * cx - c2, (3 * c2 - 5) * (3 * cx * cx - c2),
        cy * cy - cz * cz, (3 * c2 - 5) * (cy * cy - cz * cz),
        cx * cy, cy * cz, cx * cz,
        (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz,
    ]
    assert np.array_equal(M, np.array(rows))


def test_moment_matrix_orthogonal(lattice):
    M, _, _ = lattice
    G = M @ M.T
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert np.array_equal(G, np.diag(norms).astype(float))


def test_equilibrium_moments_match_printed_forms():
    """M f^eq against eq:mom_eq; rows 2, 4, 6, 8 against the reading A1/A2."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.08 * rng.standard_normal(3)
        ux, uy, uz = u
        uu = u @ u
        m = cell_api.moments(cell_api.feq(rho, u))
        printed = {
            0: rho, 1: -11 * rho + 19 * rho * uu, 3: rho * ux, 5: rho * uy, 7: rho * uz,
            9: 2 * rho * ux ** 2 - rho * uy ** 2 - rho * uz ** 2,
            10: -rho * ux ** 2 + 0.5 * rho * uy ** 2 + 0.5 * rho * uz ** 2,
            11: rho * uy ** 2 - rho * uz ** 2, 12: -0.5 * rho * uy ** 2 + 0.5 * rho * uz ** 2,
            13: rho * ux * uy, 14: rho * uy * uz, 15: rho * ux * uz, 16: 0.0, 17: 0.0, 18: 0.0,
        }
        for k, v in printed.items():
            assert abs(m[k] - v) < 1e-14, (k, m[k], v)
        # garbled rows: the reading is d'Humieres' 3 rho - 11/2 rho u^2 and -2/3 rho u
        assert abs(m[2] - (3 * rho - 5.5 * rho * uu)) < 1e-14
        for k, a in ((4, 0), (6, 1), (8, 2)):
            assert abs(m[k] - (-2.0 / 3.0) * rho * u[a]) < 1e-15


# --------------------------------------------------------------------------
# Collision (eq:lbe_mrt, eq:bodyforce, Sec. 2.2)
# --------------------------------------------------------------------------
def _random_pops(rng, rho=1.0, u=(0.04, -0.01, 0.02), eps=0.02):
    fe = cell_api.feq(rho, np.array(u))
    return fe * (1.0 + eps * rng.uniform(-1, 1, Q))


def test_equilibrium_is_a_fixed_point():
    for tau0 in (0.5001, 0.8, 1.3):
        for cs in (0.0, 0.01):
            fe = cell_api.feq(1.03, np.array([0.05, -0.02, 0.01]))
            out, rho, u = cell_api.collide(fe, tau0=tau0, c_smag=cs)
            assert np.max(np.abs(out - fe)) < 1e-15


def test_collision_conserves_mass_and_adds_the_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = _random_pops(rng)
        F = 1e-4 * rng.standard_normal(3)
        _, _, c = cell_api.matrix()
        out, rho, u = cell_api.collide(p, F=F, tau0=0.51 + rng.random(), c_smag=0.01)
        assert abs(out.sum() - p.sum()) < 1e-15
        assert np.allclose(out @ c, p @ c + F, atol=1e-16, rtol=0)
        # eq:momentum: u = (sum f c + F/2) / rho
        assert np.allclose(u, (p @ c + 0.5 * F) / p.sum(), atol=1e-16, rtol=0)


def test_single_rate_mrt_is_bgk_with_guo_force():
    """Sec. 2.1: with every omega_i equal the MRT operator is BGK, and the force
    term must be eq:bodyforce with that omega, written here in population space."""
    rng = np.random.default_rng(11)
    _, w, c = cell_api.matrix()
    for _ in range(20):
        p = _random_pops(rng)
        F = 1e-4 * rng.standard_normal(3)
        tau = 0.5 + rng.random()
        out, rho, u = cell_api.collide(p, F=F, tau0=tau, c_smag=0.0, mrt=False)
        rho_ref = p.sum()
        u_ref = (p @ c + 0.5 * F) / rho_ref
        cu = c @ u_ref
        fe = w * rho_ref * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u_ref @ u_ref) / (2 * CS2))
        Fi = (1 - 0.5 / tau) * w * (((c - u_ref) / CS2 + (cu / CS2 ** 2)[:, None] * c) @ F)
        ref = p - (p - fe) / tau + Fi
        assert np.max(np.abs(out - ref)) < 2e-16


def test_viscous_moments_relax_at_tau_eff():
    """Sec. 2.2: tau_eff replaces only the viscosity-related rates."""
    rng = np.random.default_rng(5)
    M, w, c = cell_api.matrix()
    p = _random_pops(rng, eps=0.05)
    tau0, cs = 0.52, 0.01
    out, rho, u = cell_api.collide(p, tau0=tau0, c_smag=cs)
    fe = cell_api.feq(rho, u)
    pineq = np.einsum("ia,ib,i->ab", c, c, p - fe)
    te = cell_api.tau_eff(tau0, cs, rho, [pineq[0, 0], pineq[1, 1], pineq[2, 2],
                                          pineq[0, 1], pineq[1, 2], pineq[0, 2]])
    assert te > tau0
    m, me, ms = M @ p, M @ fe, M @ out
    for k in (9, 11, 13, 14, 15):
        assert abs((ms[k] - me[k]) - (1 - 1 / te) * (m[k] - me[k])) < 1e-16
    for k, s in ((1, 1.19), (2, 1.6), (4, 1.2), (6, 1.2), (8, 1.2), (10, 1.6), (12, 1.6),
                 (16, 1.98), (17, 1.98), (18, 1.98)):
        assert abs((ms[k] - me[k]) - (1 - s) * (m[k] - me[k])) < 1e-14, k


def test_smagorinsky_tau_eff_identity():
    """eq:tau_eff (reading A6) solves nu_eff = nu0 + C |S| with Pi_neq = -2 rho cs^2 tau_eff S."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        A = 1e-3 * rng.standard_normal((3, 3))
        Pi = A + A.T
        rho = 1.0 + 0.02 * rng.standard_normal()
        tau0 = 0.5 + 0.2 * rng.random()
        C = 0.01 * (1 + rng.random())
        te = cell_api.tau_eff(tau0, C, rho, [Pi[0, 0], Pi[1, 1], Pi[2, 2], Pi[0, 1], Pi[1, 2], Pi[0, 2]])
        S = -Pi / (2 * rho * CS2 * te)
        Snorm = math.sqrt(2 * np.sum(S * S))
        assert abs(CS2 * (te - 0.5) - (CS2 * (tau0 - 0.5) + C * Snorm)) < 1e-15
        assert cell_api.tau_eff(tau0, 0.0, rho, [Pi[0, 0], Pi[1, 1], Pi[2, 2], Pi[0, 1],
                                                 Pi[1, 2], Pi[0, 2]]) == pytest.approx(tau0, abs=1e-16)


# --------------------------------------------------------------------------
# Wall law (Sec. 2.3)
# --------------------------------------------------------------------------
def test_reichardt_limits():
    # viscous sublayer: u+ -> y+ as y+ -> 0
    for y in (1e-6, 1e-4):
        assert abs(cell_api.reichardt(y) / y - 1.0) < 1e-3 * y / 1e-4 + 1e-5
    # log layer: u+ - (ln y+ / kappa + B + ln(kappa)/kappa) -> 0
    for kap, B in ((0.4, 7.8), (0.41, 7.1)):
        y = 1e7
        ref = math.log(y) / kap + B + math.log(kap) / kap
        assert abs(cell_api.reichardt(y, kap, B) - ref) < 1e-5


def test_reichardt_matches_printed_law_where_it_holds():
    """eq:reichard as printed agrees with the reading at the paper's first-cell y+."""
    for y in (50.0, 86.7, 100.0, 130.0, 260.0, 1000.0):
        printed = 2.5 * math.log(1 + 0.4 * y) + 7.8 * (1 - math.exp(-y / 11)) - y * math.exp(-y / 3)
        assert abs(cell_api.reichardt(y) - printed) < 1e-6 * printed


def test_newton_round_trip():
    nu = 4e-5
    for ut in (1e-3, 2.46e-3, 5e-3):
        for kap, B in ((0.4, 7.8), (0.38, 8.2)):
            uhat = ut * cell_api.reichardt(0.5 * ut / nu, kap, B)
            got = cell_api.solve_utau(uhat, 0.5, nu, kap, B, guess=3 * ut)
            assert abs(got - ut) < 1e-13 * ut


def test_first_cell_yplus_matches_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "first_cell_yplus.txt"))
            if l.strip() and not l.startswith("#")]
    for re_tau, H, yp in rows:
        re_tau, H, yp = float(re_tau), int(H), float(yp)
        cfg = default_config(4, H, 2, re_tau=re_tau, n_modes=0, inlet=0)
        o = Oracle(cfg)
        k = o.constants()
        y1p = 0.5 * k["utau_ref"] / k["nu"]
        assert abs(y1p - yp) <= 0.05 * 1.0 + 1e-3 * yp, (re_tau, H, y1p, yp)


# --------------------------------------------------------------------------
# Inlet (Sec. 3.1)
# --------------------------------------------------------------------------
def _neq_from_pi(w, c, Pi):
    Qi = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    return w / (2 * CS2 ** 2) * np.einsum("iab,ab->i", Qi, Pi), Qi


def test_regularized_projection_identity(lattice):
    """eq:f_i_neq with the 1/2 (reading A14): sum_i Q_i f_i^neq gives Pi back."""
    M, w, c = lattice
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 3))
    Pi = A + A.T
    fneq, Qi = _neq_from_pi(w, c, Pi)
    assert np.allclose(np.einsum("iab,i->ab", Qi, fneq), Pi, atol=1e-14)
    assert abs(fneq.sum()) < 1e-14
    assert np.allclose(fneq @ c, 0, atol=1e-14)


def test_inlet_reconstruction_is_idempotent_and_uses_known_populations(lattice):
    M, w, c = lattice
    rng = np.random.default_rng(9)
    for _ in range(10):
        rho = 1.0 + 0.02 * rng.standard_normal()
        u = np.array([0.05, 0.0, 0.0]) + 0.005 * rng.standard_normal(3)
        A = 1e-4 * rng.standard_normal((3, 3))
        fneq, _ = _neq_from_pi(w, c, A + A.T)
        p = cell_api.feq(rho, u) + fneq
        out, rho_in = cell_api.inlet(p, u)
        assert abs(rho_in - rho) < 1e-14
        assert np.max(np.abs(out - p)) < 1e-15
        # populations entering the domain (c_x > 0) are unknown and must not matter
        q = p.copy()
        q[c[:, 0] > 0] += rng.uniform(-0.1, 0.1, (c[:, 0] > 0).sum())
        out2, rho2 = cell_api.inlet(q, u)
        assert np.array_equal(out2, out) and rho2 == rho_in


def test_zou_he_density_at_rest(lattice):
    """Reading A13: the fluid at rest with f = w must give rho_in = 1 (the
    printed (2 rho_perp + rho_par)/(1 + u) would give 1.5)."""
    M, w, c = lattice
    out, rho = cell_api.inlet(w.copy(), [0.0, 0.0, 0.0])
    assert abs(rho - 1.0) < 1e-15 and np.allclose(out, w, atol=1e-16)


# --------------------------------------------------------------------------
# STG tables and statistics (Sec. 3.1, eq:cholesky, eq:aux_vec; reading A16)
# --------------------------------------------------------------------------
def _stg(ny=48, nz=16, N=100, seed=1, theta=(0.4, 1.0, 0.4, 7.8), re_tau=1000.0):
    cfg = default_config(3, ny, nz, re_tau=re_tau, n_modes=N)
    return Oracle(cfg, theta=theta, uniforms=stg_uniforms(N, seed))


def test_stg_tables_structure():
    o = _stg(theta=(0.4, 1.7, 0.4, 7.8))
    t = o.tables()
    k = o.constants()
    # eq:cholesky: a a^T = A^2 R with R = R+ u_tau^2
    for j in range(o.ny):
        a11, a21, a22, a31, a32, a33 = t["a"][j]
        L = np.array([[a11, 0, 0], [a21, a22, 0], [a31, a32, a33]])
        r = t["Rp"][j] * k["utau_ref"] ** 2
        R = np.array([[r[0], r[3], r[4]], [r[3], r[1], r[5]], [r[4], r[5], r[2]]])
        assert np.allclose(L @ L.T, 1.7 ** 2 * R, rtol=1e-13, atol=1e-20)
    # normalized spectrum weights, unit mode vectors, sigma . d = 0
    assert np.allclose((t["sqrtq"] ** 2).sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(np.linalg.norm(t["dn"], axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.linalg.norm(t["sn"], axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.einsum("na,na->n", t["dn"], t["sn"]), 0.0, atol=1e-14)
    assert np.all((t["phin"] >= 0) & (t["phin"] < 2 * math.pi))
    assert np.allclose(t["kn"][1:] / t["kn"][:-1], 1.01, rtol=1e-13)


def test_stg_length_scale_limits():
    """Reading A16 (iii): the energetic length scale is a smooth stand-in for
    min(2 d_w, l_e delta): it follows twice the wall distance at the wall
    (within 0.2% at the first cell) and saturates at l_e delta in the core
    (within 0.1%), growing monotonically in between, and is symmetric about
    the centre line."""
    ny, le = 96, 0.4
    o = _stg(ny=ny, N=16, theta=(le, 1.0, 0.4, 7.8))
    ell = o.tables()["ell"]
    delta = ny / 2
    y = np.arange(ny) + 0.5
    d = np.minimum(y, ny - y)
    assert abs(ell[0] / (2 * d[0]) - 1.0) < 2e-3
    assert abs(ell[ny // 2] / (le * delta) - 1.0) < 1e-3
    assert np.all(np.diff(ell[: ny // 2]) > 0)
    assert np.allclose(ell, ell[::-1], rtol=0, atol=1e-12)
    assert np.all(ell <= np.minimum(2 * d, le * delta) * (1 + 1e-12))


def test_stg_spectrum_has_no_energy_past_the_kolmogorov_scale():
    """Reading A16 (ii): the Kolmogorov factor removes the modes finer than
    the dissipation scale.  At Re_tau = 100 on 96 cells the Kolmogorov
    wavenumber k_eta = 2 pi (eps / nu^3)^(1/4), eps = u_tau^3 / (kappa d_w),
    falls inside the resolved range in the core; the modes with
    k_eta / 3 < k < 0.9 pi (below the grid cut-off) carry less than 1e-6 of
    the energy there, where the bare von Karman shape puts over 1%."""
    ny = 96
    o = _stg(ny=ny, N=400, re_tau=100.0)
    t, c = o.tables(), o.constants()
    k = t["kn"]
    j = 40
    d = j + 0.5
    keta = 2 * math.pi * (c["utau_ref"] ** 3 / (0.4 * d) / c["nu"] ** 3) ** 0.25
    fine = (k > keta / 3) & (k < 0.9 * math.pi)     # resolved, before the grid cut-off
    assert fine.sum() > 20
    assert (t["sqrtq"][j, fine] ** 2).sum() < 1e-6
    # the von Karman shape alone puts a visible share there
    ke = 2 * math.pi / t["ell"][j]
    r = k / ke
    vk = r ** 4 / (1 + 2.4 * r * r) ** (17 / 6) * k
    assert vk[fine].sum() / vk[k < 0.9 * math.pi].sum() > 0.01


def test_stg_inlet_signal_has_the_convective_frequencies():
    """Reading A16 (iv): the modes are frozen patterns convected through the
    inlet plane, x'_n = (x - U_b t) 2 pi / (k_n max l_e), so at x = 0 mode n
    oscillates in time at f_n = |d_n,x| U_b / max l_e cycles per step,
    whatever its wavenumber.  With three modes the velocity at one cell is a
    constant plus three tones: a least-squares fit on those frequencies
    leaves no residual (a missing U_b, a wrong time scale or a wrong
    component of d_n would)."""
    ny, nz, N, T = 32, 4, 3, 6000
    o = _stg(ny=ny, nz=nz, N=N)
    t, c = o.tables(), o.constants()
    f = np.abs(t["dn"][:, 0]) * 0.05 / c["maxl"]
    assert np.all(f * T > 10)                 # many periods in the record
    x = np.array([o.inlet_velocity(s)[1, 9, 0] for s in range(T)])
    ts = np.arange(T)
    basis = np.concatenate([np.ones((T, 1))] +
                           [np.stack([np.cos(2 * math.pi * fn * ts), np.sin(2 * math.pi * fn * ts)], 1)
                            for fn in f], axis=1)
    x = x - x.mean()
    coef, *_ = np.linalg.lstsq(basis, x, rcond=None)
    resid = x - basis @ coef
    assert np.sum(resid ** 2) < 1e-20 * np.sum(x ** 2)


def test_stg_spectrum_shape():
    """Modified von Karman spectrum: E ~ k^4 well below k_e, ~ k^(-5/3) well
    above it (before the cut-offs), peak at k = k_e."""
    o = _stg(ny=96, N=400, re_tau=1000.0)
    t = o.tables()
    k = t["kn"]
    j = 40                                   # a cell well away from the wall
    E = t["sqrtq"][j] ** 2 / k               # q_n / dk_n, dk_n proportional to k_n
    ke = 2 * math.pi / t["ell"][j]
    lo = k < 0.2 * ke
    if lo.sum() >= 3:
        slope = np.polyfit(np.log(k[lo]), np.log(E[lo]), 1)[0]
        assert abs(slope - 4.0) < 0.25
    hi = (k > 5 * ke) & (k < 0.5 * math.pi)
    if hi.sum() >= 3:
        slope = np.polyfit(np.log(k[hi]), np.log(E[hi]), 1)[0]
        assert abs(slope + 5.0 / 3.0) < 0.25
    # peak at k_e (the damping factors are ~1 there)
    kpk = k[np.argmax(E)]
    assert abs(math.log(kpk / ke)) < 0.05
    # the cut-off exp(-(4 (k - 0.9 k_cut)/k_cut)^3) removes modes beyond the grid
    # limit k_cut = pi: below 1e-30 of the total for k > 2 k_cut
    assert np.all(t["sqrtq"][:, k > 2.0 * math.pi] ** 2 < 1e-30)


@pytest.mark.slow
def test_stg_reproduces_prescribed_reynolds_stress():
    """Over independent mode draws, <u'> = 0 and <u' u'^T> = A^2 R within
    sampling error (Sec. 3.1: sum q_n = 1 and sigma_n . d_n = 0 make
    <v' v'^T> = I)."""
    ny, nz, N, nseed = 24, 8, 100, 400
    A = 1.0
    samples = []
    for s in range(nseed):
        o = _stg(ny=ny, nz=nz, N=N, seed=1000 + s, theta=(0.4, A, 0.4, 7.8), re_tau=1000.0)
        uin = o.inlet_velocity(t=37 * s)
        samples.append(uin[s % nz] - np.c_[o.tables()["UR"], np.zeros((ny, 2))])
        k = o.constants()
        Rp = o.tables()["Rp"]
    X = np.array(samples)                   # (nseed, ny, 3)
    u2 = k["utau_ref"] ** 2
    for j in (2, 6, 11, 17, 21):
        R = np.array([[Rp[j, 0], Rp[j, 3], Rp[j, 4]], [Rp[j, 3], Rp[j, 1], Rp[j, 5]],
                      [Rp[j, 4], Rp[j, 5], Rp[j, 2]]]) * u2 * A * A
        x = X[:, j, :]
        mean = x.mean(axis=0)
        cov = x.T @ x / nseed
        for a in range(3):
            assert abs(mean[a]) < 5 * math.sqrt(R[a, a] / nseed)
            for b in range(3):
                sd = math.sqrt((R[a, a] * R[b, b] + R[a, b] ** 2) / nseed)
                assert abs(cov[a, b] - R[a, b]) < 5 * sd, (j, a, b, cov[a, b], R[a, b])


# --------------------------------------------------------------------------
# Closed-form flows and conservation over whole lattices
# --------------------------------------------------------------------------
def _poiseuille(ny, tau, steps, Fx=1e-6):
    cfg = default_config(2, ny, 2, n_modes=0, inlet=0, walls=1, wall_model=0, c_smag=0.0,
                         tau0=tau, body_force=(Fx, 0.0, 0.0))
    o = Oracle(cfg)
    f = o.state()
    _, w, _ = cell_api.matrix()
    o.set_state(np.broadcast_to(w[:, None, None, None], f.shape).copy())
    o.step(steps)
    rho, u = o.fields()
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    exact = Fx / (2 * nu) * y * (ny - y)
    return u[0, :, 0, 0], exact, rho


def test_poiseuille_closed_form():
    """Laminar channel under a body force with halfway bounce-back walls (test
    only): u(y) = F y (H - y) / (2 rho nu); second-order in the resolution."""
    errs = []
    for ny in (8, 16):
        tau = 0.8
        nu = (tau - 0.5) / 3.0
        steps = int(6 * ny * ny / nu)
        ux, exact, rho = _poiseuille(ny, tau, steps)
        errs.append(np.max(np.abs(ux - exact)) / exact.max())
        assert np.allclose(rho, 1.0, atol=1e-12)
    assert errs[1] < 0.02
    assert 3.0 < errs[0] / errs[1] < 5.0       # second order


def test_mass_and_momentum_conservation_periodic():
    cfg = default_config(8, 6, 5, n_modes=0, inlet=0, walls=2, wall_model=0, c_smag=0.01)
    o = Oracle(cfg)
    f0 = o.state() * (1.0 + 0.05 * noise((Q, 5, 6, 8), seed=3))
    o.set_state(f0)
    _, _, c = cell_api.matrix()
    m0 = f0.sum()
    j0 = np.einsum("qkji,qa->a", f0, c)
    o.step(10)
    f = o.state()
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.allclose(np.einsum("qkji,qa->a", f, c), j0, atol=1e-13)
    # a uniform body force adds F per cell per step
    cfg2 = default_config(8, 6, 5, n_modes=0, inlet=0, walls=2, wall_model=0, c_smag=0.01,
                          body_force=(1e-5, -2e-5, 3e-5))
    o2 = Oracle(cfg2)
    o2.set_state(f0)
    o2.step(4)
    f = o2.state()
    assert np.allclose(np.einsum("qkji,qa->a", f, c),
                       j0 + 4 * 8 * 6 * 5 * np.array([1e-5, -2e-5, 3e-5]), atol=1e-13)


def test_streaming_moves_the_mass_centroid_by_the_momentum():
    """Streaming carries each post-collision population f*_q from x to x + c_q,
    and the collision keeps every cell's mass and momentum when F = 0, so one
    step moves the first moment of mass, sum_x x rho(x), by exactly the total
    momentum sum_x sum_q c_q f_q.  Checked on a localized disturbance of the
    rest state in a periodic box (away from the wrap), along all three axes:
    a pull from the wrong side, or a velocity read with a wrong sign,
    reverses or scrambles the shift."""
    nx, ny, nz = 12, 10, 8
    cfg = default_config(nx, ny, nz, n_modes=0, inlet=0, walls=2, wall_model=0, c_smag=0.01)
    o = Oracle(cfg)
    _, w, c = cell_api.matrix()
    f0 = np.broadcast_to(w[:, None, None, None], (Q, nz, ny, nx)).copy()
    blob = (slice(None), slice(2, 6), slice(3, 7), slice(4, 8))
    f0[blob] *= 1.0 + 0.2 * noise((Q, 4, 4, 4), seed=11)
    o.set_state(f0)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = (ii, jj, kk)

    def centroid(f):
        rho = f.sum(axis=0)
        return np.array([(p * rho).sum() for p in pos])

    j0 = np.einsum("qkji,qa->a", f0, c)
    assert np.min(np.abs(j0)) > 1e-3                   # a shift along every axis
    x0 = centroid(f0)
    o.step(1)
    x1 = centroid(o.state())
    assert np.allclose(x1 - x0, j0, rtol=0, atol=1e-11), (x1 - x0, j0)


def test_outlet_is_transparent_to_a_streamwise_uniform_flow():
    """Reading A18: the zero-gradient outlet continues the field past x = nx-1
    as if it did not change along x.  So a state uniform in x (any y, z
    dependence) must evolve in the inlet/outlet channel exactly as in a
    periodic one wherever the inlet's disturbance has not arrived: after n
    steps on every column i > n, the outlet column included.  Checked with
    the slip walls, the wall model and the SGS closure on."""
    nx, ny, nz, n = 16, 8, 6, 5
    _, w, c = cell_api.matrix()
    base = w[:, None, None] * (1.0 + 0.05 * noise((Q, nz, ny), seed=12))
    f0 = np.broadcast_to(base[..., None], (Q, nz, ny, nx)).copy()
    runs = []
    for inlet in (1, 0):
        cfg = default_config(nx, ny, nz, n_modes=8, inlet=inlet, walls=0, wall_model=1, c_smag=0.01)
        o = Oracle(cfg, theta=(0.4, 1.0, 0.4, 7.8), uniforms=stg_uniforms(8, 2))
        o.set_state(f0)
        o.step(n)
        runs.append(o.state())
    a, b = runs
    assert np.max(np.abs(a[..., n + 1:] - b[..., n + 1:])) < 1e-15
    assert np.max(np.abs(a[..., 0] - b[..., 0])) > 1e-6      # the inlet did act


def test_slip_walls_conserve_mass_and_tangential_momentum():
    cfg = default_config(8, 6, 5, n_modes=0, inlet=0, walls=0, wall_model=0, c_smag=0.01)
    o = Oracle(cfg)
    f0 = o.state() * (1.0 + 0.05 * noise((Q, 5, 6, 8), seed=4))
    o.set_state(f0)
    _, _, c = cell_api.matrix()
    j0 = np.einsum("qkji,qa->a", f0, c)
    o.step(10)
    f = o.state()
    assert abs(f.sum() - f0.sum()) < 1e-12 * f0.sum()
    j = np.einsum("qkji,qa->a", f, c)
    assert abs(j[0] - j0[0]) < 1e-13 and abs(j[2] - j0[2]) < 1e-13


def test_wall_force_opposes_the_flow_with_reichardt_stress():
    cfg = default_config(16, 16, 8, n_modes=0)
    o = Oracle(cfg)
    o.step(1)
    F = o.force()
    rho, u = o.fields()
    k = o.constants()
    ut = o.utau()
    # both walls: force along -x, magnitude rho u_tau^2, u_tau solving the law
    assert np.all(F[:, 0, :, 0] < 0) and np.all(F[:, -1, :, 0] < 0)
    assert np.allclose(np.abs(F[:, 1:-1, :, :]), 0.0)
    _, _, c = cell_api.matrix()
    # u_tau of the bottom wall solves u_tau u+(u_tau/(2 nu)) = u_hat;
    # rebuild the first-layer velocity from the state after the step: rho u0 = rho u - F/2
    u0 = u[:, 0, :, 0] - 0.5 * F[:, 0, :, 0] / rho[:, 0, :]
    res = ut[0] * np.array([[cell_api.reichardt(0.5 * x / k["nu"]) for x in row] for row in ut[0]]) - u0
    assert np.max(np.abs(res)) < 1e-14
    assert np.allclose(-F[:, 0, :, 0], rho[:, 0, :] * ut[0] ** 2, rtol=1e-13)


def test_wall_force_follows_the_tangential_velocity_of_the_second_cell():
    """Sec. 2.3 with readings A9-A11 on a disturbed state (rho != 1 and a
    wall-normal velocity at the second cell): the force on a first-layer cell
    is -rho_w u_tau^2 e_x, e_x the unit vector of the second cell's velocity
    with its wall-normal part removed, u_tau solving the wall law for the
    first-layer velocity projected on e_x, the force's sign following that
    projection (reading A10).  The bottom first layer starts mirrored in x, so
    there it flows against the second cell and the projection turns negative.
    Everything is rebuilt from the fields the step collided with
    (rho u0 = rho u - F/2)."""
    nx, ny, nz = 8, 12, 6
    _, _, c = cell_api.matrix()
    o = Oracle(default_config(nx, ny, nz, n_modes=0))
    f0 = o.state() * (1.0 + 0.03 * noise((Q, nz, ny, nx), seed=13))
    mirror = [int(np.nonzero((c == c[q] * np.array([-1, 1, 1])).all(axis=1))[0][0]) for q in range(Q)]
    f0[:, :, 0, :] = f0[mirror, :, 0, :]
    o.set_state(f0)
    o.step(1)
    F = o.force()
    rho, u = o.fields()
    nu = o.constants()["nu"]
    ut = o.utau()
    for w, (jw, j2) in enumerate(((0, 1), (ny - 1, ny - 2))):
        u2 = u[:, j2, :, :].copy()
        assert np.max(np.abs(u2[..., 1])) > 1e-4         # a wall-normal part to remove
        u2[..., 1] = 0.0
        ex = u2 / np.linalg.norm(u2, axis=-1, keepdims=True)
        rw = rho[:, jw, :]
        assert np.max(np.abs(rw - 1.0)) > 1e-3
        u0 = u[:, jw, :, :] - 0.5 * F[:, jw, :, :] / rw[..., None]
        uhat = np.einsum("kia,kia->ki", u0, ex)
        assert (uhat < 0).mean() > 0.5 if w == 0 else (uhat > 0).all()
        t = ut[w]
        law = t * np.vectorize(cell_api.reichardt)(0.5 * t / nu)
        assert np.max(np.abs(law - np.abs(uhat))) < 1e-14
        expect = -(rw * t * t * np.sign(uhat))[..., None] * ex
        assert np.max(np.abs(F[:, jw, :, :] - expect)) < 1e-15


def test_statistics_and_objective_are_window_means_of_the_collided_fields():
    """The FP64 statistics are z-sums of (u, v, w, uu, vv, ww, uv) per (y, x)
    and of u_tau per (wall, x), one sample per step; the adjoint objective is
    J = J_tau + J_R with J_tau the mean of tau_w / u_tau,ref^2 = rho_w u_tau^2 /
    u_tau,ref^2 over the window and the wall cells i0 <= i < i1 of both walls,
    and J_R = sum_j (<u'v'>(iR, j) / u_tau,ref^2 - R12+(j))^2 with the
    prescribed R12+ of reading A16 (vi), negative in the lower half.  All of
    it is rebuilt here from the per-step fields, with R12+ from its closed
    form."""
    nx, ny, nz, N, T = 16, 12, 6, 12, 5
    i0, i1, iR = 3, 9, 7
    re_tau = 1000.0
    o = Oracle(default_config(nx, ny, nz, n_modes=N, re_tau=re_tau, stats=1),
               theta=(0.4, 1.0, 0.4, 7.8), uniforms=stg_uniforms(N, 3))
    o.step(3)
    o.stats_reset()
    o.objective_begin(i0, i1, iR)
    ur2 = o.constants()["utau_ref"] ** 2
    sums = np.zeros((ny, nx, 7))
    ut_sums = np.zeros((2, nx))
    jt, su, sv, suv = 0.0, np.zeros(ny), np.zeros(ny), np.zeros(ny)
    for _ in range(T):
        o.step(1)
        rho, u = o.fields()
        ut = o.utau()
        uu, vv, ww = u[..., 0], u[..., 1], u[..., 2]
        for a, q in enumerate((uu, vv, ww, uu * uu, vv * vv, ww * ww, uu * vv)):
            sums[..., a] += q.sum(axis=0)
        ut_sums += ut.sum(axis=1)
        jt += (rho[:, 0, i0:i1] * ut[0][:, i0:i1] ** 2).sum() + (rho[:, -1, i0:i1] * ut[1][:, i0:i1] ** 2).sum()
        su += uu[:, :, iR].sum(axis=0)
        sv += vv[:, :, iR].sum(axis=0)
        suv += (uu * vv)[:, :, iR].sum(axis=0)
    s, uts, n = o.stats()
    assert n == T
    assert np.allclose(s, sums, rtol=1e-14, atol=1e-17)
    assert np.allclose(uts, ut_sums, rtol=1e-14, atol=1e-17)
    delta = ny / 2
    y = np.arange(ny) + 0.5
    d = np.minimum(y, ny - y)
    sh = (1 - d / delta) * (1 - np.exp(-d * re_tau / delta / 26.0)) ** 2
    r12 = np.where(y < delta, -sh, sh)
    cnt = T * nz
    J_tau = jt / (T * 2 * (i1 - i0) * nz) / ur2
    J_R = (((suv / cnt - su / cnt * sv / cnt) / ur2 - r12) ** 2).sum()
    _, _, parts = o.objective()
    assert abs(parts[0] - J_tau) < 1e-12 * J_tau
    assert abs(parts[1] - J_R) < 1e-12 * J_R


# --------------------------------------------------------------------------
# Complex-step derivatives agree with central differences
# --------------------------------------------------------------------------
def test_complex_step_gradient_matches_central_differences():
    nx, ny, nz, N = 12, 8, 4, 16
    un = stg_uniforms(N, 5)
    theta = np.array([0.4, 1.0, 0.4, 7.8])
    cfg = default_config(nx, ny, nz, n_modes=N, re_tau=1000.0)

    def J(th, im=None):
        o = Oracle(cfg, theta=th, uniforms=un, complex_step=im is not None, theta_im=im)
        o.objective_begin(4, 8, 6)
        o.step(4)
        return o.objective()

    h = 1e-20
    for kk in range(4):
        e = np.zeros(4)
        e[kk] = 1.0
        _, jim, _ = J(theta, h * theta[kk] * e)
        cs = jim / (h * theta[kk])
        d = 1e-5 * theta[kk]
        jp = J(theta + d * e)[0]
        jm = J(theta - d * e)[0]
        fd = (jp - jm) / (2 * d)
        scale = max(abs(cs), 1e-8)
        assert abs(cs - fd) < 1e-6 * scale + 1e-12, (kk, cs, fd)


def test_outlet_sponge_raises_the_local_viscosity_by_its_ramp():
    """Reading A24: over the last L cells the viscosity rises by nu_s r^2.
    A shear wave u_y = U sin(k z) in a periodic box decays, column by column,
    at the local rate (nu + nu_s r(x)^2) k^2 -- checked between steps 5 and
    20 (after the start-up from equilibrium) within 3%, inside and outside
    the sponge, except the three columns on each side of the periodic wrap,
    where the sponge's most viscous end meets its start and viscous diffusion
    along x mixes their rates."""
    from oracle.oracle import Oracle, cell_api, default_config
    nx, ny, nz, L, nu_s, tau0 = 32, 4, 32, 16, 0.1, 0.8
    cfg = default_config(nx, ny, nz, n_modes=0, inlet=0, walls=2, wall_model=0, c_smag=0.0, tau0=tau0,
                         sponge_cells=L, sponge_nu=nu_s)
    o = Oracle(cfg, theta=(0.4, 1.0, 0.4, 7.8), uniforms=None)
    _, w, c = cell_api.matrix()
    k = 2 * np.pi / nz
    z = np.arange(nz) + 0.5
    uy = 1e-3 * np.sin(k * z)                         # (nz,)
    cu = c[:, 1][:, None] * uy[None, :]               # (Q, nz)
    feq = w[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uy[None, :] ** 2)
    f0 = np.broadcast_to(feq[:, :, None, None], (19, nz, ny, nx)).copy()
    o.set_state(f0)
    amp = []
    for n in (5, 15):
        o.step(n)
        _, u = o.fields()
        amp.append(np.abs((u[..., 1] * np.sin(k * z)[:, None, None]).sum(axis=(0, 1))))   # per x
    rate = -np.log(amp[1] / amp[0]) / 15
    xc = np.arange(nx) + 0.5
    ramp = np.clip((xc - (nx - L)) / L, 0, 1)
    expect = ((tau0 - 0.5) / 3 + nu_s * ramp ** 2) * k * k
    err = (rate / expect - 1)[3:nx - 3]
    assert np.max(np.abs(err)) < 0.03, np.round(err, 4)
    # the rate inside the sponge differs from outside by what the ramp adds
    assert rate[nx - 4] / rate[nx // 4] > 1.5
