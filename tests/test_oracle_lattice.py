"""Pins of the oracle's lattice, equilibrium, collision and boundary closure
against what the paper prints and what the mathematics fixes (no GPU)."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _read(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_velocity_classes_match_eq_d3q19(golden_dir):
    """Eq. (d3q19): index ranges and the sign patterns of their velocities."""
    for ln in _read(golden_dir, "eq_d3q19_velocity_classes.txt"):
        rng, pat = ln.split(":")
        a, b = (int(t) for t in rng.split())
        pat = pat.split()
        want = set()
        choices = [(-1, 1) if p == "s" else (0,) for p in pat]
        for v in itertools.product(*choices):
            want.add(v)
        got = {tuple(int(c) for c in O.XI[q]) for q in range(a, b + 1)}
        assert got == want, (ln, got)
    assert len({tuple(v) for v in O.XI}) == 19


def test_opposites_pair_up():
    for q in range(19):
        assert (O.XI[O.OPP[q]] == -O.XI[q]).all()
    # odd q pairs with q+1, as the paper's +- listing implies
    for q in range(1, 19, 2):
        assert O.OPP[q] == q + 1


def test_inlet_unknowns_are_the_xi_z_plus_one_set():
    """Section 2: at the z-inlet the unknowns are f5, f11, f14, f15, f18."""
    assert O.lbm_oracle.INLET_UNKNOWN == [5, 11, 14, 15, 18]


def test_appendix_b_momentum_rows(golden_dir):
    """Each printed Appendix B row holds identically for random f with our
    velocity order (this is what fixes the order of q = 7..18)."""
    rng = np.random.default_rng(1)
    f = rng.random((19, 50))
    rho, jx, jy, jz = O.moments(f)
    mom = {"rho": rho, "jx": jx, "jy": jy, "jz": jz}
    for ln in _read(golden_dir, "appendix_b_momentum_rows.txt"):
        _, rest = ln.split(":", 1)
        lhs, m, rhs = (p.strip() for p in rest.split(";"))
        L = sum(int(t[0] + "1") * f[abs(int(t))] for t in lhs.split())
        R = mom[m] - sum(int(t[0] + "1") * f[abs(int(t))] for t in rhs.split())
        np.testing.assert_allclose(L, R, rtol=0, atol=1e-13)


def test_eq_inlet_consistency(golden_dir):
    """Eq. (inlet): rho0 u_z = rho - K at any node, K as printed."""
    rng = np.random.default_rng(2)
    f = rng.random((19, 40))
    coef = dict(tuple(int(x) for x in t.split(":")) for t in _read(golden_dir, "eq_inlet_consistency.txt")[0].split())
    K = sum(c * f[q] for q, c in coef.items())
    rho, _, _, jz = O.moments(f)
    np.testing.assert_allclose(jz, rho - K, atol=1e-13)
    np.testing.assert_allclose(O.inlet_known_sum(f), K, atol=1e-13)


def test_weights_and_isotropy():
    """Textbook D3Q19 lattice tensors: sum w = 1, sum w xi = 0, sum w xi xi = c_s^2 I,
    sum w xi^4 = c_s^4 (dd + dd + dd), odd moments vanish."""
    W, X = O.W, O.XI.astype(float)
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W @ X, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", W, X, X), np.eye(3) / 3.0, atol=1e-16)
    T4 = np.einsum("q,qa,qb,qc,qd->abcd", W, X, X, X, X)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(T4, iso, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", W, X, X, X), 0.0, atol=1e-16)
    # Appendix B: f_q^eq - f_opp^eq = 6 rho0 w_q (xi_q . u) has coefficient 1/3 on the
    # axes and 1/6 on the diagonals
    assert np.allclose(6 * W[1:7], 1 / 3) and np.allclose(6 * W[7:], 1 / 6)


def test_equilibrium_moments():
    """sum f^eq = rho, sum f^eq xi = j, sum f^eq xi xi = c_s^2 rho I + j j / rho0."""
    rng = np.random.default_rng(3)
    rho = 1 + 0.1 * rng.standard_normal(30)
    j = 0.05 * rng.standard_normal((3, 30))
    f = O.equilibrium(rho, j[0], j[1], j[2])
    r, jx, jy, jz = O.moments(f)
    np.testing.assert_allclose(r, rho, atol=1e-14)
    np.testing.assert_allclose(np.stack([jx, jy, jz]), j, atol=1e-15)
    P = np.einsum("qn,qa,qb->abn", f, O.XI.astype(float), O.XI.astype(float))
    want = np.eye(3)[:, :, None] * rho / 3.0 + np.einsum("an,bn->abn", j, j)
    np.testing.assert_allclose(P, want, atol=1e-14)
    # the equilibrium at rest is the weight times rho
    np.testing.assert_allclose(O.equilibrium(np.array(2.0), 0.0, 0.0, 0.0), 2 * O.W)


def test_moment_matrix_orthogonal_and_conserved_rows():
    M = O.moment_matrix()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    np.testing.assert_array_equal(M[0], 1)
    np.testing.assert_array_equal(M[3], O.XI[:, 0])
    np.testing.assert_array_equal(M[5], O.XI[:, 1])
    np.testing.assert_array_equal(M[7], O.XI[:, 2])
    # every row is even or odd under xi -> -xi (parity-pure), which is what makes
    # the paper's rate choice a two-relaxation-time scheme
    for k in range(19):
        row_opp = M[k, O.OPP]
        assert np.array_equal(row_opp, M[k]) or np.array_equal(row_opp, -M[k])


def test_equilibrium_moments_match_dhumieres_and_appendix_a():
    """M f^eq equals the published d'Humieres et al. (2002) incompressible
    equilibria (w_eps = 3, w_epsj = -11/2, w_xx = -1/2); its stress rows equal
    the Appendix A forms (2jx^2 - jy^2 - jz^2, jy^2 - jz^2, jx jy, jy jz, jx jz)
    with the interfacial term set to zero."""
    rng = np.random.default_rng(4)
    rho = 1 + 0.1 * rng.standard_normal(20)
    jx, jy, jz = 0.05 * rng.standard_normal((3, 20))
    m = O.moment_matrix() @ O.equilibrium(rho, jx, jy, jz)
    j2 = jx * jx + jy * jy + jz * jz
    want = np.stack([
        rho, -11 * rho + 19 * j2, 3 * rho - 5.5 * j2,
        jx, -2 / 3 * jx, jy, -2 / 3 * jy, jz, -2 / 3 * jz,
        2 * jx * jx - jy * jy - jz * jz, -0.5 * (2 * jx * jx - jy * jy - jz * jz),
        jy * jy - jz * jz, -0.5 * (jy * jy - jz * jz),
        jx * jy, jy * jz, jx * jz, 0 * jx, 0 * jx, 0 * jx])
    np.testing.assert_allclose(m, want, atol=1e-14)


def _trt(F, s_plus, s_minus):
    rho, jx, jy, jz = O.moments(F)
    E = O.equilibrium(rho, jx, jy, jz)
    D = F - E
    Dp = 0.5 * (D + D[O.OPP])
    Dm = 0.5 * (D - D[O.OPP])
    return F - s_plus * Dp - s_minus * Dm


@pytest.mark.parametrize("tau", [0.55, 0.7, 1.0, 1.5, 3.0])
def test_mrt_conserves_and_equals_trt(tau):
    """Appendix A collision conserves rho and j; with s_e = s_eps = s_pi = s_nu and
    s_q = s_m it equals the two-relaxation-time form with s+ = s_nu, s- = s_q,
    i.e. magic parameter (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 for every tau."""
    rng = np.random.default_rng(5)
    F = O.equilibrium(1 + 0.01 * rng.standard_normal(64), *(0.02 * rng.standard_normal((3, 64))))
    F = F + 1e-3 * rng.standard_normal(F.shape)
    G = O.collide_mrt(F, tau)
    for a, b in zip(O.moments(F), O.moments(G)):
        np.testing.assert_allclose(a, b, atol=1e-15)
    s_nu = 1 / tau
    s_q = 8 * (2 - s_nu) / (8 - s_nu)
    np.testing.assert_allclose(G, _trt(F, s_nu, s_q), atol=2e-15)
    lam = (1 / s_nu - 0.5) * (1 / s_q - 0.5)
    assert abs(lam - 3 / 16) < 1e-14


def test_mrt_with_equal_rates_is_bgk():
    rng = np.random.default_rng(6)
    F = O.equilibrium(np.ones(10), *(0.03 * rng.standard_normal((3, 10)))) + 1e-3 * rng.standard_normal((19, 10))
    tau = 0.8
    np.testing.assert_allclose(O.collide_mrt(F, tau, s_q=1 / tau), O.collide_bgk(F, tau), atol=2e-15)


def test_equilibrium_is_collision_fixed_point():
    F = O.equilibrium(np.full(5, 1.02), 0.01, -0.02, 0.03)
    np.testing.assert_allclose(O.collide_mrt(F, 0.7), F, atol=1e-16)
    np.testing.assert_allclose(O.collide_bgk(F, 0.7), F, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stream_pull_matches_voxel_loops(seed):
    """Brute force: the vectorised pull equals a voxel-by-voxel loop."""
    from lbm_inputs import random_mask, uniform_field
    m = random_mask(5, 4, 6, 0.3, seed)
    f = uniform_field((19,) + m.shape, seed + 10, 0.0, 1.0)
    f[:, m.astype(bool)] = 0
    a = O.stream_pull(f, m)
    b = O.stream_pull_loops(f, m)
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(np.nan_to_num(a, nan=-7), np.nan_to_num(b, nan=-7))


def _frac(s):
    return float(Fraction(s))


def test_hh_closure_rows_and_moments(golden_dir):
    """After the inlet closure: the printed rows hold, sum f = rho, sum f xi_x =
    sum f xi_y = 0 and sum f xi_z = rho0 u_z with u_z from Eq. (inlet); the
    mirrored outlet closure gives sum f = rho_out with zero tangential momentum."""
    rng = np.random.default_rng(7)
    P = rng.random((19, 6, 5)) * 0.1
    rho = 1.03
    Q = P.copy()
    uz = O.hh_closure_inlet(Q, rho)
    Nx = 0.5 * (Q[1] + Q[7] + Q[9] - Q[2] - Q[10] - Q[8])
    Ny = 0.5 * (Q[3] + Q[7] + Q[10] - Q[4] - Q[9] - Q[8])
    for ln in _read(golden_dir, "appendix_b_hh_closure.txt"):
        t = ln.split()
        if t[0] in ("Nx", "Ny"):
            continue
        qu, qk, cux, cuy, cuz, cN, which = t
        N = Nx if which == "x" else Ny if which == "y" else 0.0
        np.testing.assert_allclose(Q[int(qu)] - Q[int(qk)], _frac(cuz) * uz + _frac(cN) * N, atol=1e-15)
    r, jx, jy, jz = O.moments(Q)
    np.testing.assert_allclose(r, rho, atol=1e-15)
    np.testing.assert_allclose(jx, 0, atol=1e-15)
    np.testing.assert_allclose(jy, 0, atol=1e-15)
    np.testing.assert_allclose(jz, uz, atol=1e-15)
    # known values untouched
    known = [q for q in range(19) if q not in (5, 11, 14, 15, 18)]
    np.testing.assert_array_equal(Q[known], P[known])

    R = P.copy()
    uo = O.hh_closure_outlet(R, 0.98)
    r, jx, jy, jz = O.moments(R)
    np.testing.assert_allclose(r, 0.98, atol=1e-15)
    np.testing.assert_allclose(jx, 0, atol=1e-15)
    np.testing.assert_allclose(jy, 0, atol=1e-15)
    np.testing.assert_allclose(jz, uo, atol=1e-15)
    known = [q for q in range(19) if q not in (6, 12, 13, 16, 17)]
    np.testing.assert_array_equal(R[known], P[known])


def test_flux_density_closed_form():
    """Eq. (potential) on a plane with uniform known sum K: rho = Q/A + K."""
    K = np.full((3, 4), 0.9)
    pore = np.ones((3, 4), bool)
    pore[0, 0] = False
    rho, A, S = O.flux_density(K, pore, 0.22)
    assert A == 11 and abs(rho - (0.22 / 11 + 0.9)) < 1e-15
