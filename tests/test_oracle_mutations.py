"""Plant plausible mistakes in the oracle (on the CPU) and check that the
independent pins catch each one. A pin that a wrong oracle also passes would
be worthless; these tests show that the pins are sharp enough."""
import numpy as np
import pytest

from oracle import dwf, force, gamma, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.brute import dwf_dense, wilson_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)
DIMS = (4, 2, 2, 4)


def _wilson_brute_error():
    U = gauge_field(DIMS, "haar", 301)
    psi = gaussian_spinor(DIMS, 302)
    D = wilson_dense(U, DIMS, 0.2, BC_AP)
    out = wilson.dirac(U, psi, 0.2, BC_AP)
    return np.abs(out.reshape(-1) - D @ psi.reshape(-1)).max()


def test_unmutated_oracle_passes():
    assert _wilson_brute_error() < 1e-12


@pytest.mark.parametrize("mutation", ["swap_projectors", "drop_conj", "bc_forward_only",
                                      "link_not_shifted", "gamma_sign"])
def test_wilson_mutations_are_caught(monkeypatch, mutation):
    if mutation == "swap_projectors":
        monkeypatch.setattr(wilson, "one_minus_gamma", gamma.one_plus_gamma)
    elif mutation == "drop_conj":
        monkeypatch.setattr(wilson, "colour_apply_dag",
                            lambda u, f: np.einsum("...ba,...sb->...sa", u, f))
    elif mutation == "bc_forward_only":
        orig = wilson.shift
        monkeypatch.setattr(wilson, "shift",
                            lambda f, mu, sign, bc: orig(f, mu, sign, bc if sign > 0 else (1, 1, 1, 1)))
    elif mutation == "link_not_shifted":
        monkeypatch.setattr(wilson.np, "roll", _roll_no_links(np.roll))
    elif mutation == "gamma_sign":
        g = gamma.GAMMA.copy()
        g[2] = -g[2]
        monkeypatch.setattr(gamma, "GAMMA", g)
        monkeypatch.setattr(wilson, "one_minus_gamma", lambda mu: gamma.ID4 - g[mu])
        monkeypatch.setattr(wilson, "one_plus_gamma", lambda mu: gamma.ID4 + g[mu])
    assert _wilson_brute_error() > 1e-3


def _roll_no_links(orig_roll):
    def roll(a, shift, axis=None):
        if a.ndim >= 6 and a.shape[-1] == 3 and a.shape[-2] == 3 and shift == 1:
            return a  # the link array: forget to take U(x - mu)
        return orig_roll(a, shift, axis=axis)
    return roll


def test_dwf_chirality_swap_is_caught(monkeypatch):
    dims, Ls = (2, 2, 2, 4), 4
    U = gauge_field(dims, "haar", 303)
    psi = gaussian_spinor(dims, 304, lead=(Ls,))
    D = dwf_dense(U, dims, Ls, 1.8, 0.02, BC_AP)
    good = dwf.dirac(U, psi, 1.8, 0.02, BC_AP)
    assert np.abs(good.reshape(-1) - D @ psi.reshape(-1)).max() < 1e-12
    monkeypatch.setattr(dwf, "P_MINUS", gamma.P_PLUS)
    monkeypatch.setattr(dwf, "P_PLUS", gamma.P_MINUS)
    bad = dwf.dirac(U, psi, 1.8, 0.02, BC_AP)
    assert np.abs(bad.reshape(-1) - D @ psi.reshape(-1)).max() > 1e-3


@pytest.mark.parametrize("mutation", ["sign", "no_phase", "transpose"])
def test_force_mutations_are_caught(monkeypatch, mutation):
    """A wrong force formula fails the finite-difference pin."""
    dims = (2, 2, 2, 4)
    m = 0.05
    U = gauge_field(dims, "haar", 305)
    phi = gaussian_spinor(dims, 306)
    if mutation == "transpose":
        orig_outer = force._outer_spin_sum
        monkeypatch.setattr(force, "_outer_spin_sum", lambda a, b: np.swapaxes(orig_outer(a, b), -1, -2))
    X, _ = force.solve_normal(U, phi, m, BC_AP, tol=1e-14)
    Y = wilson.dirac(U, X, m, BC_AP)
    if mutation == "no_phase":
        orig = wilson.shift
        monkeypatch.setattr(force.wilson, "shift", lambda f, mu, s, bc: orig(f, mu, s, (1, 1, 1, 1)))
    _, F = force.force_terms(U, X, Y, BC_AP)
    if mutation == "sign":
        F = -F
    rng = np.random.default_rng(307)
    from synthetic import random_su3_algebra
    T = random_su3_algebra(rng, U.size // 9).reshape(U.shape)
    analytic = np.einsum("...ab,...ba->...", T, F).sum().real
    D0 = wilson_dense
    eps = 1e-5

    def S(u):
        D = D0(u, dims, m, BC_AP)
        return np.vdot(phi.reshape(-1), np.linalg.solve(D.conj().T @ D, phi.reshape(-1))).real

    def ex(h, e):
        w, v = np.linalg.eigh(h)
        return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * e * w), v.conj())

    fd = (S(ex(T, eps) @ U) - S(ex(T, -eps) @ U)) / (2 * eps)
    assert abs(fd - analytic) > 1e-3 * abs(fd)


def _gauge_fd_error(g_module):
    from synthetic import make_rng, random_su3_algebra
    dims = (2, 4, 2, 4)
    U = gauge_field(dims, "exp", 1504, eps=0.5)
    T = random_su3_algebra(make_rng(1505), U.size // 9).reshape(U.shape)
    analytic = np.einsum("...ij,...ji->...", T, g_module.force(U, 5.6)).real.sum()
    h = 1e-5
    fd = (g_module.action(g_module.update_links(U, T, h), 5.6) -
          g_module.action(g_module.update_links(U, T, -h), 5.6)) / (2 * h)
    return abs(fd - analytic) / abs(fd)


@pytest.mark.parametrize("mutation", ["lower_staple_unshifted", "staple_dagger", "force_sign", "half_coupling"])
def test_gauge_force_mutations_are_caught(monkeypatch, mutation):
    from oracle import gauge
    assert _gauge_fd_error(gauge) < 1e-6
    if mutation == "lower_staple_unshifted":
        monkeypatch.setattr(gauge, "_bwd", lambda f, mu: f)
    elif mutation == "staple_dagger":
        orig = gauge.staple
        monkeypatch.setattr(gauge, "staple", lambda U, mu: gauge.dag(orig(U, mu)))
    elif mutation == "force_sign":
        orig = gauge.force
        monkeypatch.setattr(gauge, "force", lambda U, beta: -orig(U, beta))
    elif mutation == "half_coupling":
        orig = gauge.force
        monkeypatch.setattr(gauge, "force", lambda U, beta: orig(U, beta / 2))
    assert _gauge_fd_error(gauge) > 1e-3


def _gparity_doubled_error(gp):
    dims, bc, mu_g = (2, 4, 2, 4), (1.0, 1.0, 1.0, -1.0), 1
    U = gauge_field(dims, "haar", 1801)
    psi2 = gaussian_spinor(dims, 1802, lead=(2,))
    out = gp.dirac(U, psi2, 0.1, bc, (mu_g,))
    ax = 3 - mu_g
    ref = wilson.dirac(np.concatenate([U, np.conj(U)], axis=ax), np.concatenate([psi2[0], psi2[1]], axis=ax), 0.1,
                       (1.0, -1.0, 1.0, -1.0))
    return np.abs(np.concatenate([out[0], out[1]], axis=ax) - ref).max()


@pytest.mark.parametrize("mutation", ["twist_sign", "backward_link_owner", "no_conjugate_links"])
def test_gparity_mutations_are_caught(monkeypatch, mutation):
    from oracle import gparity
    assert _gparity_doubled_error(gparity) < 1e-12
    if mutation == "twist_sign":
        orig = gparity._neighbour

        def flipped(psi2, mu, sign, bc, twisted):
            out = orig(psi2, mu, sign, bc, twisted)
            if twisted:
                ax = wilson.site_axis(mu)
                edge = [slice(None)] * psi2.ndim
                edge[psi2.ndim + ax] = psi2.shape[ax] - 1 if sign > 0 else 0
                out[tuple(edge)] *= -1
            return out
        monkeypatch.setattr(gparity, "_neighbour", flipped)
    elif mutation == "backward_link_owner":
        orig = gparity._backward_links
        monkeypatch.setattr(gparity, "_backward_links", lambda U, mu, twisted: orig(U, mu, False))
    elif mutation == "no_conjugate_links":
        monkeypatch.setattr(gparity, "_flavour_links", lambda u: np.stack([u, u]))
    assert _gparity_doubled_error(gparity) > 1e-3


def _galerkin_error(mg_mod):
    from tests.test_oracle_mg import _coarse_random, _dense_prolongator
    dims, b, nv, m = (4, 2, 2, 4), 2, 2, 0.1
    U = gauge_field(dims, "haar", 2011)
    P = mg_mod.orthonormalize(gaussian_spinor(dims, 2012, lead=(nv,)), b)
    Y = mg_mod.coarse_operator(U, m, BC_AP, P, b)
    Pm = _dense_prolongator(P, dims, b)
    Dc = Pm.conj().T @ wilson_dense(U, dims, m, BC_AP) @ Pm
    c = _coarse_random(mg_mod.coarse_dims(dims, b), 2 * nv, 2013)
    return np.abs(mg_mod.coarse_apply(Y, c).reshape(-1) - Dc @ c.reshape(-1)).max()


@pytest.mark.parametrize("mutation", ["no_boundary_phase", "backward_link_unshifted"])
def test_coarse_operator_mutations_are_caught(monkeypatch, mutation):
    from oracle import mg
    assert _galerkin_error(mg) < 1e-11
    if mutation == "no_boundary_phase":
        orig = mg.wilson.shift
        monkeypatch.setattr(mg.wilson, "shift", lambda f, mu, sign, bc: orig(f, mu, sign, (1, 1, 1, 1)))
    elif mutation == "backward_link_unshifted":
        orig_roll = mg.np.roll
        monkeypatch.setattr(mg.np, "roll", lambda a, s, axis=None: a if a.ndim == 6 else orig_roll(a, s, axis=axis))
    assert _galerkin_error(mg) > 1e-3


def test_mixed_chirality_aggregation_is_caught(monkeypatch):
    """Aggregates that mix chiralities still give a Galerkin operator, but lose
    gamma_5-hermiticity: the gamma_5 pin catches that reading error."""
    from oracle import mg
    from tests.test_oracle_mg import test_coarse_gamma5_hermiticity
    test_coarse_gamma5_hermiticity()
    monkeypatch.setattr(mg, "CHIRAL_SPINS", ((0, 2), (1, 3)))
    with pytest.raises(AssertionError):
        test_coarse_gamma5_hermiticity()


# ------------------------------------------------------------ source mutants
# A one-token change planted in a copy of an oracle function's source: the copy
# is compiled against the module's own globals and swapped in for the test.
# Each mutant lists the pins (existing pin tests) of which at least one must
# fail; they run in order and stop at the first failure.

def _plant(monkeypatch, module, fname, old, new):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(module, fname)))
    assert src.count(old) == 1, (fname, old)
    scope = {}
    exec(compile(src.replace(old, new), f"<mutant of {module.__name__}.{fname}>", "exec"), module.__dict__, scope)
    monkeypatch.setattr(module, fname, scope[fname])


def _some_pin_fails(pins):
    for pin in pins:
        try:
            with np.errstate(all="ignore"):
                pin()
        except AssertionError:
            return True
    return False


def _eo_pins():
    from tests import test_oracle_eo as t
    return [t.test_schur_adjoint, t.test_schur_determinant_identity, t.test_schur_solve_gives_full_solution]


@pytest.mark.parametrize("fname,old,new", [
    ("schur", "/ (4.0 * c)", "/ (2.0 * c)"),                                   # Schur term without the 1/2 of each hop
    ("schur", "hop_eo(U, tmp, bc, 0, dagger)", "hop_eo(U, tmp, bc, 0)"),       # adjoint forgets the second hop
    ("prepare_source", "restrict(b, 0) + hop_eo", "restrict(b, 0) - hop_eo"),  # source sign
    ("prepare_source", "(2.0 * c)", "(4.0 * c)"),                              # source factor
    ("reconstruct", "0.5 * hop_eo", "-0.5 * hop_eo"),                          # odd-half sign
])
def test_wilson_even_odd_mutants_are_caught(monkeypatch, fname, old, new):
    assert not _some_pin_fails(_eo_pins())
    _plant(monkeypatch, wilson, fname, old, new)
    assert _some_pin_fails(_eo_pins())


def _dwf_pins():
    from tests import test_oracle_dwf as t
    return [lambda: t.test_m5_inverse(False), lambda: t.test_m5_inverse(True), t.test_ls1_reduces_to_wilson,
            lambda: t.test_free_field_determinant_closed_form(3, 0.5, -0.3),
            lambda: t.test_dense_brute_force(False), lambda: t.test_dense_brute_force(True),
            t.test_gamma5_reflection_hermiticity, t.test_eo_solve_gives_full_solution]


@pytest.mark.parametrize("fname,old,new", [
    ("s_up", "out[-1] *= -mf", "out[-1] *= mf"),                               # wall coupling sign
    ("s_down", "out[0] *= -mf", "out[0] *= 0.0 * mf"),                         # wall coupling dropped on one side
    ("m5op", "(5.0 - M5)", "(4.0 - M5)"),                                      # diagonal of D_W(-M5) without the +1
    ("m5op_matrix", "up[s, 0] = -mf", "up[s, 0] = mf"),                        # inverse built with the wrong twist
    ("m5op_inv", "m5op_matrix(Ls, M5, mf, chir, dagger)", "m5op_matrix(Ls, M5, mf, chir)"),  # adjoint inverse
    ("schur", "0.25 *", "0.5 *"),                                              # Schur term factor
    ("reconstruct", "0.5 * wilson.hop_eo", "0.25 * wilson.hop_eo"),            # odd-half factor
])
def test_dwf_mutants_are_caught(monkeypatch, fname, old, new):
    _plant(monkeypatch, dwf, fname, old, new)
    assert _some_pin_fails(_dwf_pins())


def _cg_pins():
    from tests import test_oracle_cg as t
    return [t.test_cg_on_hermitian_matrix_exact_termination, t.test_cg_matches_dense_solve]


@pytest.mark.parametrize("fname,old,new", [
    ("cg", "p = r + (rr_new / rr) * p", "p = r + (rr / rr_new) * p"),          # beta inverted
    ("cg", "alpha = rr / _dot(p, ap).real", "alpha = rr / _dot(ap, ap).real"), # alpha of the wrong inner product
    ("cg", "r -= alpha * ap", "r += alpha * ap"),                              # residual update sign
    ("cg", "x += alpha * p", "x += alpha * r"),                                # solution updated along r
    ("true_residual", "b - apply_a(x)", "b - x"),                              # exit check without the operator
])
def test_cg_mutants_are_caught(monkeypatch, fname, old, new):
    from oracle import cg
    assert not _some_pin_fails(_cg_pins())
    _plant(monkeypatch, cg, fname, old, new)
    assert _some_pin_fails(_cg_pins())


@pytest.mark.parametrize("fname,old,new,integrator", [
    ("trajectory", "kick(eps / 2)", "kick(eps)", 0),                           # leapfrog opens with a full kick
    ("trajectory", "drift(eps)", "drift(eps / 2)", 0),                         # leapfrog drift of half a step
    ("trajectory", "kick(2 * lam * eps if", "kick(lam * eps if", 1),           # merged kicks of neighbouring steps
    ("trajectory", "kick((1 - 2 * lam) * eps)", "kick((1 - lam) * eps)", 1),   # middle kick weight
    ("total_force", "F = gauge.force(U, beta)", "F = 2.0 * gauge.force(U, beta)", 0),  # force of another action
    ("hamiltonian", "K + Sg + Sf", "K + 0.5 * Sg + Sf", 0),                    # energy without the full action
])
def test_hmc_mutants_are_caught(monkeypatch, fname, old, new, integrator):
    """Gauge-only trajectories (the fermion force has its own pins above)."""
    from oracle import hmc
    from tests import test_oracle_hmc as t
    pins = [lambda: t.test_energy_violation_is_second_order(integrator, False),
            lambda: t.test_reversibility(integrator, False)]
    assert not _some_pin_fails(pins)
    _plant(monkeypatch, hmc, fname, old, new)
    assert _some_pin_fails(pins)


def _mg_pins():
    from tests import test_oracle_mg as t
    return [lambda: t.test_restriction_and_prolongation((4, 2, 2, 4), 2, 2),
            lambda: t.test_coarse_operator_is_galerkin_product((4, 2, 2, 4), 2, 2),
            t.test_coarse_gamma5_hermiticity]


@pytest.mark.parametrize("fname,old,new", [
    ("restrict", "np.conj(Gp[..., sp, :])", "Gp[..., sp, :]"),                 # restriction without P^dag
    ("prolong", "c[..., s * Nv:(s + 1) * Nv]", "c[..., (1 - s) * Nv:(2 - s) * Nv]"),  # chiral halves swapped
    ("orthonormalize", "Q = Q * (d / np.abs(d))[..., None, :]", "Q = Q"),      # QR sign convention left to LAPACK
    ("_blocked", "n + 1, n + 3, n + 5, n + 7", "n + 3, n + 1, n + 5, n + 7"),  # in-block axes out of order
    ("coarse_operator", "fwd_out = (coord % b) == b - 1", "fwd_out = (coord % b) == 0"),  # aggregate edge
    ("coarse_operator", "(4.0 + mass) * B", "(4.0 - mass) * B"),              # site term
    ("coarse_apply", "ym = np.roll(Y[2 + 2 * mu], -1, axis=ax - 1)", "ym = Y[2 + 2 * mu]"),  # adjoint stencil
    ("coarse_apply", 'np.einsum("...ji,...j->...i", np.conj(yp), cm)',
     'np.einsum("...ij,...j->...i", np.conj(yp), cm)'),                        # adjoint without the transpose
])
def test_mg_mutants_are_caught(monkeypatch, fname, old, new):
    from oracle import mg
    assert not _some_pin_fails(_mg_pins())
    _plant(monkeypatch, mg, fname, old, new)
    assert _some_pin_fails(_mg_pins())


def _gauge_pins():
    from tests import test_oracle_gauge as t
    return [t.test_unit_links, lambda: t.test_single_twisted_link_closed_form(0, 0.3),
            t.test_staple_counts_every_plaquette_four_times, t.test_gauge_invariance,
            t.test_force_matches_central_finite_difference, t.test_exponential_against_series,
            t.test_kinetic_energy]


@pytest.mark.parametrize("fname,old,new", [
    ("plaquette_field", "dag(_fwd(u_mu, nu)) @ dag(u_nu)", "dag(u_nu) @ dag(_fwd(u_mu, nu))"),  # path order
    ("mean_plaquette", "/ 3.0", "/ 2.0"),                                      # colour normalisation
    ("action", "n_plaq = 6 *", "n_plaq = 4 *"),                                # plaquette count
    ("expm_i", "np.exp(1j * eps * w)", "np.exp(-1j * eps * w)"),               # exponent sign
    ("expm_i", "v.conj())", "v)"),                                             # eigenvectors not conjugated
    ("update_links", "expm_i(P, eps) @ U", "U @ expm_i(P, eps)"),              # update from the right
    ("kinetic", "0.5 *", "1.0 *"),                                             # kinetic normalisation
])
def test_gauge_mutants_are_caught(monkeypatch, fname, old, new):
    from oracle import gauge
    assert not _some_pin_fails(_gauge_pins())
    _plant(monkeypatch, gauge, fname, old, new)
    assert _some_pin_fails(_gauge_pins())


def test_su3_operand_swap_is_caught(monkeypatch):
    from oracle import su3
    from tests import test_oracle_su3 as t
    pins = [t.test_explicit_loop, t.test_identity_and_order]
    assert not _some_pin_fails(pins)
    _plant(monkeypatch, su3, "su3_mul", "np.matmul(x, y)", "np.matmul(y, x)")
    assert _some_pin_fails(pins)
