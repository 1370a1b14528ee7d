"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numpy's own
FFT or an explicit triple sum, closed forms (homogeneous media, the exact
layered-medium solution), a dense displacement-based solve of the same
Galerkin problem, rigorous bounds, the paper's printed tables, and the special
cases of the two-level scheme. The mutation tests at the end plant plausible
mistakes in the oracle and confirm that a pin catches each one.
"""

import os

import numpy as np
import pytest

import synth
from oracle import hh_oracle as O

RNG = np.random.default_rng(20220804)


def rand_spd6(rng, scale=50.0):
    A = rng.standard_normal((6, 6))
    return scale * (A @ A.T / 6.0 + np.eye(6))


# ---------------------------------------------------------------- FFT ------

@pytest.mark.parametrize("shape", [(3, 5, 7), (4, 6, 8), (2, 1, 9), (1, 1, 1), (12, 10, 15)])
def test_fft_matches_numpy(shape):
    a = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    ref = np.fft.fftn(a)
    got = O.fft3(a)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    back = O.ifft3(got)
    assert np.abs(back - a).max() <= 1e-12


def test_fft_explicit_sum():
    shape = (2, 3, 4)
    a = RNG.standard_normal(shape)
    nz, ny, nx = shape
    got = O.fft3(a)
    for kz in range(nz):
        for ky in range(ny):
            for kx in range(nx):
                s = 0.0
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            s += a[z, y, x] * np.exp(-2j * np.pi * (kz * z / nz + ky * y / ny + kx * x / nx))
                assert abs(got[kz, ky, kx] - s) < 1e-12


# --------------------------------------------------------- projection ------

def _rand_hat(shape):
    return RNG.standard_normal((6,) + shape) + 1j * RNG.standard_normal((6,) + shape)


def _cinner(a, b):
    return np.sum(O.FROB_W[:, None, None, None] * a * np.conj(b))


@pytest.mark.parametrize("shape", [(5, 7, 3), (4, 6, 8)])
@pytest.mark.parametrize("rule", ["component", "mode"])
def test_projection_is_orthogonal_projection(shape, rule):
    xi, zero = O.wave_vectors(shape, rule)
    a = _rand_hat(shape)
    b = _rand_hat(shape)
    Pa = O.project_sym(a, xi, zero)
    assert np.abs(O.project_sym(Pa, xi, zero) - Pa).max() < 1e-12
    lhs = _cinner(Pa, b)
    rhs = _cinner(a, O.project_sym(b, xi, zero))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    assert np.all(Pa[:, 0, 0, 0] == 0)


def test_projection_range_and_kernel():
    shape = (5, 5, 5)
    xi, zero = O.wave_vectors(shape)
    norm = np.sqrt((xi ** 2).sum(0))
    n = xi / np.where(norm > 0, norm, 1)
    a = RNG.standard_normal((3,) + shape) + 1j * RNG.standard_normal((3,) + shape)
    # compatible: sym(a (x) n) is kept unchanged
    S = 0.5 * (np.einsum("i...,j...->ij...", a, n) + np.einsum("i...,j...->ij...", n, a))
    s6 = O.from_full(S)
    P = O.project_sym(s6, xi, zero)
    assert np.abs(P - np.where(zero, 0, s6)).max() < 1e-12
    # equilibrated: tau with tau n = 0 is annihilated; build tau = Q M Q with Q = I - n n
    M = RNG.standard_normal((3, 3) + shape)
    M = M + np.swapaxes(M, 0, 1)
    Q = np.eye(3)[:, :, None, None, None] - np.einsum("i...,j...->ij...", n, n)
    T = np.einsum("ik...,kl...,lj...->ij...", Q, M, Q)
    assert np.abs(O.project_sym(O.from_full(T), xi, zero)).max() < 1e-12


@pytest.mark.parametrize("shape", [(4, 6, 8), (6, 6, 6)])
def test_projection_keeps_real_fields_real_on_even_grids(shape):
    xi, zero = O.wave_vectors(shape, "component")
    tau = RNG.standard_normal((6,) + shape)
    out = O.ifft3(O.project_sym(O.fft3(tau), xi, zero))
    assert np.abs(out.imag).max() < 1e-12 * np.abs(out.real).max()


# ------------------------------------------------- solver vs brute force ---

def _displacement_solve(medium, E):
    """Dense solve of the same Galerkin problem in displacement form.

    Unknown: periodic displacement u (3 per voxel); strain fluctuation
    eps*(u) = sym grad u by spectral differentiation (numpy FFT); minimise the
    total strain energy sum_x gamma^T C gamma with gamma the engineering
    Voigt strain of E + eps*(u). Odd grids only (no Nyquist modes).
    """
    shape = medium.shape
    V = int(np.prod(shape))
    nz, ny, nx = shape
    f = [np.fft.fftfreq(nx), np.fft.fftfreq(ny), np.fft.fftfreq(nz)]
    XI = np.zeros((3,) + shape)
    XI[0] = f[0][None, None, :]
    XI[1] = f[1][None, :, None]
    XI[2] = f[2][:, None, None]

    def strain(uvec):
        u = uvec.reshape((3,) + shape)
        uh = np.fft.fftn(u, axes=(1, 2, 3))
        G = 1j * np.einsum("i...,j...->ij...", uh, XI)  # du_i/dx_j
        eh = 0.5 * (G + np.swapaxes(G, 0, 1))
        e = np.real(np.fft.ifftn(eh, axes=(2, 3, 4)))
        return O.from_full(e)

    B = np.zeros((6 * V, 3 * V))
    for m in range(3 * V):
        e = np.zeros(3 * V)
        e[m] = 1.0
        B[:, m] = strain(e).ravel()
    Cv = medium.voigt()  # (6,6,...)
    Wt = np.repeat(O.FROB_W, V)
    DB = Wt[:, None] * B
    Cblk = np.zeros((6 * V, 6 * V))
    for i in range(6):
        for j in range(6):
            Cblk[i * V:(i + 1) * V, j * V:(j + 1) * V] = np.diag(Cv[i, j].ravel())
    gE = np.repeat(O.FROB_W * E, V)
    H = DB.T @ Cblk @ DB
    g = DB.T @ Cblk @ gE
    u, *_ = np.linalg.lstsq(H, -g, rcond=None)
    return (B @ u).reshape((6,) + shape)


def _bruteforce_error(n, phases, a):
    img = (RNG.random((n, n, n)) < 0.4).astype(np.uint8)
    med = O.IsoMedium.from_labels(img, phases)
    E = O.unit_load(a)
    x, it, _ = O.solve_cg(med, E, tol=1e-13, max_iter=5000)
    ref = _displacement_solve(med, E)
    return np.abs(x - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("n,a", [(3, 0), (3, 3), (5, 4)])
def test_cg_matches_dense_displacement_solve(n, a):
    assert _bruteforce_error(n, synth.PHASES_APPENDIX_B, a) < 1e-9


@pytest.mark.parametrize("n", [3, 5, 7])
def test_six_and_nine_component_forms_agree(n):
    img = (RNG.random((n, n, n)) < 0.5).astype(np.uint8)
    med = O.IsoMedium.from_labels(img, synth.PHASES_APPENDIX_B)
    for a in (0, 5):
        x6, _, _ = O.solve_cg(med, O.unit_load(a), tol=1e-13)
        x9 = O.solve_cg_grad(med, O.unit_load(a), tol=1e-13)
        assert np.abs(x6 - x9).max() < 1e-10 * np.abs(x6).max()


def test_fixed_iterations_reproduce_converged_path():
    img = synth.grf_two_phase(n=8, ell=2.0)
    med = O.IsoMedium.from_labels(img, synth.PHASES_SOLID_PORE)
    x1, it1, r1 = O.solve_cg(med, O.unit_load(1), fixed_iters=7)
    assert it1 == 7
    x2, it2, _ = O.solve_cg(med, O.unit_load(1), tol=r1 * 1.0000001)
    assert it2 == 7 and np.array_equal(x1, x2)


def test_basic_scheme_reaches_the_cg_solution():
    img = (RNG.random((7, 7, 7)) < 0.5).astype(np.uint8)
    ph = synth.PHASES_APPENDIX_B
    med = O.IsoMedium.from_labels(img, ph)
    lam = ph[:, 0] - 2 * ph[:, 1] / 3
    lam0 = 0.5 * (lam.min() + lam.max())
    mu0 = 0.5 * (ph[:, 1].min() + ph[:, 1].max())
    E = O.unit_load(2)
    xb, it, res = O.solve_basic(med, E, lam0, mu0, tol=1e-11)
    xc, _, _ = O.solve_cg(med, E, tol=1e-12)
    assert res <= 1e-11 and it > 5
    assert np.abs(xb - xc).max() < 1e-8 * np.abs(xc).max()


# ------------------------------------- accelerated scheme (Eyre and Milton)

def _layer_recurrence(labels, ph, E, lam0, mu0, steps):
    """The accelerated scheme on a laminate along z, written out per layer by
    hand: every field depends on z only and is constant in each phase's
    layers, so each layer keeps one strain (6 tensor components). For such
    fields Gamma0 with n = e_z keeps only the 33, 23 and 13 components of the
    polarization and maps them to (tau_33 - <tau_33>) / (lam0 + 2 mu0) and
    (tau_i3 - <tau_i3>) / (2 mu0) (the in-plane components vanish since
    n_i = 0 for i = 1, 2). B = E - eps - Gamma0 tau; the local factor
    2 (C + C0)^-1 C0 scales the spherical part of B by 2 K0 / (K + K0) and
    the deviatoric part by 2 mu0 / (mu + mu0)."""
    nz = len(labels)
    K = ph[labels, 0]
    mu = ph[labels, 1]
    lam = K - 2 * mu / 3
    K0 = lam0 + 2 * mu0 / 3
    eps = np.tile(E, (nz, 1))
    for _ in range(steps):
        tr = eps[:, 0] + eps[:, 1] + eps[:, 2]
        tau = 2 * (mu - mu0)[:, None] * eps
        tau[:, :3] += ((lam - lam0) * tr)[:, None]
        g = np.zeros_like(eps)
        g[:, 2] = (tau[:, 2] - tau[:, 2].mean()) / (lam0 + 2 * mu0)
        g[:, 3] = (tau[:, 3] - tau[:, 3].mean()) / (2 * mu0)
        g[:, 4] = (tau[:, 4] - tau[:, 4].mean()) / (2 * mu0)
        B = E - eps - g
        sph = (B[:, 0] + B[:, 1] + B[:, 2]) / 3
        fs = 2 * K0 / (K + K0)
        fd = 2 * mu0 / (mu + mu0)
        upd = fd[:, None] * B
        upd[:, :3] += ((fs - fd) * sph)[:, None]
        eps = eps + upd
    return eps


@pytest.mark.parametrize("load", [2, 4])
def test_eyre_milton_on_a_laminate_matches_the_layer_recurrence(load):
    labels = np.array([0, 0, 1, 2, 1, 1, 0])  # odd nz: no Nyquist plane
    ph = np.array([[37.0, 44.0], [2.5, 1.5], [21.0, 7.0]])
    img = synth.laminate((7, 2, 3), labels)
    med = O.IsoMedium.from_labels(img, ph)
    lam0, mu0 = O.eyre_milton_reference(ph)
    E = O.unit_load(load)
    for steps in (1, 2, 3):
        x, it, _ = O.solve_eyre_milton(med, E, lam0, mu0, fixed_iters=steps)
        assert it == steps
        want = _layer_recurrence(labels, ph, E, lam0, mu0, steps)
        got = (x + E[:, None, None, None])[:, :, 0, 0].T  # (nz, 6)
        assert np.abs(got - want).max() < 1e-12
        assert np.ptp(x, axis=(2, 3)).max() < 1e-12  # constant in x and y


def test_eyre_milton_reaches_the_cg_solution_faster_than_the_basic_scheme():
    img = (RNG.random((7, 7, 7)) < 0.5).astype(np.uint8)
    ph = np.array([[37.0, 44.0], [0.37, 0.44]])  # contrast 100
    med = O.IsoMedium.from_labels(img, ph)
    E = O.unit_load(3)
    lam0, mu0 = O.eyre_milton_reference(ph)
    xe, ite, res = O.solve_eyre_milton(med, E, lam0, mu0, tol=1e-10)
    xc, _, _ = O.solve_cg(med, E, tol=1e-12)
    assert res <= 1e-10
    assert np.abs(xe - xc).max() < 1e-7 * np.abs(xc).max()
    lam = ph[:, 0] - 2 * ph[:, 1] / 3
    _, itb, _ = O.solve_basic(med, E, 0.5 * (lam.min() + lam.max()), 0.5 * (ph[:, 1].min() + ph[:, 1].max()),
                              tol=1e-6, max_iter=5000)
    _, ite6, _ = O.solve_eyre_milton(med, E, lam0, mu0, tol=1e-6)
    assert 3 * ite6 < itb


def test_eyre_milton_reference_is_the_geometric_mean():
    ph = np.array([[37.0, 44.0], [1e-4, 1e-4], [21.0, 7.0]])
    lam0, mu0 = O.eyre_milton_reference(ph)
    assert np.isclose(mu0, np.sqrt(1e-4 * 44.0)) and np.isclose(lam0 + 2 * mu0 / 3, np.sqrt(1e-4 * 37.0))


# ------------------------------------------ Green operator of the basic scheme
# The basic scheme's Gamma0 is the Green operator of an isotropic reference
# medium C0 = (lam0, mu0). Per mode with unit wave vector n it is fixed by
# three facts that do not depend on how it is written out: it inverts C0 on
# compatible strains (Gamma0 : C0 : sym(a (x) n) = sym(a (x) n)), it vanishes
# on equilibrated polarizations (tau n = 0), and Gamma0 C0 Gamma0 = Gamma0.
# The reference medium below has mu0 != 1 and lam0 != mu0, so a dropped or
# misplaced factor of mu0 or (lam0 + 2 mu0) changes the result.

LAM0, MU0 = 5.3, 3.7


def _hooke0(e6, lam0=LAM0, mu0=MU0):
    """Isotropic Hooke's law of the reference medium on six stored components."""
    tr = e6[0] + e6[1] + e6[2]
    s = 2.0 * mu0 * e6
    s[0:3] = s[0:3] + lam0 * tr
    return s


def _sym_outer(a, n):
    """Six stored components of sym(a (x) n) per mode (a, n shaped (3, ...))."""
    return np.stack([0.5 * (a[i] * n[j] + a[j] * n[i]) for (i, j) in O.PAIRS])


def _unit(xi):
    norm = np.sqrt(np.sum(xi * xi, axis=0))
    return xi / np.where(norm > 0, norm, 1.0)


def _rand_c(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


@pytest.mark.parametrize("shape", [(5, 6, 7), (4, 4, 6)])
def test_gamma0_inverts_the_reference_medium_on_compatible_strains(shape):
    xi, zero = O.wave_vectors(shape)
    eps = _sym_outer(_rand_c((3,) + shape), _unit(xi))
    got = O.gamma0_apply(_hooke0(eps), xi, zero, LAM0, MU0)
    eps[:, zero] = 0.0
    assert np.abs(got - eps).max() < 1e-12 * np.abs(eps).max()


@pytest.mark.parametrize("shape", [(5, 6, 7), (4, 4, 6)])
def test_gamma0_vanishes_on_equilibrated_polarizations(shape):
    xi, zero = O.wave_vectors(shape)
    n = _unit(xi)
    # t1, t2: an orthonormal pair perpendicular to n (through the coordinate
    # axis least aligned with n); tau built from them has tau n = 0
    e = np.zeros_like(n)
    ax = np.argmin(np.abs(n), axis=0)
    for i in range(3):
        e[i] = (ax == i)
    t1 = np.cross(n, e, axis=0)
    t1 = t1 / np.where(np.linalg.norm(t1, axis=0) > 0, np.linalg.norm(t1, axis=0), 1.0)
    t2 = np.cross(n, t1, axis=0)
    c = _rand_c((3,) + shape)
    tau = c[0] * _sym_outer(t1, t1) + c[1] * _sym_outer(t1, t2) + c[2] * _sym_outer(t2, t2)
    tau[:, zero] = 0.0
    assert np.abs(np.einsum("ij...,j...->i...", O.to_full(tau), n)).max() < 1e-12 * np.abs(tau).max()
    got = O.gamma0_apply(tau, xi, zero, LAM0, MU0)
    assert np.abs(got).max() < 1e-12 * np.abs(tau).max()


@pytest.mark.parametrize("rule", ["component", "mode"])
def test_gamma0_is_a_projection_in_the_reference_metric(rule):
    shape = (4, 5, 6)
    xi, zero = O.wave_vectors(shape, rule)
    tau = _rand_c((6,) + shape)
    g = O.gamma0_apply(tau, xi, zero, LAM0, MU0)
    gg = O.gamma0_apply(_hooke0(g), xi, zero, LAM0, MU0)
    assert np.abs(gg - g).max() < 1e-12 * np.abs(g).max()
    # symmetric in the Frobenius product, mode by mode
    sig = _rand_c((6,) + shape)
    w = O.FROB_W[:, None, None, None]
    lhs = np.sum(w * sig * g, axis=0)
    rhs = np.sum(w * O.gamma0_apply(sig, xi, zero, LAM0, MU0) * tau, axis=0)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()
    assert np.all(g[:, zero] == 0.0)


# --------------------------------------------------------- closed forms ----

def test_homogeneous_isotropic_returns_phase_moduli_exactly():
    img = np.zeros((6, 5, 4), dtype=np.uint8)
    for K, G in [(37.0, 44.0), (36.0, 45.0), (1e-4, 1e-4)]:
        ph = np.array([[K, G]])
        res = O.homogenize_direct(img, ph)
        assert np.all(res["iters"] == 0)
        assert np.abs(res["C"] - O.iso_voigt(K, G)).max() <= 4e-16 * (K + 2 * G)
        assert abs(res["K"] - K) <= 1e-12 * K and abs(res["G"] - G) <= 1e-12 * G


def test_homogeneous_anisotropic_returns_its_stiffness():
    C = rand_spd6(RNG)
    shape = (5, 4, 6)
    med = O.AnisoMedium(np.broadcast_to(C[:, :, None, None, None], (6, 6) + shape).copy())
    res = O.homogenize_box(med, (slice(None),) * 3)
    assert np.all(res["iters"] == 0)
    assert np.abs(res["C"] - C).max() <= 1e-13 * np.abs(C).max()


def test_paper_phase_moduli(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "phase_moduli.txt")) if not l.startswith("#")]
    for name, K, G, C11, C12, C44 in rows:
        C = O.iso_voigt(float(K), float(G))
        assert C[0, 0] == pytest.approx(float(C11), rel=1e-12)
        assert C[0, 1] == pytest.approx(float(C12), rel=1e-12)
        assert C[3, 3] == pytest.approx(float(C44), rel=1e-12)
        k, g = O.moduli_voigt(C)
        kr, gr = O.moduli_reuss(C)
        assert k == pytest.approx(float(K), rel=1e-12) and g == pytest.approx(float(G), rel=1e-12)
        assert kr == pytest.approx(float(K), rel=1e-10) and gr == pytest.approx(float(G), rel=1e-10)


NORM = [2, 3, 4]   # Voigt 33, 23, 13: traction components on a z-normal plane
TANG = [0, 1, 5]   # Voigt 11, 22, 12: in-plane strains


def backus(Cs, f):
    """Exact effective stiffness of a z-layered medium (layer stiffness Cs[l],
    volume fraction f[l]): traction sigma_N and in-plane strain gamma_T are
    uniform across layers."""
    f = np.asarray(f) / np.sum(f)
    iNN = [np.linalg.inv(C[np.ix_(NORM, NORM)]) for C in Cs]
    A = sum(fl * m for fl, m in zip(f, iNN))
    CNN = np.linalg.inv(A)
    B = sum(fl * m @ C[np.ix_(NORM, TANG)] for fl, m, C in zip(f, iNN, Cs))
    D = sum(fl * C[np.ix_(TANG, NORM)] @ m for fl, m, C in zip(f, iNN, Cs))
    T = sum(fl * (C[np.ix_(TANG, TANG)] - C[np.ix_(TANG, NORM)] @ m @ C[np.ix_(NORM, TANG)])
            for fl, m, C in zip(f, iNN, Cs))
    out = np.zeros((6, 6))
    out[np.ix_(NORM, NORM)] = CNN
    out[np.ix_(NORM, TANG)] = CNN @ B
    out[np.ix_(TANG, NORM)] = D @ CNN
    out[np.ix_(TANG, TANG)] = T + D @ CNN @ B
    return out


def test_isotropic_laminate_matches_backus_closed_form():
    labels = [0, 0, 1, 0, 1, 1, 1]
    img = synth.laminate((7, 3, 5), labels)
    ph = synth.PHASES_APPENDIX_B
    res = O.homogenize_direct(img, ph, tol=1e-13)
    ref = backus([O.iso_voigt(*ph[l]) for l in labels], np.ones(7))
    assert np.abs(res["C"] - ref).max() <= 1e-9 * np.abs(ref).max()
    # the scalar form of the same closed form: Reuss across, Voigt along
    Ms = [ph[l, 0] + 4 * ph[l, 1] / 3 for l in labels]
    mus = [ph[l, 1] for l in labels]
    assert res["C"][2, 2] == pytest.approx(1 / np.mean([1 / m for m in Ms]), rel=1e-9)
    assert res["C"][3, 3] == pytest.approx(1 / np.mean([1 / m for m in mus]), rel=1e-9)
    assert res["C"][5, 5] == pytest.approx(np.mean(mus), rel=1e-9)


def test_anisotropic_laminate_matches_backus_closed_form():
    nz = 5
    Cs = [rand_spd6(RNG) for _ in range(nz)]
    shape = (nz, 3, 3)
    C = np.zeros((6, 6) + shape)
    for z in range(nz):
        C[:, :, z] = Cs[z][:, :, None, None]
    res = O.homogenize_box(O.AnisoMedium(C), (slice(None),) * 3, tol=1e-13)
    ref = backus(Cs, np.ones(nz))
    assert np.abs(res["C"] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_buffered_laminate_core_averages():
    """A layered box with a buffer: core averages of the exact layered solution
    give Sigma and Eps (Eps != I), and C_R = Sigma Eps^-1."""
    labels = [1, 0, 0, 1, 0, 1, 1, 0, 1]
    nz = len(labels)
    ph = synth.PHASES_APPENDIX_B
    img = synth.laminate((nz, 3, 3), labels)
    core = (slice(2, 7), slice(0, 3), slice(0, 3))
    med = O.IsoMedium.from_labels(img, ph)
    res = O.homogenize_box(med, core, tol=1e-13)
    Cs = [O.iso_voigt(*ph[l]) for l in labels]
    Sig = np.zeros((6, 6))
    Eps = np.zeros((6, 6))
    iNN = [np.linalg.inv(C[np.ix_(NORM, NORM)]) for C in Cs]
    A = np.mean(iNN, axis=0)
    for a in range(6):
        gE = np.zeros(6)
        gE[a] = 1.0
        gT = gE[TANG]
        sN = np.linalg.solve(A, gE[NORM] + np.mean([m @ C[np.ix_(NORM, TANG)] @ gT for m, C in zip(iNN, Cs)], 0))
        g_layers = []
        s_layers = []
        for m, C in zip(iNN, Cs):
            g = np.zeros(6)
            g[TANG] = gT
            g[NORM] = m @ (sN - C[np.ix_(NORM, TANG)] @ gT)
            g_layers.append(g)
            s_layers.append(C @ g)
        Eps[:, a] = np.mean(g_layers[2:7], axis=0)
        Sig[:, a] = np.mean(s_layers[2:7], axis=0)
    assert np.abs(Eps - np.eye(6)).max() > 1e-2
    ref = Sig @ np.linalg.inv(Eps)
    assert np.abs(res["Eps"] - Eps).max() < 1e-9
    assert np.abs(res["C"] - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(res["C"] - np.linalg.inv(Eps) @ Sig).max() > 1e-3 * np.abs(ref).max()


# --------------------------------------------------------------- bounds ----

@pytest.mark.parametrize("shape,ph", [((6, 6, 6), synth.PHASES_APPENDIX_B),
                                      ((5, 7, 6), synth.PHASES_SOLID_CLAY_PORE)])
def test_voigt_reuss_bounds_and_symmetry(shape, ph):
    img = (RNG.random(shape) * len(ph)).astype(np.uint8)
    med = O.IsoMedium.from_labels(img, ph)
    res = O.homogenize_box(med, (slice(None),) * 3, tol=1e-10, max_iter=50000)
    C = res["C"]
    Cv = med.voigt().reshape(6, 6, -1)
    CV = Cv.mean(axis=2)
    CR = np.linalg.inv(np.mean([np.linalg.inv(Cv[:, :, i]) for i in range(Cv.shape[2])], axis=0))
    s = np.abs(C).max()
    assert np.linalg.norm(C - C.T) / np.linalg.norm(C) <= 1e-8
    Cs = O.symmetrize(C)
    assert np.linalg.eigvalsh(CV - Cs).min() >= -1e-8 * s
    assert np.linalg.eigvalsh(Cs - CR).min() >= -1e-8 * s
    K, G = O.moduli_voigt(Cs)
    KR, GR = O.moduli_reuss(Cs)
    assert KR <= K + 1e-12 and GR <= G + 1e-12
    KV, GV = O.moduli_voigt(CV)
    KRR, GRR = O.moduli_reuss(CR)
    assert KRR - 1e-9 <= K <= KV + 1e-9 and GRR - 1e-9 <= G <= GV + 1e-9


def test_hashin_shtrikman_bounds_two_phase_isotropic():
    """Soft check on a statistically isotropic field: K and G within the
    two-phase Hashin-Shtrikman bounds."""
    img = synth.grf_two_phase(n=16, ell=2.0, porosity=0.4, seed=7)
    ph = synth.PHASES_APPENDIX_B
    res = O.homogenize_direct(img, ph, tol=1e-8)
    f2 = img.mean()
    f1 = 1 - f2
    (K1, G1), (K2, G2) = ph

    def hs(Ka, Ga, Kb, Gb, fa, fb):
        K = Ka + fb / (1 / (Kb - Ka) + fa / (Ka + 4 * Ga / 3))
        z = Ga / 6 * (9 * Ka + 8 * Ga) / (Ka + 2 * Ga)
        G = Ga + fb / (1 / (Gb - Ga) + fa / (Ga + z))
        return K, G

    Ku, Gu = hs(K1, G1, K2, G2, f1, f2)
    Kl, Gl = hs(K2, G2, K1, G1, f2, f1)
    assert Kl <= res["K"] <= Ku
    assert Gl <= res["G"] <= Gu


# --------------------------------------------------- hierarchical scheme ---

def test_single_box_hierarchical_equals_direct():
    img = synth.grf_two_phase(n=8, ell=2.0)
    ph = synth.PHASES_APPENDIX_B
    d = O.homogenize_direct(img, ph, tol=1e-10)
    h = O.homogenize_hierarchical(img, ph, synth.uniform_partition(8, 8, 0), unit=8, tol=1e-10)
    assert np.all(h["level2"]["iters"] == 0)
    assert np.abs(h["C_sym"] - d["C_sym"]).max() <= 1e-13 * np.abs(d["C_sym"]).max()


def test_voxel_boxes_hierarchical_equals_direct():
    img = (RNG.random((5, 5, 5)) < 0.5).astype(np.uint8)
    ph = synth.PHASES_APPENDIX_B
    d = O.homogenize_direct(img, ph, tol=1e-12)
    h = O.homogenize_hierarchical(img, ph, synth.uniform_partition(5, 1, 0), unit=1, tol=1e-12)
    for r, lab in zip(h["per_box"], img.ravel()):
        assert np.all(r["iters"] == 0)
    assert np.abs(h["coarse"][:, :, 2, 3, 1] - O.iso_voigt(*ph[img[2, 3, 1]])).max() < 1e-12
    assert np.abs(h["C_sym"] - d["C_sym"]).max() <= 1e-9 * np.abs(d["C_sym"]).max()
    K, G = O.moduli_voigt(np.mean([O.iso_voigt(*ph[l]) for l in img.ravel()], axis=0))
    assert h["K_am"] == pytest.approx(K, rel=1e-12) and h["G_am"] == pytest.approx(G, rel=1e-12)


def test_extract_box_wraps_periodically():
    img = RNG.integers(0, 3, size=(6, 7, 8)).astype(np.uint8)
    box = (6, 0, 4, 2, 3, 2, 2)  # ox oy oz nx ny nz b
    sub = O.extract_box(img, box)
    assert sub.shape == (2 + 4, 3 + 4, 2 + 4)
    for k in range(sub.shape[0]):
        for j in range(sub.shape[1]):
            for i in range(sub.shape[2]):
                assert sub[k, j, i] == img[(4 - 2 + k) % 6, (0 - 2 + j) % 7, (6 - 2 + i) % 8]


def test_uneven_partition_tiles_the_image():
    boxes = synth.uneven_partition()
    assert boxes.shape == (27000, 7)
    assert set(np.unique(boxes[:, 3:6])) == {16, 24, 32}
    assert boxes[:, 6].min() == 0 and boxes[:, 6].max() == 8
    cover = np.zeros((64, 64, 64), dtype=np.int32)
    for ox, oy, oz, nx, ny, nz, b in boxes:
        cover[oz // 8:(oz + nz) // 8, oy // 8:(oy + ny) // 8, ox // 8:(ox + nx) // 8] += 1
    assert np.all(cover == 1)
    sizes = boxes[:, 3:6] + 2 * boxes[:, 6:7]
    assert sizes.min() == 16 and sizes.max() == 48


def test_clip_spd_is_the_nearest_tensor_above_the_floor():
    D = np.array([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)])
    Q, _ = np.linalg.qr(RNG.standard_normal((6, 6)))
    w = np.array([-3.0, -1e-3, 2e-4, 0.5, 7.0, 40.0])
    M = (Q * w) @ Q.T                  # Mandel form
    A = M / D[:, None] / D[None, :]    # Voigt form
    B = O.clip_spd(A, 1e-2)
    MB = D[:, None] * B * D[None, :]
    assert np.allclose(np.sort(np.linalg.eigvalsh(MB)), np.sort(np.maximum(w, 1e-2)), atol=1e-12)
    for lam in (0.5, 7.0, 40.0):
        v = Q[:, list(w).index(lam)]
        assert np.allclose(MB @ v, lam * v, atol=1e-12)
    d0 = np.linalg.norm(M - MB)
    for _ in range(200):
        P = RNG.standard_normal((6, 6))
        P = P @ P.T + 1e-2 * np.eye(6)
        assert np.linalg.norm(M - P) >= d0 - 1e-12
    # isotropic tensor eigenvalues are 3K and 2G: phases at the floor pass unchanged
    for K, G in [(37.0, 44.0), (1e-4, 1e-4), (9.8, 3.76)]:
        C = O.iso_voigt(K, G)
        assert O.clip_spd(C, min(3 * K, 2 * G)) is C
    assert O.stiffness_floor([[37.0, 44.0], [1e-4, 1e-4]]) == pytest.approx(2e-4)


def test_unbuffered_subimage_stiffness_is_positive_definite():
    img = synth.grf_two_phase(n=8, ell=2.0, porosity=0.3, seed=31)
    res = O.homogenize_hierarchical(img, synth.PHASES_APPENDIX_B, synth.uniform_partition(8, 4, 0), unit=4,
                                    tol=1e-10)
    assert res["n_clipped"] == 0
    for C in res["C_boxes"]:
        assert np.linalg.eigvalsh(C).min() > 0


# ---------------------------------------------------------- power law ------

def test_fit_inverse_n_exact():
    ns = [16, 24, 32, 64, 128]
    M = [3.0 + 5.0 / n for n in ns]
    Mi, C = O.fit_inverse_n(ns, M)
    assert Mi == pytest.approx(3.0, abs=1e-12) and C == pytest.approx(5.0, abs=1e-10)
    n1, n2, m1, m2 = 16, 32, 4.1, 3.7
    Mi, C = O.fit_inverse_n([n1, n2], [m1, m2])
    assert Mi == pytest.approx((n2 * m2 - n1 * m1) / (n2 - n1), rel=1e-13)


def test_fit_reproduces_paper_tables(golden_dir):
    ns = np.array([75, 90, 100, 150, 180, 225, 300], dtype=float)
    A = np.stack([np.ones_like(ns), 1 / ns], axis=1)
    W = np.linalg.pinv(A)
    # tolerance from the printed rounding: inputs and outputs carry +-0.005
    tol_m = np.abs(W[0]).sum() * 0.005 + 0.005
    tol_c = np.abs(W[1]).sum() * 0.005 + 0.005
    count = 0
    for line in open(os.path.join(golden_dir, "power_law_fit.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        M = np.array([float(v) for v in f[3:10]])
        Mi, C = O.fit_inverse_n(ns, M)
        assert abs(Mi - float(f[10])) <= tol_m, line
        assert abs(C - float(f[11])) <= tol_c, line
        count += 1
    assert count == 17


# ------------------------------------------------------------ mutations ----

def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle and check that a pin fails."""
    good = O.project_sym

    def dropped_term(tau_hat, xi, zero):
        norm = np.sqrt(np.sum(xi * xi, axis=0))
        n = xi / np.where(norm > 0, norm, 1.0)
        T = O.to_full(tau_hat)
        v = np.einsum("ij...,j...->i...", T, n)
        P = np.einsum("i...,j...->ij...", n, v) + np.einsum("i...,j...->ij...", v, n)
        out = O.from_full(P)
        out[:, zero] = 0
        return out

    # 1. projection without the n n (n.v) term: same kernel, but no longer a
    #    projection; the orthogonal-projection pin catches it.
    monkeypatch.setattr(O, "project_sym", dropped_term)
    with pytest.raises(AssertionError):
        test_projection_is_orthogonal_projection((5, 7, 3), "component")
    monkeypatch.setattr(O, "project_sym", good)

    # 2. shear components 23 and 13 swapped when the 3x3 tensor is formed
    good_full = O.to_full

    def swapped_full(t6):
        t = t6.copy()
        t[[3, 4]] = t6[[4, 3]]
        return good_full(t)

    monkeypatch.setattr(O, "to_full", swapped_full)
    assert _bruteforce_error(3, synth.PHASES_APPENDIX_B, 0) > 1e-3
    monkeypatch.setattr(O, "to_full", good_full)

    # 3. wave-vector components x and z transposed: the laminate pin catches it
    good_wv = O.wave_vectors

    def swapped(shape, nyquist="component"):
        xi, zero = good_wv(shape, nyquist)
        return np.stack([xi[2], xi[1], xi[0]]), zero

    monkeypatch.setattr(O, "wave_vectors", swapped)
    labels = [0, 1, 1, 0, 1]
    img = synth.laminate((5, 3, 3), labels)
    ph = synth.PHASES_APPENDIX_B
    res = O.homogenize_direct(img, ph, tol=1e-12)
    ref = backus([O.iso_voigt(*ph[l]) for l in labels], np.ones(5))
    assert np.abs(res["C"] - ref).max() > 1e-3 * np.abs(ref).max()
    monkeypatch.setattr(O, "wave_vectors", good_wv)

    # 4. Eps^-1 Sigma instead of Sigma Eps^-1: the buffered laminate catches it
    good_hb = O.homogenize_box

    def transposed(*a, **k):
        r = good_hb(*a, **k)
        r["C"] = np.linalg.inv(r["Eps"]) @ r["Sigma"]
        return r

    monkeypatch.setattr(O, "homogenize_box", transposed)
    with pytest.raises(AssertionError):
        test_buffered_laminate_core_averages()
    monkeypatch.setattr(O, "homogenize_box", good_hb)

    # 5. plain instead of engineering shear in the strain weights
    monkeypatch.setattr(O, "FROB_W", np.array([1.0, 1, 1, 1, 1, 1]))
    with pytest.raises(AssertionError):
        test_homogeneous_isotropic_returns_phase_moduli_exactly()
    monkeypatch.setattr(O, "FROB_W", np.array([1.0, 1, 1, 2, 2, 2]))

    # 6, 7. Green operator of the basic scheme with a wrong factor: the n n
    #    coefficient (lam0 + mu0) / (lam0 + 2 mu0) without its 1 / mu0, and
    #    the symmetric part without its 1 / (2 mu0)
    good_g0 = O.gamma0_apply

    def g0_with(ca, cb):
        def g0(tau_hat, xi, zero, lam0, mu0):
            n = _unit(xi)
            v = np.einsum("ij...,j...->i...", O.to_full(tau_hat), n)
            s = np.einsum("i...,i...->...", n, v)
            out = (ca(lam0, mu0) * (np.einsum("i...,j...->ij...", n, v) + np.einsum("i...,j...->ij...", v, n))
                   - cb(lam0, mu0) * np.einsum("i...,j...->ij...", n, n) * s)
            o6 = O.from_full(out)
            o6[:, zero] = 0.0
            return o6
        return g0

    g0_factor = g0_with(lambda l, m: 1.0 / (2.0 * m), lambda l, m: (l + m) / (l + 2.0 * m))
    g0_half = g0_with(lambda l, m: 1.0, lambda l, m: (l + m) / (m * (l + 2.0 * m)))
    # the same helper with the right coefficients passes
    monkeypatch.setattr(O, "gamma0_apply", g0_with(lambda l, m: 1.0 / (2.0 * m),
                                                   lambda l, m: (l + m) / (m * (l + 2.0 * m))))
    test_gamma0_inverts_the_reference_medium_on_compatible_strains((5, 6, 7))
    for bad in (g0_factor, g0_half):
        monkeypatch.setattr(O, "gamma0_apply", bad)
        with pytest.raises(AssertionError):
            test_gamma0_inverts_the_reference_medium_on_compatible_strains((5, 6, 7))
    monkeypatch.setattr(O, "gamma0_apply", good_g0)

    # 8, 9. accelerated scheme with the relaxation factor 1 instead of 2, or
    #    with the basic scheme's increment E - <eps> - Gamma0 * (C : eps) in
    #    place of the Lippmann-Schwinger residual (equal only on compatible
    #    iterates): the laminate recurrence catches both
    good_em = O.solve_eyre_milton

    def em_with(relax, lippmann_schwinger):
        def em(medium, E, lam0, mu0, tol=1e-6, max_iter=100000, nyquist="component", fixed_iters=None):
            xi, zero = O.wave_vectors(medium.shape, nyquist)
            K0 = lam0 + 2.0 * mu0 / 3.0
            fs, fd = relax * K0 / (medium.K + K0), relax * mu0 / (medium.mu + mu0)
            eps = np.broadcast_to(E[:, None, None, None], (6,) + tuple(medium.shape)).copy()
            for _ in range(fixed_iters):
                if lippmann_schwinger:
                    tau = O.IsoMedium(medium.K - K0, medium.mu - mu0).stress(eps)
                    B = E[:, None, None, None] - eps - np.real(O.ifft3(O.gamma0_apply(O.fft3(tau), xi, zero, lam0, mu0)))
                else:
                    B = (E - eps.mean(axis=(1, 2, 3)))[:, None, None, None] - np.real(
                        O.ifft3(O.gamma0_apply(O.fft3(medium.stress(eps)), xi, zero, lam0, mu0)))
                upd = fd * B
                upd[0:3] += (fs - fd) * (B[0] + B[1] + B[2]) / 3.0
                eps = eps + upd
            return eps - E[:, None, None, None], fixed_iters, 0.0
        return em

    monkeypatch.setattr(O, "solve_eyre_milton", em_with(2.0, True))
    test_eyre_milton_on_a_laminate_matches_the_layer_recurrence(2)
    for bad in (em_with(1.0, True), em_with(2.0, False)):
        monkeypatch.setattr(O, "solve_eyre_milton", bad)
        with pytest.raises(AssertionError):
            test_eyre_milton_on_a_laminate_matches_the_layer_recurrence(2)
    monkeypatch.setattr(O, "solve_eyre_milton", good_em)


# ------------------------------------------------- multi-level renormalisation

def test_multilevel_one_level_is_hierarchical():
    img = synth.grf_two_phase(n=12, ell=2.0, porosity=0.3, seed=4)
    ph = synth.PHASES_APPENDIX_B
    a = O.homogenize_multilevel(img, ph, [(6, 1)], tol=1e-11)
    b = O.homogenize_hierarchical(img, ph, O.uniform_boxes(img.shape, 6, 1), unit=6, tol=1e-11)
    assert np.abs(a["C_sym"] - b["C_sym"]).max() < 1e-9 * np.abs(b["C_sym"]).max()


def test_multilevel_unit_boxes_reproduce_the_direct_solve():
    # one-voxel cores without buffer return the voxel's own stiffness at every
    # level, so any number of such levels equals the direct solve
    img = (RNG.random((4, 4, 4)) < 0.4).astype(np.uint8)
    ph = synth.PHASES_APPENDIX_B
    a = O.homogenize_multilevel(img, ph, [(1, 0), (1, 0), (1, 0)], tol=1e-12)
    d = O.homogenize_direct(img, ph, tol=1e-12)
    assert np.abs(a["C_sym"] - d["C_sym"]).max() < 1e-8 * np.abs(d["C_sym"]).max()


def test_multilevel_laminate_exact_at_every_level():
    # a laminate along z: every core is itself a laminate (odd edges, so no
    # Nyquist mode is lost), its periodic solve is the exact layered (Backus)
    # average, and Backus averages of groups of layers compose exactly
    lab = synth.laminate((9, 9, 9), [0, 1, 1, 0, 0, 1, 1, 0, 1])
    ph = synth.PHASES_APPENDIX_B
    a = O.homogenize_multilevel(lab, ph, [(3, 0), (3, 0)], tol=1e-12)
    d = O.homogenize_direct(lab, ph, tol=1e-12)
    assert np.abs(a["C_sym"] - d["C_sym"]).max() < 1e-8 * np.abs(d["C_sym"]).max()


def test_extract_field_wraps_like_extract_box():
    C = RNG.standard_normal((6, 6, 5, 4, 3))
    box = (2, 3, 4, 2, 1, 2, 1)
    sub = O.extract_field(C, box)
    lab = np.arange(60).reshape(5, 4, 3)
    idx = O.extract_box(lab, box)
    flat = C.reshape(6, 6, -1)
    assert np.array_equal(sub, flat[:, :, idx])


# ------------------------------------------------------ correlation length ----

def test_correlation_counts_brute_force():
    img = (RNG.random((5, 6, 7)) < 0.6).astype(np.uint8)
    cnt = O.correlation_counts(img, 1, 4)
    M = (img != 1).astype(int)
    for l in range(5):
        sx = sum(M[k, j, i] * M[k, j, i + l] for k in range(5) for j in range(6) for i in range(7 - l))
        sy = sum(M[k, j, i] * M[k, j + l, i] for k in range(5) for j in range(6 - l) for i in range(7))
        sz = sum(M[k, j, i] * M[k + l, j, i] for k in range(5 - l) for j in range(6) for i in range(7))
        assert list(cnt[:, l]) == [sx, sy, sz]


def test_correlation_function_special_values():
    img = synth.grf_two_phase(n=20, ell=2.0, porosity=0.3, seed=9)
    corr = O.correlation_function(img, 1, 8)
    assert np.allclose(corr[:, 0], 1.0, atol=1e-12)  # Corr(0) = 1
    # a laminate along z of period 4: pairs one period apart coincide
    lab = synth.laminate((12, 5, 5), [0, 1, 1, 0] * 3)
    cz = O.correlation_function(lab, 1, 4)[2]
    assert abs(cz[4] - 1.0) < 1e-12
    cx = O.correlation_function(lab, 1, 3)[0]  # uniform along x
    assert np.allclose(cx, 1.0, atol=1e-12)


def test_fit_recovers_an_exponential():
    for xi in (2.5, 7.0, 13.1):
        l = np.arange(60)
        assert abs(O.fit_correlation_length(np.exp(-l / xi)) - xi) < 1e-6 * xi
