"""Plain FP64 CPU oracle of hierarchical homogenization (Ahmad et al., 2022).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
module: only the test suite, the package's smoke check and the CPU-baseline leg
of the benchmark use it. It shares no code, table or helper with the CUDA path.

Every function is slow and direct on purpose: fields are complex128/float64
numpy arrays, the discrete Fourier transform is this module's own (a DFT
matrix applied along each axis, i.e. the definition of the transform), and
the conjugate-gradient loop follows the textbook recurrences with x0 = 0.

Notation and conventions
------------------------
* Images are uint8 label arrays indexed [z, y, x]. A phase table maps a label
  to its (K, mu) pair (Section 4: isotropic C(x) from bulk and shear moduli).
* A symmetric strain or stress field is stored as six tensor components in the
  order 11, 22, 33, 23, 13, 12 with shape (6, nz, ny, nx). Vector index 0 is x,
  1 is y, 2 is z.
* Voigt vectors (Section 4, Voigt notation) list stress as (s11, s22, s33, s23,
  s13, s12) and strain with engineering shear (e11, e22, e33, 2e23, 2e13,
  2e12), so an isotropic phase has C44 = mu.
* The inner product of two tensor fields is the Frobenius product summed over
  voxels, i.e. weights (1, 1, 1, 2, 2, 2) on the six stored components.

Readings of the paper taken here (where it is silent or ambiguous)
------------------------------------------------------------------
* Projection: Appendix A defines G^(k) on 3x3 (gradient) fields. The six-
  component operator used by `project_sym` is the orthogonal projection of a
  symmetric tensor onto {sym(a (x) k)}; its kernel is {tau : tau k = 0}, the
  same equilibrium condition, and its range is the same set of compatible
  strains, so both give the same discrete solution. `project_grad` carries the
  paper's own form for the equivalence check.
* Wave vector: xi_d = m_d / N_d with m_d the signed integer frequency in
  (-N_d/2, N_d/2] (the scale cancels in the projection; dividing by N_d keeps
  the direction right on non-cubic boxes).
* Even N (Section 6 and Appendix A treat odd N): by default the component of
  the wave vector that sits at the Nyquist index is set to zero
  ("component" rule); the "mode" rule instead zeroes the projection on every
  Nyquist mode.
* Stopping rule (Appendix A names conjugate gradients only): stop when
  ||r_k|| <= tol * ||r_0||, r_0 = b = -G*(C:E), in the Frobenius norm above.
* Buffer at the image edge (Section 4, Fig. 4): indices wrap periodically.
* K and G of an anisotropic stiffness: the isotropic Voigt projection (Reuss
  projection also given).
* Uneven partitions are assembled on a regular coarse grid of `unit` voxels;
  each subimage fills its block of coarse voxels with its stiffness.
* The arithmetic mean (AM) of subimage moduli is weighted by core volume
  (a plain mean for a uniform partition).
* Level-2 voxel stiffness: sym(C_R). With a buffer, Sigma Eps^-1 need not be
  symmetric and its symmetric part can be indefinite when the core is not much
  larger than the correlation length; the conjugate-gradient solve of the
  intermediate image needs positive-definite voxels, so sym(C_R) is projected
  onto {C >= c_min I} (as a tensor, i.e. in Mandel form) by raising its
  eigenvalues to c_min, the smallest tensor eigenvalue min(3K, 2G) over the
  phases (the Frobenius-nearest tensor in that set). Positive-definite sym(C_R) (always the case without a
  buffer) passes unchanged.
"""

from __future__ import annotations

import numpy as np

PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
FROB_W = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


# --------------------------------------------------------------------------
# Discrete Fourier transform (Appendix A: trigonometric-polynomial basis,
# convolution evaluated as F^-1[G^ . zeta^]).
# --------------------------------------------------------------------------

def dft_matrix(n: int) -> np.ndarray:
    """Forward DFT matrix F[k, j] = exp(-2 pi i k j / n)."""
    j = np.arange(n)
    t = np.outer(j, j) % n  # exact integer phase index
    ang = 2.0 * np.pi * t / n
    return np.cos(ang) - 1j * np.sin(ang)


def _along(a: np.ndarray, mat: np.ndarray, axis: int) -> np.ndarray:
    a = np.moveaxis(a, axis, -1)
    a = a @ mat.T
    return np.moveaxis(a, -1, axis)


def fft3(a: np.ndarray) -> np.ndarray:
    """Unnormalised forward 3D DFT over the last three axes [z, y, x]."""
    a = np.asarray(a, dtype=np.complex128)
    for axis in (-1, -2, -3):
        a = _along(a, dft_matrix(a.shape[axis]), axis)
    return a


def ifft3(a: np.ndarray) -> np.ndarray:
    """Inverse 3D DFT (conjugate matrix, scaled by 1/V)."""
    a = np.asarray(a, dtype=np.complex128)
    V = a.shape[-1] * a.shape[-2] * a.shape[-3]
    for axis in (-1, -2, -3):
        a = _along(a, np.conj(dft_matrix(a.shape[axis])), axis)
    return a / V


# --------------------------------------------------------------------------
# Wave vectors and projections (Appendix A).
# --------------------------------------------------------------------------

def wave_vectors(shape, nyquist: str = "component"):
    """Return (xi, zero_mask): xi has shape (3, nz, ny, nx) with components
    (x, y, z); zero_mask marks modes where the projection is zero (k = 0, and
    every Nyquist mode under the "mode" rule)."""
    nz, ny, nx = shape

    def axis_freq(n):
        i = np.arange(n)
        m = np.where(i <= n // 2, i, i - n).astype(np.float64)
        nyq = (n % 2 == 0) & (i == n // 2)
        return m / n, nyq

    fx, qx = axis_freq(nx)
    fy, qy = axis_freq(ny)
    fz, qz = axis_freq(nz)
    if nyquist == "component":
        fx = np.where(qx, 0.0, fx)
        fy = np.where(qy, 0.0, fy)
        fz = np.where(qz, 0.0, fz)
    elif nyquist != "mode":
        raise ValueError(nyquist)
    XI = np.zeros((3, nz, ny, nx))
    XI[0] = fx[None, None, :]
    XI[1] = fy[None, :, None]
    XI[2] = fz[:, None, None]
    zero = np.all(XI == 0.0, axis=0)
    if nyquist == "mode":
        zero = zero | qx[None, None, :] | qy[None, :, None] | qz[:, None, None]
    return XI, zero


def to_full(t6: np.ndarray) -> np.ndarray:
    """Six stored components -> full symmetric 3x3 field (3, 3, ...)."""
    T = np.empty((3, 3) + t6.shape[1:], dtype=t6.dtype)
    for c, (i, j) in enumerate(PAIRS):
        T[i, j] = t6[c]
        T[j, i] = t6[c]
    return T


def from_full(T: np.ndarray) -> np.ndarray:
    return np.stack([T[i, j] for (i, j) in PAIRS])


def project_sym(tau_hat: np.ndarray, xi: np.ndarray, zero: np.ndarray) -> np.ndarray:
    """Orthogonal projection of symmetric tau^(k) onto {sym(a (x) n)}, n = xi/|xi|:

        (P tau)_ij = n_i v_j + v_i n_j - n_i n_j (n . v),  v = tau n,

    and 0 on `zero` modes. Its kernel is tau n = 0 (equilibrium of Eq.
    (equilibrium/compatibility)); its range is the compatible strains.
    """
    norm = np.sqrt(np.sum(xi * xi, axis=0))
    safe = np.where(norm > 0, norm, 1.0)
    n = xi / safe
    T = to_full(tau_hat)
    v = np.einsum("ij...,j...->i...", T, n)
    s = np.einsum("i...,i...->...", n, v)
    P = (np.einsum("i...,j...->ij...", n, v) + np.einsum("i...,j...->ij...", v, n)
         - np.einsum("i...,j...->ij...", n, n) * s)
    out = from_full(P)
    out[:, zero] = 0.0
    return out


def project_grad(zeta_hat: np.ndarray, xi: np.ndarray, zero: np.ndarray) -> np.ndarray:
    """The paper's operator on a 3x3 field zeta^(k) of shape (3, 3, ...):
    G^_ijlm = delta_im g^_jl with g^_jl = k_j k_l / |k|^2 (0 at k = 0), which
    contracts to (G^ zeta^)_ij = (zeta^ n)_i n_j."""
    norm = np.sqrt(np.sum(xi * xi, axis=0))
    safe = np.where(norm > 0, norm, 1.0)
    n = xi / safe
    zn = np.einsum("ik...,k...->i...", zeta_hat, n)
    out = np.einsum("i...,j...->ij...", zn, n)
    out[:, :, zero] = 0.0
    return out


# --------------------------------------------------------------------------
# Constitutive law (Section 4).
# --------------------------------------------------------------------------

class IsoMedium:
    """Per-voxel isotropic C(x) from bulk and shear moduli:
    sigma = K tr(eps) I + 2 mu (eps - tr(eps) I / 3)."""

    def __init__(self, K: np.ndarray, mu: np.ndarray):
        self.K = np.asarray(K, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.shape = self.K.shape

    @classmethod
    def from_labels(cls, labels: np.ndarray, phases: np.ndarray):
        ph = np.asarray(phases, dtype=np.float64)
        return cls(ph[labels, 0], ph[labels, 1])

    def stress(self, eps: np.ndarray) -> np.ndarray:
        tr = eps[0] + eps[1] + eps[2]
        lam = self.K - 2.0 * self.mu / 3.0
        s = 2.0 * self.mu * eps
        s[0:3] += lam * tr
        return s

    def voigt(self) -> np.ndarray:
        """Per-voxel 6x6 Voigt stiffness (6, 6, nz, ny, nx)."""
        lam = self.K - 2.0 * self.mu / 3.0
        C = np.zeros((6, 6) + self.shape)
        for i in range(3):
            for j in range(3):
                C[i, j] = lam
            C[i, i] = lam + 2.0 * self.mu
            C[3 + i, 3 + i] = self.mu
        return C


class AnisoMedium:
    """Per-voxel anisotropic 6x6 Voigt stiffness (stress Voigt = C . engineering strain)."""

    def __init__(self, C: np.ndarray):
        self.C = np.asarray(C, dtype=np.float64)  # (6, 6, nz, ny, nx)
        self.shape = self.C.shape[2:]

    def stress(self, eps: np.ndarray) -> np.ndarray:
        gamma = eps * FROB_W[:, None, None, None]
        return np.einsum("ij...,j...->i...", self.C, gamma)

    def voigt(self) -> np.ndarray:
        return self.C


def inner(a: np.ndarray, b: np.ndarray) -> float:
    """Frobenius inner product of two symmetric tensor fields."""
    return float(np.sum(FROB_W[:, None, None, None] * a * b))


def unit_load(a: int) -> np.ndarray:
    """Load case a (0..5): engineering-Voigt unit macro-strain as tensor components."""
    E = np.zeros(6)
    E[a] = 1.0 / FROB_W[a]
    return E


# --------------------------------------------------------------------------
# Solvers (Appendix A: G*(C:eps*) = -G*(C:E), conjugate gradients).
# --------------------------------------------------------------------------

def apply_operator(medium, p: np.ndarray, xi, zero) -> np.ndarray:
    """q = G*(C : p) with G the symmetric projection."""
    return np.real(ifft3(project_sym(fft3(medium.stress(p)), xi, zero)))


RHS_FLOOR = 1e-14


def solve_cg(medium, E: np.ndarray, tol: float = 1e-6, max_iter: int = 20000,
             nyquist: str = "component", fixed_iters: int | None = None):
    """Solve G*(C:eps*) = -G*(C:E) for the fluctuation eps* by conjugate gradients.

    x0 = 0, r0 = b = -G*(C:E), p0 = r0. Each iteration applies the operator
    once. Stops when ||r|| <= tol ||b|| (or after `fixed_iters` iterations if
    given, regardless of tol). A right-hand side at the transform's round-off
    floor, ||b|| <= RHS_FLOOR ||C:E||, counts as zero (a homogeneous box):
    eps* = 0 after 0 iterations. Returns (eps_star, iterations, ||r||/||b||).
    """
    shape = medium.shape
    xi, zero = wave_vectors(shape, nyquist)
    Ef = np.broadcast_to(E[:, None, None, None], (6,) + tuple(shape)).copy()
    tauE = medium.stress(Ef)
    b = -np.real(ifft3(project_sym(fft3(tauE), xi, zero)))
    x = np.zeros_like(b)
    r = b.copy()
    rho = inner(r, r)
    rho0 = rho
    if rho0 <= (RHS_FLOOR ** 2) * inner(tauE, tauE):
        return x, 0, 0.0
    p = r.copy()
    it = 0
    limit = fixed_iters if fixed_iters is not None else max_iter
    while it < limit:
        q = apply_operator(medium, p, xi, zero)
        alpha = rho / inner(p, q)
        x = x + alpha * p
        r = r - alpha * q
        rho_new = inner(r, r)
        it += 1
        if rho_new == 0.0 or (fixed_iters is None and np.sqrt(rho_new) <= tol * np.sqrt(rho0)):
            rho = rho_new
            break
        beta = rho_new / rho
        p = r + beta * p
        rho = rho_new
    return x, it, float(np.sqrt(rho / rho0))


def solve_cg_grad(medium, E: np.ndarray, tol: float = 1e-12, max_iter: int = 5000):
    """The same problem in the paper's nine-component form: unknown F* in the
    range of G (a displacement gradient), residual G*(C:(E + sym F*)), CG in
    the plain Frobenius product on 3x3 fields. Returns sym(F*) as six
    components. Odd grids only (no Nyquist modes)."""
    shape = medium.shape
    assert all(s % 2 == 1 for s in shape)
    xi, zero = wave_vectors(shape)

    def op(F):
        sig = medium.stress(from_full(0.5 * (F + np.swapaxes(F, 0, 1))))
        return np.real(ifft3(project_grad(fft3(to_full(sig)), xi, zero)))

    Ef = np.broadcast_to(to_full(E[:, None, None, None] * np.ones((1,) + tuple(shape))),
                         (3, 3) + tuple(shape)).copy()
    b = -op(Ef)
    x = np.zeros_like(b)
    r = b.copy()
    rho = float(np.sum(r * r))
    rho0 = rho
    if rho0 == 0.0:
        return from_full(x)
    p = r.copy()
    for _ in range(max_iter):
        q = op(p)
        alpha = rho / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        rho_new = float(np.sum(r * r))
        if np.sqrt(rho_new) <= tol * np.sqrt(rho0):
            break
        p = r + (rho_new / rho) * p
        rho = rho_new
    return from_full(0.5 * (x + np.swapaxes(x, 0, 1)))


def gamma0_apply(tau_hat: np.ndarray, xi, zero, lam0: float, mu0: float) -> np.ndarray:
    """Green operator of an isotropic reference medium (lam0, mu0) applied to tau^:
    [n (x) tau n + tau n (x) n] / (2 mu0) - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) (n.tau n) n (x) n."""
    norm = np.sqrt(np.sum(xi * xi, axis=0))
    safe = np.where(norm > 0, norm, 1.0)
    n = xi / safe
    T = to_full(tau_hat)
    v = np.einsum("ij...,j...->i...", T, n)
    s = np.einsum("i...,i...->...", n, v)
    out = ((np.einsum("i...,j...->ij...", n, v) + np.einsum("i...,j...->ij...", v, n)) / (2.0 * mu0)
           - (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)) * np.einsum("i...,j...->ij...", n, n) * s)
    o6 = from_full(out)
    o6[:, zero] = 0.0
    return o6


def solve_basic(medium, E: np.ndarray, lam0: float, mu0: float, tol: float = 1e-6,
                max_iter: int = 100000, nyquist: str = "component", fixed_iters: int | None = None):
    """Basic Lippmann-Schwinger fixed point with an isotropic reference medium
    (Moulinec and Suquet, cited in Appendix A):

        eps^{k+1}^(xi) = eps^k^(xi) - Gamma0^(xi) : sigma^k^(xi)  (xi != 0),
        eps^{k+1}^(0)  = V E.

    Stops when ||G*sigma||/||<sigma>|| <= tol (equilibrium residual in the
    symmetric projection, Frobenius norms). Returns (eps_star, iterations, residual).
    """
    shape = medium.shape
    xi, zero = wave_vectors(shape, nyquist)
    V = float(np.prod(shape))
    eps = np.broadcast_to(E[:, None, None, None], (6,) + tuple(shape)).copy()
    it = 0
    limit = fixed_iters if fixed_iters is not None else max_iter
    res = np.inf
    while True:
        sig = medium.stress(eps)
        sh = fft3(sig)
        mean_sig = np.real(sh[:, 0, 0, 0]) / V
        eq = np.real(ifft3(project_sym(sh, xi, zero)))
        den = np.sqrt(np.sum(FROB_W * mean_sig * mean_sig) * V)
        res = np.sqrt(inner(eq, eq)) / den if den > 0 else 0.0
        if it >= limit or (fixed_iters is None and res <= tol):
            break
        eh = fft3(eps) - gamma0_apply(sh, xi, zero, lam0, mu0)
        eh[:, 0, 0, 0] = E * V
        eps = np.real(ifft3(eh))
        it += 1
    return eps - E[:, None, None, None], it, float(res)


def solve_eyre_milton(medium, E: np.ndarray, lam0: float, mu0: float, tol: float = 1e-6,
                      max_iter: int = 100000, nyquist: str = "component", fixed_iters: int | None = None):
    """Accelerated fixed point of Eyre and Milton (from the FFT-scheme
    literature cited in Appendix A), in strain form with an isotropic
    reference medium C0 (lam0, mu0). With the polarization
    tau^k = (C - C0) : eps^k and the Lippmann-Schwinger residual

        B^k = E - eps^k - Gamma0 * tau^k          (Gamma0 vanishes at xi = 0),

    each iteration sets eps^{k+1} = eps^k + 2 (C + C0)^-1 C0 : B^k. The
    iterates need not be compatible; a fixed point (B = 0) is the solution
    eps = E - Gamma0 * (C - C0) eps of the basic scheme. For isotropic C (K,
    mu) and C0 (K0 = lam0 + 2 mu0 / 3, mu0) the local factor scales the
    spherical part of B by 2 K0 / (K + K0) and the deviatoric part by
    2 mu0 / (mu + mu0). The iteration that computes a residual
    ||B^k|| / ||E|| <= tol (Frobenius norms over the box) still applies its
    update and is the last. Returns (eps - E, iterations, residual)."""
    shape = medium.shape
    xi, zero = wave_vectors(shape, nyquist)
    V = float(np.prod(shape))
    K0 = lam0 + 2.0 * mu0 / 3.0
    pol = IsoMedium(medium.K - K0, medium.mu - mu0)  # tau = (C - C0) : eps
    fs = 2.0 * K0 / (medium.K + K0)
    fd = 2.0 * mu0 / (medium.mu + mu0)
    normE = np.sqrt(np.sum(FROB_W * E * E) * V)
    eps = np.broadcast_to(E[:, None, None, None], (6,) + tuple(shape)).copy()
    it = 0
    limit = fixed_iters if fixed_iters is not None else max_iter
    while True:
        q = np.real(ifft3(gamma0_apply(fft3(pol.stress(eps)), xi, zero, lam0, mu0)))
        B = E[:, None, None, None] - eps - q
        res = np.sqrt(inner(B, B)) / normE
        sph = (B[0] + B[1] + B[2]) / 3.0
        upd = fd * B
        upd[0:3] += (fs - fd) * sph
        eps = eps + upd
        it += 1
        if it >= limit or (fixed_iters is None and res <= tol):
            break
    return eps - E[:, None, None, None], it, float(res)


def eyre_milton_reference(phases):
    """Default reference medium of the accelerated scheme: the geometric means
    K0 = sqrt(K_min K_max), mu0 = sqrt(mu_min mu_max) of the phase moduli
    (the choice that gives the contraction factor (sqrt(k) - 1) / (sqrt(k) + 1)
    for a contrast k). Returns (lam0, mu0)."""
    ph = np.asarray(phases, dtype=np.float64)
    K0 = np.sqrt(ph[:, 0].min() * ph[:, 0].max())
    mu0 = np.sqrt(ph[:, 1].min() * ph[:, 1].max())
    return K0 - 2.0 * mu0 / 3.0, mu0


# --------------------------------------------------------------------------
# Averages and effective stiffness (Section 4).
# --------------------------------------------------------------------------

def voigt_strain(e6: np.ndarray) -> np.ndarray:
    return e6 * FROB_W


def homogenize_box(medium, core, tol: float = 1e-6, max_iter: int = 20000,
                   nyquist: str = "component", fixed_iters: int | None = None,
                   scheme: str = "cg", ref=None):
    """Six load cases on the buffered box, averages over the core region.

    `core` is a tuple of three slices (z, y, x) selecting Omega_R inside the box
    (Omega_B). Returns dict with Sigma, Eps (6x6, columns = load cases), C
    (raw Sigma Eps^-1), iters (6,), resid (6,).
    """
    Sig = np.zeros((6, 6))
    Eps = np.zeros((6, 6))
    iters = np.zeros(6, dtype=int)
    resid = np.zeros(6)
    for a in range(6):
        E = unit_load(a)
        if scheme == "cg":
            x, it, rr = solve_cg(medium, E, tol, max_iter, nyquist, fixed_iters)
        elif scheme == "em":
            lam0, mu0 = ref
            x, it, rr = solve_eyre_milton(medium, E, lam0, mu0, tol, max_iter, nyquist, fixed_iters)
        else:
            lam0, mu0 = ref
            x, it, rr = solve_basic(medium, E, lam0, mu0, tol, max_iter, nyquist, fixed_iters)
        eps = x + E[:, None, None, None]
        sig = medium.stress(eps)
        cs = (slice(None),) + tuple(core)
        Sig[:, a] = sig[cs].mean(axis=(1, 2, 3))
        Eps[:, a] = voigt_strain(eps[cs].mean(axis=(1, 2, 3)))
        iters[a] = it
        resid[a] = rr
    C = Sig @ np.linalg.inv(Eps)
    return dict(Sigma=Sig, Eps=Eps, C=C, iters=iters, resid=resid)


def symmetrize(C: np.ndarray) -> np.ndarray:
    return 0.5 * (C + C.T)


def stiffness_floor(phases) -> float:
    """Smallest tensor eigenvalue min(3K, 2G) over the phases."""
    ph = np.asarray(phases, dtype=np.float64)
    return float(np.min(np.minimum(3.0 * ph[:, 0], 2.0 * ph[:, 1])))


MANDEL = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])


def clip_spd(C: np.ndarray, floor: float) -> np.ndarray:
    """Symmetric Voigt stiffness C with every tensor eigenvalue below `floor`
    raised to `floor`: eigenvalues are taken in the Mandel form D C D,
    D = diag(1, 1, 1, sqrt2, sqrt2, sqrt2), an orthonormal basis of symmetric
    tensors. C is returned unchanged when no eigenvalue is below
    floor (1 - 1e-12)."""
    M = MANDEL[:, None] * C * MANDEL[None, :]
    w, V = np.linalg.eigh(M)
    if w.min() >= floor * (1.0 - 1e-12):
        return C
    Mc = (V * np.maximum(w, floor)) @ V.T
    return Mc / MANDEL[:, None] / MANDEL[None, :]


def moduli_voigt(C: np.ndarray):
    """Isotropic Voigt projection: K = (C11+C22+C33+2(C12+C13+C23))/9,
    G = (C11+C22+C33-(C12+C13+C23)+3(C44+C55+C66))/15."""
    a = C[0, 0] + C[1, 1] + C[2, 2]
    b = C[0, 1] + C[0, 2] + C[1, 2]
    c = C[3, 3] + C[4, 4] + C[5, 5]
    return (a + 2.0 * b) / 9.0, (a - b + 3.0 * c) / 15.0


def moduli_reuss(C: np.ndarray):
    """Isotropic Reuss projection from S = C^-1."""
    S = np.linalg.inv(C)
    a = S[0, 0] + S[1, 1] + S[2, 2]
    b = S[0, 1] + S[0, 2] + S[1, 2]
    c = S[3, 3] + S[4, 4] + S[5, 5]
    return 1.0 / (a + 2.0 * b), 15.0 / (4.0 * a - 4.0 * b + 3.0 * c)


def iso_voigt(K: float, mu: float) -> np.ndarray:
    return IsoMedium(np.array([[[K]]]), np.array([[[mu]]])).voigt()[:, :, 0, 0, 0]


# --------------------------------------------------------------------------
# Partition, extraction, assembly and the two-level scheme (Section 3).
# --------------------------------------------------------------------------

def extract_box(image: np.ndarray, box) -> np.ndarray:
    """Omega_B = core grown by b on every side, wrapped periodically at the image edge."""
    ox, oy, oz, nx, ny, nz, b = (int(v) for v in box)
    Nz, Ny, Nx = image.shape
    iz = np.mod(np.arange(oz - b, oz + nz + b), Nz)
    iy = np.mod(np.arange(oy - b, oy + ny + b), Ny)
    ix = np.mod(np.arange(ox - b, ox + nx + b), Nx)
    return image[np.ix_(iz, iy, ix)]


def core_slices(box):
    ox, oy, oz, nx, ny, nz, b = (int(v) for v in box)
    return (slice(b, b + nz), slice(b, b + ny), slice(b, b + nx))


def assemble_coarse(image_shape, boxes, C_list, unit: int) -> np.ndarray:
    """Coarse grid of `unit`-voxel cells; each box fills its cells with its
    symmetric stiffness. Returns (6, 6, Nz/unit, Ny/unit, Nx/unit)."""
    Nz, Ny, Nx = image_shape
    G = np.full((6, 6, Nz // unit, Ny // unit, Nx // unit), np.nan)
    for box, C in zip(boxes, C_list):
        ox, oy, oz, nx, ny, nz, _ = (int(v) for v in box)
        G[:, :, oz // unit:(oz + nz) // unit, oy // unit:(oy + ny) // unit,
          ox // unit:(ox + nx) // unit] = C[:, :, None, None, None]
    assert not np.isnan(G).any(), "partition does not tile the image"
    return G


def homogenize_direct(image, phases, tol=1e-6, max_iter=20000, nyquist="component",
                      fixed_iters=None):
    """Brute-force solve of the whole image (Section 5, the reference M_N)."""
    med = IsoMedium.from_labels(image, phases)
    core = (slice(None),) * 3
    res = homogenize_box(med, core, tol, max_iter, nyquist, fixed_iters)
    Cs = symmetrize(res["C"])
    K, G = moduli_voigt(Cs)
    KR, GR = moduli_reuss(Cs)
    res.update(C_sym=Cs, K=K, G=G, K_reuss=KR, G_reuss=GR)
    return res


def homogenize_hierarchical(image, phases, boxes, unit, tol=1e-6, max_iter=20000,
                            nyquist="component", fixed_iters=None, level2_fixed_iters=None):
    """Two-level hierarchical homogenization (Section 3, Fig. 2; Section 4).

    Level 1: every box (core + buffer, periodic) -> C_R = Sigma Eps^-1 over its
    core. Assembly: symmetric C_R fills the box's coarse cells. Level 2: the
    anisotropic coarse image is homogenized once more (no buffer). Also the
    core-volume-weighted arithmetic mean (AM) of the subimage moduli.
    """
    boxes = np.asarray(boxes)
    per_box = []
    Cs = []
    Ks, Gs, w = [], [], []
    cmin = stiffness_floor(phases)
    clipped = 0
    for box in boxes:
        sub = extract_box(image, box)
        med = IsoMedium.from_labels(sub, phases)
        r = homogenize_box(med, core_slices(box), tol, max_iter, nyquist, fixed_iters)
        per_box.append(r)
        C = symmetrize(r["C"])
        Cc = clip_spd(C, cmin)
        clipped += int(Cc is not C)
        Cs.append(Cc)
        k, g = moduli_voigt(C)
        Ks.append(k)
        Gs.append(g)
        w.append(float(box[3]) * box[4] * box[5])
    coarse = assemble_coarse(image.shape, boxes, Cs, unit)
    med2 = AnisoMedium(coarse)
    res2 = homogenize_box(med2, (slice(None),) * 3, tol, max_iter, nyquist, level2_fixed_iters)
    Ceff = symmetrize(res2["C"])
    K, G = moduli_voigt(Ceff)
    KR, GR = moduli_reuss(Ceff)
    w = np.array(w)
    return dict(C=res2["C"], C_sym=Ceff, K=K, G=G, K_reuss=KR, G_reuss=GR,
                K_am=float(np.sum(w * Ks) / w.sum()), G_am=float(np.sum(w * Gs) / w.sum()),
                per_box=per_box, C_boxes=np.array(Cs), coarse=coarse, level2=res2, n_clipped=clipped)


def uniform_boxes(shape, n: int, b: int) -> np.ndarray:
    """Cubic cores of edge n tiling an image of the given (z, y, x) shape,
    each with buffer b; rows (ox, oy, oz, nx, ny, nz, b), x fastest."""
    Nz, Ny, Nx = shape
    assert Nz % n == 0 and Ny % n == 0 and Nx % n == 0
    return np.array([(i * n, j * n, k * n, n, n, n, b) for k in range(Nz // n) for j in range(Ny // n)
                     for i in range(Nx // n)], dtype=np.int64)


def extract_field(C: np.ndarray, box) -> np.ndarray:
    """extract_box for a stiffness field (6, 6, Z, Y, X): the buffered box with
    periodic wrap."""
    ox, oy, oz, nx, ny, nz, b = (int(v) for v in box)
    Nz, Ny, Nx = C.shape[2:]
    iz = np.mod(np.arange(oz - b, oz + nz + b), Nz)
    iy = np.mod(np.arange(oy - b, oy + ny + b), Ny)
    ix = np.mod(np.arange(ox - b, ox + nx + b), Nx)
    return C[:, :, iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def homogenize_multilevel(image, phases, levels, tol=1e-6, max_iter=20000, nyquist="component",
                          fixed_iters=None):
    """Hierarchical homogenization repeated over several levels (Section 3:
    the renormalisation is applied repeatedly until the image is small).
    levels = [(n1, b1), (n2, b2), ...]: level 1 cuts the label image into
    n1-cubes with buffer b1 and assembles the symmetric stiffnesses (raised
    to the stiffness floor) into a coarse anisotropic image; every further
    level does the same to the previous coarse image with (n_k, b_k); the last
    coarse image is solved whole."""
    cmin = stiffness_floor(phases)
    n1, b1 = levels[0]
    Cs = []
    for box in uniform_boxes(image.shape, n1, b1):
        med = IsoMedium.from_labels(extract_box(image, box), phases)
        r = homogenize_box(med, core_slices(box), tol, max_iter, nyquist, fixed_iters)
        Cs.append(clip_spd(symmetrize(r["C"]), cmin))
    coarse = assemble_coarse(image.shape, uniform_boxes(image.shape, n1, b1), Cs, n1)
    coarses = [coarse]
    for n, b in levels[1:]:
        shape = coarse.shape[2:]
        boxes = uniform_boxes(shape, n, b)
        Cs = []
        for box in boxes:
            r = homogenize_box(AnisoMedium(extract_field(coarse, box)), core_slices(box), tol, max_iter, nyquist,
                               fixed_iters)
            Cs.append(clip_spd(symmetrize(r["C"]), cmin))
        coarse = assemble_coarse(shape, boxes, Cs, n)
        coarses.append(coarse)
    res = homogenize_box(AnisoMedium(coarse), (slice(None),) * 3, tol, max_iter, nyquist, fixed_iters)
    Ceff = symmetrize(res["C"])
    K, G = moduli_voigt(Ceff)
    KR, GR = moduli_reuss(Ceff)
    return dict(C=res["C"], C_sym=Ceff, K=K, G=G, K_reuss=KR, G_reuss=GR, coarse=coarses)


# --------------------------------------------------------------------------
# Correlation length (Section 2, Eq. eq_correlation) and the subimage size.
# --------------------------------------------------------------------------

def correlation_counts(image, pore_label: int, lmax: int):
    """Pair counts of the material indicator M = [label != pore_label]
    (mineral 1, pore 0) along x, y, z: count[a][l] = sum of M(v) M(v + l e_a)
    over the voxel pairs that lie inside the image, l = 0..lmax (integers)."""
    M = (np.asarray(image) != pore_label).astype(np.int64)
    out = np.zeros((3, lmax + 1), dtype=np.int64)
    for a, axis in enumerate((2, 1, 0)):  # x, y, z
        n = M.shape[axis]
        for l in range(min(lmax, n - 1) + 1):
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[axis] = slice(0, n - l)
            hi[axis] = slice(l, n)
            out[a, l] = int(np.sum(M[tuple(lo)] * M[tuple(hi)]))
    return out


def correlation_function(image, pore_label: int, lmax: int):
    """Corr_a(l) = (<M(v) M(v + l e_a)> - <M>^2) / (<M^2> - <M>^2), the pair
    average over the pairs inside the image, <M> and <M^2> = <M> over all
    voxels. Returns (3, lmax + 1)."""
    M = (np.asarray(image) != pore_label)
    m = float(M.mean())
    counts = correlation_counts(image, pore_label, lmax)
    corr = np.zeros((3, lmax + 1))
    Nz, Ny, Nx = M.shape
    for a, n in enumerate((Nx, Ny, Nz)):
        other = M.size // n
        for l in range(min(lmax, n - 1) + 1):
            pairs = (n - l) * other
            corr[a, l] = (counts[a, l] / pairs - m * m) / (m - m * m)
    return corr


def fit_correlation_length(corr_l):
    """xi of the least-squares fit of exp(-l / xi) to corr(l) over l = 0 up to
    the first l where corr drops below 0.05 (the paper's range of useful
    correlation), by golden-section search on xi in (0.01, 1e4)."""
    c = np.asarray(corr_l, dtype=np.float64)
    below = np.flatnonzero(c < 0.05)
    L = int(below[0]) if below.size else len(c) - 1
    L = max(L, 1)
    l = np.arange(L + 1, dtype=np.float64)
    f = lambda lx: float(np.sum((c[:L + 1] - np.exp(-l / np.exp(lx))) ** 2))
    a, b = np.log(0.01), np.log(1e4)
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = f(x1), f(x2)
    for _ in range(200):
        if f1 < f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - g * (b - a)
            f1 = f(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (b - a)
            f2 = f(x2)
    return float(np.exp(0.5 * (a + b)))


# --------------------------------------------------------------------------
# Power law in 1/n and Richardson extrapolation (Section 5, Eq. fit_power_law).
# --------------------------------------------------------------------------

def fit_inverse_n(ns, M):
    """Ordinary least squares of M(n) = M_inf + C / n. Returns (M_inf, C)."""
    ns = np.asarray(ns, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    A = np.stack([np.ones_like(ns), 1.0 / ns], axis=1)
    sol, *_ = np.linalg.lstsq(A, M, rcond=None)
    return float(sol[0]), float(sol[1])


# --------------------------------------------------------------------------
# Choice of subimage edge and buffer (Section 2, Section 3 Eq. 2, Section 5).
# --------------------------------------------------------------------------

def largest_prime_factor(m: int) -> int:
    """Trial division (m >= 1; 1 for m = 1)."""
    p, big = 2, 1
    while p * p <= m:
        while m % p == 0:
            big, m = p, m // p
        p += 1
    return max(big, m) if m > 1 else big


def plan_partition(shape, n_min: int, bs, c_rel, a: float, eps: float):
    """Every candidate (n, b) written out and the best one picked.

    n runs over the common divisors of the image edges with n >= n_min
    (Section 2: subimages of at least 3 xi), b over the buffers whose fitted
    constant is known, skipping buffered edges n + 2b with a prime factor
    above 31 (FFT lengths the solver does not take). Predicted relative
    error: c_rel / n (Section 5, the C / n term of Eq. fit_power_law, one
    constant per buffer width as in Table fit_pad). Predicted cost: the
    number of subimages (N/n)^3 times the single-solve time of a box of edge
    n + 2b, taken as (n + 2b)^a (Section 3, Eq. 2 with the buffered box).
    Rule: cheapest among those meeting eps (ties: smaller error, larger n,
    smaller b); if none meets eps, least error (ties: cheaper).
    Returns (n, b, err, cost, met, table) with table the list of all
    candidates as (n, b, err, cost)."""
    nz, ny, nx = shape
    V = float(nx) * float(ny) * float(nz)
    table = []
    for n in range(max(n_min, 1), min(nx, ny, nz) + 1):
        if nx % n or ny % n or nz % n:
            continue
        for b, c in zip(bs, c_rel):
            if largest_prime_factor(n + 2 * b) > 31:
                continue
            table.append((n, int(b), c / n, V / float(n) ** 3 * float(n + 2 * b) ** a))
    if not table:
        raise ValueError("no candidate: no edge n >= n_min divides the image with a supported box")
    met = [t for t in table if t[2] <= eps]
    if met:
        best = min(met, key=lambda t: (t[3], t[2], -t[0], t[1]))
    else:
        best = min(table, key=lambda t: (t[2], t[3], -t[0], t[1]))
    return best[0], best[1], best[2], best[3], bool(met), table
