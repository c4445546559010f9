"""Seeded synthetic inputs for block lower triangular Toeplitz (BLTT) all-at-once systems.

This module defines *problems*, not the solver: the block coefficients of the BLTT matrix that a
time discretisation produces (Sec. 5: backward Euler / Crank-Nicolson heat equations, the L1
scheme for the time-fractional sub-diffusion equation) and seeded right-hand sides.  It holds none
of the solver's arithmetic (no transforms, no preconditioner, no Krylov recurrences).  Both the
CPU oracle and the CUDA path take their inputs from here, so neither depends on the other.

Conventions (Sec. 5 and Sec. 2):
  * every block is A_(k) = a_k I + b_k L, with L = -Delta_h the SPD finite-difference Dirichlet
    Laplacian on a uniform grid with m interior points per axis, h = length/(m+1);
  * unknowns are time-major: u[n*M + i], n = 0..N-1 the time step, i the lexicographic spatial
    index with x fastest; M = m**d.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "l1_weights", "fractional_problem", "heat_bdf_problem", "heat_cn_problem",
    "heat_cn_varcoeff_problem", "fractional_varcoeff_problem", "nonlocal_diffusion_problem",
    "commuting_blocks_problem",
    "paper_data_fractional", "paper_data_frac_var", "paper_data_heat_var",
    "rhs_uniform", "rhs_smoothed_field", "WORKLOADS", "workload", "batched_systems",
    "alpha_training_problems",
]


@dataclass
class Problem:
    """One BLTT system A u = f with blocks A_(k) = a[k] I + b[k] L (eq. amatdef)."""
    N: int                      # number of time steps (blocks per block row)
    d: int                      # spatial dimension (1, 2 or 3)
    m: tuple                    # interior points per axis, length d
    h: tuple                    # grid spacing per axis, length d
    a: np.ndarray               # (N,) identity coefficients of the blocks
    b: np.ndarray               # (N,) Laplacian coefficients of the blocks
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(np.prod(self.m))

    @property
    def n(self) -> int:
        return self.N * self.M


def l1_weights(gamma: float, N: int) -> np.ndarray:
    """L1-scheme weights l_k^(gamma), k = 0..N-1 (Sec. 5.2, the L1 discretisation).

    l_0 = 1/Gamma(2-gamma);  l_k = [(k+1)^(1-gamma) - 2 k^(1-gamma) + (k-1)^(1-gamma)]/Gamma(2-gamma).
    At k = 1 the term 0^(1-gamma) is taken as 0 for every gamma in (0, 1]; this is also its
    gamma -> 1 limit, under which the weights become (1, -1, 0, ...), the backward-Euler ones.
    """
    if not (0.0 < gamma <= 1.0):
        raise ValueError("gamma must lie in (0, 1]")
    p = 1.0 - gamma
    k = np.arange(N, dtype=np.float64)

    def pw(x):
        out = np.zeros_like(x)
        pos = x > 0
        out[pos] = x[pos] ** p
        return out

    g = math.gamma(2.0 - gamma)
    l = (pw(k + 1) - 2.0 * pw(k) + pw(k - 1)) / g
    l[0] = 1.0 / g
    return l


def _grid(d, m, length):
    m = tuple([m] * d) if np.isscalar(m) else tuple(m)
    if len(m) != d:
        raise ValueError("m must have d entries")
    h = tuple(length / (mi + 1) for mi in m)
    return m, h


def fractional_problem(d, m, N, gamma, T=1.0, length=1.0, name=None) -> Problem:
    """L1-scheme time-fractional sub-diffusion: A_(0) = l_0/tau^g I + L, A_(k) = l_k/tau^g I."""
    m, h = _grid(d, m, length)
    tau = T / N
    a = l1_weights(gamma, N) / tau ** gamma
    b = np.zeros(N)
    b[0] = 1.0
    return Problem(N, d, m, h, a, b, name or f"frac{d}d_N{N}_m{m[0]}_g{gamma}",
                   dict(kind="fractional", gamma=gamma, tau=tau))


def heat_bdf_problem(d, m, N, T=1.0, length=1.0, name=None) -> Problem:
    """Backward-Euler heat equation: A_(0) = I/tau + L, A_(1) = -I/tau (Sec. 5.1, BDF)."""
    m, h = _grid(d, m, length)
    tau = T / N
    a = np.zeros(N)
    a[0] = 1.0 / tau
    if N > 1:
        a[1] = -1.0 / tau
    b = np.zeros(N)
    b[0] = 1.0
    return Problem(N, d, m, h, a, b, name or f"heat{d}d_bdf_N{N}_m{m[0]}",
                   dict(kind="heat_bdf", gamma=1.0, tau=tau))


def heat_cn_problem(d, m, N, T=1.0, length=1.0, name=None) -> Problem:
    """Crank-Nicolson heat equation: A_(0) = I/tau + L/2, A_(1) = -I/tau + L/2 (Sec. 5.1, CN)."""
    m, h = _grid(d, m, length)
    tau = T / N
    a = np.zeros(N)
    b = np.zeros(N)
    a[0], b[0] = 1.0 / tau, 0.5
    if N > 1:
        a[1], b[1] = -1.0 / tau, 0.5
    return Problem(N, d, m, h, a, b, name or f"heat{d}d_cn_N{N}_m{m[0]}",
                   dict(kind="heat_cn", gamma=1.0, tau=tau))


def heat_cn_varcoeff_problem(m, N, T=1.0, name=None) -> Problem:
    """Crank-Nicolson heat equation with the variable coefficient of the paper's Example
    heateqvarcoeff: d = 2, Omega = (0,1)^2, a(x) = (20 + x_1^2)(20 + x_2^2).  Blocks
    A_(0) = I/tau + L_a/2, A_(1) = -I/tau + L_a/2 with L_a = -Delta_{a,h} (eq.
    cnheatvarcoeff_tssystem); meta["faces"] holds a at the cell faces along x and y (arrays
    (m, m+1) and (m+1, m), y-major), meta["abar"] the mean of a over the interior grid points
    (the preconditioner's constant coefficient, eq. meancoeffheateqtsmat)."""
    p = heat_cn_problem(2, m, N, T=T)
    mm = p.m[0]
    h = p.h[0]
    pts = (np.arange(mm) + 1.0) * h                   # interior points
    fcs = (np.arange(mm + 1) + 0.5) * h               # faces: before point f, and after the last
    coef = lambda x1, x2: (20.0 + x1 ** 2) * (20.0 + x2 ** 2)
    fx = coef(fcs[None, :], pts[:, None])             # rows y, columns x faces: (m, m+1)
    fy = coef(pts[None, :], fcs[:, None])             # rows y faces, columns x: (m+1, m)
    abar = float(np.mean(coef(pts[None, :], pts[:, None])))
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name or f"heat2d_cnvar_N{N}_m{mm}",
                   dict(kind="heat_cn_var", gamma=1.0, tau=p.meta["tau"], faces=(fx, fy),
                        abar=abar))


def fractional_varcoeff_problem(m, N, gamma, name=None) -> Problem:
    """The paper's Example 4 (Sec. 5.2): L1 time-fractional blocks (as fractional_problem, d = 2,
    Omega = (0,1)^2, T = 1) with the variable coefficient a(x, y) = 35 + x^3.5 + y^3.5, i.e. the
    blocks a_k I + b_k L_a with L_a = -Delta_{a,h}.  meta["faces"] holds a at the cell faces along
    x and y (arrays (m, m+1) and (m+1, m), y-major), meta["abar"] the mean of a over the interior
    grid points (the preconditioner's constant coefficient)."""
    p = fractional_problem(2, m, N, gamma)
    mm, h = p.m[0], p.h[0]
    pts = (np.arange(mm) + 1.0) * h
    fcs = (np.arange(mm + 1) + 0.5) * h
    coef = lambda x1, x2: 35.0 + x1 ** 3.5 + x2 ** 3.5
    fx = coef(fcs[None, :], pts[:, None])
    fy = coef(pts[None, :], fcs[:, None])
    abar = float(np.mean(coef(pts[None, :], pts[:, None])))
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name or f"fracvar2d_N{N}_m{mm}_g{gamma}",
                   dict(p.meta, kind="fractional_var", faces=(fx, fy), abar=abar))


def nonlocal_diffusion_problem(m, N, gamma, delta_cells=3.0, name=None) -> Problem:
    """The L1 time-fractional blocks of fractional_problem (d = 2, Omega = (0,1)^2) with a dense
    non-local spatial operator K in place of -Delta_h: the blocks become a_k I + b_k K, which
    commute (Sec. 3).  K is the volume-constrained non-local diffusion operator with the Gaussian
    kernel J(r) = C exp(-r^2/delta^2), u = 0 outside the domain:
      (K u)_i = C pi delta^2 u_i - h^2 sum_j J(|x_i - x_j|) u_j,
    C = 4/(pi delta^4) so that K u -> -Delta u for smooth u as delta -> 0, delta = delta_cells h.
    K is dense (every pair of grid points interacts) and SPD.  meta["K"]: the M x M matrix."""
    p = fractional_problem(2, m, N, gamma)
    mm, h = p.m[0], p.h[0]
    delta = delta_cells * h
    C = 4.0 / (math.pi * delta ** 4)
    pts = (np.arange(mm) + 1.0) * h
    # the Gaussian separates over the axes: J(|x_i - x_j|) = C E[iy, jy] E[ix, jx] (x fastest)
    E = np.exp(-((pts[:, None] - pts[None, :]) / delta) ** 2)
    K = np.kron(E, E)
    K *= -(h * h * C)
    K[np.diag_indices_from(K)] += C * math.pi * delta * delta
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name or f"nonlocal2d_N{N}_m{mm}_g{gamma}",
                   dict(p.meta, kind="nonlocal", K=K, delta=delta))


def commuting_blocks_problem(M, N, seed=0, kind="modal", T=1.0, name=None) -> Problem:
    """General commuting symmetric blocks (Assumption 1 (i), Sec. 3): A_(k) = U diag(lam_k) U^T
    with one orthonormal U for every block, not tied to a grid or a single operator.

    U is the Q factor of a seeded Gaussian M x M matrix (default_rng(seed)).  lam[k, i] is the
    eigenvalue of A_(k) on column i of U:
      kind "modal": every eigenmode carries its own L1 time-fractional order and diffusion rate,
        lam[0, i] = l_0^(g_i)/tau^(g_i) + nu_i, lam[k, i] = l_k^(g_i)/tau^(g_i) (k >= 1), with
        g_i ~ U[0.3, 0.9] and log10 nu_i ~ U[0, 3];
      kind "poly": blocks a_k I + b_k K + c_k K^2 of one SPD K = U diag(nu) U^T (L1 weights
        of order 0.6 in a, b = e_0, c = 1e-3 e_0: a fourth-order term in the first block).
    Assumption 1 (ii) holds for both (the L1 weights' sums are positive, nu > 0).  meta["U"],
    meta["lam"] are what the library takes; meta["blocks"] holds the (N, M, M) matrices the
    oracle works from.  The grid fields describe a 1-D line of M points (unused by the blocks)."""
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((M, M)))
    U = Q * np.sign(np.diag(R))[None, :]
    tau = T / N
    nu = 10.0 ** rng.uniform(0.0, 3.0, M)
    if kind == "modal":
        g = rng.uniform(0.3, 0.9, M)
        lam = np.stack([l1_weights(gi, N) / tau ** gi for gi in g], axis=1)
        lam[0] += nu
    elif kind == "poly":
        a = l1_weights(0.6, N) / tau ** 0.6
        lam = np.repeat(a[:, None], M, axis=1)
        lam[0] += nu + 1e-3 * nu ** 2
    else:
        raise ValueError(kind)
    blocks = np.einsum("ij,kj,lj->kil", U, lam, U)
    blocks = 0.5 * (blocks + np.transpose(blocks, (0, 2, 1)))
    m, h = _grid(1, M, 1.0)
    return Problem(N, 1, m, h, np.zeros(N), np.zeros(N), name or f"commuting_{kind}_N{N}_M{M}_s{seed}",
                   dict(kind="commuting", U=U, lam=lam, blocks=blocks, tau=tau))


def paper_data_fractional(prob, gamma: float) -> np.ndarray:
    """Right-hand side of the paper's non-local Example 3 (Sec. 5.2: Omega = (0, pi)^2, T = 1,
    u = sin x sin y t^2, a = 1): f(x, y, t_n) = sin x sin y [2 t^(2-gamma)/Gamma(3-gamma) + 2 t^2]
    at the interior grid points and t_n = n tau, n = 1..N (u_0 = 0 adds nothing)."""
    import math
    m, h, N = prob.m[0], prob.h[0], prob.N
    x = (np.arange(m) + 1.0) * h
    S = np.outer(np.sin(x), np.sin(x)).reshape(-1)
    t = (np.arange(N) + 1.0) / N
    ft = 2.0 * t ** (2.0 - gamma) / math.gamma(3.0 - gamma) + 2.0 * t ** 2
    return (ft[:, None] * S[None, :]).reshape(-1)


def paper_data_frac_var(prob, gamma: float) -> np.ndarray:
    """Right-hand side of the paper's Example 4 (Sec. 5.2; the example writes alpha for the
    fractional order gamma): u = sin(pi x) sin(pi y) t^2 and a = 35 + x^3.5 + y^3.5 give
    f = sin(pi x) sin(pi y) [2 t^(2-gamma)/Gamma(3-gamma) + 2 pi^2 a t^2]
        - pi t^2 [a_x cos(pi x) sin(pi y) + a_y sin(pi x) cos(pi y)],
    a_x = 3.5 x^2.5, a_y = 3.5 y^2.5, at the interior grid points and t_n = n tau, n = 1..N
    (u_0 = 0 adds nothing)."""
    m, h, N = prob.m[0], prob.h[0], prob.N
    x = (np.arange(m) + 1.0) * h
    X, Y = np.meshgrid(x, x)                          # rows y, columns x: x fastest
    a = 35.0 + X ** 3.5 + Y ** 3.5
    S = np.sin(np.pi * X) * np.sin(np.pi * Y)
    G = np.pi * (3.5 * X ** 2.5 * np.cos(np.pi * X) * np.sin(np.pi * Y)
                 + 3.5 * Y ** 2.5 * np.sin(np.pi * X) * np.cos(np.pi * Y))
    t = (np.arange(N) + 1.0) / N
    c = 2.0 * t ** (2.0 - gamma) / math.gamma(3.0 - gamma)
    F = c[:, None] * S.reshape(-1)[None, :] + (t * t)[:, None] * (2 * np.pi ** 2 * a * S - G).reshape(-1)[None, :]
    return F.reshape(-1)


def paper_data_heat_var(prob):
    """Data of the paper's Example heateqvarcoeff on the interior grid (x fastest): the source
    f(x, t_{n-1/2}), n = 1..N, as an (N, M) array, and u_0 as an (M,) array.  f is the one of the
    exact solution u = e^t x_1(1-x_1) x_2(1-x_2) for a = (20 + x_1^2)(20 + x_2^2) (the printed f
    has (20 + x_2^2) in its third term, where the exact solution gives (20 + x_1^2))."""
    m, h, N = prob.m[0], prob.h[0], prob.N
    x = (np.arange(m) + 1.0) * h
    X1, X2 = np.meshgrid(x, x)                        # X1 along rows' entries: x fastest
    a = (20.0 + X1 ** 2) * (20.0 + X2 ** 2)
    s = X1 * (1 - X1) * X2 * (1 - X2)
    g = (s - 2 * X1 * (20 + X2 ** 2) * (1 - 2 * X1) * X2 * (1 - X2)
         - 2 * X2 * (20 + X1 ** 2) * (1 - 2 * X2) * X1 * (1 - X1)
         + 2 * a * (X1 * (1 - X1) + X2 * (1 - X2))).reshape(-1)
    t = (np.arange(N) + 0.5) / N
    return np.exp(t)[:, None] * g[None, :], s.reshape(-1)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Seeded U[-1, 1] right-hand side of length n (float64)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def rhs_smoothed_field(N: int, d: int, m, seed: int, sigma: float = 2.0) -> np.ndarray:
    """Seeded Gaussian-smoothed random field, one independent field per time slice.

    iid N(0,1) per grid point, separable Gaussian smoothing in space (sigma grid cells,
    truncated at 3 sigma, zero outside the domain), normalised to unit RMS over the whole vector.
    """
    from scipy.ndimage import gaussian_filter1d
    m = tuple([m] * d) if np.isscalar(m) else tuple(m)
    rng = np.random.default_rng(seed)
    shape = (N,) + tuple(reversed(m))          # (time, z, y, x): x fastest
    f = rng.standard_normal(shape)
    for ax in range(1, f.ndim):
        gaussian_filter1d(f, sigma, axis=ax, mode="constant", cval=0.0, truncate=3.0, output=f)
    f /= np.sqrt(np.mean(f * f))
    return f.reshape(-1)


# Named workloads, each with its sizes.  A workload bundles a problem, its right-hand-side recipe
# and the seed; the solver tolerance is 1e-8 relative residual throughout.
def _w_frac1d():
    p = fractional_problem(1, 63, 64, 0.5)
    return p, (lambda: rhs_uniform(p.n, 1))


def _w_frac2d():
    p = fractional_problem(2, 255, 1024, 0.7)
    return p, (lambda: rhs_uniform(p.n, 2))


def _w_heat3d():
    p = heat_bdf_problem(3, 127, 256)
    return p, (lambda: rhs_smoothed_field(p.N, 3, p.m, 3))


WORKLOADS = {
    "frac1d_N64_m63_g0.5": _w_frac1d,      # 1-D L1 fractional, 4,032 unknowns
    "frac2d_N1024_m255_g0.7": _w_frac2d,   # 2-D L1 fractional, 66,585,600 unknowns
    "heat3d_bdf_N256_m127": _w_heat3d,     # 3-D backward-Euler heat, 524,386,048 unknowns
}


def workload(name: str):
    """Return (Problem, rhs_factory) for a named workload."""
    return WORKLOADS[name]()


_BATCH_N = (128, 256, 512, 1024, 2048)
_BATCH_SPACE = ((1, 127), (2, 63), (2, 127), (2, 255))   # M = 127, 63^2, 127^2, 255^2


def batched_systems(nsys: int = 96, nrhs: int = 4, seed: int = 4, scale: float = 1.0):
    """Mixed batch of L1 fractional systems with uneven N and M, nrhs seeded U[-1,1] RHS each.

    Draws N from {128,...,2048}, the space from {1-D m=127, 2-D m=63, 127, 255} and
    gamma ~ U[0.2, 0.9] from default_rng(seed); RHS r of system s uses seed + 1000 s + r.
    `scale` < 1 shrinks N (never below 8) for reduced test batches.
    Returns a list of (Problem, [rhs factories]).
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys):
        N = int(rng.choice(_BATCH_N))
        d, m = _BATCH_SPACE[int(rng.integers(len(_BATCH_SPACE)))]
        gamma = float(rng.uniform(0.2, 0.9))
        if scale != 1.0:
            N = max(8, int(N * scale))
        p = fractional_problem(d, m, N, gamma, name=f"batch{s}_{d}d_N{N}_m{m}_g{gamma:.3f}")
        rhs = [(lambda p=p, r=r, s=s: rhs_uniform(p.n, seed + 1000 * s + r)) for r in range(nrhs)]
        out.append((p, rhs))
    return out


def alpha_training_problems(count: int, seed: int = 5):
    """Problems for learning alpha: half 1-D L1 fractional, half 3-D backward-Euler heat.

    1-D fractional: m in {31, 63, 127, 255}, N in {32, ..., 1024}, gamma ~ U[0.2, 0.9].
    3-D heat:       m in {15, 31, 63},       N in {32, ..., 256}  (gamma := 1 as a feature).
    Each comes with a seeded U[-1,1] right-hand side.  Returns a list of (Problem, rhs_factory).
    """
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        if j % 2 == 0:
            m = int(rng.choice((31, 63, 127, 255)))
            N = int(rng.choice((32, 64, 128, 256, 512, 1024)))
            gamma = float(rng.uniform(0.2, 0.9))
            p = fractional_problem(1, m, N, gamma)
        else:
            m = int(rng.choice((15, 31, 63)))
            N = int(rng.choice((32, 64, 128, 256)))
            p = heat_bdf_problem(3, m, N)
        sd = int(rng.integers(1 << 30))
        out.append((p, (lambda p=p, sd=sd: rhs_uniform(p.n, sd))))
    return out
