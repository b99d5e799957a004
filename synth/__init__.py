"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the sweeping method itself: only velocity
fields c(x), right-hand sides f(x) and receiver/source placements, evaluated on
the interior grid p_{i,j} = (i h, j h), 1 <= i, j <= n, h = 1/(n+1) (Section 2.1).

Arrays are laid out row by row, x1 fastest: a field is an (n, n) array F with
F[j-1, i-1] = F(i h, j h), matching the unknown ordering of Section 2.1.

The paper's own velocity fields are only pictured (Section 3), so these are
stand-ins with the same character: a converging Gaussian lens, a random smooth
medium and point/Gaussian sources.
"""
import numpy as np

__all__ = [
    "grid", "velocity_constant", "velocity_lens", "smooth_noise", "velocity_random",
    "source_gaussian", "source_delta", "source_positions", "workload",
]


def grid(n):
    """Node coordinates x = (k+1) h, k = 0..n-1, and the spacing h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    return (np.arange(n, dtype=np.float64) + 1.0) * h, h


def velocity_constant(n, c0=1.0):
    return np.full((n, n), float(c0))


def velocity_lens(n):
    """Converging Gaussian lens c = (4/3)(1 - 0.5 exp(-32 |x - (0.5, 0.5)|^2))."""
    x, _ = grid(n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    r2 = (X1 - 0.5) ** 2 + (X2 - 0.5) ** 2
    return (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * r2))


def _gauss_filter_1d(n, h, width):
    """Truncated (4 width) Gaussian taps of standard deviation `width` (physical units)."""
    rad = int(np.ceil(4.0 * width / h))
    t = np.arange(-rad, rad + 1) * h
    return np.exp(-0.5 * (t / width) ** 2)


def smooth_noise(n, width, seed):
    """Unit-std smooth field: i.i.d. N(0,1) on the nodes, separable Gaussian filter
    with zero padding, divided by its population standard deviation."""
    rng = np.random.default_rng(seed)
    g0 = rng.standard_normal((n, n))
    _, h = grid(n)
    k = _gauss_filter_1d(n, h, width)
    rad = (k.size - 1) // 2

    def conv(v):  # zero-padded, centred, length n even when the taps outnumber v
        return np.convolve(v, k, mode="full")[rad:rad + n]

    g = np.apply_along_axis(conv, 1, g0)
    g = np.apply_along_axis(conv, 0, g)
    return g / g.std()


def velocity_random(n, width, seed, amp=0.2):
    """Random smooth medium c = 1 + amp * g."""
    return 1.0 + amp * smooth_noise(n, width, seed)


def velocity_linear_x2(n, c0=0.5, slope=1.0):
    """c(x1, x2) = c0 + slope * x2 (rows are x2, columns x1)."""
    x, _ = grid(n)
    return np.tile((c0 + slope * x)[:, None], (1, n))


def velocity_waveguide(n):
    """A vertical waveguide with a Gaussian cross section: c = (4/3)(1 - 0.5 exp(-32 (x1 - 1/2)^2)),
    constant along x2 (the same profile as velocity_lens, in x1 only)."""
    x, _ = grid(n)
    row = (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * (x - 0.5) ** 2))
    return np.tile(row[None, :], (n, 1))


def velocity_random_modes(n, seed=7, kmax=8, amp=0.2):
    """A random smooth medium that is the same function of x on every grid (for tables over
    n): c = 1 + amp * g / gmax, g = sum_{j,k <= kmax} a_jk cos(pi j x1 + p_jk) cos(pi k x2 + q_jk),
    a_jk ~ N(0, 1) / (1 + j^2 + k^2), phases uniform, gmax = max |g| on the 255 x 255 grid."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((kmax + 1, kmax + 1))
    j = np.arange(kmax + 1)
    a = a / (1.0 + j[:, None] ** 2 + j[None, :] ** 2)
    ph = rng.uniform(0, 2 * np.pi, (2, kmax + 1, kmax + 1))

    def g_on(m):
        x, _ = grid(m)
        g = np.zeros((m, m))
        for jj in range(kmax + 1):
            for kk in range(kmax + 1):
                g += a[jj, kk] * np.cos(np.pi * jj * x[None, :] + ph[0, jj, kk]) * np.cos(np.pi * kk * x[:, None] + ph[1, jj, kk])
        return g

    return 1.0 + amp * g_on(n) / np.abs(g_on(255)).max()


def source_wavepacket(n, center, direction, k, sigma):
    """Gaussian wave packet exp(-|x - x0|^2 / (2 sigma^2)) exp(i k d.(x - x0)), d the unit
    vector along `direction` (complex128)."""
    x, _ = grid(n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    r1, r2 = X1 - center[0], X2 - center[1]
    return np.exp(-(r1 * r1 + r2 * r2) / (2.0 * sigma * sigma) + 1j * k * (d[0] * r1 + d[1] * r2))


def source_gaussian(n, center=(0.5, 0.5), sigma=1.0 / 64.0):
    """Unnormalised Gaussian f = exp(-|x - x0|^2 / (2 sigma^2)) (complex128)."""
    x, _ = grid(n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    r2 = (X1 - center[0]) ** 2 + (X2 - center[1]) ** 2
    return np.exp(-r2 / (2.0 * sigma * sigma)).astype(np.complex128)


def _nearest_node(n, t):
    _, h = grid(n)
    k = int(np.floor(t / h + 0.5)) - 1
    return min(max(k, 0), n - 1)


def source_delta(n, point):
    """Discrete delta of mass one: 1/h^2 at the node nearest to `point`."""
    _, h = grid(n)
    f = np.zeros((n, n), dtype=np.complex128)
    f[_nearest_node(n, point[1]), _nearest_node(n, point[0])] = 1.0 / (h * h)
    return f


def source_positions(n, count, pml_width, seed):
    """`count` points uniform in [eta, 1 - eta]^2 with eta = pml_width * h."""
    _, h = grid(n)
    eta = pml_width * h
    rng = np.random.default_rng(seed)
    return rng.uniform(eta, 1.0 - eta, size=(count, 2))


def workload(name):
    """Named synthetic workloads (sizes, frequencies and inputs of the five
    configurations the build is measured on).  Returns a dict with the
    velocity field `c` (n, n), the right-hand sides `f` (nrhs, n, n) and the
    solver settings.  `omega` is the angular frequency 2 pi (omega / 2 pi)."""
    two_pi = 2.0 * np.pi
    if name == "n64_const":
        n = 64
        return dict(name=name, n=n, omega=two_pi * 4, pml=8, eps_H=1e-9, tol=1e-8,
                    c=velocity_constant(n), f=source_gaussian(n)[None])
    if name == "n511_lens":
        n = 511
        return dict(name=name, n=n, omega=two_pi * 32, pml=12, eps_H=1e-6, tol=1e-6,
                    c=velocity_lens(n), f=source_gaussian(n)[None])
    if name in ("n1023_random", "n2047_random"):
        big = name == "n2047_random"
        n = 2047 if big else 1023
        w, seed_c, seed_s, ns = (1 / 64, 5, 6, 16) if big else (1 / 32, 1, 2, 64)
        pml = 16
        pts = source_positions(n, ns, pml, seed_s)
        f = np.stack([source_delta(n, p) for p in pts])
        return dict(name=name, n=n, omega=two_pi * (128 if big else 64), pml=pml,
                    eps_H=1e-6, tol=1e-7, c=velocity_random(n, w, seed_c), f=f)
    if name == "n511_grad":
        n = 511
        _, h = grid(n)
        pml = 12
        eta = pml * h
        xs = eta + (np.arange(32) + 0.5) * (1.0 - 2.0 * eta) / 32.0
        f = np.stack([source_delta(n, (x, 0.9)) for x in xs])
        rec_row = _nearest_node(n, 0.85)
        rec_idx = rec_row * n + np.arange(n)
        c_true = velocity_lens(n)
        c = c_true + 0.05 * smooth_noise(n, 1 / 32, 3)
        return dict(name=name, n=n, omega=two_pi * 32, pml=pml, eps_H=1e-6, tol=1e-8,
                    c=c, c_true=c_true, f=f, rec_idx=rec_idx)
    if name.startswith("dir_n"):
        # the sweeping-direction test of Section 3.1: c = 1/2 + x2, a narrow Gaussian point
        # source at (0.125, 0.5), q = 8 points per wavelength, fixed rank R = 2 (r_max = 2,
        # no truncation threshold), GMRES tolerance 1e-3; PML one wavelength (8 cells)
        n = int(name[len("dir_n"):])
        return dict(name=name, n=n, omega=two_pi * (n + 1) / 8.0, pml=8, eps_H=0.0, r_max=2, tol=1e-3,
                    c=velocity_linear_x2(n), f=source_gaussian(n, (0.125, 0.5))[None])
    if name.startswith(("pml1_n", "pml2_n", "pml3_n")):
        # Section 3.1, dependence on omega: PML on all sides, q = 8 (omega / 2 pi = (n + 1) / 8,
        # relative to c = 1), fixed rank R = 2, tol 1e-3; velocity 1: the converging lens,
        # 2: the vertical waveguide, 3: a random smooth medium (the same function for every
        # n); two forces: a narrow Gaussian at (0.5, 0.125) and a Gaussian wave packet at
        # (0.125, 0.125) towards (1, 1) with the wavelength of c = 1
        kind, n = name.split("_n")
        n = int(n)
        omega = two_pi * (n + 1) / 8.0
        c = {"pml1": velocity_lens, "pml2": velocity_waveguide, "pml3": velocity_random_modes}[kind](n)
        f = np.stack([source_gaussian(n, (0.5, 0.125)),
                      source_wavepacket(n, (0.125, 0.125), (1.0, 1.0), omega, 1.0 / 16.0)])
        return dict(name=name, n=n, omega=omega, pml=8, eps_H=0.0, r_max=2, tol=1e-3, c=c, f=f)
    if name.startswith(("qpml1_n", "qpml2_n", "qpml3_n")):
        # Section 3.1, dependence on q: omega / 2 pi = 32 fixed, q = (n + 1) / 32 points per
        # wavelength (n = 255, 511, 1023, 2047 for q = 8 .. 64), a PML of one wavelength
        # (q cells), R = 2, tol 1e-3; the fields and forces of the pml workloads
        kind, n = name.split("_n")
        n = int(n)
        w = workload("pml%s_n%d" % (kind[-1], n))
        omega = two_pi * 32.0
        q = (n + 1) // 32
        f = np.stack([source_gaussian(n, (0.5, 0.125)),
                      source_wavepacket(n, (0.125, 0.125), (1.0, 1.0), omega, 1.0 / 16.0)])
        return dict(w, name=name, omega=omega, pml=max(2, q), f=f)
    if name.startswith(("depth1_n", "depth2_n", "mixed1_n", "mixed2_n")):
        # Section 3.2, other boundary conditions; q = 8, fixed rank R = 2, tol 1e-3, PML of
        # one wavelength (8 cells) on the sides in `pml_sides` (1: x1 = 0, 2: x1 = 1,
        # 4: x2 = 0, 8: x2 = 1), zero Dirichlet on the others.
        #   depth1/depth2: waveguide, Dirichlet data b on x2 = 1 (b = 1, resp. the slant wave
        #     exp(i omega x1 / 2)), f = 0 otherwise (the data enters through `b_top`);
        #   mixed1: c = 1, Dirichlet at x1 = 0 and x1 = 1, packet at (0.5, 0.125) towards
        #     (cos pi/8, sin pi/8); mixed2: c = 1, Dirichlet at x1 = 1 and x2 = 1, packet at
        #     (0.5, 0.125) towards (1, 1).
        kind, n = name.split("_n")
        n = int(n)
        omega = two_pi * (n + 1) / 8.0
        x, _ = grid(n)
        base = dict(name=name, n=n, omega=omega, pml=8, eps_H=0.0, r_max=2, tol=1e-3)
        if kind in ("depth1", "depth2"):
            b = np.ones(n, np.complex128) if kind == "depth1" else np.exp(1j * omega * x / 2.0)
            return dict(base, pml_sides=1 | 2 | 4, c=velocity_waveguide(n), f=np.zeros((1, n, n), np.complex128),
                        b_top=b[None, :])
        direction = (np.cos(np.pi / 8), np.sin(np.pi / 8)) if kind == "mixed1" else (1.0, 1.0)
        sides = (4 | 8) if kind == "mixed1" else (1 | 4)
        f = source_wavepacket(n, (0.5, 0.125), direction, omega, 1.0 / 16.0)
        return dict(base, pml_sides=sides, c=velocity_constant(n), f=f[None])
    raise KeyError(name)
