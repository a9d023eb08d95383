"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: it only draws the initial
states and problem lists of the five workloads, with numpy's PCG64 generator,
so that the CUDA path and the FP64 oracle are fed identical arrays.

Workloads (grid conventions: periodic axes store the N unique points
x_i = lo + i*h, h = (hi-lo)/N; Dirichlet axes store all nodes including both
boundary nodes, h = (hi-lo)/(n-1)):

* ``heat_modes``   -- 2-D periodic [0,1]^2, u0 = sum of 8 Fourier modes
                      a_m cos(2 pi (kx_m x + ky_m y)), (kx, ky) ~ U{1..8}^2,
                      a_m ~ N(0,1).
* ``wave_bumps``   -- 3-D [0,1]^3 Dirichlet, u0 = sum of 16 Gaussian bumps
                      exp(-|x-x_k|^2 / (2 s_k^2)), x_k ~ U[0,1]^3,
                      s_k ~ U[0.02, 0.1]; boundary nodes set to 0; u_t = 0.
* ``batched_sides``-- 64 side lengths drawn uniformly from
                      {128, 256, 512, 1024, 2048}.
* ``hj_initial``   -- 2-D periodic [0,2pi]^2, u0 = -cos x - cos y plus iid
                      1e-3 N(0,1) noise per node.
* ``mlp_stencils`` -- raw 5-value stencils of the kinds the learned weight
                      path meets: smooth data sampled at h = 2 pi / 4096 on an
                      O(1) level, the same with 1e-3 noise, kinks and jumps.
* ``mlp_initial_params`` -- seeded He-style initial network parameters.
* ``mlp_positions`` -- seeded flat grid indices for harvesting stencils.
* the test problems of Sec. 5.1 on [0,2pi]^2, periodic (analytic, no seed):
  ``advection_initial`` (Example 1) u0 = (1 - cos x)(1 - cos y)/4;
  ``diffusion_initial`` (Example 2) u0 = sin x + sin y;
  ``manufactured_hj_solution`` / ``manufactured_hj_source`` (Example 3)
  u = t (sin x + sin y) for u_t + (1 + u_x + u_y)^2/2 = F, so that
  F = sin x + sin y + (1 + t cos x + t cos y)^2/2
    = [sin x + sin y + 1/2] + t [cos x + cos y] + t^2 [(cos x + cos y)^2/2].
* ``burgers_initial`` -- 2-D viscous Burgers (Sec. 2.5 flux splitting):
  [0,2pi]^2 periodic, u0 = 0.3 + 0.5 sin x sin y (|u| <= 0.8).
"""
import numpy as np

SEED_HEAT = 1
SEED_WAVE = 2
SEED_BATCH = 3
SEED_HJ = 4
SEED_HJ_LARGE = 5
SEED_MLP = 50


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def heat_mode_params(seed=SEED_HEAT, nmodes=8, kmax=8):
    """Wavenumbers (nmodes x 2: kx, ky) and amplitudes of ``heat_modes``."""
    g = rng(seed)
    k = g.integers(1, kmax + 1, size=(nmodes, 2))
    a = g.standard_normal(nmodes)
    return k, a


def heat_modes(n, seed=SEED_HEAT, nmodes=8, kmax=8):
    k, a = heat_mode_params(seed, nmodes, kmax)
    x = np.arange(n) / n
    u = np.zeros((n, n))          # [y][x]
    for m in range(nmodes):
        u += a[m] * np.cos(2 * np.pi * (k[m, 0] * x[None, :] + k[m, 1] * x[:, None]))
    return u


def wave_bump_params(seed=SEED_WAVE, nbumps=16):
    g = rng(seed)
    centres = g.uniform(0.0, 1.0, size=(nbumps, 3))
    widths = g.uniform(0.02, 0.1, size=nbumps)
    return centres, widths


def wave_bumps(n, seed=SEED_WAVE, nbumps=16, dtype=np.float64):
    """[z][y][x] array of n^3 nodes on [0,1]^3 (h = 1/(n-1))."""
    centres, widths = wave_bump_params(seed, nbumps)
    x = np.arange(n) / (n - 1)
    u = np.zeros((n, n, n), dtype=dtype)
    for (cx, cy, cz), s in zip(centres, widths):
        gx = np.exp(-(x - cx) ** 2 / (2 * s * s))
        gy = np.exp(-(x - cy) ** 2 / (2 * s * s))
        gz = np.exp(-(x - cz) ** 2 / (2 * s * s))
        u += (gz[:, None, None] * gy[None, :, None]) * gx[None, None, :]
    zero_boundary(u)
    return u


def zero_boundary(u):
    for ax in range(u.ndim):
        sl = [slice(None)] * u.ndim
        sl[ax] = 0
        u[tuple(sl)] = 0.0
        sl[ax] = -1
        u[tuple(sl)] = 0.0
    return u


def batched_sides(seed=SEED_BATCH, count=64):
    g = rng(seed)
    return [int(s) for s in g.choice([128, 256, 512, 1024, 2048], size=count)]


def batched_heat(seed=SEED_BATCH, count=64, sides=None):
    sides = sides if sides is not None else batched_sides(seed, count)
    return [heat_modes(s, seed=3000 + i) for i, s in enumerate(sides)]


def hj_initial(n, seed=SEED_HJ, noise=1e-3):
    g = rng(seed)
    x = 2 * np.pi * np.arange(n) / n
    u = -np.cos(x)[None, :] - np.cos(x)[:, None]
    return u + noise * g.standard_normal((n, n))


def random_lines(shape, seed=0):
    """Generic seeded test field, N(0,1) iid."""
    return rng(seed).standard_normal(shape)


def mlp_stencils(n, seed=SEED_MLP, h=2 * np.pi / 4096):
    """(n, 5) float32 raw stencils: a quarter each of smooth samples
    a sin(k x + phi) + c, the same plus 1e-3 N(0,1) noise, kinks
    a |x - x0| + c and jumps a [x > x0] + c, x on five nodes spaced h (smooth)
    or 1 (kinks, jumps)."""
    g = rng(seed)
    q = n // 4
    kinds = np.repeat(np.arange(4), [q, q, q, n - 3 * q])
    g.shuffle(kinds)
    j = np.arange(-2, 3, dtype=np.float64)
    a = g.uniform(0.5, 2.0, size=(n, 1)) * g.choice([-1.0, 1.0], size=(n, 1))
    c = g.uniform(-2.0, 2.0, size=(n, 1))
    k = g.uniform(0.5, 4.0, size=(n, 1))
    phi = g.uniform(0.0, 2 * np.pi, size=(n, 1))
    x0 = g.uniform(-2.0, 2.0, size=(n, 1))
    noise = 1e-3 * g.standard_normal((n, 5))
    smooth = a * np.sin(k * h * j[None, :] + phi) + c
    out = np.where((kinds == 0)[:, None], smooth, 0.0)
    out = np.where((kinds == 1)[:, None], smooth + noise, out)
    out = np.where((kinds == 2)[:, None], a * np.abs(j[None, :] - x0) + c, out)
    out = np.where((kinds == 3)[:, None], a * (j[None, :] > x0) + c, out)
    return out.astype(np.float32)


def mlp_initial_params(seed=SEED_MLP):
    """1347 FP32 network parameters (order W1 32x5, b1, W2 32x32, b2, W3 3x32,
    b3): weights N(0, 2/fan_in) (last layer N(0, 1/fan_in)), biases zero."""
    g = rng(seed)
    w1 = g.standard_normal((32, 5)) * np.sqrt(2.0 / 5)
    w2 = g.standard_normal((32, 32)) * np.sqrt(2.0 / 32)
    w3 = g.standard_normal((3, 32)) * np.sqrt(1.0 / 32)
    return np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(32), w3.ravel(),
                           np.zeros(3)]).astype(np.float32)


def mlp_positions(count, nx, ny, seed=SEED_MLP):
    """`count` flat indices drawn uniformly from an ny x nx grid (int64)."""
    return rng(seed).integers(0, nx * ny, size=count, dtype=np.int64)


def paper_grid(n):
    """x_i = 2 pi i / n, i < n, as a (y, x) pair of broadcastable arrays."""
    x = 2 * np.pi * np.arange(n) / n
    return x[None, :], x[:, None]


def advection_initial(n):
    x, y = paper_grid(n)
    return 0.25 * (1 - np.cos(x)) * (1 - np.cos(y))


def advection_solution(n, t):
    """u0(x - t, y - t) of u_t + u_x + u_y = 0."""
    x, y = paper_grid(n)
    return 0.25 * (1 - np.cos(x - t)) * (1 - np.cos(y - t))


def diffusion_initial(n):
    x, y = paper_grid(n)
    return np.sin(x) + np.sin(y) + 0.0 * x * y


def diffusion_solution(n, t):
    return np.exp(-t) * diffusion_initial(n)


def manufactured_hj_solution(n, t):
    return t * diffusion_initial(n)


def manufactured_hj_source(n):
    """The coefficients (F_0, F_1, F_2) of the Example 3 source, shape (3, n, n)."""
    x, y = paper_grid(n)
    c = np.cos(x) + np.cos(y)
    return np.stack([np.sin(x) + np.sin(y) + 0.5, c, 0.5 * c * c])


def burgers_initial(n):
    x, y = paper_grid(n)
    return 0.3 + 0.5 * np.sin(x) * np.sin(y)
