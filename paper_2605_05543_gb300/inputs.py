"""Seeded synthetic inputs for EM-PP runs: relativistic Gaussian electron bunches and trajectory
histories.

This module is the one piece shared by the CUDA path's callers and the oracle's tests: it only
draws and lays out input data. It holds none of the method's arithmetic (no retarded time, field or
push).

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used as a counter-based
generator: output k of stream `seed` is the SplitMix64 finaliser applied to
``seed + (k + 1) * 0x9E3779B97F4A7C15`` (mod 2^64). Uniforms take the top 53 bits; normals use the
Box-Muller transform on consecutive uniform pairs.

Bunch recipe (the paper's Gaussian phase-space initialisation of Sec. 2.5, with the widths given in
momentum as the benchmark workloads state them). Particle i consumes normals 6i..6i+5 in the order
x, y, z, K, u_x, u_y:
    x, y, z ~ N(0, sigma^2);  K ~ N(K0, (dE_rel K0)^2) with K0 = (gamma0 - 1) m_e c^2;
    u_x, u_y ~ N(0, (du_perp_rel u0)^2) with u0 = c sqrt(gamma0^2 - 1);
    gamma = 1 + K / (m_e c^2);  u_z = sqrt((gamma^2 - 1) c^2 - u_x^2 - u_y^2)  (beam along +z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# CODATA 2018, for the kinematics of the input recipe only
C_LIGHT = 299792458.0
M_E = 9.1093837015e-31
Q_E = 1.602176634e-19
R_EARTH = 6.371e6

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream started at `seed`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on uniform pairs (2m, 2m+1) -> normals (2m, 2m+1)."""
    m0 = offset // 2
    npairs = (offset + count + 1) // 2 - m0
    u = uniforms(seed, 2 * npairs, 2 * m0)
    u1 = u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    th = 2.0 * np.pi * u2
    out = np.empty(2 * npairs)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    s = offset - 2 * m0
    return out[s:s + count]


@dataclass
class Bunch:
    x: np.ndarray  # (N, 3) positions, m
    u: np.ndarray  # (N, 3) proper velocities gamma*v, m/s
    sigma: float
    gamma0: float
    seed: int


def gaussian_bunch(N: int, sigma: float, gamma0: float, dE_rel: float = 1e-3, du_perp_rel: float = 1e-4,
                   seed: int = 0, center=(0.0, 0.0, 0.0)) -> Bunch:
    """Isotropic Gaussian bunch of N electrons moving along +z (recipe in the module docstring)."""
    g = normals(seed, 6 * N).reshape(N, 6)
    mc2 = M_E * C_LIGHT * C_LIGHT
    K0 = (gamma0 - 1.0) * mc2
    u0 = C_LIGHT * math.sqrt(gamma0 * gamma0 - 1.0)
    x = np.empty((N, 3))
    x[:, 0] = center[0] + sigma * g[:, 0]
    x[:, 1] = center[1] + sigma * g[:, 1]
    x[:, 2] = center[2] + sigma * g[:, 2]
    K = K0 * (1.0 + dE_rel * g[:, 3])
    ux = du_perp_rel * u0 * g[:, 4]
    uy = du_perp_rel * u0 * g[:, 5]
    gam = 1.0 + K / mc2
    uz = np.sqrt((gam * gam - 1.0) * C_LIGHT * C_LIGHT - ux * ux - uy * uy)
    u = np.stack([ux, uy, uz], axis=1)
    return Bunch(x=x, u=u, sigma=sigma, gamma0=gamma0, seed=seed)


def beam_kinematics(E0: float):
    """gamma0 = 1 + E0 / (m_e c^2) and beta = sqrt(1 - 1 / gamma0^2) of a kinetic energy E0 (J) (Sec. 2.5)."""
    g0 = 1.0 + E0 / (M_E * C_LIGHT * C_LIGHT)
    return g0, math.sqrt(1.0 - 1.0 / (g0 * g0))


def rotation(theta: float, phi: float) -> np.ndarray:
    """R(theta, phi) = R_z(phi) R_y(theta): beam frame to laboratory frame (Sec. 2.5)."""
    ct, st, cp, sp = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    Ry = np.array([[ct, 0.0, st], [0.0, 1.0, 0.0], [-st, 0.0, ct]])
    Rz = np.array([[cp, -sp, 0.0], [sp, cp, 0.0], [0.0, 0.0, 1.0]])
    return Rz @ Ry


def paper_bunch(Np: int, E0_MeV: float, r_perp: float = 2e-3, r_par: float = 2e-3, delta_E: float = 0.01,
                eps_r: float = 1e-6, theta: float = 0.0, phi: float = 0.0, center=(0.0, 0.0, 0.0), seed: int = 0,
                weight: float = 1.0) -> Bunch:
    """The paper's own bunch (Sec. 2.5, Table 1): Np macroparticles with
    x, y ~ N(0, r_perp^2), z ~ N(0, r_par^2); v_x, v_y ~ N(0, sigma_perp^2) with sigma_perp = eps_r v0 / r_perp;
    E ~ N(E0, (delta_E E0)^2), gamma(E) = 1 + E / (m_e c^2), v_z = c sqrt(1 - 1 / gamma(E)^2); then v_z is
    shifted so that its sample mean is v0, and positions and velocities are rotated by R(theta, phi) and
    the positions translated to `center`. Particle i consumes normals 6i..6i+5 in the order x, y, z, v_x,
    v_y, E. The returned u is the proper velocity v / sqrt(1 - v.v / c^2). `weight` is the number of
    electrons per macroparticle (w_p = n0 V / Np; the paper does not state n0)."""
    g = normals(seed, 6 * Np).reshape(Np, 6)
    mc2 = M_E * C_LIGHT * C_LIGHT
    E0 = E0_MeV * 1e6 * Q_E
    g0, beta0 = beam_kinematics(E0)
    v0 = beta0 * C_LIGHT
    sig_perp = eps_r * v0 / r_perp
    x = np.stack([r_perp * g[:, 0], r_perp * g[:, 1], r_par * g[:, 2]], axis=1)
    E = E0 + delta_E * E0 * g[:, 5]
    gam = 1.0 + E / mc2
    vz = C_LIGHT * np.sqrt(1.0 - 1.0 / (gam * gam))
    vz = vz - (vz.mean() - v0)
    v = np.stack([sig_perp * g[:, 3], sig_perp * g[:, 4], vz], axis=1)
    R = rotation(theta, phi)
    x = x @ R.T + np.asarray(center, dtype=float)[None, :]
    v = v @ R.T
    vv = np.sum(v * v, axis=1) / (C_LIGHT * C_LIGHT)
    if np.any(vv >= 1.0):
        raise ValueError("sampled speed at or above c")
    u = v / np.sqrt(1.0 - vv)[:, None]
    b = Bunch(x=x, u=u, sigma=r_perp, gamma0=g0, seed=seed)
    b.weights = np.full(Np, float(weight))
    return b


# Geometry of the paper's runs (Sec. 2.5, Sec. 2.6): injection at (-10 R_E, 0, 0) in a centred dipole of
# moment 8.6e22 A m^2 along +z.
PAPER_M0 = 8.6e22
PAPER_R0 = (-10.0 * R_EARTH, 0.0, 0.0)


def velocity_of(u: np.ndarray) -> np.ndarray:
    """v = u / sqrt(1 + u.u / c^2): the relativistic relation the recipe needs to lay out a history."""
    uu = np.sum(u * u, axis=-1)
    return u / np.sqrt(1.0 + uu / (C_LIGHT * C_LIGHT))[..., None]


def time_stamps(nslots: int, dt: float, t0: float = 0.0) -> np.ndarray:
    """t_0 = t0 and t_{k+1} = t_k + dt, accumulated one step at a time."""
    T = np.empty(nslots)
    t = float(t0)
    for k in range(nslots):
        T[k] = t
        t = t + dt
    return T


@dataclass
class History:
    T: np.ndarray  # (S,) slot time stamps, s
    W: np.ndarray  # (S, N, 3) positions, m
    V: np.ndarray  # (S, N, 3) velocities, m/s
    u: np.ndarray  # (N, 3) present proper velocity, m/s
    n: int  # index of the present slot (slots 0..n are held)


def synthetic_history(x: np.ndarray, u: np.ndarray, n: int, dt: float, wiggle: float = 1e-4,
                      period_steps: float = 160.0, seed: int = 7) -> History:
    """History of slots 0..n that ends at the present state (x, u) at slot n.

    Each particle j follows w_j(t) = x_j + v_j s + (A_j / omega^2)(1 - cos(omega s)) with
    s = t - t_n, so that its present position and velocity are (x_j, v_j) and its acceleration at
    t_n is A_j. |A_j| / omega = wiggle * c (random direction, seeded), omega = 2 pi / (period_steps
    dt). This gives stored samples with non-zero acceleration and the bunch's drift, so that the
    bracket visits every branch.
    """
    N = x.shape[0]
    v = velocity_of(u)
    T = time_stamps(n + 1, dt)
    s = T - T[n]
    omega = 2.0 * math.pi / (period_steps * dt)
    d = normals(seed, 3 * N).reshape(N, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    A = d * (wiggle * C_LIGHT * omega)
    W = x[None, :, :] + v[None, :, :] * s[:, None, None] + (A[None] / omega ** 2) * (
        1.0 - np.cos(omega * s))[:, None, None]
    V = v[None, :, :] + (A[None] / omega) * np.sin(omega * s)[:, None, None]
    V[n] = v
    W[n] = x
    return History(T=T, W=np.ascontiguousarray(W), V=np.ascontiguousarray(V), u=u.copy(), n=n)


# ------------------------------------------------------------------------------------------------
# Workloads (sizes and settings of the benchmark configurations)
# ------------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    N: int
    sigma: float
    gamma0: float
    dt: float
    steps: int
    depth: int
    bext: str  # "none" | "uniform" | "dipole"
    b_uniform: tuple = (0.0, 0.0, 0.0)
    seed: int = 0


FREE_EXPANSION_256 = Workload("free-expansion N=256 sigma=10um gamma0=3 fp64", 256, 10e-6, 3.0, 1e-15, 200, 256,
                              "none")
UNIFORM_B_4096 = Workload("uniform-Bx N=4096 sigma=10um gamma0=3 fp64", 4096, 10e-6, 3.0, 1e-15, 2000, 512,
                          "uniform", (5e-5, 0.0, 0.0))
BUNCH_65536 = Workload("free-expansion N=65536 sigma=20um gamma0=3", 65536, 20e-6, 3.0, 1e-15, 500, 1024, "none")


def batch_bunches(nbunch: int = 64, nmin: int = 512, nmax: int = 16384, smin: float = 5e-6, smax: float = 50e-6,
                  gmin: float = 2.0, gmax: float = 20.0):
    """Per-bunch (N, sigma, gamma0, seed) of the batched two-stage workload: bunch b draws three
    uniforms from stream 1000 + b, and its particles come from stream b."""
    out = []
    for b in range(nbunch):
        r = uniforms(1000 + b, 3)
        N = nmin + int(r[0] * (nmax - nmin + 1))
        out.append((min(N, nmax), smin + r[1] * (smax - smin), gmin + r[2] * (gmax - gmin), b))
    return out


# ------------------------------------------------------------------------------------------------
# Proposal network (10-64-64-1): seeded initial parameters
# ------------------------------------------------------------------------------------------------
MLP_IN, MLP_H = 10, 64
MLP_NUM_PARAMS = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Initial parameters, float32: W1 and W2 and w3 uniform in +-1/sqrt(fan in), biases zero, in the
    layout W1[10][64], b1[64], W2[64][64], b2[64], w3[64], b3."""
    u = uniforms(2000 + seed, MLP_IN * MLP_H + MLP_H * MLP_H + MLP_H)
    k = MLP_IN * MLP_H
    W1 = (2 * u[:k] - 1) / math.sqrt(MLP_IN)
    W2 = (2 * u[k:k + MLP_H * MLP_H] - 1) / math.sqrt(MLP_H)
    w3 = (2 * u[k + MLP_H * MLP_H:] - 1) / math.sqrt(MLP_H)
    z = np.zeros(MLP_H)
    return np.concatenate([W1, z, W2, z, w3, [0.0]]).astype(np.float32)
