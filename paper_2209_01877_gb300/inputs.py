"""Seeded synthetic inputs: meshes, initial fields and random directions.

This module holds no part of the discretisation.  It builds the arrays a
user would hand to the library (tetrahedra, vertex coordinates, boundary
tags) and pointwise analytic fields; the modal projection, quadrature and
residual live in the library (and, independently, in the test oracle).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of a generator
seeded with s is mix(s + (i+1)*0x9E3779B97F4A7C15), which this module
evaluates vectorised.  A uniform double in [0,1) is (z >> 11) * 2**-53.

Mesh recipe (stands in for the paper's unstructured 2D grids, Tab. 3):
the box is cut into nx*ny*nz hexahedra, each split into 6 Kuhn tetrahedra
(one per ordering of the three axis steps from the low corner to the high
corner), interior vertices are jittered by U(-a, a)*h per component,
boundary vertices only tangentially, each tetrahedron's local vertex order
is shuffled by a random even permutation (so every face orientation
occurs) and the element order is shuffled (the paper's "original"
unrenumbered ordering, Sec. III-B).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds used by the standard workloads.
SEED_PERM = 1        # element order
SEED_PERTURB = 2     # 1% state perturbation
SEED_PULSE = 3       # Gaussian pulse centre
SEED_DIRS = 4        # adjoint test directions
SEED_JITTER = 5      # vertex jitter
SEED_LOCAL = 6       # local vertex order of each tetrahedron


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of SplitMix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) from SplitMix64."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, n: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, n, offset)


@dataclass
class TetMesh:
    """A tetrahedral mesh in the form the C-ABI takes.

    tet_vid  int32 [ne][4]    global vertex ids (periodic images share ids)
    tet_xyz  float64 [ne][4][3] unwrapped vertex coordinates of each tet
    bc_tag   int8 [ne][4]     per local face (opposite local vertex f):
                              0 interior/periodic, 1 slip wall, 2 far field
    lengths  box edge lengths; periodic per-axis flags
    """
    tet_vid: np.ndarray
    tet_xyz: np.ndarray
    bc_tag: np.ndarray
    lengths: tuple
    periodic: tuple
    dims: tuple

    @property
    def ne(self) -> int:
        return int(self.tet_vid.shape[0])


def _kuhn_local():
    """The 6 Kuhn tetrahedra of the unit cube as integer corner offsets [6][4][3],
    each with positive orientation."""
    tets = []
    for perm in itertools.permutations(range(3)):
        v = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            w = v[-1].copy()
            w[ax] += 1
            v.append(w)
        e = np.array(v)
        d = np.linalg.det((e[1:] - e[0]).T.astype(float))
        if d < 0:
            e[[2, 3]] = e[[3, 2]]
        tets.append(e)
    return np.array(tets)


_EVEN_PERMS = np.array([p for p in itertools.permutations(range(4))
                        if sum(1 for i in range(4) for j in range(i + 1, 4) if p[i] > p[j]) % 2 == 0],
                       dtype=np.int64)


def make_box_mesh(dims, lengths=(1.0, 1.0, 1.0), periodic=(True, True, True),
                  jitter=0.10, seed_jitter=SEED_JITTER, shuffle_elements=True,
                  seed_perm=SEED_PERM, shuffle_local=True, seed_local=SEED_LOCAL) -> TetMesh:
    """Kuhn-split jittered box mesh.  Non-periodic faces get bc_tag 1 (slip
    wall) on the y and z sides and 2 (characteristic far field) on the x
    sides; periodic faces are matched by shared vertex ids."""
    nx, ny, nz = (int(d) for d in dims)
    n = np.array([nx, ny, nz])
    L = np.array(lengths, dtype=np.float64)
    h = L / n
    per = np.array(periodic, dtype=bool)
    # unique vertex lattice: periodic axes have n points, others n+1
    nv_ax = np.where(per, n, n + 1)

    def vid_of(ijk):
        w = np.where(per, ijk % n, ijk)
        return (w[..., 0] * nv_ax[1] + w[..., 1]) * nv_ax[2] + w[..., 2]

    nverts = int(np.prod(nv_ax))
    # jitter per unique vertex; boundary vertices of non-periodic axes move tangentially only
    jit = uniform(seed_jitter, nverts * 3, -jitter, jitter).reshape(nverts, 3)
    vi = np.stack(np.meshgrid(np.arange(nv_ax[0]), np.arange(nv_ax[1]), np.arange(nv_ax[2]),
                              indexing="ij"), axis=-1).reshape(-1, 3)
    for ax in range(3):
        if not per[ax]:
            on_b = (vi[:, ax] == 0) | (vi[:, ax] == n[ax])
            jit[on_b, ax] = 0.0

    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hexes = np.stack([hi, hj, hk], axis=-1).reshape(-1, 1, 1, 3)     # [nh,1,1,3]
    corners = hexes + _kuhn_local()[None]                              # [nh,6,4,3]
    corners = corners.reshape(-1, 4, 3)
    vid = vid_of(corners).astype(np.int64)
    xyz = (corners + jit[vid]) * h
    ne = vid.shape[0]

    # boundary tags of the local faces (face f is opposite local vertex f)
    tag = np.zeros((ne, 4), dtype=np.int8)
    for f in range(4):
        others = [k for k in range(4) if k != f]
        c = corners[:, others, :]
        for ax in range(3):
            if per[ax]:
                continue
            for side in (0, n[ax]):
                on = np.all(c[:, :, ax] == side, axis=1)
                tag[on, f] = 2 if ax == 0 else 1

    if shuffle_local:
        pick = (splitmix64(seed_local, ne) % np.uint64(len(_EVEN_PERMS))).astype(np.int64)
        lp = _EVEN_PERMS[pick]                                          # [ne,4]
        rows = np.arange(ne)[:, None]
        vid = vid[rows, lp]
        xyz = xyz[rows, lp]
        tag = tag[rows, lp]
    if shuffle_elements:
        order = np.argsort(uniform01(seed_perm, ne), kind="stable")
        vid, xyz, tag = vid[order], xyz[order], tag[order]
    return TetMesh(tet_vid=np.ascontiguousarray(vid, dtype=np.int32),
                   tet_xyz=np.ascontiguousarray(xyz, dtype=np.float64),
                   bc_tag=np.ascontiguousarray(tag, dtype=np.int8),
                   lengths=tuple(float(x) for x in L), periodic=tuple(bool(x) for x in per),
                   dims=(nx, ny, nz))


def make_periodic_cube(n, jitter=0.10, **kw) -> TetMesh:
    """n^3 hexes x 6 tets on the periodic unit cube."""
    return make_box_mesh((n, n, n), (1.0, 1.0, 1.0), (True, True, True), jitter=jitter, **kw)


def make_box_channel(nx=96, ny=48, nz=48, lengths=(2.0, 1.0, 1.0), jitter=0.15, **kw) -> TetMesh:
    """Channel box with slip walls at y, z and far-field faces at x."""
    return make_box_mesh((nx, ny, nz), lengths, (False, False, False), jitter=jitter, **kw)


# ----------------------------------------------------------------------------------------------
# Pointwise fields (conserved variables rho, rho u, rho v, rho w, E), x: [..., 3]
# ----------------------------------------------------------------------------------------------

def prim_to_cons(rho, u, v, w, p, gamma=GAMMA):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=-1)


def uniform_flow(x, rho=1.0, vel=(0.3, 0.2, 0.1), p=1.0 / GAMMA, gamma=GAMMA):
    one = np.ones(x.shape[:-1])
    return prim_to_cons(rho * one, vel[0] * one, vel[1] * one, vel[2] * one, p * one, gamma)


def isentropic_vortex(x, t=0.0, centre=(0.5, 0.5), radius=1.0 / 16.0, beta=5.0,
                      mach=0.5, gamma=GAMMA, period=1.0):
    """Shu's isentropic vortex in the x-y plane, uniform in z, advected along
    +x at speed mach*sqrt(gamma) (free stream rho = p = 1).  The exact solution
    at time t is the initial field translated by u_inf*t (periodic images
    beyond the nearest one are below 1e-13 for radius 1/16)."""
    uinf = mach * math.sqrt(gamma)
    xc = centre[0] + uinf * t
    dx = x[..., 0] - xc
    dy = x[..., 1] - centre[1]
    if period is not None:
        dx = dx - period * np.round(dx / period)
        dy = dy - period * np.round(dy / period)
    r2 = (dx * dx + dy * dy) / (radius * radius)
    g = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2.0 * math.pi) * (dy / radius) * g
    dv = beta / (2.0 * math.pi) * (dx / radius) * g
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi * math.pi) * g * g
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return prim_to_cons(rho, uinf + du, dv, 0.0 * du, p, gamma)


def entropy_wave(x, t=0.0, amp=0.2, vel=(0.3, 0.2, 0.1), p=1.0, k=(1, 0, 0), gamma=GAMMA):
    """rho = 1 + amp*sin(2 pi k.(x - vel t)), constant velocity and pressure:
    an exact solution of the Euler equations on the periodic unit cube."""
    ph = 2.0 * math.pi * sum(k[d] * (x[..., d] - vel[d] * t) for d in range(3))
    rho = 1.0 + amp * np.sin(ph)
    one = np.ones_like(rho)
    return prim_to_cons(rho, vel[0] * one, vel[1] * one, vel[2] * one, p * one, gamma)


def gaussian_pulse(x, centre, mach=0.3, amp=0.1, width=0.05, gamma=GAMMA):
    """Mach-0.3 uniform stream (rho = p = 1) carrying a Gaussian density pulse."""
    r2 = sum((x[..., d] - centre[d]) ** 2 for d in range(3))
    rho = 1.0 + amp * np.exp(-r2 / (width * width))
    one = np.ones_like(rho)
    return prim_to_cons(rho, mach * math.sqrt(gamma) * one, 0 * one, 0 * one, one, gamma)


def pulse_centre(seed=SEED_PULSE):
    u = uniform01(seed, 3)
    return (0.6 + 0.8 * u[0], 0.35 + 0.3 * u[1], 0.35 + 0.3 * u[2])


def freestream_state(mach=0.3, gamma=GAMMA):
    """Conserved free-stream state (rho = p = 1, velocity mach*c along +x)."""
    return prim_to_cons(np.array(1.0), np.array(mach * math.sqrt(gamma)), np.array(0.0),
                        np.array(0.0), np.array(1.0), gamma)


def perturb_coefficients(U, amp=0.01, seed=SEED_PERTURB):
    """Seeded 1% perturbation of modal state coefficients U[ne][5][nb]: every
    element's density coefficients are scaled by (1 + amp*xi1) and its
    momentum coefficients by (1 + amp*xi1)(1 + amp*xi2), xi ~ U(-1, 1) per
    element (density and velocity each perturbed by up to amp)."""
    ne = U.shape[0]
    xi = uniform(seed, 2 * ne, -1.0, 1.0).reshape(ne, 2)
    a = 1.0 + amp * xi[:, 0]
    b = 1.0 + amp * xi[:, 1]
    out = U.copy()
    out[:, 0, :] *= a[:, None]
    out[:, 1:4, :] *= (a * b)[:, None, None]
    return out


def random_directions(shape, count, seed=SEED_DIRS):
    """``count`` seeded directions with entries U(-1, 1)."""
    n = int(np.prod(shape))
    return uniform(seed, n * count, -1.0, 1.0).reshape((count,) + tuple(shape))


def n_basis(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6
