"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds none of the method's arithmetic: it only describes meshes,
material parameters, the fibre field, right-hand sides and stimuli, so that
both sides of every parity test receive bit-identical inputs.

The workloads stand in for the paper's meshes (Section 3: an idealised
ventricle and a patient mesh that is not public): box slabs meshed by uniform
Q1 hexahedra, with the transmural fibre rotation of Section 2 ("fibres
rotating counterclockwise from epi- to endocardium") made linear in z.
"""
from __future__ import annotations

import math

import numpy as np

#: intracellular / extracellular conductivities (mS/cm), surface-to-volume
#: ratio chi (1/cm), membrane capacitance Cm (uF/cm^2), time step dt (ms).
DEFAULT_PARAMS = dict(sil=3.0, sit=0.31525, sel=2.0, set=1.3514, chi=1000.0, cm=1.0, dt=0.05)

#: slab sizes (elements and cm)
SLAB_SMALL = dict(nx=24, ny=24, nz=12, lx=1.0, ly=1.0, lz=0.5)        # 16,250 unknowns
SLAB_PAPER = dict(nx=128, ny=128, nz=32, lx=1.0, ly=1.0, lz=0.5)      # 1,098,306 unknowns
SLAB_LARGE = dict(nx=256, ny=256, nz=64, lx=1.0, ly=1.0, lz=0.5)      # 8,586,370 unknowns


def n_nodes(mesh: dict) -> int:
    return (mesh["nx"] + 1) * (mesh["ny"] + 1) * (mesh["nz"] + 1)


def mesh(nx, ny, nz, lx=None, ly=None, lz=None) -> dict:
    """A slab with the given element counts; default extent keeps cube elements
    of side 1/24 cm along x."""
    h = 1.0 / 24.0
    return dict(nx=nx, ny=ny, nz=nz, lx=lx if lx else nx * h, ly=ly if ly else ny * h,
                lz=lz if lz else nz * h)


def fibre_table(mesh: dict, rot_deg: float = 120.0, off_deg: float = 0.0) -> np.ndarray:
    """Fibre direction a_l at the two Gauss z-levels of every element layer.

    Shape (nz, 2, 3), float64.  theta(z) = off + rot * (z/lz - 1/2), fibre
    (cos theta, sin theta, 0).  Gauss z-levels of layer ez are
    z = (ez + (1 -/+ 1/sqrt3)/2) * lz/nz.
    """
    nz, lz = mesh["nz"], mesh["lz"]
    hz = lz / nz
    g = np.array([(1.0 - 1.0 / math.sqrt(3.0)) * 0.5, (1.0 + 1.0 / math.sqrt(3.0)) * 0.5])
    z = (np.arange(nz)[:, None] + g[None, :]) * hz
    th = np.deg2rad(off_deg) + np.deg2rad(rot_deg) * (z / lz - 0.5)
    out = np.zeros((nz, 2, 3))
    out[..., 0] = np.cos(th)
    out[..., 1] = np.sin(th)
    return out


def fibre_offset_from_seed(seed: int) -> float:
    """Seeded transmural offset angle in [-30, 30) degrees."""
    return float(np.random.Generator(np.random.PCG64(seed)).uniform(-30.0, 30.0))


def rhs(n_unknowns: int, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) right-hand side with the u_e part's mean removed, so that
    it is consistent with the null vector (0, 1)."""
    f = np.random.Generator(np.random.PCG64(seed)).standard_normal(n_unknowns)
    f[1::2] -= f[1::2].mean()
    return f


def stimulus(mesh: dict, amplitude: float = 8.0e4, corner: float = 0.1) -> np.ndarray:
    """Per-node applied current (uA/cm^3) on the corner cube [0, corner]^3."""
    nx, ny, nz = mesh["nx"], mesh["ny"], mesh["nz"]
    x = np.arange(nx + 1) * (mesh["lx"] / nx)
    y = np.arange(ny + 1) * (mesh["ly"] / ny)
    z = np.arange(nz + 1) * (mesh["lz"] / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    inside = (X <= corner + 1e-12) & (Y <= corner + 1e-12) & (Z <= corner + 1e-12)
    return np.where(inside, amplitude, 0.0).reshape(-1)


def random_slab(rng: np.random.Generator, lo=(16, 16, 8), hi=(64, 64, 16)):
    """Seeded slab for the batched workload: element counts, fibre rotation in
    [60, 150) degrees and a conductivity scale in [0.8, 1.2)."""
    nx = int(rng.integers(lo[0], hi[0] + 1))
    ny = int(rng.integers(lo[1], hi[1] + 1))
    nz = int(rng.integers(lo[2], hi[2] + 1))
    rot = float(rng.uniform(60.0, 150.0))
    scale = float(rng.uniform(0.8, 1.2))
    return mesh(nx, ny, nz), rot, scale


def batch_slabs(count: int = 64, seed: int = 2) -> list:
    """Seeded uneven slabs for the batched form: nx, ny ~ U{16..64},
    nz ~ U{8..16} (cube elements of side 1/24 cm), fibre rotation
    U[60, 150] degrees with offset U[-30, 30), every conductivity scaled by
    its own U[0.8, 1.2].  Returns (mesh, params, fibre table) per slab."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        nx, ny = (int(v) for v in rng.integers(16, 65, 2))
        nz = int(rng.integers(8, 17))
        rot = float(rng.uniform(60.0, 150.0))
        off = float(rng.uniform(-30.0, 30.0))
        sc = rng.uniform(0.8, 1.2, 4)
        m = mesh(nx, ny, nz)
        p = dict(DEFAULT_PARAMS)
        for key, f in zip(("sil", "sit", "sel", "set"), sc):
            p[key] = DEFAULT_PARAMS[key] * float(f)
        out.append((m, p, fibre_table(m, rot, off)))
    return out
