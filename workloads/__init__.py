"""Seeded synthetic problem descriptions and inputs.

This module is shared by the oracle side and the CUDA side. It holds problem
data only: mesh vertex coordinates, boundary tags, physical parameters and
seeded random states. It holds none of the discontinuous Galerkin arithmetic.

Face tags (one byte per boundary face):
  1 WALL, 2 INLET, 3 OUTLET, 4 DIRICHLET, 5 + j ELECTRODE number j (j < 4).
Boundary sides are ordered x-, x+, y-, y+, (z-, z+); the faces of one side are
numbered lexicographically over the remaining axes, lowest axis fastest.

The shapes follow the paper's workloads: the manufactured-solution test of
Sec. 5.1 (unit cube, two ions, parabolic velocity) and the parallel-plate flow
reactor of Sec. 5.2 (plate flow, Butler-Volmer electrodes, a J_0 profile
across the channel width). The paper's meshes and data files are not public,
so these structured boxes stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
import torch

WALL, INLET, OUTLET, DIRICHLET, ELECTRODE0 = 1, 2, 3, 4, 5
VEL_CONSTANT, VEL_PLATE = 0, 1
MAX_SPECIES = 4


@dataclasses.dataclass
class Problem:
    """A structured tensor-product box mesh plus CNP physics parameters."""
    dim: int
    n_el: List[int]
    coords: List[np.ndarray]          # per axis: n_el[a] + 1 vertex coordinates
    tags: List[np.ndarray]            # per boundary side: uint8 tag per face
    m: int                            # number of ionic species (c_m eliminated)
    z: List[float]
    D: List[float]
    c_in: List[float]
    p: int
    q: int
    F: float = 1.0
    RT: float = 1.0
    vel_kind: int = VEL_CONSTANT
    vel_params: List[float] = dataclasses.field(default_factory=lambda: [0.0] * 8)
    bv_oxidant: int = -1              # species index of the oxidant, -1 = no electrode reaction
    bv_J0: float = 0.0
    bv_alpha1: float = 0.5
    bv_alpha2: float = 0.5
    bv_n: float = 1.0
    bv_gamma: float = 1.0
    bv_c_ref: float = 1.0
    bv_phi_app: List[float] = dataclasses.field(default_factory=lambda: [0.0] * 4)
    bv_J0_axis: int = -1              # axis of the J_0 profile, -1 = constant J_0
    bv_J0_lo: float = 0.0
    bv_J0_hi: float = 1.0
    C_IP: float = 10.0
    name: str = ""

    @property
    def n_fields(self) -> int:
        return self.m

    @property
    def E(self) -> int:
        return int(np.prod(self.n_el[: self.dim]))

    @property
    def Np(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def Nq(self) -> int:
        return self.q ** self.dim

    @property
    def Nfq(self) -> int:
        return self.q ** (self.dim - 1)

    @property
    def n_bfaces(self) -> int:
        return int(sum(len(t) for t in self.tags))

    @property
    def n_dof(self) -> int:
        return self.n_fields * self.E * self.Np

    def bv_params(self) -> np.ndarray:
        """The 13 Butler-Volmer reals in the order both C interfaces take them."""
        return np.array([self.bv_J0, self.bv_alpha1, self.bv_alpha2, self.bv_n, self.bv_gamma,
                         self.bv_c_ref, *self.bv_phi_app[:4], float(self.bv_J0_axis),
                         self.bv_J0_lo, self.bv_J0_hi], dtype=np.float64)

    def side_faces(self, s: int) -> List[int]:
        a = s // 2
        return [b for b in range(self.dim) if b != a]


def _side_shape(dim, n_el, s):
    a = s // 2
    others = [b for b in range(dim) if b != a]
    return [n_el[b] for b in others], others


def box_tags(dim, n_el, coords, fill=WALL):
    tags = []
    for s in range(2 * dim):
        shape, _ = _side_shape(dim, n_el, s)
        tags.append(np.full(int(np.prod(shape)), fill, dtype=np.uint8))
    return tags


def face_centres(dim, n_el, coords, s):
    """Centres of the faces of boundary side s, in face order: array [nf, dim]."""
    a = s // 2
    shape, others = _side_shape(dim, n_el, s)
    mids = [0.5 * (coords[b][1:] + coords[b][:-1]) for b in others]
    grids = np.meshgrid(*mids, indexing="ij")  # others[0] first
    out = np.zeros((int(np.prod(shape)), dim))
    for j, b in enumerate(others):
        out[:, b] = grids[j].transpose().reshape(-1) if dim == 3 else grids[j].reshape(-1)
    out[:, a] = coords[a][-1] if (s & 1) else coords[a][0]
    return out


def _linspace_coords(n_el, lengths):
    return [np.linspace(0.0, L, n + 1) for n, L in zip(n_el, lengths)]


def _reactor_tags(dim, n_el, coords, x_lo, x_hi, anode=True):
    """Inlet at x-, outlet at x+, cathode (electrode 0) on y- and anode (electrode 1)
    on y+ over x in [x_lo, x_hi], walls elsewhere."""
    tags = box_tags(dim, n_el, coords, WALL)
    tags[0][:] = INLET
    tags[1][:] = OUTLET
    for s, j in ((2, 0), (3, 1)):
        if s == 3 and not anode:
            continue
        cen = face_centres(dim, n_el, coords, s)
        sel = (cen[:, 0] > x_lo) & (cen[:, 0] < x_hi)
        tags[s][sel] = ELECTRODE0 + j
    return tags


def config(name: str, p: Optional[int] = None) -> Problem:
    """The synthetic workloads, by name.

    mms2d_8x8_p2      2D unit square, 8x8 quads, p=2, binary electrolyte z=(+1,-1),
                      D=(1e-3,2e-3), u=(1,0.5), all faces DIRICHLET.
    cube16_p3         3D unit cube, 16^3 hex, p=3, binary electrolyte, plate flow
                      u_x = 6y(1-y), inlet/outlet, two electrodes on y faces.
    channel64_p3      (0,4)x(0,2)x(0,1), 64x32x16 hex, p=3, three ions
                      z=(+1,-1,+2), D=(5e-4,1e-3,2e-3), plate flow u_avg=5.
    cube24_p2         3D unit cube, 24^3 hex, p=2, as cube16.
    reactor192_p{2,4} (0,12)x(0,3)x(0,1), 192x48x16 hex, CuSO4-like binary
                      z=(+2,-2), D=(1e-4,1.48e-4), Butler-Volmer cathode on y=0 and
                      anode (phi_app = 0) on y=3 for x in [5,7] (electrode length
                      between inlet and outlet regions 5:2:5 as in Sec. 5.2), with
                      a J_0 profile across z.
    Small variants for tests take a suffix, e.g. 'cube_n4_p3' (n^3 elements).
    """
    if name == "mms2d_8x8_p2" or name.startswith("mms2d_n"):
        n = 8 if name == "mms2d_8x8_p2" else int(name.split("_n")[1].split("_")[0])
        pp = 2 if p is None else p
        n_el = [n, n, 1]
        coords = _linspace_coords(n_el[:2], [1.0, 1.0])
        tags = box_tags(2, n_el, coords, DIRICHLET)
        return Problem(dim=2, n_el=n_el, coords=coords, tags=tags, m=2, z=[1.0, -1.0],
                       D=[1e-3, 2e-3], c_in=[1.0, 1.0], p=pp, q=pp + 2,
                       vel_kind=VEL_CONSTANT, vel_params=[1.0, 0.5, 0.0] + [0.0] * 5, name=name)
    if name in ("cube16_p3", "cube24_p2") or name.startswith("cube_n"):
        if name == "cube16_p3":
            n, pp = 16, 3
        elif name == "cube24_p2":
            n, pp = 24, 2
        else:
            n = int(name.split("_n")[1].split("_")[0])
            pp = int(name.split("_p")[1]) if "_p" in name else 3
        if p is not None:
            pp = p
        n_el = [n, n, n]
        coords = _linspace_coords(n_el, [1.0, 1.0, 1.0])
        tags = _reactor_tags(3, n_el, coords, 1.0 / 3.0, 2.0 / 3.0)
        return Problem(dim=3, n_el=n_el, coords=coords, tags=tags, m=2, z=[1.0, -1.0],
                       D=[1e-3, 2e-3], c_in=[1.0, 1.0], p=pp, q=pp + 2,
                       vel_kind=VEL_PLATE, vel_params=[0, 1, 0.0, 1.0, 1.0, 0, 0, 0],
                       bv_oxidant=0, bv_J0=0.1, bv_alpha1=0.5, bv_alpha2=0.5, bv_n=1.0,
                       bv_gamma=1.0, bv_c_ref=1.0, bv_phi_app=[1.17, 0.0, 0.0, 0.0], name=name)
    if name == "channel64_p3" or name.startswith("channel_n"):
        if name == "channel64_p3":
            n_el = [64, 32, 16]
        else:
            k = int(name.split("_n")[1].split("_")[0])  # scale: (4k, 2k, k)
            n_el = [4 * k, 2 * k, k]
        pp = 3 if p is None else p
        coords = _linspace_coords(n_el, [4.0, 2.0, 1.0])
        tags = _reactor_tags(3, n_el, coords, 4.0 / 3.0, 8.0 / 3.0)
        return Problem(dim=3, n_el=n_el, coords=coords, tags=tags, m=3, z=[1.0, -1.0, 2.0],
                       D=[5e-4, 1e-3, 2e-3], c_in=[1.0, 2.0, 0.5], p=pp, q=pp + 2,
                       vel_kind=VEL_PLATE, vel_params=[0, 1, 0.0, 2.0, 5.0, 0, 0, 0],
                       bv_oxidant=2, bv_J0=0.1, bv_alpha1=0.5, bv_alpha2=0.5, bv_n=2.0,
                       bv_gamma=1.0, bv_c_ref=0.5, bv_phi_app=[1.17, 0.0, 0.0, 0.0], name=name)
    if name.startswith("reactor192") or name.startswith("reactor_n"):
        if name.startswith("reactor192"):
            n_el = [192, 48, 16]
        else:
            k = int(name.split("_n")[1].split("_")[0])  # scale: (12k, 3k, k)
            n_el = [12 * k, 3 * k, k]
        pp = int(name.split("_p")[1]) if "_p" in name else 2
        if p is not None:
            pp = p
        coords = _linspace_coords(n_el, [12.0, 3.0, 1.0])
        tags = _reactor_tags(3, n_el, coords, 5.0, 7.0, anode=True)
        return Problem(dim=3, n_el=n_el, coords=coords, tags=tags, m=2, z=[2.0, -2.0],
                       D=[1e-4, 1.48e-4], c_in=[1.0, 1.0], p=pp, q=pp + 2,
                       vel_kind=VEL_PLATE, vel_params=[0, 1, 0.0, 3.0, 1.0, 0, 0, 0],
                       bv_oxidant=0, bv_J0=0.05, bv_alpha1=0.5, bv_alpha2=0.5, bv_n=2.0,
                       bv_gamma=1.0, bv_c_ref=1.0, bv_phi_app=[0.1 * 38.92, 0.0, 0.0, 0.0],
                       bv_J0_axis=2, bv_J0_lo=0.0, bv_J0_hi=1.0, name=name)
    raise KeyError(name)


def reactor_initial_state(P: Problem, phi_app) -> np.ndarray:
    """Initial guess of the reactor solves: c = c_in and Phi = phi_app / 2 (between
    the anode at 0 and the cathode), one block per operating point."""
    out = []
    for ph in np.atleast_1d(phi_app):
        u = np.zeros((P.n_fields, P.E, P.Np))
        u[0] = 0.5 * ph
        for k in range(1, P.n_fields):
            u[k] = P.c_in[k - 1]
        out.append(u.reshape(-1))
    return np.concatenate(out)


def random_state(P: Problem, seed: int, c_mean: float = 1.0, c_amp: float = 0.1,
                 phi_amp: float = 0.1) -> np.ndarray:
    """u[f][e][i]: Phi ~ phi_amp U(-1,1); c_k ~ c_mean_k (1 + c_amp U(-1,1)), where
    c_mean_k is the inlet value scaled by c_mean."""
    g = torch.Generator().manual_seed(seed)
    r = torch.rand((P.n_fields, P.E, P.Np), generator=g, dtype=torch.float64) * 2 - 1
    u = r.numpy().copy()
    u[0] *= phi_amp
    for k in range(1, P.n_fields):
        u[k] = P.c_in[k - 1] * c_mean * (1.0 + c_amp * u[k])
    return u.reshape(-1)


def random_vector(P: Problem, seed: int, n: Optional[int] = None) -> np.ndarray:
    """A direction ~ U(-1,1) of n entries (default: one state vector)."""
    g = torch.Generator().manual_seed(seed)
    n = P.n_dof if n is None else n
    return (torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1).numpy().copy()


def random_sources(P: Problem, seed: int, amp: float = 1.0) -> np.ndarray:
    """Volume source values at quadrature points, [NF][E][Nq]."""
    return amp * random_vector(P, seed, P.n_fields * P.E * P.Nq)


def random_dirichlet(P: Problem, seed: int, base: float = 1.0, amp: float = 0.1) -> np.ndarray:
    """Exterior Dirichlet data at boundary-face quadrature points, [NF][NBF][Nfq]."""
    v = random_vector(P, seed, P.n_fields * P.n_bfaces * P.Nfq).reshape(
        P.n_fields, P.n_bfaces, P.Nfq)
    out = v * amp
    out[1:] += base
    return out.reshape(-1)
