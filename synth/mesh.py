"""Surface meshes of linear triangles (inputs only).

Nodes are numbered ring by ring (circumferential index fastest), which keeps every
node's neighbours within one ring of it; that ordering is what the device gather
relies on for cache locality, so generators here produce it directly.
Triangle corners are ordered so that (X2-X1) x (X3-X1) points out of the lumen.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class Mesh:
    xyz: np.ndarray                 # [N][3] float64, metres
    tri: np.ndarray                 # [E][3] int32, outward orientation
    fixed: np.ndarray               # [N][3] uint8, 1 = dof held at zero
    name: str = "mesh"
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.tri.shape[0])

    def check(self) -> None:
        assert self.xyz.dtype == np.float64 and self.xyz.ndim == 2 and self.xyz.shape[1] == 3
        assert self.tri.dtype == np.int32 and self.tri.ndim == 2 and self.tri.shape[1] == 3
        assert self.fixed.dtype == np.uint8 and self.fixed.shape == self.xyz.shape
        assert self.tri.min() >= 0 and self.tri.max() < self.n_nodes


def _ring_tube(nc: int, na: int, length: float, radius_of_z, z0: float = 0.0,
               clamp_ends: bool = True, name: str = "tube") -> Mesh:
    """Tube along +z with nc nodes per ring and na rings; radius_of_z(z) gives the wall radius."""
    if nc < 3 or na < 2:
        raise ValueError("need nc >= 3 and na >= 2")
    z = z0 + length * np.arange(na, dtype=np.float64) / (na - 1)
    th = 2.0 * np.pi * np.arange(nc, dtype=np.float64) / nc
    r = np.asarray(radius_of_z(z), dtype=np.float64) * np.ones(na)
    xyz = np.empty((na, nc, 3), dtype=np.float64)
    xyz[:, :, 0] = r[:, None] * np.cos(th)[None, :]
    xyz[:, :, 1] = r[:, None] * np.sin(th)[None, :]
    xyz[:, :, 2] = z[:, None]
    xyz = xyz.reshape(-1, 3)
    a = np.arange(na - 1)[:, None]
    c = np.arange(nc)[None, :]
    p0 = a * nc + c
    p1 = a * nc + (c + 1) % nc
    p2 = (a + 1) * nc + (c + 1) % nc
    p3 = (a + 1) * nc + c
    t1 = np.stack([p0, p1, p2], axis=-1).reshape(-1, 3)
    t2 = np.stack([p0, p2, p3], axis=-1).reshape(-1, 3)
    tri = np.empty((t1.shape[0] * 2, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    fixed = np.zeros((nc * na, 3), dtype=np.uint8)
    if clamp_ends:
        fixed[:nc, :] = 1
        fixed[(na - 1) * nc:, :] = 1
    m = Mesh(xyz=xyz, tri=tri, fixed=fixed, name=name,
             meta={"nc": nc, "na": na, "length": length, "z0": z0})
    m.check()
    return m


def tube_mesh(nc: int = 40, na: int = 40, radius: float = 0.01, length: float = 0.10,
              clamp_ends: bool = True) -> Mesh:
    """Straight circular tube (defaults: R = 1 cm, L = 10 cm, 40 x 40 nodes, 3120 triangles)."""
    m = _ring_tube(nc, na, length, lambda z: np.full_like(z, radius), clamp_ends=clamp_ends,
                   name=f"tube_{nc}x{na}")
    m.meta["radius"] = radius
    return m


def aneurysm_mesh(nc: int = 400, na: int = 500, radius: float = 0.01, length: float = 0.12,
                  bulge_center: float = 0.06, bulge_width: float = 0.015,
                  max_radius: float = 0.02) -> Mesh:
    """Tube with a Gaussian bulge r(z) = R + (Rmax - R) exp(-(z - zc)^2 / (2 w^2)), ends clamped."""
    def rz(z):
        return radius + (max_radius - radius) * np.exp(-((z - bulge_center) ** 2) / (2.0 * bulge_width ** 2))
    m = _ring_tube(nc, na, length, rz, name=f"aneurysm_{nc}x{na}")
    m.meta.update(radius=radius, max_radius=max_radius)
    return m


def tube_for_nodes(n_nodes: int, radius: float = 0.01, length: float = 0.10) -> Mesh:
    """Straight clamped tube with about n_nodes nodes and near-square quads."""
    nc = max(8, int(round(np.sqrt(n_nodes * 2.0 * np.pi * radius / length))))
    na = max(2, int(round(n_nodes / nc)))
    return tube_mesh(nc=nc, na=na, radius=radius, length=length)


def plate_mesh(nx: int = 5, ny: int = 4, lx: float = 0.04, ly: float = 0.03,
               jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Flat plate in the z = 0 plane (normal +z), optional interior node jitter; nothing fixed."""
    x = lx * np.arange(nx) / (nx - 1)
    y = ly * np.arange(ny) / (ny - 1)
    X, Y = np.meshgrid(x, y, indexing="xy")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=-1)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.Philox(key=seed))
        interior = np.ones((ny, nx), dtype=bool)
        interior[0, :] = interior[-1, :] = interior[:, 0] = interior[:, -1] = False
        d = rng.uniform(-jitter, jitter, size=(ny, nx, 2))
        d[~interior] = 0.0
        xyz[:, 0] += d[..., 0].ravel() * lx / (nx - 1)
        xyz[:, 1] += d[..., 1].ravel() * ly / (ny - 1)
    tri = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            p0, p1 = j * nx + i, j * nx + i + 1
            p3, p2 = (j + 1) * nx + i, (j + 1) * nx + i + 1
            tri.append((p0, p1, p2))
            tri.append((p0, p2, p3))
    m = Mesh(xyz=xyz.astype(np.float64), tri=np.asarray(tri, dtype=np.int32),
             fixed=np.zeros((nx * ny, 3), dtype=np.uint8), name=f"plate_{nx}x{ny}",
             meta={"nx": nx, "ny": ny})
    m.check()
    return m


def single_triangle(points=None) -> Mesh:
    """One element (default: a scalene triangle tilted out of every coordinate plane)."""
    if points is None:
        points = [[0.0, 0.0, 0.0], [0.003, 0.0005, 0.001], [0.0007, 0.0025, -0.0004]]
    xyz = np.asarray(points, dtype=np.float64)
    m = Mesh(xyz=xyz, tri=np.array([[0, 1, 2]], dtype=np.int32),
             fixed=np.zeros((3, 3), dtype=np.uint8), name="one_triangle")
    m.check()
    return m


def _rotation(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def arch_mesh(target_elems: int = 500_000, arch_radius: float = 0.03, radius: float = 0.012,
              branch_radii=(0.006, 0.005, 0.004), branch_length: float = 0.04,
              straight: float = 0.03) -> Mesh:
    """Synthetic arch: a curved tube (half torus between two straight legs) plus three side
    branches rising from the top of the arch.

    Each branch is its own tube whose root ring sits just outside the arch wall and is
    clamped, as is its outlet ring and both arch ends; branches are not stitched into the
    arch surface. The mesh exercises uneven node degrees and several disconnected
    components in one launch, with consistent outward orientation; it is a synthetic
    stand-in, not an anatomical model.
    """
    # Arc length of the centreline: leg + half circle + leg.
    s_total = 2 * straight + np.pi * arch_radius
    # Element budget: main tube gets ~80 %, branches share the rest.
    main_elems = int(target_elems * 0.8)
    nc = max(16, int(round(np.sqrt(main_elems / 2 * 2 * np.pi * radius / s_total))))
    na = max(2, int(round(main_elems / (2 * nc))) + 1)
    s = s_total * np.arange(na) / (na - 1)
    # centreline points and frames
    cen = np.zeros((na, 3))
    tan = np.zeros((na, 3))
    nor = np.zeros((na, 3))
    for k, sk in enumerate(s):
        if sk <= straight:  # up leg along +z at x = -arch_radius
            cen[k] = [-arch_radius, 0.0, sk]
            tan[k] = [0, 0, 1]
        elif sk <= straight + np.pi * arch_radius:
            phi = (sk - straight) / arch_radius  # 0..pi
            cen[k] = [-arch_radius * np.cos(phi), 0.0, straight + arch_radius * np.sin(phi)]
            tan[k] = [np.sin(phi), 0.0, np.cos(phi)]
        else:
            cen[k] = [arch_radius, 0.0, straight - (sk - straight - np.pi * arch_radius)]
            tan[k] = [0, 0, -1]
        nor[k] = [0.0, 1.0, 0.0]
    binor = np.cross(tan, nor)
    th = 2 * np.pi * np.arange(nc) / nc
    xyz = (cen[:, None, :] + radius * (np.cos(th)[None, :, None] * binor[:, None, :]
                                         + np.sin(th)[None, :, None] * nor[:, None, :]))
    xyz = xyz.reshape(-1, 3)
    a = np.arange(na - 1)[:, None]
    c = np.arange(nc)[None, :]
    p0 = a * nc + c
    p1 = a * nc + (c + 1) % nc
    p2 = (a + 1) * nc + (c + 1) % nc
    p3 = (a + 1) * nc + c
    t1 = np.stack([p0, p1, p2], axis=-1).reshape(-1, 3)
    t2 = np.stack([p0, p2, p3], axis=-1).reshape(-1, 3)
    tris = [t1, t2]
    # orientation: make the first triangle outward w.r.t. the centreline
    def outward(tt, pts, cref):
        e1 = pts[tt[:, 1]] - pts[tt[:, 0]]
        e2 = pts[tt[:, 2]] - pts[tt[:, 0]]
        n = np.cross(e1, e2)
        cg = pts[tt].mean(axis=1)
        return np.einsum("ij,ij->i", n, cg - cref)
    nodes = [xyz]
    fixed_rows = [np.r_[np.arange(nc), np.arange((na - 1) * nc, na * nc)]]
    offset = xyz.shape[0]
    centres = []
    branch_elems = (target_elems - main_elems) // max(1, len(branch_radii))
    for b, rb in enumerate(branch_radii):
        phi_b = np.pi * (b + 1) / (len(branch_radii) + 1)
        base = np.array([-arch_radius * np.cos(phi_b), 0.0, straight + arch_radius * np.sin(phi_b)])
        up = np.array([-np.cos(phi_b), 0.0, np.sin(phi_b)])  # radial out of the arch circle
        ncb = max(8, int(round(np.sqrt(branch_elems / 2 * 2 * np.pi * rb / branch_length))))
        nab = max(2, int(round(branch_elems / (2 * ncb))) + 1)
        sb = radius + branch_length * np.arange(nab) / (nab - 1)
        e_a = np.array([0.0, 1.0, 0.0])
        e_b = np.cross(up, e_a)
        thb = 2 * np.pi * np.arange(ncb) / ncb
        pts = (base[None, None, :] + sb[:, None, None] * up[None, None, :]
               + rb * (np.cos(thb)[None, :, None] * e_b[None, None, :]
                       + np.sin(thb)[None, :, None] * e_a[None, None, :])).reshape(-1, 3)
        ab = np.arange(nab - 1)[:, None]
        cb = np.arange(ncb)[None, :]
        q0 = ab * ncb + cb
        q1 = ab * ncb + (cb + 1) % ncb
        q2 = (ab + 1) * ncb + (cb + 1) % ncb
        q3 = (ab + 1) * ncb + cb
        bt = np.concatenate([np.stack([q0, q1, q2], -1).reshape(-1, 3),
                             np.stack([q0, q2, q3], -1).reshape(-1, 3)])
        # orient outward from the branch axis
        proj = base + (np.einsum("ij,j->i", pts[bt].mean(axis=1) - base, up))[:, None] * up[None, :]
        e1 = pts[bt[:, 1]] - pts[bt[:, 0]]
        e2 = pts[bt[:, 2]] - pts[bt[:, 0]]
        sgn = np.einsum("ij,ij->i", np.cross(e1, e2), pts[bt].mean(axis=1) - proj)
        bt[sgn < 0] = bt[sgn < 0][:, [0, 2, 1]]
        nodes.append(pts)
        tris.append(bt + offset)
        fixed_rows.append(offset + np.arange(ncb))                      # root ring (joined)
        fixed_rows.append(offset + np.arange((nab - 1) * ncb, nab * ncb))  # outlet ring
        offset += pts.shape[0]
        centres.append(base)
    xyz_all = np.concatenate(nodes)
    tri_all = np.concatenate(tris).astype(np.int32)
    # orient main-tube triangles outward from the centreline point of their ring
    main_n = 2 * nc * (na - 1)
    mt = tri_all[:main_n]
    ring = np.minimum(mt[:, 0] // nc, na - 1)
    sgn = outward(mt, xyz_all, cen[ring])
    mt[sgn < 0] = mt[sgn < 0][:, [0, 2, 1]]
    tri_all[:main_n] = mt
    fixed = np.zeros(xyz_all.shape, dtype=np.uint8)
    fixed[np.concatenate(fixed_rows)] = 1
    m = Mesh(xyz=xyz_all, tri=tri_all, fixed=fixed, name="arch",
             meta={"nc": nc, "na": na, "centreline": cen, "s": s})
    m.check()
    return m
