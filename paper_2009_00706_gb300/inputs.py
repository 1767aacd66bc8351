"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers and builds the
input surfaces and parameter sets.  Both sides of every parity test receive the very same
arrays from here.

* Random numbers: SplitMix64 (Steele, Lea, Flood 2014), used counter-style: the i-th draw of
  stream `seed` is mix(seed * 2^32 + i).  Normals by the Box-Muller transform.
* Surfaces: a subdivided icosahedron projected on a sphere, every shared vertex jittered once,
  so the surface stays closed; and a filleted box ("rounded box") meshed as a mapped grid,
  the bluff bodies of the truck-like workload.  Triangles are counter-clockwise seen from
  outside the body.
* Workloads: the mesh parameters, physical parameters and state vectors of the five
  workloads (small sphere, sphere LES step, bluff-body pair, batched spheres, learned
  preconditioner), each with the sizes of the paper's runs (Sec. "Validation: flow past a
  sphere", Sec. "Scaling", Sec. "Platooning").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n 64-bit outputs of SplitMix64 stream `seed` starting at draw `offset`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0x100000000) + i * _GOLD
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in (0, 1): (top 53 bits + 0.5) * 2^-53."""
    z = splitmix64(seed, n, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, sigma: float = 1.0, offset: int = 0) -> np.ndarray:
    """n N(0, sigma^2) draws by Box-Muller (one normal per pair of uniforms)."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ------------------------------------------------------------------------------------------
# surfaces
# ------------------------------------------------------------------------------------------
def icosphere(level: int, radius: float, center, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Closed triangulated sphere: icosahedron subdivided `level` times (20 * 4^level
    triangles), vertices projected on the sphere, then every vertex coordinate jittered by
    N(0, jitter^2) (shared vertices once).  Returns [n_tri, 3, 3] float64, CCW from outside."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache: dict = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    if jitter > 0.0:
        V = V + normal(seed, V.size, jitter).reshape(V.shape)
    F = np.array(faces, dtype=np.int64)
    tri = V[F]
    # orient counter-clockwise seen from outside
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    out = np.einsum("ij,ij->i", n, tri.mean(axis=1) - np.asarray(center))
    flip = out < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return np.ascontiguousarray(tri)


def rounded_box(lo, hi, fillet: float, n_per_edge: int, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Closed filleted box [lo, hi] meshed as a cube-sphere mapped grid: each face of the unit
    cube carries an n x n grid, every grid point p of the cube surface is mapped to the
    rounded box by  x = clamp(p) + fillet * (p - clamp(p)) / |p - clamp(p)|  where clamp()
    projects on the inner box shrunk by `fillet`.  Returns [12 n^2 ... , 3, 3], CCW from outside."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    inner = half - fillet
    n = n_per_edge
    s = np.linspace(-1.0, 1.0, n + 1)
    key_of: dict = {}
    verts: list = []
    faces: list = []

    def vid(p):
        k = tuple(np.round(p * n).astype(np.int64))
        if k not in key_of:
            key_of[k] = len(verts)
            verts.append(p.copy())
        return key_of[k]

    for axis in range(3):
        for sign in (-1.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            grid = np.empty((n + 1, n + 1), dtype=np.int64)
            for i in range(n + 1):
                for j in range(n + 1):
                    p = np.zeros(3)
                    p[axis] = sign
                    p[u_ax] = s[i]
                    p[v_ax] = s[j]
                    grid[i, j] = vid(p)
            for i in range(n):
                for j in range(n):
                    a, b, cc, d = grid[i, j], grid[i + 1, j], grid[i + 1, j + 1], grid[i, j + 1]
                    faces.append((a, b, cc))
                    faces.append((a, cc, d))
    P = np.array(verts)
    # map cube-surface points: scale to the box, then round the corners/edges
    X = P * half
    cl = np.clip(X, -inner, inner)
    d = X - cl
    nd = np.linalg.norm(d, axis=1)
    nd[nd == 0] = 1.0
    V = cl + fillet * d / nd[:, None] + c
    if jitter > 0.0:
        V = V + normal(seed, V.size, jitter).reshape(V.shape)
    F = np.array(faces, dtype=np.int64)
    tri = V[F]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    out = np.einsum("ij,ij->i", nrm, tri.mean(axis=1) - c)
    flip = out < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return np.ascontiguousarray(tri)


# ------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------
def grid_box(lo, hi, grid: float, apex=(0.6180339887498949, 0.2763932022500210)) -> np.ndarray:
    """Surface of the axis-aligned box [lo, hi], counter-clockwise seen from outside.  Each face is
    cut into rectangles by its own edges and by the planes at whole multiples of `grid` between
    them; each rectangle into 4 triangles around an interior vertex at the fractions `apex` of its
    sides.  With the faces on sub-cell planes of an octree and `grid` its finest element size,
    every triangle lies in one element face patch and no volume point is cut, so the quadrature of
    the body is exact.  The interior vertex lies on neither diagonal of its rectangle, so rays cast
    from element centres, which project onto rectangle centres, meet no triangle edge there."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)

    def breaks(a, b):
        k0, k1 = int(np.floor(a / grid)) + 1, int(np.ceil(b / grid)) - 1
        inner = [k * grid for k in range(k0, k1 + 1) if a < k * grid < b]
        return [a] + inner + [b]

    tris = []
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3          # e_a x e_b = e_k
        ba, bb = breaks(lo[a], hi[a]), breaks(lo[b], hi[b])
        for side in (0, 1):
            x = hi[k] if side else lo[k]
            for i in range(len(ba) - 1):
                for j in range(len(bb) - 1):
                    def P(sa, sb):
                        p = np.zeros(3)
                        p[k] = x
                        p[a] = sa
                        p[b] = sb
                        return p
                    c = [P(ba[i], bb[j]), P(ba[i + 1], bb[j]), P(ba[i + 1], bb[j + 1]), P(ba[i], bb[j + 1])]
                    v = P(ba[i] + apex[0] * (ba[i + 1] - ba[i]), bb[j] + apex[1] * (bb[j + 1] - bb[j]))
                    for q in range(4):
                        p0, p1 = c[q], c[(q + 1) % 4]
                        tris.append((p0, p1, v) if side else (p1, p0, v))   # outward +e_k / -e_k
    return np.array(tris, dtype=np.float64)


REGION_SPHERE_BAND, REGION_BOX, REGION_CONE = 0, 1, 2
SCHEME_BE, SCHEME_CN, SCHEME_BDF2 = 0, 1, 2


@dataclass
class Region:
    kind: int
    level: int
    par: tuple  # up to 8 doubles

    def packed(self):
        p = list(self.par) + [0.0] * (8 - len(self.par))
        return p[:8]


@dataclass
class Physics:
    rho: float = 1.0
    mu: float = 0.02
    dt: float = 0.01
    scheme: int = SCHEME_BE
    Cb: float = 4.0
    CI: float = 36.0
    g: tuple = (0.0, 0.0, 0.0)
    uinf: tuple = (1.0, 0.0, 0.0)
    drop_visc: int = 0

    def packed(self):
        return [self.rho, self.mu, self.dt, float(self.scheme), self.Cb, self.CI, *self.g, *self.uinf,
                float(self.drop_visc)]


@dataclass
class Workload:
    name: str
    lo: tuple
    hi: tuple
    base_level: int
    regions: list
    lmax: int
    physics: Physics
    surface: callable = field(repr=False, default=None)
    seed: int = 0

    def triangles(self) -> np.ndarray:
        return self.surface() if self.surface is not None else np.zeros((0, 3, 3))


def small_sphere(seed: int = 0) -> Workload:
    """Unit cube, level 3 far field, level 6 within 0.05 of a sphere r = 0.1 at the centre
    (icosphere 1280 triangles, jitter 1e-4), Re 10 on the diameter, BE dt 0.01, C_b 4, L_max 3."""
    c = (0.5, 0.5, 0.5)
    return Workload(
        name="small_sphere", lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), base_level=3,
        regions=[Region(REGION_SPHERE_BAND, 6, (*c, 0.1, 0.05))], lmax=3,
        physics=Physics(rho=1.0, mu=0.02, dt=0.01, scheme=SCHEME_BE),
        surface=lambda: icosphere(3, 0.1, c, 1e-4, seed), seed=seed)


def sphere_les(seed: int = 0) -> Workload:
    """Box 32 x 16 x 16 diameters, sphere D = 1 at (8, 8, 8) (icosphere level 6, 81920
    triangles), level 4 background, level 10 within 0.25 D of the surface, a wake cone behind
    the sphere at levels 9 (length 11, radius 1 at the centre) and 8 (length 20, radius 2.25),
    half-angle 15 degrees; Re 1e4, BDF2 dt 0.01.  2,001,176 elements."""
    c = (8.0, 8.0, 8.0)
    return Workload(
        name="sphere_les", lo=(0.0, 0.0, 0.0), hi=(32.0, 16.0, 16.0), base_level=4,
        regions=[Region(REGION_SPHERE_BAND, 10, (*c, 0.5, 0.25)),
                 Region(REGION_CONE, 9, (8.0, 8.0, 8.0, 11.0, 1.0, 0.2679491924)),
                 Region(REGION_CONE, 8, (8.0, 8.0, 8.0, 20.0, 2.25, 0.2679491924))],
        lmax=3, physics=Physics(rho=1.0, mu=1e-4, dt=0.01, scheme=SCHEME_BDF2),
        surface=lambda: icosphere(6, 0.5, c, 1e-5, seed), seed=seed)


TRUCK_L = 5.05   # truck length: cab 1, gap 0.05, trailer 4


def truck(x0: float, yc: float, zb: float, n_per_edge: int, jitter: float, seed: int) -> np.ndarray:
    """Two disjoint closed filleted boxes (fillet 0.05), bottom-aligned at z = zb and centred on
    y = yc: a cab 1 x 1 x 0.8 at x in [x0, x0 + 1] in front of a trailer 4 x 1 x 1 at
    x in [x0 + 1.05, x0 + 5.05].  CCW from outside."""
    cab = rounded_box((x0, yc - 0.5, zb), (x0 + 1.0, yc + 0.5, zb + 0.8), 0.05, n_per_edge, jitter, seed)
    trailer = rounded_box((x0 + 1.05, yc - 0.5, zb), (x0 + TRUCK_L, yc + 0.5, zb + 1.0), 0.05, n_per_edge, jitter,
                          seed + 1)
    return np.concatenate([cab, trailer])


def bluff_pair(seed: int = 0, levels: int = 0, n_per_edge: int = 91) -> Workload:
    """Two trucks in tandem at a 0.5 L gap (L = 5.05), the first 5 L behind the inlet of a
    16 L x 2 L x 2 L box, both centred in y and z; each body two rounded boxes of 12 n^2 triangles
    (n = 91: 198,744 triangles per truck), jitter 1e-5.  Levels 5 (far field) to 11: level 11 in a
    box around both trucks and the near wake, 10 and 9 in longer wake boxes, 8 around those.
    `levels` < 0 lowers every refinement level by -levels, not below the far field's 5 (same geometry,
    smaller mesh).  Re 1e6 on
    L (mu = L / 1e6), BDF2 dt 0.01.  At full size: 19,791,080 elements, 19,520,852 nodes."""
    L = TRUCK_L
    Lx, Ly, Lz = 16 * L, 2 * L, 2 * L
    yc, zc = 0.5 * Ly, 0.5 * Lz
    zb = zc - 0.5
    x1 = 5 * L
    x2 = x1 + L + 0.5 * L
    d = levels

    def box(lev, xa, xb, half):
        return Region(REGION_BOX, max(5, lev + d), (xa, yc - half, zc - half, xb, yc + half, zc + half))

    regions = [box(11, x1 - 0.25, x2 + L + 12.0, 3.1), box(10, x1 - 1.0, x2 + L + 30.0, 3.6),
               box(9, x1 - 5.0, Lx, 4.5), box(8, 0.0, Lx, 6.0)]
    return Workload(
        name="bluff_pair", lo=(0.0, 0.0, 0.0), hi=(Lx, Ly, Lz), base_level=5, regions=regions, lmax=3,
        physics=Physics(rho=1.0, mu=L / 1e6, dt=0.01, scheme=SCHEME_BDF2),
        surface=lambda: np.concatenate([truck(x1, yc, zb, n_per_edge, 1e-5, seed),
                                        truck(x2, yc, zb, n_per_edge, 1e-5, seed + 2)]), seed=seed)


def inout_truck(level: int, seed: int = 0, n_per_edge: int = 32) -> Workload:
    """The in/out comparison of Table in-out on a uniform grid: one truck (cab and trailer, fillet
    0.05, 0.05 gap between them; 12 n^2 triangles per box, n = 32: 24,576 triangles, jitter 1e-5)
    centred in a cube of edge 6.4, meshed uniformly at `level` (6, 7, 8: the paper's 64^3, 128^3,
    256^3 grids), no refinement regions."""
    edge = 6.4
    c = 0.5 * edge
    return Workload(
        name="inout_truck_%d" % (1 << level), lo=(0.0, 0.0, 0.0), hi=(edge, edge, edge), base_level=level,
        regions=[], lmax=3, physics=Physics(),
        surface=lambda: truck(c - 0.5 * TRUCK_L, c, c - 0.5, n_per_edge, 1e-5, seed), seed=seed)


def state(n_nodes: int, seed: int = 0, sigma: float = 0.01):
    """u_prev = uniform inflow (1, 0, 0), p = 0; u = u_prev + N(0, sigma^2) on the velocity;
    v ~ N(0, 1) on every dof.  Node-major [n_nodes, 4] float64 (u, v, w, p)."""
    up = np.zeros((n_nodes, 4))
    up[:, 0] = 1.0
    u = up.copy()
    u[:, :3] += normal(seed * 4 + 1, n_nodes * 3, sigma).reshape(n_nodes, 3)
    v = normal(seed * 4 + 2, n_nodes * 4).reshape(n_nodes, 4)
    return u, up, v


def _sphere_band_model(level: int, w: float, r: float = 0.1) -> float:
    """Element-count model of a unit-cube sphere mesh (level 3 far field, `level` within w of the
    sphere): 512 base elements plus ~1.9 x the band volume over the fine element volume (the factor
    accounts for the 2:1 transition layers; 1.9 reproduces the small-sphere workload)."""
    shell = 4.0 / 3.0 * math.pi * ((r + w) ** 3 - max(r - w, 0.0) ** 3)
    return 512.0 + 1.9 * shell * 8.0 ** level


def batched_spheres(n: int = 64, seed0: int = 0):
    """n independent unit-cube sphere problems (seeds seed0 .. seed0+n-1): target element counts
    log-uniform in [5k, 200k], Reynolds numbers log-uniform in [1, 1e6] on the diameter 0.2 (mu = 0.2 /
    Re), BE dt 0.01.  For each problem the finest level (5..8) and the band width are chosen by
    bisection on the element-count model so that the model meets the target.
    Returns a list of (Workload, target elements, Re)."""
    out = []
    for k in range(n):
        s = seed0 + k
        u = uniform(1000 + s, 2)
        target = math.exp(math.log(5e3) + u[0] * (math.log(2e5) - math.log(5e3)))
        Re = 10.0 ** (6.0 * u[1])
        level, w = 8, 0.01
        for L in (5, 6, 7, 8):
            if _sphere_band_model(L, 0.09) >= target:
                level = L
                break
        lo, hi = 1e-4, 0.09
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if _sphere_band_model(level, mid) < target:
                lo = mid
            else:
                hi = mid
        w = 0.5 * (lo + hi)
        c = (0.5, 0.5, 0.5)
        wl = Workload(name=f"sphere_{s}", lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), base_level=3,
                      regions=[Region(REGION_SPHERE_BAND, level, (*c, 0.1, w))], lmax=3,
                      physics=Physics(rho=1.0, mu=0.2 / Re, dt=0.01, scheme=SCHEME_BE),
                      surface=(lambda s=s: icosphere(3, 0.1, (0.5, 0.5, 0.5), 1e-4, s)), seed=s)
        out.append((wl, target, Re))
    return out
