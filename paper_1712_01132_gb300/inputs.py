"""Seeded synthetic porous geometries (solid masks), shared by the tests, the smoke check and the
benchmark.  This module holds only geometry generation; none of the solver's arithmetic.

Masks are numpy bool arrays, True = solid, shape (n2, n1) in 2D or (n3, n2, n1) in 3D (x1 is the
fastest index and the flow direction).  Every random generator takes an explicit seed and uses
numpy's default_rng.

Workloads (the paper's digital-rock images are not available, so these stand in for them):
  * ``cylinder_cell``      -- periodic unit cell with one centred circular cylinder.
  * ``random_discs``       -- overlapping discs with uniform radii and periodic wrap, added until a
                              target solid fraction is reached (stands in for the random-cylinder
                              image of Sec. 4.1).
  * ``gaussian_rock``      -- a 3D Gaussian random field (white noise convolved periodically with a
                              Gaussian of the given correlation length) thresholded at the target
                              porosity (stands in for the bead-pack image of Sec. 4.2).
  * ``sierpinski_carpet``  -- the level-3 carpet of Sec. 4.1 (removed squares are solid).
  * ``sphere_quadrant``    -- the quadrant of the cubic sphere array of Sec. 4.2.
  * ``keep_percolating``   -- fills every fluid region that does not connect x1-periodic images.
  * ``disc_batch``         -- many disc packings of uneven sizes and porosities, each with its own
                              Knudsen number (the batched workload).
"""
import math

import numpy as np


def cylinder_cell(n=32, porosity=0.7):
    """n x n cell-centred grid with a centred disc of area (1 - porosity) n^2."""
    r = math.sqrt((1.0 - porosity) * n * n / math.pi)
    c = np.arange(n) + 0.5
    x, y = np.meshgrid(c, c, indexing="xy")
    return (x - n / 2) ** 2 + (y - n / 2) ** 2 <= r * r


def random_discs(n1, n2, seed, rmin=6.0, rmax=20.0, solid_fraction=0.5, percolating=True):
    """Overlapping discs, centres uniform in [0,n1) x [0,n2), radii uniform in [rmin, rmax],
    periodic wrap, added one at a time until the solid fraction reaches ``solid_fraction``."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((n2, n1), dtype=bool)
    c1 = np.arange(n1) + 0.5
    c2 = np.arange(n2) + 0.5
    while solid.mean() < solid_fraction:
        x0 = rng.uniform(0, n1)
        y0 = rng.uniform(0, n2)
        r = rng.uniform(rmin, rmax)
        dx = np.abs(c1 - x0)
        dx = np.minimum(dx, n1 - dx)
        dy = np.abs(c2 - y0)
        dy = np.minimum(dy, n2 - dy)
        solid |= dy[:, None] ** 2 + dx[None, :] ** 2 <= r * r
    if percolating:
        solid = keep_percolating(solid)
    return solid


def disc_batch(count=64, seed0=1000, nmin=64, nmax=512, eps=(0.4, 0.7), rmin=6.0, rmax=20.0,
               kn_log10=(-2.0, 1.0)):
    """``count`` seeded disc packings: for seed = seed0, seed0 + 1, ..., n1 and n2 uniform integers
    in [nmin, nmax], target porosity uniform in ``eps``, disc radii uniform in [rmin, rmax],
    Kn = 10**U(kn_log10).  A packing with no fluid path along x1 (nothing left after
    ``keep_percolating``) has k = 0 and is skipped; the next seed takes its place.  Returns a list
    of (mask, kn, seed)."""
    out = []
    seed = seed0
    while len(out) < count:
        rng = np.random.default_rng(seed)
        n1 = int(rng.integers(nmin, nmax + 1))
        n2 = int(rng.integers(nmin, nmax + 1))
        porosity = float(rng.uniform(*eps))
        kn = float(10.0 ** rng.uniform(*kn_log10))
        mask = random_discs(n1, n2, seed=seed, rmin=rmin, rmax=rmax, solid_fraction=1.0 - porosity)
        if not mask.all():
            out.append((mask, kn, seed))
        seed += 1
    return out


def gaussian_rock(n, seed, corr_len=8.0, porosity=0.35, percolating=True):
    """n^3 Gaussian random field: white noise N(0,1) convolved periodically (FFT) with a Gaussian of
    standard deviation corr_len voxels, fluid where the field is below its porosity quantile."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kernel = np.exp(-2.0 * (math.pi * corr_len) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * kernel))
    thr = np.quantile(field, porosity)
    solid = field >= thr
    if percolating:
        solid = keep_percolating(solid)
    return solid


def sierpinski_carpet(n=540, level=3):
    """Level-`level` Sierpinski carpet on n x n pixels; the removed squares are solid, so the
    porosity is (8/9)^level (0.702 at level 3, the value of Sec. 4.1)."""
    solid = np.zeros((n, n), dtype=bool)
    idx = np.arange(n)
    for lev in range(1, level + 1):
        cell = n // (3 ** lev)
        if cell * 3 ** lev != n:
            raise ValueError("n must be divisible by 3^level")
        digit = (idx // cell) % 3
        mid = digit == 1
        solid |= mid[:, None] & mid[None, :]
    return solid


def sphere_quadrant(n1=200, n2=100, n3=100, porosity=0.75):
    """Quadrant of the cubic sphere array (Sec. 4.2): an n1 x (2 n2) x (2 n3) unit cell with a
    centred sphere of volume (1 - porosity) of the cell; the quadrant keeps the half-planes
    x2 >= centre and x3 >= centre, so the sphere centre sits on the (x2, x3) mirror corner."""
    vol = (1.0 - porosity) * n1 * (2 * n2) * (2 * n3)
    r = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
    c1 = np.arange(n1) + 0.5 - n1 / 2
    c2 = np.arange(n2) + 0.5
    c3 = np.arange(n3) + 0.5
    z, y, x = np.meshgrid(c3, c2, c1, indexing="ij")
    return x ** 2 + y ** 2 + z ** 2 <= r * r


class _DisplacedUnionFind:
    """Union-find over component labels that tracks the x1 period offset between a node and its
    root, so a merge that closes a loop with nonzero offset marks a percolating cluster."""

    def __init__(self, n):
        self.parent = list(range(n))
        self.disp = [0] * n
        self.perc = [False] * n

    def find(self, a):
        path = []
        while self.parent[a] != a:
            path.append(a)
            a = self.parent[a]
        root = a
        # compress: accumulate displacement from the end of the path
        acc = 0
        for node in reversed(path):
            acc += self.disp[node]
            self.disp[node] = acc
            self.parent[node] = root
        return root

    def offset(self, a):
        self.find(a)
        return self.disp[a] if self.parent[a] != a else 0

    def union(self, a, b, d):
        """b's image sits d periods (along x1) away from a's."""
        ra, rb = self.find(a), self.find(b)
        da, db = self.offset(a), self.offset(b)
        if ra == rb:
            if da + d - db != 0:
                self.perc[ra] = True
            return
        # attach rb under ra: position(rb) relative to ra = da + d - db
        self.parent[rb] = ra
        self.disp[rb] = da + d - db
        self.perc[ra] = self.perc[ra] or self.perc[rb]


def keep_percolating(solid, lateral_periodic=True):
    """Fill with solid every fluid voxel whose face-connected fluid cluster (on the domain that is
    periodic along x1, and laterally periodic when lateral_periodic) does not connect a voxel to
    its own image one x1 period away."""
    from scipy import ndimage

    fluid = ~np.asarray(solid, dtype=bool)
    dims = fluid.ndim
    structure = ndimage.generate_binary_structure(dims, 1)
    labels, nlab = ndimage.label(fluid, structure=structure)
    if nlab == 0:
        return np.ones_like(fluid)
    uf = _DisplacedUnionFind(nlab + 1)
    # axis order in numpy arrays: last axis is x1
    for ax in range(dims):
        is_x1 = ax == dims - 1
        if not is_x1 and not lateral_periodic:
            continue
        lo = np.take(labels, 0, axis=ax)
        hi = np.take(labels, labels.shape[ax] - 1, axis=ax)
        both = (lo > 0) & (hi > 0)
        pairs = np.unique(np.stack([hi[both], lo[both]], axis=1), axis=0)
        for a, b in pairs:
            uf.union(int(a), int(b), 1 if is_x1 else 0)
    keep = np.zeros(nlab + 1, dtype=bool)
    for lab in range(1, nlab + 1):
        keep[lab] = uf.perc[uf.find(lab)]
    return ~keep[labels]
