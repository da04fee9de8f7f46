"""Seeded synthetic inputs for the multiphase lattice Boltzmann workloads.

This module holds no arithmetic of the lattice Boltzmann method itself: it
draws random numbers and builds initial density fields and solid masks with the
shapes of the paper's workloads (droplets with a tanh interface, Section 3.1;
Gaussian-random-field porous media and overlapping sphere packs standing in for
the Digital Rocks Portal geometries of Section 3.4, which are not available
here). Both the CUDA path (tests, bench) and the oracle (tests) consume its
arrays.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written
out below so that every array is reproducible from its seed on any machine.
Arrays are numpy, shaped (nz, ny, nx) (x fastest in memory).
"""
import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed, n):
    """n successive SplitMix64 outputs (uint64) from the given 64-bit seed."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & _MASK
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def splitmix64_vec(seed, n):
    """Vectorised SplitMix64 stream: identical values to ``splitmix64`` for the same seed."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n):
    """n doubles in [0, 1): the top 53 bits of each SplitMix64 output."""
    return (splitmix64_vec(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal(seed, n):
    """n standard normal doubles (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


# ---------------------------------------------------------------------------
# Droplets (Section 3.1: tanh interface of width w between liquid and vapour)
# ---------------------------------------------------------------------------

def _periodic_distance(grids, center, shape):
    d2 = 0.0
    for g, c, n in zip(grids, center, shape):
        dd = np.abs(g - c)
        dd = np.minimum(dd, n - dd)
        d2 = d2 + dd * dd
    return np.sqrt(d2)


def droplet_field(shape_xyz, centers, radii, rho_l, rho_g, width, periodic=True):
    """Density field of liquid droplets in vapour.

    Each droplet i contributes s_i(d) = (1 - tanh(2 (d - r_i) / w)) / 2, the
    profile of the paper's initial condition read with the vapour density added
    back (rho = (rho_l + rho_g)/2 - (rho_l - rho_g)/2 tanh(2(d - r)/w)); the field
    is rho_g + (rho_l - rho_g) max_i s_i. Distances use the minimum image when
    periodic. Returns float64 (nz, ny, nx) (nz = 1 for 2-D shapes)."""
    nx, ny, nz = shape_xyz
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.zeros((nz, ny, nx))
    for c, r in zip(centers, radii):
        c = list(c) + [0.0] * (3 - len(c))
        if periodic:
            d = _periodic_distance((xx, yy, zz), c, (nx, ny, nz))
        else:
            d = np.sqrt((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2)
        s = np.maximum(s, 0.5 * (1.0 - np.tanh(2.0 * (d - r) / width)))
    return rho_g + (rho_l - rho_g) * s


def random_droplets(shape_xyz, count, rmin, rmax, width, seed, max_tries=100000, gap_widths=3.0):
    """Centres and radii of `count` droplets with radii U[rmin, rmax], placed at
    uniformly random positions in a periodic box by rejection so that any two
    are separated by at least r_i + r_j + gap_widths * w (minimum image): with
    three interface widths between surfaces the tanh tails leave no bridge of
    intermediate (spinodal) density between neighbours."""
    nx, ny, nz = shape_xyz
    dims = [nx, ny, nz] if nz > 1 else [nx, ny]
    u = uniform(seed, max_tries * 4)
    centers, radii = [], []
    t = 0
    while len(radii) < count:
        if t + 4 > u.size:
            raise RuntimeError("could not place droplets")
        r = rmin + (rmax - rmin) * u[t]
        c = [u[t + 1 + a] * dims[a] for a in range(len(dims))]
        t += 4
        ok = True
        for c2, r2 in zip(centers, radii):
            d2 = 0.0
            for a in range(len(dims)):
                dd = abs(c[a] - c2[a])
                dd = min(dd, dims[a] - dd)
                d2 += dd * dd
            if d2 < (r + r2 + gap_widths * width) ** 2:
                ok = False
                break
        if ok:
            centers.append(c)
            radii.append(r)
    return centers, radii


# ---------------------------------------------------------------------------
# Porous media
# ---------------------------------------------------------------------------

def gaussian_random_field(shape_xyz, corr_length, seed):
    """White noise smoothed by a periodic Gaussian filter of standard deviation
    `corr_length` (lattice units), normalised to zero mean and unit variance."""
    nx, ny, nz = shape_xyz
    z = normal(seed, nx * ny * nz).reshape(nz, ny, nx)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = (2 * np.pi) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2)
    g = np.fft.irfftn(np.fft.rfftn(z) * np.exp(-0.5 * corr_length ** 2 * k2), s=(nz, ny, nx),
                      axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def _label_6(pore):
    from scipy import ndimage
    st = ndimage.generate_binary_structure(pore.ndim, 1)
    return ndimage.label(pore, structure=st)


def percolating_pores(pore):
    """Keep only the pore cluster(s) (6-connected) touching both x faces.
    Returns (pore mask, percolates?)."""
    lab, n = _label_6(pore)
    if n == 0:
        return pore & False, False
    a = set(np.unique(lab[..., 0])) - {0}
    b = set(np.unique(lab[..., -1])) - {0}
    keep = sorted(a & b)
    if not keep:
        return pore & False, False
    return np.isin(lab, keep), True


def periodic_percolating_pores(pore):
    """Keep only the pore cluster(s) (6-connected) joined to their own periodic image
    along x, i.e. the clusters that carry flow through a box periodic in x. The box
    is doubled along x and labelled; a cluster percolates when some voxel and its copy
    one period further share a label. Returns (pore mask, percolates?)."""
    n = pore.shape[-1]
    lab, count = _label_6(np.concatenate([pore, pore], axis=-1))
    if count == 0:
        return pore & False, False
    a, b = lab[..., :n], lab[..., n:]
    keep = np.unique(a[(a == b) & (a != 0)])
    if keep.size == 0:
        return pore & False, False
    return np.isin(a, keep), True


def grf_porous_medium(shape_xyz, porosity, corr_length, seed, buffer=8, max_seeds=50, periodic_x=False):
    """Solid mask (uint8, 1 = solid) of a thresholded Gaussian random field.

    The porous block fills x in [buffer, nx - buffer); pores are the lowest
    `porosity` quantile of the field; pores not connected inlet-to-outlet are
    filled; `buffer` fluid layers sit at both x ends. With periodic_x (and no
    buffer) the pores kept are those joined to their periodic image along x. If a
    seed does not percolate the next seed (seed + 1, ...) is taken. Returns
    (solid, seed_used)."""
    nx, ny, nz = shape_xyz
    for s in range(seed, seed + max_seeds):
        g = gaussian_random_field((nx - 2 * buffer, ny, nz), corr_length, s)
        thr = np.quantile(g, porosity)
        pore = g <= thr
        pore, ok = periodic_percolating_pores(pore) if periodic_x else percolating_pores(pore)
        if not ok:
            continue
        solid = np.zeros((nz, ny, nx), dtype=np.uint8)
        solid[:, :, buffer:nx - buffer] = (~pore).astype(np.uint8)
        return solid, s
    raise RuntimeError("no percolating seed found")


def sphere_pack(shape_xyz, rmin, rmax, porosity, seed, max_spheres=10 ** 6):
    """Boolean model of overlapping spheres (radius U[rmin, rmax], centres
    uniform in the box), added until the porosity falls to `porosity` or below.
    Returns uint8 solid mask (nz, ny, nx)."""
    nx, ny, nz = shape_xyz
    solid = np.zeros((nz, ny, nx), dtype=bool)
    total = nx * ny * nz
    u = uniform(seed, 4 * 65536)
    t = 0
    count = 0
    nsolid = 0
    while 1.0 - nsolid / total > porosity and count < max_spheres:
        if t + 4 > u.size:
            u = uniform(seed + 1 + count, 4 * 65536)
            t = 0
        r = rmin + (rmax - rmin) * u[t]
        cx, cy, cz = u[t + 1] * nx, u[t + 2] * ny, u[t + 3] * nz
        t += 4
        count += 1
        x0, x1 = max(0, int(cx - r) - 1), min(nx, int(cx + r) + 2)
        y0, y1 = max(0, int(cy - r) - 1), min(ny, int(cy + r) + 2)
        z0, z1 = max(0, int(cz - r) - 1), min(nz, int(cz + r) + 2)
        zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1),
                                 indexing="ij")
        inside = (xx + 0.5 - cx) ** 2 + (yy + 0.5 - cy) ** 2 + (zz + 0.5 - cz) ** 2 <= r * r
        nsolid += int(np.count_nonzero(inside & ~solid[z0:z1, y0:y1, x0:x1]))
        solid[z0:z1, y0:y1, x0:x1] |= inside
    return solid.astype(np.uint8)


def random_solids(shape_xyz, fraction, seed):
    """Independent random solid voxels (for small parity cases)."""
    nx, ny, nz = shape_xyz
    return (uniform(seed, nx * ny * nz) < fraction).astype(np.uint8).reshape(nz, ny, nx)


def random_field(shape_xyz, lo, hi, seed):
    """Uniform random scalar field in [lo, hi)."""
    nx, ny, nz = shape_xyz
    return (lo + (hi - lo) * uniform(seed, nx * ny * nz)).reshape(nz, ny, nx)
