"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module only builds initial conditions and work lists; it holds no step
of the solver.  Both the CUDA path's tests/benchmarks and the CPU oracle take
their inputs from here.  Fields are numpy float64 arrays [5, Z, Y, X] of the
conserved variables (rho, rho u, rho v, rho w, E) of an ideal gas, built from
primitive initial data with E = p / (gamma - 1) + rho |v|^2 / 2 (the
definition of the initial state, not part of the update).

Workloads (Sec. 5 of the paper uses a 3D blast wave and a cosmological AMR
run; their data are not available, so these stand in for them):
  * sod(n, axis)             Sod shock tube, rho/p = 1/1 | 0.125/0.1
  * lognormal(n, seed, ...)  periodic lognormal density (sigma 0.5, k^-3
                             Gaussian field), p = 1, random k^-3 velocities
                             scaled to an rms Mach number
  * sedov(n)                 Sedov-Taylor blast: E = 1 in r < 2 cells
  * sound_wave / advection / uniform: small analytic cases for the pins
"""
import numpy as np


def conserved(rho, vx, vy, vz, p, gamma):
    """Initial conserved state [5, ...] from primitive initial data."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    vx, vy, vz, p = (np.broadcast_to(np.asarray(a, dtype=np.float64), shape) for a in (vx, vy, vz, p))
    U = np.empty((5,) + shape)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return U


def cell_centres(n, length=1.0):
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    return x, dx


def uniform(shape, rho=1.0, v=(0.3, -0.2, 0.1), p=0.7, gamma=1.4):
    r = np.full(shape, rho)
    return conserved(r, v[0], v[1], v[2], p, gamma)


def sod(n, axis=0, gamma=1.4, ny=None, nz=None, diagonal=False):
    """Sod tube on [0,1]^3 (interface x_axis = 0.5, or x+y+z = 1.5 if diagonal)."""
    nx = n
    ny = ny or n
    nz = nz or n
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    coord = (X, Y, Z)[axis]
    left = (X + Y + Z < 1.5) if diagonal else (coord < 0.5)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return conserved(rho, 0.0, 0.0, 0.0, p, gamma)


def gaussian_field(n, seed, slope=-3.0):
    """Unit-variance periodic Gaussian random field with P(k) ~ k^slope on n^3."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (slope / 2.0)
    f = np.fft.ifftn(np.fft.fftn(white) * amp).real
    f -= f.mean()
    f /= f.std()
    return f


def lognormal(n, seed=1, sigma=0.5, mach=1.5, gamma=1.4, p0=1.0, vel_seeds=None, p_index=0.0):
    """Periodic lognormal box: rho = exp(sigma d - sigma^2/2), p = p0 rho^p_index
    (uniform by default), and three independent k^-3 velocity components
    scaled so that sqrt(<|v|^2/c^2>) = mach."""
    d = gaussian_field(n, seed)
    rho = np.exp(sigma * d - 0.5 * sigma * sigma)
    p = p0 * rho ** p_index if p_index else p0
    vs = vel_seeds or (seed + 1, seed + 2, seed + 3)
    v = [gaussian_field(n, s) for s in vs]
    c2 = gamma * p / rho
    m2 = (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / c2
    scale = mach / np.sqrt(m2.mean())
    return conserved(rho, scale * v[0], scale * v[1], scale * v[2], p, gamma)


def sedov(n, gamma=5.0 / 3.0, E=1.0, rho0=1.0, p0=1.0e-5, r_cells=2.0, window=None):
    """Sedov-Taylor blast on [0,1]^3: E spread uniformly over the cells whose
    centre lies within r_cells cell widths of the box centre.  With
    window = w, only the central w^3 cells of the n^3 box are returned (the
    rest of the box is the uniform background state)."""
    x, dx = cell_centres(n)
    if window is not None:
        a = n // 2 - window // 2
        x = x[a:a + window]
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    inside = r < r_cells * dx
    U = conserved(np.full(X.shape, rho0), 0.0, 0.0, 0.0, p0, gamma)
    U[4][inside] += E / (inside.sum() * dx ** 3)
    return U


def sound_wave(n, amp=1.0e-6, gamma=1.4, direction=(1, 0, 0), shape=None):
    """Right-moving linear sound wave, rho0 = 1, c = 1 (p0 = 1/gamma), wave
    vector 2 pi direction on the periodic unit box."""
    shape = shape or (n, n, n)
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    kd = np.asarray(direction, dtype=np.float64)
    phase = 2 * np.pi * (kd[0] * X + kd[1] * Y + kd[2] * Z)
    nhat = kd / np.linalg.norm(kd)
    s = amp * np.sin(phase)
    return conserved(1.0 + s, nhat[0] * s, nhat[1] * s, nhat[2] * s, 1.0 / gamma + s, gamma)


def advection(shape, velocity=(1.0, 0.0, 0.0), gamma=1.4, kind="sine", axis=0):
    """Density profile carried by a uniform velocity at uniform pressure."""
    nz, ny, nx = shape
    n_ax = (nx, ny, nz)[axis]
    s = (np.arange(n_ax) + 0.5) / n_ax
    if kind == "sine":
        prof = 1.0 + 0.5 * np.sin(2 * np.pi * s)
    else:  # square pulse
        prof = np.where((s > 0.25) & (s < 0.5), 2.0, 1.0)
    sh = [1, 1, 1]
    sh[2 - axis] = n_ax
    rho = np.broadcast_to(prof.reshape(sh), shape).copy()
    return conserved(rho, velocity[0], velocity[1], velocity[2], 1.0, gamma)


def group_origins(X, Y, Z, N=16):
    """Interior corners (x0, y0, z0) of the N^3 groups tiling an X x Y x Z box,
    group index (gz * GY + gy) * GX + gx."""
    assert X % N == 0 and Y % N == 0 and Z % N == 0
    o = [(gx * N, gy * N, gz * N) for gz in range(Z // N) for gy in range(Y // N) for gx in range(X // N)]
    return np.asarray(o, dtype=np.int32).reshape(-1, 3)


def column_origins(X, Y, Z, N=16):
    """The origins of group_origins in column order: z fastest, then x, then
    y, so that z-neighbouring groups are consecutive."""
    o = [(gx * N, gy * N, gz * N) for gy in range(Y // N) for gx in range(X // N) for gz in range(Z // N)]
    return np.asarray(o, dtype=np.int32).reshape(-1, 3)


def runs_from_links(nxt):
    """zrun[g] = 1 + zrun[g+1] where group g+1 continues group g along +z
    (nxt[g] true), else 1: the run of z-continuations starting at g."""
    nxt = np.asarray(nxt, dtype=bool)
    z = np.ones(len(nxt), dtype=np.int32)
    for g in range(len(nxt) - 2, -1, -1):
        if nxt[g]:
            z[g] = z[g + 1] + 1
    return z


def scatter_groups(U_groups, X, Y, Z):
    """Inverse of the interior tiling: [G,5,N,N,N] -> [5,Z,Y,X]."""
    G, _, N = U_groups.shape[:3]
    GX, GY, GZ = X // N, Y // N, Z // N
    a = U_groups.reshape(GZ, GY, GX, 5, N, N, N)
    return a.transpose(3, 0, 4, 1, 5, 2, 6).reshape(5, Z, Y, X)


def poisson_arrivals(rate=200.0, n=2000, seed=6):
    """Serving requests: arrival time, box size, rms Mach, step count, seed."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    sizes = rng.choice([32, 64, 128, 256], size=n, p=[0.4, 0.3, 0.2, 0.1])
    mach = rng.uniform(0.5, 3.0, n)
    steps = rng.integers(5, 51, n)
    seeds = rng.integers(0, 2 ** 31 - 1, n)
    return [dict(t=float(t[i]), n=int(sizes[i]), mach=float(mach[i]), steps=int(steps[i]), seed=int(seeds[i]))
            for i in range(n)]


def _pad_periodic(U, g):
    return np.pad(U, ((0, 0), (g, g), (g, g), (g, g)), mode="wrap")


def _grad_score(rho):
    """max over cells of |grad rho| / rho (central differences, unit spacing)."""
    gx = 0.5 * (rho[..., 2:] - rho[..., :-2])[1:-1, 1:-1]
    gy = 0.5 * (rho[:, 2:, :] - rho[:, :-2, :])[1:-1, :, 1:-1]
    gz = 0.5 * (rho[2:, :, :] - rho[:-2, :, :])[:, 1:-1, 1:-1]
    return np.sqrt(gx * gx + gy * gy + gz * gz) / rho[1:-1, 1:-1, 1:-1]


def amr_levels(counts=(4096, 2500, 1500, 800), n0=128, seed=5, N=16, g=3, mach=1.5, gamma=1.4, threshold=0.3,
               dtype=np.float32):
    """AMR-shaped batch: per level a list of halo-prepared patch groups [G,5,M,M,M].

    Level 0 tiles a periodic lognormal root of n0^3 cells (seed `seed`); the
    stated per-level counts are authoritative, so the root's groups are
    repeated on seeded periodic shifts of the root until count[0] is reached.
    Level l+1 refines the groups of level l that score highest in
    max |grad rho|/rho (cells above `threshold` flag a group); each refined
    group yields its 8 children (16^3 cells at twice the resolution) by
    trilinear interpolation of the parent's halo-padded data, with a seeded
    1% k^-3 density perturbation.  Ghost zones are prepared (filled from the
    parent), as the AMR ghost interpolation itself is not part of this path.
    Groups that continue one another along z are consecutive: level 0 column
    by column (z fastest) within each shifted root, the children of a refined
    group as four z-pairs; `zrun` gives the runs (hydro_params.zrun).
    Returns a list of dicts {U: groups, dx, score, flagged_fraction, zrun}.
    """
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    root = lognormal(n0, seed=seed, mach=mach, gamma=gamma)
    M = N + 2 * g
    levels = []
    # level 0
    groups, scores, nxt = [], [], []
    shift = np.zeros(3, dtype=int)
    while len(groups) < counts[0]:
        f = np.roll(root, tuple(-shift[::-1]), axis=(1, 2, 3))
        fp = _pad_periodic(f, g)
        sc = _grad_score(fp[0])
        for (x0, y0, z0) in column_origins(n0, n0, n0, N):
            if len(groups) >= counts[0]:
                break
            groups.append(fp[:, z0:z0 + M, y0:y0 + M, x0:x0 + M])
            scores.append(sc[z0:z0 + M - 2, y0:y0 + M - 2, x0:x0 + M - 2].max())
            nxt.append(z0 + N < n0)  # the next group of this root's column lies above
        shift = rng.integers(0, n0, 3)
    U0 = np.stack(groups).astype(dtype)
    levels.append({"U": U0, "dx": 1.0 / n0, "score": np.asarray(scores),
                   "flagged_fraction": float(np.mean(np.asarray(scores) > threshold)),
                   "zrun": runs_from_links(nxt[:len(groups) - 1] + [False])})
    # refined levels
    for l in range(1, len(counts)):
        prev = levels[-1]
        need = int(np.ceil(counts[l] / 8))
        order = np.argsort(-prev["score"], kind="stable")
        parents = [order[k % len(order)] for k in range(need)]
        kids, ksc, nxt = [], [], []
        for pi in parents:
            P = prev["U"][pi].astype(np.float64)
            fine = np.stack([ndimage.zoom(P[v], 2, order=1, mode="nearest", grid_mode=True) for v in range(5)])
            pert = gaussian_field(2 * M, int(rng.integers(0, 2 ** 31 - 1)))
            fine[0] *= 1.0 + 0.01 * pert
            sc = _grad_score(fine[0])
            for cy in (0, 1):
                for cx in (0, 1):
                    for cz in (0, 1):
                        a = (N * cz + 2 * g - g, N * cy + 2 * g - g, N * cx + 2 * g - g)
                        kids.append(fine[:, a[0]:a[0] + M, a[1]:a[1] + M, a[2]:a[2] + M])
                        ksc.append(sc[a[0]:a[0] + M - 2, a[1]:a[1] + M - 2, a[2]:a[2] + M - 2].max())
                        nxt.append(cz == 0)  # the upper child of the pair follows
        G = counts[l]
        Ul = np.stack(kids[:G]).astype(dtype)
        sl = np.asarray(ksc[:G])
        levels.append({"U": Ul, "dx": prev["dx"] / 2.0, "score": sl,
                       "flagged_fraction": float(np.mean(sl > threshold)),
                       "zrun": runs_from_links(nxt[:G - 1] + [False])})
    return levels


def smooth_field(x, y, z, seed=7, mach=1.0, gamma=1.4, modes=6, kmax=3):
    """Smooth periodic state [5][nz][ny][nx] on the tensor grid of the 1-D
    coordinate arrays x, y, z (unit box): density and pressure exp/affine in
    a few random Fourier modes of integer wavevector (|k_i| <= kmax, seeded),
    three velocity components from further modes, scaled so the peak |v| is
    about `mach` sound speeds.  Resolution-free, so every AMR level samples
    the same field at its own cell centres.  Each mode sin(2 pi k.x + phi) is
    evaluated as the imaginary part of a product of 1-D complex exponentials."""
    rng = np.random.default_rng(seed)
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))

    def series(amp):
        k = rng.integers(-kmax, kmax + 1, size=(modes, 3))
        k[np.all(k == 0, axis=1)] = (1, 0, 0)
        ph = rng.uniform(0.0, 2.0 * np.pi, modes)
        a = rng.uniform(0.5, 1.0, modes) * amp / modes
        s = np.zeros((z.size, y.size, x.size))
        for m in range(modes):
            ex = np.exp(1j * (2.0 * np.pi * k[m, 0] * x + ph[m]))
            ey = np.exp(2j * np.pi * k[m, 1] * y)
            ez = np.exp(2j * np.pi * k[m, 2] * z)
            s = s + a[m] * (ez[:, None, None] * (ey[None, :, None] * ex[None, None, :])).imag
        return s

    rho = np.exp(series(0.6))
    p = 1.0 + series(0.4)
    c = np.sqrt(gamma)
    v = [mach * c * series(1.0) for _ in range(3)]
    return conserved(rho, v[0], v[1], v[2], p, gamma)


def amr_hierarchy(n0=48, radii=(0.2,), center=(0.5, 0.5, 0.5), seed=7, mach=1.0, gamma=1.4, N=16, full=None,
                  counts=None):
    """Static AMR hierarchy on the periodic unit box, as a list of levels
    {U [G][5][N][N][N], origin [G][3] (x, y, z corner in the level's cells),
    box (X, Y, Z), dx (3 floats)}.

    Level 0 tiles the n0^3 box.  Level l+1 refines, as octets (the 8 groups
    of twice the resolution covering one level-l group), every level-l group
    whose centre lies within radii[l] of `center` (periodic distance) and
    whose 26 neighbour groups all exist at level l (proper nesting); with
    full = l, level l+1 refines every group of level l instead; with counts
    (groups wanted per refined level), level l+1 refines the ceil(counts[l] /
    8) eligible level-l groups nearest to `center` instead of using radii.  The data of
    every level are smooth_field sampled at that level's cell centres, so
    coarse and fine data are independent samples (not averages) of one field.
    Group order, every level: column by column (y, then x, then z fastest),
    so that the z-neighbours of a column are consecutive (the runs of
    z-continuations that the unsplit kernels stream as chains)."""
    levels = []
    origin = column_origins(n0, n0, n0, N)
    nref = len(counts) if counts is not None else len(radii)
    for l in range(nref + 1):
        n = n0 * 2 ** l
        if l > 0:
            prev = levels[-1]
            pn = n // 2
            slots = {tuple(o // N) for o in prev["origin"]}
            gp = pn // N
            kids = []
            dist = []
            eligible = []
            for o in prev["origin"]:
                s = o // N
                cen = (o + N / 2) / pn
                dvec = np.abs(cen - np.asarray(center))
                dvec = np.minimum(dvec, 1.0 - dvec)
                dist.append(np.sqrt((dvec ** 2).sum()))
                eligible.append(all(((s[0] + i) % gp, (s[1] + j) % gp, (s[2] + k) % gp) in slots
                                    for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)))
            dist = np.asarray(dist)
            if counts is not None:
                order = [i for i in np.argsort(dist, kind="stable") if eligible[i]]
                pick = set(order[:int(np.ceil(counts[l - 1] / 8))])
            else:
                pick = {i for i in range(len(dist))
                        if eligible[i] and (full == l - 1 or dist[i] <= radii[l - 1])}
            for i, o in enumerate(prev["origin"]):
                if i in pick:
                    for dz in range(2):
                        for dy in range(2):
                            for dx_ in range(2):
                                kids.append((2 * o[0] + dx_ * N, 2 * o[1] + dy * N, 2 * o[2] + dz * N))
            if not kids:
                break
            origin = np.asarray(kids, dtype=np.int32).reshape(-1, 3)
            origin = origin[np.lexsort((origin[:, 2], origin[:, 0], origin[:, 1]))]
        r = (np.arange(N) + 0.5) / n
        U = np.empty((len(origin), 5, N, N, N))
        for k, (x0, y0, z0) in enumerate(origin):
            U[k] = smooth_field(x0 / n + r, y0 / n + r, z0 / n + r, seed=seed, mach=mach, gamma=gamma)
        levels.append({"U": U, "origin": np.asarray(origin, dtype=np.int32), "box": (n, n, n),
                       "dx": (1.0 / n,) * 3})
    return levels
