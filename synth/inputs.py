"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module builds the *data* of the transport-constrained registration problems of
He & Mang (arXiv 2510.08782, Sec. 2 and Sec. 3): template/reference images m0, m1
(or densities pi0, pi1) on the periodic box [0, 2*pi)^d and smooth velocity fields.
It deliberately holds none of the method's arithmetic: no semi-Lagrangian step,
no cubic interpolation, no spectral differential operator, no objective or gradient.
Images are analytic Gaussian mixtures or trigonometric polynomials, so a warped reference is an
exact evaluation of the same analytic function at displaced centres or points; velocities are band-limited random
Fourier series (synthesised with a plain inverse FFT, a library primitive).

Layout convention (shared by every consumer): a scalar field has shape n = (n_1,...,n_d)
in C order (last axis contiguous); a vector field has shape (d, n_1, ..., n_d) and
component c points along axis c. Grid point l sits at x_l = 2*pi*l/n (Sec. 2.2).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def spacing(n):
    """Cell sizes h_i = 2*pi/n_i of the periodic grid (Sec. 2.2)."""
    return tuple(TWO_PI / float(ni) for ni in n)


def coords(n):
    """1D coordinate arrays x_i = 2*pi*l/n_i, l = 0..n_i-1, one per axis."""
    return [TWO_PI * np.arange(ni) / ni for ni in n]


def _int_freqs(ni):
    return np.fft.fftfreq(ni, d=1.0 / ni)


def random_fourier_field(n, ncomp, kmax, rng, norm="euclid"):
    """Band-limited random real field(s) on the grid n.

    Each component is the real part of a sum over modes 0 < |k| <= kmax (Euclidean
    norm, or max-norm with norm='inf') with i.i.d. complex N(0,1) coefficients.
    Returns an array of shape (ncomp, *n), float64, unit max-abs per component set.
    """
    n = tuple(int(x) for x in n)
    ks = np.meshgrid(*[_int_freqs(ni) for ni in n], indexing="ij")
    if norm == "inf":
        kn = np.max(np.abs(np.stack(ks)), axis=0)
    else:
        kn = np.sqrt(sum(k * k for k in ks))
    mask = (kn > 0) & (kn <= kmax)
    out = np.empty((ncomp,) + n)
    for c in range(ncomp):
        coef = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * mask
        out[c] = np.real(np.fft.ifftn(coef)) * np.prod(n)
    return out


def _scale_max(v, target):
    """Scale a vector field so that max over the grid of |v(x)|_2 equals target."""
    mag = np.sqrt(np.sum(v * v, axis=0)).max()
    return v * (target / mag) if mag > 0 else v


def _curl_field(n, kmax, rng):
    """Divergence-free random field as the curl of a random band-limited potential.

    In 2D the stream function psi gives v = (d psi/d x_1, -d psi/d x_0); in 3D a
    vector potential A gives v = curl A. The derivatives are taken mode by mode on
    the random coefficients (not with the method's Leray projector).
    """
    n = tuple(int(x) for x in n)
    d = len(n)
    ks = np.meshgrid(*[_int_freqs(ni) for ni in n], indexing="ij")
    kn = np.sqrt(sum(k * k for k in ks))
    mask = (kn > 0) & (kn <= kmax)
    # Zero the Nyquist planes so that each mode's derivative stays real.
    for ax, ni in enumerate(n):
        if ni % 2 == 0:
            mask &= ks[ax] != -(ni // 2)
    npts = float(np.prod(n))
    if d == 2:
        psi = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * mask
        v0 = np.real(np.fft.ifftn(1j * ks[1] * psi)) * npts
        v1 = np.real(np.fft.ifftn(-1j * ks[0] * psi)) * npts
        return np.stack([v0, v1])
    a = [(rng.standard_normal(n) + 1j * rng.standard_normal(n)) * mask for _ in range(3)]
    curl = [ks[1] * a[2] - ks[2] * a[1], ks[2] * a[0] - ks[0] * a[2], ks[0] * a[1] - ks[1] * a[0]]
    return np.stack([np.real(np.fft.ifftn(1j * c)) * npts for c in curl])


def eval_fourier_at(field_grid, points):
    """Evaluate the trigonometric interpolant of a band-limited grid field at points.

    Used only to move Gaussian centres by a known velocity; points is (npts, d).
    The field must be band-limited well below Nyquist (true for the generators here).
    """
    n = field_grid.shape
    fh = np.fft.fftn(field_grid) / np.prod(n)
    idx = np.nonzero(np.abs(fh) > 1e-13 * np.abs(fh).max())
    ks = [(_int_freqs(ni))[ix] for ni, ix in zip(n, idx)]
    coef = fh[idx]
    phase = sum(np.outer(points[:, a], ks[a]) for a in range(len(n)))
    return np.real(np.exp(1j * phase) @ coef)


def gaussian_mixture(n, centers, inv_covs, weights, radius):
    """Sum of periodic Gaussians w_i * exp(-0.5 (x-c_i)^T S_i (x-c_i)) on the grid.

    Distances use the periodic minimum image; Gaussian i is evaluated in a box of half-width
    radius[i] (physical units; a scalar applies to all) around its centre, covering its support.
    Boxes are accumulated into a padded array that is folded back periodically at the end.
    """
    n = tuple(int(x) for x in n)
    d = len(n)
    h = spacing(n)
    radii = np.broadcast_to(np.asarray(radius, dtype=float), (len(centers),))
    cells = [[min(int(np.ceil(r / h[a])), n[a]) for a in range(d)] for r in radii]
    pad = [max([c[a] for c in cells] + [0]) + 1 for a in range(d)]
    acc = np.zeros(tuple(n[a] + 2 * pad[a] for a in range(d)))
    for c, S, w, rc in zip(centers, inv_covs, weights, cells):
        offs, sl = [], []
        for a in range(d):
            length = min(2 * rc[a] + 2, n[a])
            start = int(np.floor(c[a] / h[a])) - rc[a]
            j = np.arange(start, start + length)
            dx = j * h[a] - c[a]
            dx = (dx + np.pi) % TWO_PI - np.pi
            shape = [1] * d
            shape[a] = length
            offs.append(dx.reshape(shape))
            sl.append(slice(start + pad[a], start + pad[a] + length))
        q = 0.0
        for a in range(d):
            q = q + S[a, a] * offs[a] * offs[a]
            for b in range(a + 1, d):
                if S[a, b] != 0.0:
                    q = q + 2.0 * S[a, b] * offs[a] * offs[b]
        acc[tuple(sl)] += w * np.exp(-0.5 * q)
    # fold the padding back onto the periodic grid, one axis at a time
    for a in range(d):
        core = [slice(None)] * d
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        p, m = pad[a], n[a]
        core[a] = slice(p, p + m)
        out = acc[tuple(core)].copy()
        lo[a] = slice(0, p)
        hi[a] = slice(p + m, 2 * p + m)
        low, high = acc[tuple(lo)], acc[tuple(hi)]
        for k in range(p):  # wrap index k - p -> k - p + m, and p + m + k -> k
            dst = [slice(None)] * d
            src = [slice(None)] * d
            dst[a] = (k - p) % m
            src[a] = k
            out[tuple(dst)] += low[tuple(src)]
            dst[a] = k % m
            out[tuple(dst)] += high[tuple(src)]
        acc = out
    return acc


def _random_rotation(d, rng):
    qm, r = np.linalg.qr(rng.standard_normal((d, d)))
    qm = qm * np.sign(np.diag(r))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    return qm


def smooth_velocity(n, kmax, max_disp_voxels, rng, divergence_free=False):
    """Random smooth stationary velocity with max |v|_2 = max_disp_voxels * h.

    Over the unit time interval a stationary field of this size moves material by at
    most about max_disp_voxels cells.
    """
    n = tuple(int(x) for x in n)
    if divergence_free:
        v = _curl_field(n, kmax, rng)
    else:
        v = random_fourier_field(n, len(n), kmax, rng)
    return _scale_max(v, max_disp_voxels * min(spacing(n)))


def blob_image_pair(n, v_true, count, sigma_vox, rng, amplitude_sign=False, normalize=True):
    """Template/reference images from isotropic Gaussian blobs.

    The template is sum_i a_i G_sigma_i(x - c_i); the reference uses the same blobs with
    centres displaced by v_true(c_i) (unit time). With amplitude_sign the amplitudes are
    N(0,1) (a shot-noise realisation of low-pass Gaussian noise), else all ones.
    Both images are then mapped by the same affine min-max map of the template to [0,1].
    """
    n = tuple(int(x) for x in n)
    d = len(n)
    h = min(spacing(n))
    centers = rng.uniform(0.0, TWO_PI, size=(count, d))
    sig = rng.uniform(sigma_vox[0], sigma_vox[1], size=count) * h
    amps = rng.standard_normal(count) if amplitude_sign else np.ones(count)
    disp = np.stack([eval_fourier_at(v_true[a], centers) for a in range(d)], axis=1)
    inv = [np.eye(d) / (s * s) for s in sig]
    rad = 5.0 * sig
    m0 = gaussian_mixture(n, centers, inv, amps, rad)
    m1 = gaussian_mixture(n, (centers + disp) % TWO_PI, inv, amps, rad)
    if normalize:
        lo, hi = m0.min(), m0.max()
        m0 = (m0 - lo) / (hi - lo)
        m1 = (m1 - lo) / (hi - lo)
    return m0, m1


def sinusoid_image_pair(n, v_true, kmax, rng):
    """Template/reference images from a smooth trigonometric polynomial (the sinusoidal data of the
    incompressible experiments, Sec. 3.6).

    m(x) = sum over integer k with 0 < |k| <= kmax of a_k cos(k . x) + b_k sin(k . x), a_k, b_k ~ N(0,1).
    The template is m on the grid; the reference is the same analytic m evaluated at the grid points
    displaced by v_true (unit time, one explicit step back along the flow: m1(x) = m(x - v_true(x))).
    Both are mapped by the template's affine min-max map to [0, 1].
    """
    n = tuple(int(x) for x in n)
    d = len(n)
    rng_k = range(-kmax, kmax + 1)
    ks = np.array([k for k in np.ndindex(*(len(rng_k),) * d)]) - kmax
    ks = ks[(np.sum(ks * ks, axis=1) > 0) & (np.sum(ks * ks, axis=1) <= kmax * kmax)]
    a = rng.standard_normal(len(ks))
    b = rng.standard_normal(len(ks))
    grids = np.meshgrid(*coords(n), indexing="ij")
    pts = np.stack([g.ravel() for g in grids], axis=1)

    def evaluate(points):
        out = np.zeros(points.shape[0])
        for start in range(0, len(ks), 32):  # modest temporaries
            ph = points @ ks[start:start + 32].T.astype(np.float64)
            out += np.cos(ph) @ a[start:start + 32] + np.sin(ph) @ b[start:start + 32]
        return out.reshape(n)

    m0 = evaluate(pts)
    disp = np.stack([v_true[c].ravel() for c in range(d)], axis=1)
    m1 = evaluate(pts - disp)
    lo, hi = m0.min(), m0.max()
    return (m0 - lo) / (hi - lo), (m1 - lo) / (hi - lo)


def density_pair(n, v_true, count, sigma_vox, rng, floor=1e-3):
    """Probability densities pi0, pi1 from anisotropic Gaussians (mass-preserving model).

    pi0 = sum of `count` Gaussians with random rotations, axis std ~ U[sigma_vox] voxels
    and weights ~ U[0.5, 1]; pi1 moves each centre by v_true(c_i). A floor of
    floor*max is added and both are normalised to unit mass sum(pi) * prod(h) = 1.
    """
    n = tuple(int(x) for x in n)
    d = len(n)
    h = spacing(n)
    hmin = min(h)
    centers = rng.uniform(0.0, TWO_PI, size=(count, d))
    weights = rng.uniform(0.5, 1.0, size=count)
    inv = []
    rad = []
    for _ in range(count):
        s = rng.uniform(sigma_vox[0], sigma_vox[1], size=d) * hmin
        rad.append(4.5 * s.max())
        r = _random_rotation(d, rng)
        inv.append(r @ np.diag(1.0 / (s * s)) @ r.T)
    disp = np.stack([eval_fourier_at(v_true[a], centers) for a in range(d)], axis=1)
    p0 = gaussian_mixture(n, centers, inv, weights, rad)
    p1 = gaussian_mixture(n, (centers + disp) % TWO_PI, inv, weights, rad)
    cell = float(np.prod(h))
    out = []
    for p in (p0, p1):
        p = p + floor * p.max()
        out.append(p / (p.sum() * cell))
    return out[0], out[1]


# ---------------------------------------------------------------------------
# Named workloads (the five problem configurations the library is measured on)
# ---------------------------------------------------------------------------

def workload(name, seed=0, n=None):
    """Problem data and solver settings for a named workload.

    name: 'adv2d64'   2D 64^2 advection, 8 blobs, |k|<=3 velocity of 0.5 px, nt=4, H1, alpha=1e-2, w=5
          'adv3d64'   3D 64^3 advection, low-pass template, |k|<=4 velocity of 2 voxels, nt=4, H2, alpha=1e-3, w=5
          'inc3d128'  3D 128^3 incompressible, nt=8, H1, alpha=1e-2
          'cont3d256' 3D 256^3 mass-preserving (continuity), nt=16, H1, alpha=1e-3, w=10, checkpoint every 4
          'inc2d256'  2D 256^2 incompressible, sinusoidal images, divergence-free velocity of 4 px, nt=16, H3,
                      alpha=1e-4, tolerance 1e-3
          'batch'     see batch_workloads()
    n overrides the grid (same recipe at another size, used for small test cases).
    Returns a dict with float64 arrays and the problem/solver settings.
    """
    rng = np.random.default_rng(seed)
    if name == "adv2d64":
        n = tuple(n or (64, 64))
        v_true = _scale_max(random_fourier_field(n, 2, 3, rng, norm="inf"), 0.5 * min(spacing(n)))
        m0, m1 = blob_image_pair(n, v_true, 8, (4.0, 8.0), rng)
        return dict(name=name, dim=2, n=n, nt=4, model="advection", reg_order=1, alpha=1e-2,
                    window=5, sigma=4, tau=2, max_iter=20, rel_tol=1e-2, ckpt_every=0,
                    m0=m0, m1=m1, v_true=v_true)
    if name == "adv3d64":
        n = tuple(n or (64, 64, 64))
        v_true = smooth_velocity(n, 4, 2.0, rng)
        m0, m1 = blob_image_pair(n, v_true, 256, (2.0, 3.0) if n[0] <= 64 else (2.0 * n[0] / 64, 3.0 * n[0] / 64),
                                 rng, amplitude_sign=True)
        return dict(name=name, dim=3, n=n, nt=4, model="advection", reg_order=2, alpha=1e-3,
                    window=5, sigma=4, tau=2, max_iter=200, rel_tol=1e-2, ckpt_every=0,
                    m0=m0, m1=m1, v_true=v_true)
    if name == "inc3d128":
        n = tuple(n or (128, 128, 128))
        v_true = smooth_velocity(n, 4, 2.0, rng, divergence_free=True)
        s = n[0] / 64.0
        m0, m1 = blob_image_pair(n, v_true, 256, (2.0 * s, 3.0 * s), rng, amplitude_sign=True)
        return dict(name=name, dim=3, n=n, nt=8, model="incompressible", reg_order=1, alpha=1e-2,
                    window=5, sigma=4, tau=2, max_iter=200, rel_tol=1e-2, ckpt_every=0,
                    m0=m0, m1=m1, v_true=v_true)
    if name == "inc2d256":  # the incompressible experiments of Sec. 3.6
        n = tuple(n or (256, 256))
        v_true = smooth_velocity(n, 4, 4.0, rng, divergence_free=True)
        m0, m1 = sinusoid_image_pair(n, v_true, 6, rng)
        return dict(name=name, dim=len(n), n=n, nt=16, model="incompressible", reg_order=3, alpha=1e-4,
                    window=10, sigma=4, tau=2, max_iter=200, rel_tol=1e-3, ckpt_every=0,
                    m0=m0, m1=m1, v_true=v_true)
    if name == "cont3d256":
        n = tuple(n or (256, 256, 256))
        v_true = smooth_velocity(n, 4, 6.0, rng)
        s = n[0] / 256.0
        p0, p1 = density_pair(n, v_true, 64, (4.0 * s, 16.0 * s), rng)
        return dict(name=name, dim=3, n=n, nt=16, model="continuity", reg_order=1, alpha=1e-3,
                    window=10, sigma=4, tau=2, max_iter=200, rel_tol=1e-2, ckpt_every=4,
                    m0=p0, m1=p1, v_true=v_true)
    raise ValueError(f"unknown workload {name!r}")


def batch_specs(count=32, seed=0, sizes=(64, 96, 128, 160)):
    """(index, grid size, alpha, data seed) of each problem of a seeded batch: sizes drawn from
    `sizes`, alpha from {1e-2, 1e-3}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ni = int(rng.choice(sizes))
        alpha = float(rng.choice([1e-2, 1e-3]))
        out.append((i, ni, alpha, seed * 1000 + i + 1))
    return out


def batch_problem(spec):
    """One problem of a batch from its spec (batch_specs): the adv3d64 recipe at that size, nt=4, H1."""
    i, ni, alpha, data_seed = spec
    w = workload("adv3d64", seed=data_seed, n=(ni, ni, ni))
    w.update(name=f"batch{i}", reg_order=1, alpha=alpha, nt=4)
    return w


def batch_workloads(count=32, seed=0, sizes=(64, 96, 128, 160)):
    """Independent 3D advection problems of uneven size (nt=4, H1, alpha in {1e-2,1e-3})."""
    return [batch_problem(sp) for sp in batch_specs(count, seed, sizes)]


def random_problem_fields(n, seed, model="advection", vel_scale_vox=1.0, kmax_img=4, kmax_vel=3):
    """Small smooth random (m0, m1, v) for operator-level tests.

    m0, m1 are band-limited fields in roughly [0, 1]; v has max displacement
    vel_scale_vox cells; for model='incompressible' v is divergence free; for
    'continuity' m0, m1 are positive.
    """
    rng = np.random.default_rng(seed)
    n = tuple(int(x) for x in n)
    f = random_fourier_field(n, 2, kmax_img, rng)
    f = f / np.abs(f).max()
    m0 = 0.5 + 0.4 * f[0]
    m1 = 0.5 + 0.4 * f[1]
    if model == "continuity":
        m0 = m0 + 0.2
        m1 = m1 + 0.2
    v = smooth_velocity(n, kmax_vel, vel_scale_vox, rng, divergence_free=(model == "incompressible"))
    return m0, m1, v
