"""Seeded synthetic inputs shaped like the paper's workloads.

This module makes images and velocity fields only.  It holds none of the
registration method's arithmetic (no transport, no spectral operators of the
method, no interpolation), so that the FP64 oracle and the CUDA path can both
consume exactly the same inputs.  All outputs are float32 numpy arrays; the
oracle reads them widened to float64.

The paper's real datasets (NIREP T1 MRI, CLARITY) are not available; these
generators stand in for them:

* ``sinusoid_pair``: template = sum of 8 random sinusoids (wavenumbers <= 4,
  amplitudes U(0,1), min-max normalised to [0, 1]); reference = the same
  analytic template evaluated at x - u(x) for a band-limited displacement u.
* ``blob_pair``: "brain-like" label images: random ellipsoids with intensities
  U(0.2, 1), later blobs overwrite earlier ones, then periodic Gaussian
  smoothing; the reference rasterises the same ellipsoids at x - u(x).
* ``bandlimited_velocity``: real fields whose Fourier coefficients vanish
  outside |k|_inf <= kmax, scaled to a stated max norm.
* ``syn_problem``: the paper's analytic SYN template and divergence-free
  velocity (Section 5).

Seeds: each named workload uses numpy's PCG64 with seed 1000 + its index.
"""
from __future__ import annotations

import math
import os

import numpy as np

TWO_PI = 2.0 * math.pi


def grid_axes(shape):
    """Coordinates x_d = 2*pi*i/N_d of each axis of the periodic grid."""
    return [TWO_PI * np.arange(n, dtype=np.float64) / n for n in shape]


def _trig_sum(shape, modes, coefs, phases=None, displacement=None, chunk=16):
    """Evaluate sum_l Re(c_l exp(i k_l . x)) on the grid, optionally at x - u(x).

    ``modes`` is an (L, 3) integer array, ``coefs`` complex (L,).  Without a
    displacement the sum is separable and is formed axis by axis; with one it
    is evaluated point by point in chunks of x1-planes.
    """
    x1, x2, x3 = grid_axes(shape)
    modes = np.asarray(modes, dtype=np.float64)
    coefs = np.asarray(coefs, dtype=np.complex128)
    out = np.empty(shape, dtype=np.float64)
    for s in range(0, shape[0], chunk):
        e = min(shape[0], s + chunk)
        X1 = x1[s:e, None, None]
        X2 = x2[None, :, None]
        X3 = x3[None, None, :]
        if displacement is not None:
            X1 = X1 - displacement[0, s:e]
            X2 = X2 - displacement[1, s:e]
            X3 = X3 - displacement[2, s:e]
        acc = np.zeros((e - s, shape[1], shape[2]), dtype=np.float64)
        for (k1, k2, k3), c in zip(modes, coefs):
            ph = k1 * X1 + k2 * X2 + k3 * X3
            acc += c.real * np.cos(ph) - c.imag * np.sin(ph)
        out[s:e] = acc
    return out


def _random_modes(rng, n_modes, kmax):
    modes = []
    while len(modes) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(k != 0):
            modes.append(k)
    return np.array(modes, dtype=np.int64)


def bandlimited_field(shape, kmax, rng, ncomp=3):
    """Random real field(s) with Fourier support |k|_inf <= kmax.

    Built from the full box of modes with k3 >= 0 (the real part of a complex
    sum covers the negative half); coefficients are complex normal with a
    1/(1+|k|^2) amplitude decay so the field is smooth."""
    ks = np.arange(-kmax, kmax + 1)
    K1, K2, K3 = np.meshgrid(ks, ks, np.arange(0, kmax + 1), indexing="ij")
    modes = np.stack([K1.ravel(), K2.ravel(), K3.ravel()], axis=1)
    amp = 1.0 / (1.0 + (modes ** 2).sum(axis=1))
    out = []
    for _ in range(ncomp):
        c = (rng.standard_normal(len(modes)) + 1j * rng.standard_normal(len(modes))) * amp
        out.append(_trig_field_separable(shape, modes, c))
    return np.stack(out, axis=0)


def _trig_field_separable(shape, modes, coefs):
    """sum_l Re(c_l exp(i k_l.x)) by three successive small contractions."""
    x1, x2, x3 = grid_axes(shape)
    ks = np.unique(modes[:, 0]), np.unique(modes[:, 1]), np.unique(modes[:, 2])
    C = np.zeros((len(ks[0]), len(ks[1]), len(ks[2])), dtype=np.complex128)
    pos = [{int(k): i for i, k in enumerate(kk)} for kk in ks]
    for (k1, k2, k3), c in zip(modes, coefs):
        C[pos[0][int(k1)], pos[1][int(k2)], pos[2][int(k3)]] += c
    E1 = np.exp(1j * np.outer(x1, ks[0]))  # [N1, K1]
    E2 = np.exp(1j * np.outer(x2, ks[1]))  # [N2, K2]
    E3 = np.exp(1j * np.outer(x3, ks[2]))  # [N3, K3]
    B = np.einsum("abc,zc->abz", C, E3)    # [K1, K2, N3]
    B = np.einsum("abz,yb->ayz", B, E2)    # [K1, N2, N3]
    out = np.empty(shape, dtype=np.float64)
    step = max(1, (1 << 24) // max(1, shape[1] * shape[2]))
    for s in range(0, shape[0], step):
        e = min(shape[0], s + step)
        out[s:e] = np.einsum("ayz,xa->xyz", B, E1[s:e]).real
    return out


def max_norm(v):
    """max over grid points of the Euclidean norm of a vector field [3, ...]."""
    return float(np.sqrt((np.asarray(v, dtype=np.float64) ** 2).sum(axis=0)).max())


def bandlimited_velocity(shape, kmax, rng, max_norm_value=None, max_disp_vox=None):
    """Band-limited velocity scaled to max |v|_2 = max_norm_value (domain units)
    or to a maximum displacement of max_disp_vox voxels over unit time."""
    v = bandlimited_field(shape, kmax, rng, 3)
    if max_disp_vox is not None:
        h = TWO_PI / min(shape)
        max_norm_value = max_disp_vox * h
    if max_norm_value is not None:
        v *= max_norm_value / max_norm(v)
    return v


# --------------------------------------------------------------------------
# sinusoid images (the 32^3 plain-method workload)
# --------------------------------------------------------------------------

def sinusoid_pair(shape, seed, n_terms=8, kmax=4, vel_kmax=3, vel_max_norm=0.5):
    """Template = normalised sum of random sinusoids; reference = the same sum
    at x - v(x) (v a band-limited velocity with max |v|_2 = 0.5, applied for
    unit time as a displacement).  Returns dict(m0, m1, v_true) in float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = _random_modes(rng, n_terms, kmax)
    amp = rng.uniform(0.0, 1.0, n_terms)
    phase = rng.uniform(0.0, TWO_PI, n_terms)
    coefs = amp * np.exp(1j * (phase - math.pi / 2))  # Re(c e^{ikx}) = a sin(kx + phi)
    raw0 = _trig_sum(shape, modes, coefs)
    lo, hi = raw0.min(), raw0.max()
    v = bandlimited_velocity(shape, vel_kmax, rng, max_norm_value=vel_max_norm)
    raw1 = _trig_sum(shape, modes, coefs, displacement=v)
    m0 = (raw0 - lo) / (hi - lo)
    m1 = (raw1 - lo) / (hi - lo)
    return dict(m0=m0.astype(np.float32), m1=m1.astype(np.float32), v_true=v.astype(np.float32))


# --------------------------------------------------------------------------
# blob images (the 128^3 / 256^3 / 768^3 workloads)
# --------------------------------------------------------------------------

def _rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _blob_params(shape, n_blobs, rng):
    n = np.array(shape, dtype=np.float64)
    blobs = []
    for _ in range(n_blobs):
        centre = rng.uniform(0.15, 0.85, 3) * n
        semi = rng.uniform(0.04, 0.12, 3) * n
        R = _rotation(rng)
        intensity = rng.uniform(0.2, 1.0)
        blobs.append((centre, semi, R, intensity))
    return blobs


def _rasterise(shape, blobs, disp_vox=None):
    """Label image: voxel p gets the intensity of the last ellipsoid containing
    p - u(p) (u in voxels, periodic minimum image), else 0."""
    img = np.zeros(shape, dtype=np.float32)
    n = np.array(shape, dtype=np.float64)
    pad = 0.0 if disp_vox is None else float(np.abs(disp_vox).max()) + 1.0
    for centre, semi, R, intensity in blobs:
        r = float(semi.max()) + pad + 1.0
        lo = np.floor(centre - r).astype(int)
        hi = np.ceil(centre + r).astype(int)
        idx = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        wrapped = [np.mod(i, shape[d]) for d, i in enumerate(idx)]
        P1, P2, P3 = np.meshgrid(*idx, indexing="ij")
        pts = np.stack([P1, P2, P3], axis=0).astype(np.float64)
        if disp_vox is not None:
            W = np.ix_(*wrapped)
            pts = pts - np.stack([disp_vox[d][W] for d in range(3)], axis=0)
        rel = pts - centre[:, None, None, None]
        rel -= n[:, None, None, None] * np.round(rel / n[:, None, None, None])
        loc = np.einsum("ji,j...->i...", R, rel)
        inside = ((loc / semi[:, None, None, None]) ** 2).sum(axis=0) <= 1.0
        sub = img[np.ix_(*wrapped)]
        sub[inside] = intensity
        img[np.ix_(*wrapped)] = sub
    return img


def gaussian_smooth(img, sigma_vox):
    """Periodic Gaussian smoothing with standard deviation sigma (voxels)."""
    shape = img.shape
    F = np.fft.rfftn(img.astype(np.float64))
    w = [TWO_PI * np.fft.fftfreq(shape[0]), TWO_PI * np.fft.fftfreq(shape[1]),
         TWO_PI * np.fft.rfftfreq(shape[2])]
    g1 = np.exp(-0.5 * (sigma_vox * w[0]) ** 2)[:, None, None]
    g2 = np.exp(-0.5 * (sigma_vox * w[1]) ** 2)[None, :, None]
    g3 = np.exp(-0.5 * (sigma_vox * w[2]) ** 2)[None, None, :]
    return np.fft.irfftn(F * g1 * g2 * g3, s=shape, axes=(0, 1, 2))


def blob_pair(shape, seed, n_blobs=12, sigma_vox=2.0, vel_kmax=6, max_disp_vox=4.0):
    """Template and reference blob images plus the velocity that relates them.

    The reference rasterises the same ellipsoids at x - u(x), u = v (unit time)
    with v band-limited (|k|_inf <= 6) and max displacement 4 voxels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    blobs = _blob_params(shape, n_blobs, rng)
    v = bandlimited_velocity(shape, vel_kmax, rng, max_disp_vox=max_disp_vox)
    h = np.array([TWO_PI / s for s in shape])
    disp_vox = v / h[:, None, None, None]
    m0 = gaussian_smooth(_rasterise(shape, blobs), sigma_vox)
    m1 = gaussian_smooth(_rasterise(shape, blobs, disp_vox), sigma_vox)
    return dict(m0=m0.astype(np.float32), m1=m1.astype(np.float32), v_true=v.astype(np.float32))


# --------------------------------------------------------------------------
# the paper's analytic SYN problem (Section 5, dataset 1)
# --------------------------------------------------------------------------

def syn_template(shape):
    """m0(x) = sum_i sin^2(x_i) / 3."""
    x1, x2, x3 = grid_axes(shape)
    return ((np.sin(x1)[:, None, None] ** 2 + np.sin(x2)[None, :, None] ** 2
             + np.sin(x3)[None, None, :] ** 2) / 3.0).astype(np.float32)


def syn_velocity(shape):
    """Divergence-free SYN velocity, read as v1 = sin x3 cos x2 sin x2,
    v2 = sin x1 cos x3 sin x3, v3 = sin x2 cos x1 sin x1 (component i does not
    depend on x_i)."""
    x1, x2, x3 = np.meshgrid(*grid_axes(shape), indexing="ij")
    v = np.stack([np.sin(x3) * np.cos(x2) * np.sin(x2),
                  np.sin(x1) * np.cos(x3) * np.sin(x3),
                  np.sin(x2) * np.cos(x1) * np.sin(x1)], axis=0)
    return v.astype(np.float32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    # name: (seed, generator, parameters)
    "sin32": dict(seed=1000, shape=(32, 32, 32), nt=4, beta=1e-2, gamma=1.0),
    "blob128": dict(seed=1001, shape=(128, 128, 128), nt=4, beta=1e-2, gamma=1.0),
    "blob256": dict(seed=1001, shape=(256, 256, 256), nt=4, beta=1e-2, gamma=1.0),
    "blob256_nt8": dict(seed=1002, shape=(256, 256, 256), nt=8, beta=1e-2, gamma=1.0),
    # the 256^3 pair with three times the displacement (12 voxels at most)
    "blob256_d12": dict(seed=1001, shape=(256, 256, 256), nt=4, beta=1e-2, gamma=1.0, max_disp_vox=12.0),
    "blob768": dict(seed=1004, shape=(768, 768, 768), nt=8, beta=1e-2, gamma=1.0),
}


def workload(name, shape=None):
    """Inputs of a named workload, optionally at another grid size (same
    generator and seed).  If the environment names a directory in
    CLAIRE_SYNTH_CACHE, generated arrays are kept there as .npy files and
    reused (the 768^3 images take minutes to make on the host)."""
    w = dict(WORKLOADS[name])
    if shape is not None:
        w["shape"] = tuple(shape)
    cache = os.environ.get("CLAIRE_SYNTH_CACHE")
    tag = f"{name}_{'x'.join(str(n) for n in w['shape'])}_s{w['seed']}"
    keys = ("m0", "m1", "v_true")
    if cache and all(os.path.exists(os.path.join(cache, f"{tag}_{k}.npy")) for k in keys):
        d = {k: np.load(os.path.join(cache, f"{tag}_{k}.npy")) for k in keys}
    else:
        if name.startswith("sin"):
            d = sinusoid_pair(w["shape"], w["seed"])
        elif name == "blob768":
            d = blob_pair(w["shape"], w["seed"], n_blobs=60, sigma_vox=3.0)
        else:
            d = blob_pair(w["shape"], w["seed"], max_disp_vox=w.get("max_disp_vox", 4.0))
        if cache:
            os.makedirs(cache, exist_ok=True)
            for k in keys:
                np.save(os.path.join(cache, f"{tag}_{k}.npy"), d[k])
    d.update(nt=w["nt"], beta=w["beta"], gamma=w["gamma"], shape=w["shape"])
    return d


def batch_workload(seed=1003, n_pairs=16, sizes=(64, 96, 128, 160)):
    """The batched form's inputs: n_pairs blob pairs (the 128^3 / 256^3
    generator: 12 ellipsoids, sigma 2 voxels, max displacement 4 voxels) on
    cubic grids drawn uniformly from ``sizes``; pair i uses seed 1000*seed + i.
    N_t = 4, beta = 1e-2, gamma = 1.  Returns a list of workload dicts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.asarray(sizes), size=n_pairs)
    out = []
    for i, n in enumerate(ns):
        shape = (int(n),) * 3
        d = blob_pair(shape, 1000 * seed + i)
        d.update(nt=4, beta=1e-2, gamma=1.0, shape=shape)
        out.append(d)
    return out


def smooth_direction(shape, seed, kmax=6):
    """A random smooth vector field with unit max norm (test directions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = bandlimited_field(shape, kmax, rng, 3)
    return (v / max_norm(v)).astype(np.float32)
