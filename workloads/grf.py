"""Gaussian random fields with an exponential variogram, and lognormal grades.

Simulation is by circulant embedding (Dietrich and Newsam; Wood and Chan): the
covariance is laid out on a periodic grid padded to at least twice the block
grid along each axis, its FFT gives the eigenvalues of the embedding, and one
complex FFT of weighted complex white noise yields two independent real fields
(real and imaginary parts).  Small negative eigenvalues of the embedding are
clipped to zero.  The nugget is added as independent Gaussian noise.

Variogram convention (practical range a):
    gamma(h) = c0 + (sill - c0) * (1 - exp(-3 h / a))   for h > 0
so the structured part has covariance (sill - c0) exp(-3 h / a) and the nugget
contributes an independent N(0, c0) term per block.
"""

from __future__ import annotations

import numpy as np

try:  # scipy's FFT is multi-threaded; numpy's is the fallback
    import scipy.fft as _fft

    def _fftn(a):
        return _fft.fftn(a, workers=-1)

except Exception:  # pragma: no cover - scipy is in the image
    _fft = None

    def _fftn(a):
        return np.fft.fftn(a)


def _good_size(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n (fast FFT lengths)."""
    best = None
    p2 = 1
    while p2 < 2 * n:
        p3 = p2
        while p3 < 2 * n:
            p5 = p3
            while p5 < 2 * n:
                if p5 >= n and (best is None or p5 < best):
                    best = p5
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best if best is not None else n


def _embedding_eigenvalues(nz: int, ny: int, nx: int, rng_a: float, c_struct: float):
    """sqrt(lambda / M) of the periodic embedding of c_struct * exp(-3h/a)."""
    pz, py, px = (_good_size(2 * n) if n > 1 else 1 for n in (nz, ny, nx))

    def torus_dist(n):
        i = np.arange(n, dtype=np.float64)
        return np.minimum(i, n - i)

    dz = torus_dist(pz)[:, None, None]
    dy = torus_dist(py)[None, :, None]
    dx = torus_dist(px)[None, None, :]
    h = np.sqrt(dz * dz + dy * dy + dx * dx)
    cov = c_struct * np.exp(-3.0 * h / rng_a)
    lam = np.real(_fftn(cov))
    lam = np.maximum(lam, 0.0)
    m = lam.size
    return np.sqrt(lam / m), (pz, py, px)


def gaussian_field(nx: int, ny: int, nz: int, n_fields: int, rng_a: float,
                   nugget: float, sill: float, seed_seq: np.random.SeedSequence) -> np.ndarray:
    """n_fields independent zero-mean Gaussian fields on an nx*ny*nz grid.

    Returns float64 [n_fields][nz][ny][nx] (x fastest, z = 0 is the top level).
    One child of ``seed_seq`` is spawned per pair of fields.
    """
    c_struct = sill - nugget
    sq, pad = _embedding_eigenvalues(nz, ny, nx, rng_a, c_struct)
    out = np.empty((n_fields, nz, ny, nx), dtype=np.float64)
    n_pairs = (n_fields + 1) // 2
    children = seed_seq.spawn(n_pairs)
    for p in range(n_pairs):
        rng = np.random.default_rng(children[p])
        w = rng.standard_normal(pad) + 1j * rng.standard_normal(pad)
        y = _fftn(sq * w)[:nz, :ny, :nx]
        nug = rng.standard_normal((2, nz, ny, nx)) * np.sqrt(nugget)
        out[2 * p] = y.real + nug[0]
        if 2 * p + 1 < n_fields:
            out[2 * p + 1] = y.imag + nug[1]
    return out


def lognormal_grades(nx: int, ny: int, nz: int, n_scen: int, mean: float, cv: float,
                     rng_a: float, nugget: float, sill: float, seed: int) -> np.ndarray:
    """Grades g[b][s] (g/t, float64, scenario fastest) for B = nx*ny*nz blocks.

    Block index b = x + nx*(y + ny*z).  g = exp(mu + sigma_L * Y) with
    sigma_L^2 = ln(1 + cv^2) and mu = ln(mean) - sigma_L^2 / 2, so each block's
    grade has the requested mean and coefficient of variation when Y has unit
    variance (sill = 1).  Stream 0 of SeedSequence(seed) drives the grades.
    """
    ss = np.random.SeedSequence(seed).spawn(2)[0]
    y = gaussian_field(nx, ny, nz, n_scen, rng_a, nugget, sill, ss)
    sig2 = np.log1p(cv * cv)
    mu = np.log(mean) - 0.5 * sig2
    g = np.exp(mu + np.sqrt(sig2) * y)  # [S][nz][ny][nx]
    return np.ascontiguousarray(g.reshape(n_scen, -1).T)  # [B][S]
