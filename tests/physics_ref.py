"""Independent numpy evaluations of Eq. 1 used to pin the oracle.

These are written from the Hamiltonian of Eq. 1 (site energies, pair term
with minimum-image distances on the torus, field term) with numpy's own
``hypot`` and dense algebra; they share nothing with the oracle's C tables.
"""
import numpy as np


def min_image_distance_matrix(Lx, Ly):
    """Euclidean minimum-image distance between every pair of sites."""
    N = Lx * Ly
    s = np.arange(N)
    x, y = s % Lx, s // Lx
    dx = np.abs(x[:, None] - x[None, :])
    dy = np.abs(y[:, None] - y[None, :])
    dx = np.minimum(dx, Lx - dx)
    dy = np.minimum(dy, Ly - dy)
    return np.hypot(dx, dy)


def coupling_matrix(Lx, Ly):
    """G[s, t] = 1 / r_st for s != t and 0 on the diagonal."""
    D = min_image_distance_matrix(Lx, Ly)
    with np.errstate(divide="ignore"):
        G = np.where(D > 0, 1.0 / np.where(D > 0, D, 1.0), 0.0)
    return G


def site_energies(n, phi, nu, G):
    """eps = phi + G (n - nu)."""
    return phi + G @ (n.astype(np.float64) - nu)


def interaction_energy(n, phi, nu, G):
    """H of Eq. 1 without the field term (well defined on the torus)."""
    s = n.astype(np.float64) - nu
    return float(phi @ n.astype(np.float64) + 0.5 * s @ (G @ s))


def interaction_energy_batch(S, phi, nu, G):
    """Rows of S are occupations; returns H_int for each."""
    Sf = S.astype(np.float64)
    c = Sf - nu
    return Sf @ phi + 0.5 * np.einsum("ij,ij->i", c @ G, c)


def coupling_kernel(L):
    """g[dy, dx] = 1 / r for the minimum-image displacement, g[0, 0] = 0."""
    d = np.arange(L)
    d = np.minimum(d, L - d)
    r = np.hypot(d[:, None], d[None, :])
    with np.errstate(divide="ignore"):
        return np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)


def site_energies_fft(n, phi, nu, L):
    """eps = phi + G (n - nu) as a circular convolution on the L x L torus."""
    g = coupling_kernel(L)
    s = (n.astype(np.float64) - nu).reshape(L, L)
    conv = np.fft.irfft2(np.fft.rfft2(g) * np.fft.rfft2(s), s=(L, L))
    return phi + conv.reshape(-1)


def min_image_distance_matrix3(Lx, Ly, Lz):
    """Euclidean minimum-image distance between every pair of sites of an
    Lx x Ly x Lz torus, site s = (z Ly + y) Lx + x."""
    N = Lx * Ly * Lz
    s = np.arange(N)
    x, y, z = s % Lx, (s // Lx) % Ly, s // (Lx * Ly)
    d = []
    for c, L in ((x, Lx), (y, Ly), (z, Lz)):
        a = np.abs(c[:, None] - c[None, :])
        d.append(np.minimum(a, L - a))
    return np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)


def coupling_matrix3(Lx, Ly, Lz):
    """G[s, t] = 1 / r_st on the three-dimensional torus, 0 on the diagonal."""
    D = min_image_distance_matrix3(Lx, Ly, Lz)
    with np.errstate(divide="ignore"):
        return np.where(D > 0, 1.0 / np.where(D > 0, D, 1.0), 0.0)


def site_energies_fft3(n, phi, nu, L):
    """eps = phi + G (n - nu) as a circular convolution on the L x L x L torus
    (site s = (z L + y) L + x), G the minimum-image 1/r with G(0) = 0."""
    a = np.minimum(np.arange(L), L - np.arange(L)).astype(np.float64)
    r = np.sqrt(a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        g = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    s = (n.astype(np.float64) - nu).reshape(L, L, L)
    conv = np.fft.irfftn(np.fft.rfftn(g) * np.fft.rfftn(s), s=(L, L, L))
    return phi + conv.reshape(-1)
