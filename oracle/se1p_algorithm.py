"""FP64 restatement of the SE1P Fourier-space algorithm (Algorithms 1-3).

TEST INFRASTRUCTURE ONLY: used by the tests, the package smoke check and the
benchmark's CPU-baseline leg.  It shares no code with the CUDA library.

The steps follow Section 3 in the paper's order and notation:

  1. h = L/M, Lt = L + P h, Mt >= M + P, eta = P xi^2 h^2 / (c^2 pi), c = 0.95
     (Eq. 3.3); one eta per axis when the grid spacings differ.
  2. Gridding (Eq. 3.4): H(x_g) = sum_n q_n W(x_g - x_n), with
     W(d) = prod_i (2 xi^2/(pi eta_i))^{1/2} exp(-2 xi^2 d_i^2 / eta_i), truncated
     to P points per axis; z wraps periodically, x,y live on [0, Lt).
  3. AFT (Algorithm 2): FFT along z; the k3 = 0 slab zero-padded to n0 x n0,
     slabs with 0 < |k3| <= 2 pi n_l / L zero-padded to nI x nI, the rest kept
     at Mt x Mt; a 2-D FFT of each slab.
  4. Scaling (Eqs. 3.5-3.7): 4 pi exp(-(1-eta)(kappa^2+k3^2)/4xi^2) G(kappa,k3), with
     G = 1/(kappa^2+k3^2) for k3 != 0 and the truncated 2-D Green's function
     (1 - J0(R kappa))/kappa^2 - R log(R) J1(R kappa)/kappa at k3 = 0,
     R^2/4 (1 - 2 log R) at kappa = 0, R = sqrt(2) Lt (Eqs. 3.9-3.10).
  5. AIFT (Algorithm 3): 2-D inverse FFT of each slab, restricted to the
     Mt x Mt spreading region, merged, inverse FFT along z.
  6. Gathering (Eq. 3.11 and Eq. 3.25):
       phi^F(x_m) = h^3 sum_g W(x_m - x_g) Ht(x_g)
       F^F(x_m)   = q_m h^3 sum_g (4 xi^2/eta_i) (x_m - x_g)_i W(x_m - x_g) Ht(x_g).

Readings of the paper used here (each is listed in the design notes):
  * The forward trapezoidal sum carries h^3 and the inverse (dk)^2/(2 pi)^2/L3;
    together they reduce to an unnormalised forward DFT and a normalised
    inverse DFT per slab, and 4 pi comes from -Laplace(phi) = 4 pi f (Eq. 3.8).
    With that the gather carries h^3 and no 2/L3 factor.
  * The free-dimension grid starts at -P h/2: a particle at x sits at x + P h/2
    on [0, Lt).  For even P the support is floor(x'/h) - P/2 + 1 ... + P/2,
    for odd P it is centred on round(x'/h).
  * The I set is {0 < |k3| <= 2 pi n_l / L_free}; for a cubic box this is
    mode indices 1..n_l.
  * Spectral indices run over numpy's FFT order (Nyquist kept, scaled by |k|).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

C_SHAPE = 0.95


def eta_of(P: int, xi: float, h: float, c: float = C_SHAPE) -> float:
    """Eq. 3.3: eta = P xi^2 h^2 / (c^2 pi)."""
    return P * xi * xi * h * h / (c * c * math.pi)


def support(xs: np.ndarray, h: float, P: int) -> tuple[np.ndarray, np.ndarray]:
    """Unwrapped grid indices of the P-point support and distances x - x_g.

    xs are coordinates measured from the grid origin.
    """
    t = xs / h
    if P % 2 == 0:
        i0 = np.floor(t).astype(np.int64) - P // 2 + 1
    else:
        i0 = np.floor(t + 0.5).astype(np.int64) - (P - 1) // 2
    idx = i0[:, None] + np.arange(P)[None, :]
    d = xs[:, None] - idx * h
    return idx, d


def window_1d(d: np.ndarray, xi: float, eta: float) -> np.ndarray:
    """One axis of the Gaussian window W (Eq. 3.4)."""
    return math.sqrt(2.0 * xi * xi / (math.pi * eta)) * np.exp(-2.0 * xi * xi * d * d / eta)


class Grid:
    """Geometry of one SE1P evaluation (step 1 of Algorithm 1)."""

    def __init__(self, L, xi, M, P, Mt, n0, nI, nl, c=C_SHAPE):
        self.L = tuple(float(v) for v in L)
        self.xi = float(xi)
        self.M = tuple(int(v) for v in M)
        self.P = int(P)
        self.Mt = int(Mt)
        self.n0 = int(n0)
        self.nI = int(nI)
        self.nl = int(nl)
        if self.L[0] != self.L[1] or self.M[0] != self.M[1]:
            raise ValueError("free dimensions must share L and M")
        if self.Mt < self.M[0] + self.P:
            raise ValueError("Mt must be >= M + P")
        self.h = self.L[0] / self.M[0]  # free dimensions
        self.hz = self.L[2] / self.M[2]
        self.eta = eta_of(self.P, self.xi, self.h, c)
        self.etaz = eta_of(self.P, self.xi, self.hz, c)
        self.offset = self.P * self.h / 2.0  # free-dimension grid origin at -P h/2
        self.Lt = self.Mt * self.h
        self.R = math.sqrt(2.0) * self.Lt

    def coords(self, x: np.ndarray):
        """Particle coordinates measured from the grid origin (z wrapped)."""
        xs = x[:, 0] + self.offset
        ys = x[:, 1] + self.offset
        zs = np.mod(x[:, 2], self.L[2])
        return xs, ys, zs

    def weights(self, x: np.ndarray):
        xs, ys, zs = self.coords(x)
        ix, dx = support(xs, self.h, self.P)
        iy, dy = support(ys, self.h, self.P)
        iz, dz = support(zs, self.hz, self.P)
        wx = window_1d(dx, self.xi, self.eta)
        wy = window_1d(dy, self.xi, self.eta)
        wz = window_1d(dz, self.xi, self.etaz)
        return (ix, dx, wx), (iy, dy, wy), (np.mod(iz, self.M[2]), dz, wz)


def spread(g: Grid, x: np.ndarray, q: np.ndarray, chunk: int = 256) -> np.ndarray:
    """Step 2 (Eq. 3.4): H on the M3 x Mt x Mt grid, stored [z][y][x]."""
    M3, Mt, P = g.M[2], g.Mt, g.P
    H = np.zeros(M3 * Mt * Mt)
    for s in range(0, x.shape[0], chunk):
        (ix, _, wx), (iy, _, wy), (iz, _, wz) = g.weights(x[s:s + chunk])
        if ix.min() < 0 or ix.max() >= Mt or iy.min() < 0 or iy.max() >= Mt:
            raise ValueError("particle support leaves the extended grid")
        w = (q[s:s + chunk, None, None, None] * wz[:, :, None, None] * wy[:, None, :, None]
             * wx[:, None, None, :])
        flat = (iz[:, :, None, None] * Mt + iy[:, None, :, None]) * Mt + ix[:, None, None, :]
        H += np.bincount(flat.ravel(), weights=w.ravel(), minlength=H.size)
    return H.reshape(M3, Mt, Mt)


def vico_green(kappa: np.ndarray, R: float) -> np.ndarray:
    """Fourier transform of the 2-D Green's function truncated at R (Eqs. 3.9-3.10)."""
    out = np.empty_like(kappa)
    z = kappa == 0.0
    k = kappa[~z]
    out[~z] = (1.0 - special.j0(R * k)) / (k * k) - R * math.log(R) * special.j1(R * k) / k
    out[z] = R * R / 4.0 * (1.0 - 2.0 * math.log(R))
    return out


def slab_size(g: Grid, jj: int) -> int:
    """Padded 2-D size for the z-mode with signed index jj (upsampling rule, Eq. 3.2)."""
    if jj == 0:
        return g.n0
    k3 = 2.0 * math.pi * abs(jj) / g.L[2]
    if k3 * g.L[0] <= 2.0 * math.pi * g.nl * (1.0 + 1e-12):
        return g.nI
    return g.Mt


def fourier_solve(g: Grid, H: np.ndarray) -> np.ndarray:
    """Steps 3-5: AFT (Algorithm 2), scaling (Eq. 3.5), AIFT (Algorithm 3)."""
    M3, Mt = g.M[2], g.Mt
    xi2 = g.xi * g.xi
    Hz = np.fft.fft(H, axis=0)  # Algorithm 2, step 1
    out = np.empty_like(Hz)
    jj_all = np.rint(np.fft.fftfreq(M3) * M3).astype(np.int64)
    for j in range(M3):
        jj = int(jj_all[j])
        n = slab_size(g, jj)
        k3 = 2.0 * math.pi * jj / g.L[2]
        A = np.zeros((n, n), dtype=np.complex128)
        A[:Mt, :Mt] = Hz[j]
        Ah = np.fft.fft2(A)  # Algorithm 2, steps 2-4
        kv = 2.0 * math.pi * np.fft.fftfreq(n, d=g.h)
        K2 = kv[None, :] ** 2 + kv[:, None] ** 2
        if jj == 0:
            G = vico_green(np.sqrt(K2), g.R)
        else:
            G = 1.0 / (K2 + k3 * k3)
        S = 4.0 * math.pi * np.exp(-((1.0 - g.eta) * K2 + (1.0 - g.etaz) * k3 * k3) / (4.0 * xi2)) * G
        out[j] = np.fft.ifft2(Ah * S)[:Mt, :Mt]  # Algorithm 3, steps 1-4
    return np.fft.ifft(out, axis=0).real  # Algorithm 3, step 5


def gather(g: Grid, Ht: np.ndarray, x: np.ndarray, q: np.ndarray, chunk: int = 256):
    """Step 6 (Eq. 3.11, Eq. 3.25): phi^F and F^F at the given particles."""
    M3, Mt = g.M[2], g.Mt
    h3 = g.h * g.h * g.hz
    flat_grid = Ht.ravel()
    n = x.shape[0]
    phi = np.empty(n)
    F = np.empty((n, 3))
    cx = 4.0 * g.xi * g.xi / g.eta
    cz = 4.0 * g.xi * g.xi / g.etaz
    for s in range(0, n, chunk):
        (ix, dx, wx), (iy, dy, wy), (iz, dz, wz) = g.weights(x[s:s + chunk])
        flat = (iz[:, :, None, None] * Mt + iy[:, None, :, None]) * Mt + ix[:, None, None, :]
        Hv = flat_grid[flat]
        W = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
        WH = W * Hv
        phi[s:s + chunk] = h3 * WH.sum(axis=(1, 2, 3))
        F[s:s + chunk, 0] = h3 * cx * np.einsum('nkji,ni->n', WH, dx)
        F[s:s + chunk, 1] = h3 * cx * np.einsum('nkji,nj->n', WH, dy)
        F[s:s + chunk, 2] = h3 * cz * np.einsum('nkji,nk->n', WH, dz)
    F *= q[:, None]
    return phi, F


def se1p_fourier(x, q, L, xi, M, P, Mt, n0, nI, nl, targets=None, c=C_SHAPE):
    """phi^F and F^F of Algorithm 1 at all particles (or at `targets`)."""
    g = Grid(L, xi, M, P, Mt, n0, nI, nl, c)
    H = spread(g, x, q)
    Ht = fourier_solve(g, H)
    if targets is None:
        return gather(g, Ht, x, q)
    t = np.asarray(targets)
    return gather(g, Ht, x[t], q[t])
