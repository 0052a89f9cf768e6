"""Grid, Fourier conventions and k-binning of the FP64 oracle (test infrastructure).

Sec. 2: an equidistant N^3 Cartesian grid; a flat voxel index stands for (r,s,t),
x slowest.  App. C.1 (Eqs. FFT, IFFT): forward transform unnormalised
(C_hat = 1), inverse carries C = 1/N_vox so that C * C_hat = 1/N_vox.  numpy's
rfftn / irfftn follow exactly this convention and serve as the FFT step.

Fourier storage is the real-to-complex half spectrum [N][N][N/2+1]: mode
(ix, iy, iz) has integer wave vector n = (ix or ix-N, iy or iy-N, iz), the
signed index running over (-N/2, N/2].  A sum over the full grid equals the sum
over the half spectrum with multiplicity w = 1 on the iz = 0 and iz = N/2 planes
and w = 2 elsewhere.

Binning (the paper leaves it open; Sec. 3.4 only says P_m belongs to the m-th
mode bin): n_bins linear bins in |n| over (0, sqrt(3) N / 2],
    bin(n2) = min(n_bins - 1, floor(n_bins * sqrt(n2) / (sqrt(3) * N / 2))),
evaluated in FP64 on the integer n2 = |n|^2.  The DC mode belongs to no bin.
"""
import numpy as np


class Geometry:
    """Static description of one grid (Sec. 2) and its mode bins (Sec. 3.4)."""

    def __init__(self, N, box, n_bins):
        self.N = int(N)
        self.box = float(box)
        self.n_bins = int(n_bins)
        self.Nv = self.N ** 3
        self.Vc = (self.box / self.N) ** 3
        N = self.N
        ix = np.arange(N)
        ns = np.where(ix <= N // 2, ix, ix - N)
        nz = np.arange(N // 2 + 1)
        self.nx = ns[:, None, None]
        self.ny = ns[None, :, None]
        self.nz = nz[None, None, :]
        self.n2 = (self.nx ** 2 + self.ny ** 2 + self.nz ** 2).astype(np.int64)
        w = np.full((N, N, N // 2 + 1), 2.0)
        w[:, :, 0] = 1.0
        w[:, :, N // 2] = 1.0
        self.w = w
        self.bin = bin_of_n2(self.n2, N, self.n_bins)
        # full-grid mode count per bin (n_m of Eq. INVERSE_GAMMA)
        self.n_modes = np.array([w[self.bin == m].sum() for m in range(self.n_bins)])
        self.kmag = 2.0 * np.pi * np.sqrt(self.n2) / self.box

    def per_mode(self, per_bin, dc=0.0):
        """Expand a per-bin array to the half-spectrum grid (DC gets `dc`)."""
        out = np.asarray(per_bin, dtype=np.float64)[np.maximum(self.bin, 0)]
        out[self.bin < 0] = dc
        return out


def bin_of_n2(n2, N, n_bins):
    """Bin index of integer |n|^2 (-1 for the DC mode)."""
    n2 = np.asarray(n2, dtype=np.int64)
    b = np.floor(float(n_bins) * np.sqrt(n2.astype(np.float64)) / (np.sqrt(3.0) * float(N) / 2.0))
    b = np.minimum(b, n_bins - 1).astype(np.int64)
    return np.where(n2 == 0, -1, b)


def forward(field):
    """Eq. FFT with C_hat = 1: real field [N]^3 -> half spectrum."""
    return np.fft.rfftn(np.asarray(field, dtype=np.float64))


def inverse(spec, N):
    """Eq. IFFT with C = 1/N_vox: half spectrum -> real field [N]^3."""
    return np.fft.irfftn(np.asarray(spec, dtype=np.complex128), s=(N, N, N), axes=(0, 1, 2))
