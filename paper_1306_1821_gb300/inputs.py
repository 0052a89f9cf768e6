"""Seeded synthetic surveys (inputs only: none of the sampler's arithmetic).

Stand-ins for the paper's SDSS-DR7-like mock (Sec. 5), whose mask, Schechter
selection and Eisenstein-Hu spectrum are not available here:

  * spectrum P(k) = A k (1 + (k / 0.02)^2)^-2, k in h/Mpc, with A chosen so the
    voxel variance (1/V) sum_{k != 0} P(k) over the grid is 0.5;
  * true field delta = IFFT(sqrt(P(k)/V_cell) FFT(xi)) with xi white noise
    (FFT forward unnormalised, inverse 1/N_vox, the App. C.1 convention);
  * observer at the box centre, voxel centres at (i + 1/2) dx - L/2; angular
    mask a spherical cap about +z, cos(theta) >= 1 - 2 f_sky; R = 0 beyond L/2;
  * radial selection linear (1 - r / (L/2)) or Gaussian exp(-(r / r0)^2);
  * counts N^l ~ Poisson(R^l Nbar^l max(0, 1 + b^l delta)) (the data model of
    Eq. data_model with Poisson rather than Gaussian noise).

Everything is drawn from numpy's PCG64 with a fixed seed, so each named
workload is reproducible bit for bit.  The step-size bounds eps_max are set for
a density-move acceptance of roughly 0.8-0.9 at the true hyperparameters (the
stable leapfrog step shrinks with the dimension, about as N_vox^(-1/4)).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    N: int
    box: float
    n_bins: int
    b: list
    nbar: list
    f_sky: float
    radial: str            # "linear", "gauss" or "schechter" (selection tables, made on the device)
    r0: float = 350.0
    n_leapfrog: int = 10
    eps_max: float = 0.3
    jump: bool = False
    jump_leapfrog: int = 10
    jump_eps_max: float = 0.05
    seed: int = 0
    alpha: float = 1.0
    fixed_bias: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_sub(self):
        return len(self.b)


def _six_nbar():
    return [8.0 * (1.0 / 16.0) ** (l / 5.0) for l in range(6)]


SIX_B = [1.0, 1.1, 1.2, 1.35, 1.5, 1.65]

WORKLOADS = {
    # 32^3, L = 500 Mpc/h, one subsample, 40% sky with linear radial fall-off
    "survey32": Workload("survey32", 32, 500.0, 16, [1.2], [5.0], 0.4, "linear",
                         n_leapfrog=10, eps_max=0.15),
    # 128^3, L = 750 Mpc/h, six luminosity subsamples, 25% sky, exp(-(r/350)^2)
    "survey128": Workload("survey128", 128, 750.0, 16, SIX_B, _six_nbar(), 0.25, "gauss",
                          n_leapfrog=10, eps_max=0.06),
    # 256^3, L = 1000 Mpc/h, six subsamples, 32 bins, 20 leapfrog steps, jump on
    "survey256": Workload("survey256", 256, 1000.0, 32, SIX_B, _six_nbar(), 0.25, "gauss",
                          n_leapfrog=20, eps_max=0.05, jump=True, jump_leapfrog=10, jump_eps_max=0.15),
}


# The paper's own test setup (Sec. 5) at 128^3, L = 750 Mpc/h: fifteen
# luminosity subsamples in absolute-magnitude bins of 0.4 from -23 to -17
# (brightest first), radial selection from the Schechter function of App. D
# with M_* - 5 log10 h = -20.44, alpha = -1.05 inside 14.5 < r < 17.77 (flat
# LCDM, Omega_m = 0.24), mean numbers Nbar^l = Phi_* int Phi dM over each bin
# with Phi_* = 19.6798... (the faintest bin has Nbar = 8), and biases from the
# luminosity law of Eq. rel_bias (b_* = 1.2, M_* = -20.83, a = 0.895,
# b = 0.105, c = -0.040) at the bin centres.  The values below are those
# definitions evaluated once in FP64: they are the table of
# tests/golden/schechter15.txt, which tests/golden/schechter15.py writes from
# the printed constants with the FP64 oracle, and the tests hold the two equal.
# The DR7 mask is replaced by a 25% cap.
SCHECHTER15_EDGES = [-23.0 + 0.4 * i for i in range(16)]
SCHECHTER15_PHI_STAR = 19.679837431231647
SCHECHTER15_B = [1.9419001265076423, 1.6843806505723544, 1.5003038561471536, 1.3670369833779648,
                 1.2689219880403695, 1.195126150195898, 1.138155058691824, 1.092823847783893,
                 1.0555454667701716, 1.023838282880806, 0.9959854257071645, 0.9707991111275014,
                 0.9474575932996266, 0.9253923629996902, 0.9042101079393786]
SCHECHTER15_NBAR = [0.0014022274046629074, 0.017877857008321816, 0.10835142812365212, 0.38647319977232125,
                    0.9463696456518819, 1.7774796502645018, 2.771610849132778, 3.794844809474923,
                    4.7459183261589715, 5.573165614259365, 6.2647350878662635, 6.831900757373581,
                    7.295583066943564, 7.678240761551859, 8.0]
WORKLOADS["schechter128"] = Workload(
    "schechter128", 128, 750.0, 16, SCHECHTER15_B, SCHECHTER15_NBAR, 0.25, "schechter",
    n_leapfrog=10, eps_max=0.06, jump=True, jump_leapfrog=10, jump_eps_max=0.15, fixed_bias=6,
    extra={"M_edges": SCHECHTER15_EDGES, "phi_star": SCHECHTER15_PHI_STAR})


def small_workload(N, box=None, n_bins=4, n_sub=1, f_sky=0.5, seed=0, **kw):
    """A small survey for parity tests (same recipe, any grid size)."""
    box = float(box if box is not None else 500.0 * N / 32.0)
    b = SIX_B[:n_sub]
    nbar = _six_nbar()[:n_sub]
    return Workload(f"small{N}", N, box, n_bins, b, nbar, f_sky, "gauss", r0=0.7 * box / 2.0,
                    seed=seed, **kw)


def spectrum_shape(k):
    k = np.asarray(k, dtype=np.float64)
    return k * (1.0 + (k / 0.02) ** 2) ** -2


def wavenumbers(N, box):
    """|k| on the half-spectrum grid [N][N][N/2+1] (h/Mpc)."""
    i = np.arange(N)
    n = np.where(i <= N // 2, i, i - N).astype(np.float64)
    nz = np.arange(N // 2 + 1, dtype=np.float64)
    n2 = n[:, None, None] ** 2 + n[None, :, None] ** 2 + nz[None, None, :] ** 2
    return 2.0 * np.pi * np.sqrt(n2) / box


def amplitude(N, box, variance=0.5):
    """A such that (1/V) sum over all non-DC grid modes of P(k) equals `variance`."""
    k = wavenumbers(N, box)
    w = np.full(k.shape, 2.0)
    w[:, :, 0] = 1.0
    w[:, :, N // 2] = 1.0
    s = np.sum(w * spectrum_shape(k))
    return variance * box ** 3 / s


def true_spectrum(k, N, box):
    return amplitude(N, box) * spectrum_shape(k)


def bin_centre_spectrum(N, box, n_bins):
    """The true spectrum at the centres of n_bins linear |n| bins over (0, sqrt(3) N/2]."""
    edges = np.sqrt(3.0) * N / 2.0 / n_bins
    nc = (np.arange(n_bins) + 0.5) * edges
    return true_spectrum(2.0 * np.pi * nc / box, N, box)


def response(N, box, f_sky, radial, r0=350.0, axis=(0.0, 0.0, 1.0)):
    """Survey response R (float32 [N]^3): spherical cap about `axis` times radial selection."""
    dx = box / N
    c = (np.arange(N) + 0.5) * dx - box / 2.0
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    proj = ax[0] * x + ax[1] * y + ax[2] * z
    cos_t = np.where(r > 0, proj / np.maximum(r, 1e-300), 1.0)
    cap = cos_t >= 1.0 - 2.0 * f_sky
    rmax = box / 2.0
    if radial == "linear":
        sel = np.maximum(0.0, 1.0 - r / rmax)
    else:
        sel = np.exp(-(r / r0) ** 2)
    R = np.where(cap & (r <= rmax), sel, 0.0)
    return R.astype(np.float32)


def make_survey(wl: Workload, seed=None):
    """(delta_true float64 [N]^3, counts int32 [n_sub,N,N,N], R float32 [n_sub,N,N,N])."""
    seed = wl.seed if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    N = wl.N
    xi = rng.standard_normal((N, N, N))
    k = wavenumbers(N, wl.box)
    vc = (wl.box / N) ** 3
    amp = np.sqrt(true_spectrum(k, N, wl.box) / vc)
    amp[0, 0, 0] = 0.0
    delta = np.fft.irfftn(amp * np.fft.rfftn(xi), s=(N, N, N), axes=(0, 1, 2))
    R1 = response(N, wl.box, wl.f_sky, wl.radial, wl.r0, wl.extra.get("axis", (0.0, 0.0, 1.0)))
    R = np.broadcast_to(R1, (wl.n_sub, N, N, N)).copy()
    counts = np.empty((wl.n_sub, N, N, N), dtype=np.int32)
    for l in range(wl.n_sub):
        lam = R[l].astype(np.float64) * wl.nbar[l] * np.maximum(0.0, 1.0 + wl.b[l] * delta)
        counts[l] = rng.poisson(lam).astype(np.int32)
    return delta, counts, R


def initial_state(wl: Workload):
    """Starting point: delta_hat = 0, P at the bin centres, b and Nbar at the truth."""
    P = bin_centre_spectrum(wl.N, wl.box, wl.n_bins)
    return P, np.array(wl.b, dtype=np.float64), np.array(wl.nbar, dtype=np.float64)


def random_spectrum(N, n_bins, seed, scale=1.0):
    """A seeded random half spectrum (complex128 [N][N][N/2+1]) of a real field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((N, N, N)) * scale
    return np.fft.rfftn(x)


def batch_workloads(sizes=(32, 64, 96), per_size=32, seed0=1000):
    """Many small independent surveys: per_size chains of each grid size, box
    L = 500 N / 32 Mpc/h (the cell size of the 32^3 survey), a spherical cap of
    20-60% of the sky about a random direction with linear radial fall-off to
    L/2, 1-4 luminosity subsamples (the first entries of the six-subsample
    lists) and 16 k bins; chain j draws its mock from seed seed0 + j."""
    out = []
    j = 0
    for N in sizes:
        for _ in range(per_size):
            rng = np.random.Generator(np.random.PCG64(seed0 + j))
            f_sky = float(rng.uniform(0.2, 0.6))
            n_sub = int(rng.integers(1, 5))
            v = rng.standard_normal(3)
            wl = Workload(f"batch{j}", N, 500.0 * N / 32.0, 16, SIX_B[:n_sub], _six_nbar()[:n_sub], f_sky,
                          "linear", n_leapfrog=10, eps_max=0.1, seed=seed0 + j,
                          extra={"axis": tuple(v / np.linalg.norm(v))})
            out.append(wl)
            j += 1
    return out
