"""Seeded synthetic inputs for the GSVD-MUSIC hot path.

This module only *generates inputs*: STFT-domain microphone frames, a preset
noise correlation, and a free-field steering table.  It holds none of the
method's arithmetic (no correlation, no whitening, no decomposition, no
spectrum); both the CUDA path and the FP64 oracle consume what it returns.

Recipe (all draws come from one ``numpy.random.Generator(PCG64(seed))``):

* Frequencies: fs = 16 kHz, 512-point STFT, bins k = 16..224 (209 bins),
  f_k = k * fs / 512 = 31.25 k Hz.  The STFT itself is upstream of the method
  (Sec. III-A, eq. 1), so frames are drawn directly in the STFT domain.
* Geometry: a uniform circular array (mic m at angle 2 pi m / M, z = 0) or M
  points uniform inside a ball.
* Directions: azimuth 0, 5, ..., 355 deg and elevation -90, -80, ..., 90 deg
  (or elevation 0 only).  Flat direction index d = el_idx * n_az + az_idx.
  Unit vector u = (cos el cos az, cos el sin az, sin el), with cos/sin of
  multiples of 90 deg exact so that the two pole rows are bit-identical.
* Steering (the transfer function H of eq. 5, measured in the paper, missing
  here): far-field free-field plane waves h_m = exp(+j 2 pi f (u . p_m) / c),
  c = 343 m/s.  The same formula places the simulated sources.
* Noise: per bin a mixing G = Q diag(sqrt(s)), Q Haar-unitary (QR of a complex
  Gaussian with the phase of diag(R) removed), s log-spaced from 1 down to
  1/cond.  Noise frames are n = G w, w ~ CN(0, I).
* Sources: i.i.d. CN(0, sigma_s^2) per (frame, bin), sigma_s^2 =
  10^(SNR/10) * tr(G G^H) / M (power against the mean per-channel noise).
* Frames: X(w, f) = sum_s h(theta_s, w) S_s(w, f) + G(w) w(w, f).
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SPEED_OF_SOUND = 343.0
FS = 16000.0
NFFT = 512
BIN_LO, BIN_HI = 16, 224  # inclusive


def bin_frequencies(lo: int = BIN_LO, hi: int = BIN_HI) -> np.ndarray:
    """Centre frequencies (Hz) of STFT bins lo..hi inclusive."""
    k = np.arange(lo, hi + 1, dtype=np.float64)
    return k * FS / NFFT


def _cos_sin_deg(deg: np.ndarray):
    """cos/sin of angles in degrees, exact at multiples of 90 degrees."""
    deg = np.asarray(deg, dtype=np.float64)
    rad = np.deg2rad(deg)
    c, s = np.cos(rad), np.sin(rad)
    q = np.mod(deg, 360.0)
    exact = np.isclose(np.mod(q, 90.0), 0.0)
    if np.any(exact):
        quad = np.round(q / 90.0).astype(int) % 4
        cq = np.array([1.0, 0.0, -1.0, 0.0])[quad]
        sq = np.array([0.0, 1.0, 0.0, -1.0])[quad]
        c = np.where(exact, cq, c)
        s = np.where(exact, sq, s)
    return c, s


@dataclasses.dataclass(frozen=True)
class Grid:
    """Direction grid: n_el elevation rows x n_az azimuth columns."""

    az_deg: np.ndarray
    el_deg: np.ndarray

    @property
    def n_az(self) -> int:
        return int(self.az_deg.size)

    @property
    def n_el(self) -> int:
        return int(self.el_deg.size)

    @property
    def D(self) -> int:
        return self.n_az * self.n_el

    def unit_vectors(self) -> np.ndarray:
        """[D][3] unit vectors, d = el_idx * n_az + az_idx."""
        ca, sa = _cos_sin_deg(self.az_deg)
        ce, se = _cos_sin_deg(self.el_deg)
        u = np.empty((self.n_el, self.n_az, 3))
        u[..., 0] = ce[:, None] * ca[None, :]
        u[..., 1] = ce[:, None] * sa[None, :]
        u[..., 2] = se[:, None] * np.ones_like(ca)[None, :]
        return u.reshape(-1, 3)


def azimuth_grid(step_deg: float = 5.0) -> Grid:
    return Grid(np.arange(0.0, 360.0, step_deg), np.array([0.0]))


def sphere_grid(az_step: float = 5.0, el_step: float = 10.0) -> Grid:
    return Grid(np.arange(0.0, 360.0, az_step), np.arange(-90.0, 90.0 + 1e-9, el_step))


@dataclasses.dataclass(frozen=True)
class DirectionSet:
    """Directions that form no grid (e.g. the paper's 2522-direction measured
    transfer functions, Sec. V), with each direction's neighbours for the peak
    search as compressed rows: neighbours of d are
    nbr_idx[nbr_ptr[d]:nbr_ptr[d + 1]] (ascending, d itself excluded).  The
    library's convention for such a set is n_az = D, n_el = 0."""

    u: np.ndarray        # [D][3] unit vectors
    nbr_ptr: np.ndarray  # [D + 1] int32
    nbr_idx: np.ndarray  # [E] int32

    @property
    def D(self) -> int:
        return int(self.u.shape[0])

    @property
    def n_az(self) -> int:
        return self.D

    @property
    def n_el(self) -> int:
        return 0

    def unit_vectors(self) -> np.ndarray:
        return self.u


def _csr(lists):
    ptr = np.zeros(len(lists) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(x) for x in lists])
    idx = np.concatenate([np.asarray(sorted(x), dtype=np.int32) for x in lists]) if lists else \
        np.zeros(0, dtype=np.int32)
    return ptr, idx.astype(np.int32)


def fibonacci_sphere(n: int = 2522, k: int = 6) -> DirectionSet:
    """n directions spread evenly over the sphere by the golden-angle spiral
    (z_i = 1 - (2 i + 1) / n, azimuth i times the golden angle), each with its
    k nearest directions (largest u . v) as neighbours, made symmetric (a
    direction lists every direction that lists it)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    u = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    dots = u @ u.T
    np.fill_diagonal(dots, -np.inf)
    knn = np.argsort(-dots, axis=1, kind="stable")[:, :k]
    sets = [set(int(j) for j in knn[d]) for d in range(n)]
    for d in range(n):
        for j in knn[d]:
            sets[int(j)].add(d)
    ptr, idx = _csr([list(x) for x in sets])
    return DirectionSet(u=u, nbr_ptr=ptr, nbr_idx=idx)


def grid_neighbours(n_az: int, n_el: int):
    """The n_el x n_az grid's 8-neighbourhood (azimuth wraps, rows outside the
    grid dropped, d itself excluded) as compressed rows (nbr_ptr, nbr_idx)."""
    lists = []
    for d in range(n_az * n_el):
        e, a = divmod(d, n_az)
        nb = set()
        for de in (-1, 0, 1):
            if not 0 <= e + de < n_el:
                continue
            for da in (-1, 0, 1):
                n = (e + de) * n_az + (a + da) % n_az
                if n != d:
                    nb.add(n)
        lists.append(list(nb))
    return _csr(lists)


def uca(M: int, radius: float) -> np.ndarray:
    """[M][3] positions of a uniform circular array in the z = 0 plane."""
    ang = 2.0 * np.pi * np.arange(M) / M
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(M)], axis=1)


def ball(M: int, radius: float, rng: np.random.Generator) -> np.ndarray:
    """[M][3] positions drawn uniformly inside a ball."""
    v = rng.standard_normal((M, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.random(M) ** (1.0 / 3.0)
    return v * r[:, None]


def steering(pos: np.ndarray, u: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """Free-field far-field plane-wave responses H[B][D][M] (complex128)."""
    delay = u @ pos.T / SPEED_OF_SOUND  # [D][M] seconds
    ph = 2.0 * np.pi * freqs[:, None, None] * delay[None, :, :]
    return np.exp(1j * ph)


def cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex Gaussian CN(0, 1) samples."""
    z = rng.standard_normal(tuple(shape) + (2,)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def haar_unitary(rng: np.random.Generator, B: int, M: int) -> np.ndarray:
    """[B][M][M] Haar-distributed unitary matrices."""
    Z = cgauss(rng, (B, M, M))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    ph = d / np.abs(d)
    return Q * ph[:, None, :]


def noise_mixing(rng: np.random.Generator, B: int, M: int, cond: float) -> np.ndarray:
    """[B][M][M] mixing G = Q diag(sqrt(s)), s log-spaced 1 .. 1/cond."""
    s = np.logspace(0.0, -np.log10(cond), M)
    return haar_unitary(rng, B, M) * np.sqrt(s)[None, None, :]


@dataclasses.dataclass
class Workload:
    """One array's synthetic input.

    X:        [nblk][T][B][M] complex frames, one non-overlapping block of T
              frames per entry of the first axis.
    Xnoise:   [N_K][B][M] noise-only frames from which K is estimated.
    K_true:   [B][M][M] population noise correlation G G^H.
    H:        [B][D][M] steering table.
    """

    X: np.ndarray
    Xnoise: np.ndarray
    K_true: np.ndarray
    H: np.ndarray
    pos: np.ndarray
    grid: "Grid | DirectionSet"
    freqs: np.ndarray
    src_dirs: np.ndarray  # [nblk][Ns][3] unit vectors of the true sources
    src_grid_idx: np.ndarray  # [nblk][Ns] grid index when on-grid, else -1
    snr_db: np.ndarray  # [Ns]
    Ns: int
    T: int

    @property
    def nblk(self) -> int:
        return int(self.X.shape[0])

    @property
    def B(self) -> int:
        return int(self.X.shape[2])

    @property
    def M(self) -> int:
        return int(self.X.shape[3])

    @property
    def D(self) -> int:
        return int(self.H.shape[1])


def _frames(rng, pos, G, freqs, dirs_per_blk, snr_db, nblk, T, dtype):
    B, M = G.shape[0], G.shape[1]
    noise_pow = np.real(np.einsum("bij,bij->b", G, G.conj())) / M  # tr(GG^H)/M per bin
    X = np.empty((nblk, T, B, M), dtype=dtype)
    for k in range(nblk):
        W = cgauss(rng, (B, M, T))
        frames = np.matmul(G, W)  # [B][M][T]
        for s, u in enumerate(dirs_per_blk[k]):
            h = steering(pos, u[None, :], freqs)[:, 0, :]  # [B][M]
            amp = np.sqrt(10.0 ** (snr_db[s] / 10.0) * noise_pow)  # [B]
            S = cgauss(rng, (B, T)) * amp[:, None]
            frames += h[:, :, None] * S[:, None, :]
        X[k] = np.transpose(frames, (2, 0, 1))
    return X


def make_workload(
    M: int,
    T: int = 50,
    nblk: int = 1,
    Ns: int = 1,
    geometry: str = "uca",
    radius: float = 0.1,
    grid: Optional[Grid] = None,
    snr_db=0.0,
    cond: float = 1e3,
    n_k: Optional[int] = None,
    bins=(BIN_LO, BIN_HI),
    on_grid: bool = True,
    max_abs_el: float = 80.0,
    drift_deg_per_blk: float = 0.0,
    seed: int = 1,
    dtype=np.complex64,
) -> Workload:
    """Generate one array's frames, noise frames, K and steering table."""
    rng = np.random.default_rng(seed)
    grid = grid if grid is not None else azimuth_grid()
    freqs = bin_frequencies(*bins)
    B = freqs.size
    if geometry == "uca":
        pos = uca(M, radius)
    elif geometry == "ball":
        pos = ball(M, radius, rng)
    else:
        raise ValueError(geometry)
    u_grid = grid.unit_vectors()
    H = steering(pos, u_grid, freqs)
    G = noise_mixing(rng, B, M, cond)
    K_true = np.matmul(G, np.conj(np.transpose(G, (0, 2, 1))))
    snr = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (Ns,)).copy()

    # Source directions (fixed over blocks unless drifting in azimuth).
    if on_grid and not isinstance(grid, Grid):
        raise ValueError("on-grid sources need a Grid")
    if on_grid:
        el_ok = np.nonzero(np.abs(grid.el_deg) <= max_abs_el + 1e-9)[0]
        idx0 = []
        while len(idx0) < Ns:
            e = int(rng.choice(el_ok))
            a = int(rng.integers(grid.n_az))
            d = e * grid.n_az + a
            if d not in idx0:
                idx0.append(d)
        az0 = np.array([grid.az_deg[d % grid.n_az] for d in idx0])
        el0 = np.array([grid.el_deg[d // grid.n_az] for d in idx0])
    else:
        az0 = rng.uniform(0.0, 360.0, Ns)
        if isinstance(grid, Grid) and grid.n_el == 1:
            el0 = np.zeros(Ns)
        else:
            el0 = np.rad2deg(np.arcsin(rng.uniform(-1.0, 1.0, Ns)))
    dirs = np.empty((nblk, Ns, 3))
    gidx = np.full((nblk, Ns), -1, dtype=np.int64)
    for k in range(nblk):
        az = az0 + drift_deg_per_blk * k
        ca, sa = _cos_sin_deg(az)
        ce, se = _cos_sin_deg(el0)
        dirs[k] = np.stack([ce * ca, ce * sa, se], axis=1)
        if on_grid:
            step = grid.az_deg[1] - grid.az_deg[0] if grid.n_az > 1 else 360.0
            for s in range(Ns):
                a = np.mod(az[s], 360.0) / step
                if np.isclose(a, np.round(a)):
                    e = int(np.argmin(np.abs(grid.el_deg - el0[s])))
                    gidx[k, s] = e * grid.n_az + int(np.round(a)) % grid.n_az
    X = _frames(rng, pos, G, freqs, dirs, snr, nblk, T, dtype)
    nk = n_k if n_k is not None else max(50, 4 * M)
    Wn = cgauss(rng, (B, M, nk))
    Xnoise = np.ascontiguousarray(np.transpose(np.matmul(G, Wn), (2, 0, 1)), dtype=dtype)
    return Workload(
        X=X,
        Xnoise=Xnoise,
        K_true=K_true,
        H=H,
        pos=pos,
        grid=grid,
        freqs=freqs,
        src_dirs=dirs,
        src_grid_idx=gidx,
        snr_db=snr,
        Ns=Ns,
        T=T,
    )


# ---------------------------------------------------------------------------
# The workloads the method is measured on (M, geometry, grid, sources, K).
# ---------------------------------------------------------------------------

def uca8_single_source(seed: int = 1, nblk: int = 1, **kw) -> Workload:
    """8-mic UCA (r = 0.1 m), 72 azimuths, one on-grid source at 0 dB, K cond 1e3,
    K from 50 noise frames, 209 bins, T = 50."""
    args = dict(M=8, T=50, nblk=nblk, Ns=1, geometry="uca", radius=0.1, grid=azimuth_grid(),
                snr_db=0.0, cond=1e3, n_k=50, seed=seed)
    args.update(kw)
    return make_workload(**args)


def ball60_three_sources(seed: int = 2, nblk: int = 100, **kw) -> Workload:
    """60 mics uniform in a 0.4 m ball, 72 x 19 sphere grid (D = 1368), three
    sources at continuous directions with per-source SNR ~ U[-5, 10] dB, K from
    240 noise frames (cond 1e3), 209 bins, T = 50, nblk consecutive blocks."""
    rng = np.random.default_rng(seed + 1000)
    snr = rng.uniform(-5.0, 10.0, 3)
    args = dict(M=60, T=50, nblk=nblk, Ns=3, geometry="ball", radius=0.4, grid=sphere_grid(),
                snr_db=snr, cond=1e3, n_k=240, on_grid=False, seed=seed)
    args.update(kw)
    return make_workload(**args)


def paper_shape(seed: int = 3, nblk: int = 100, **kw) -> Workload:
    """The paper's own shape (Sec. V): 60 mics (uniform in a 0.4 m ball),
    73 bins (k = 16..88 of the 512-point STFT, 0.5-2.75 kHz), a 2522-direction
    set over the sphere (Fibonacci spiral, 6 nearest neighbours made
    symmetric), two sources at continuous directions with per-source SNR
    U[-5, 10] dB, K from 240 noise frames (cond 1e3), T = 50."""
    rng = np.random.default_rng(seed + 1000)
    snr = rng.uniform(-5.0, 10.0, 2)
    args = dict(M=60, T=50, nblk=nblk, Ns=2, geometry="ball", radius=0.4,
                grid=fibonacci_sphere(2522), snr_db=snr, cond=1e3, n_k=240,
                bins=(16, 88), on_grid=False, seed=seed)
    args.update(kw)
    return make_workload(**args)
