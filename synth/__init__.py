"""Seeded synthetic inputs for handheld near-range SAR imaging.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds only input generation: trajectories, frequency
lists, scatterer scenes, output grids and the monostatic Born-model echoes of
Section II-A, Eq. (1):

    s(p', k) = sum_p f(p) exp(-j 2 k ||p - p'||),   k = 2 pi f / c

It contains none of the imaging method's arithmetic (no range compression,
backprojection, spectrum compression or interpolation).

Workload recipes (sizes, trajectory kinds, scenes, grids) follow the synthetic
configurations the project measures on; every random draw comes from a numpy
PCG64 generator seeded per configuration (scene seed 1000 + index, noise seed
2000 + index), so CPU and GPU runs see identical inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0  # m/s (exact SI value; the paper gives no value)


@dataclasses.dataclass
class Grid:
    """Cartesian output grid D: voxel (a, b, c) sits at (x0 + a dx, y0 + b dy, z0 + c dz).

    Images are stored as complex64[nz][ny][nx] (x fastest).
    """
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_vox(self):
        return self.nx * self.ny * self.nz

    def axes(self):
        x = self.x0 + self.dx * np.arange(self.nx)
        y = self.y0 + self.dy * np.arange(self.ny)
        z = self.z0 + self.dz * np.arange(self.nz)
        return x, y, z

    def points(self, flat_index=None):
        """Voxel centres as float64[n][3] in storage order (x fastest)."""
        if flat_index is None:
            flat_index = np.arange(self.n_vox)
        flat_index = np.asarray(flat_index, dtype=np.int64)
        a = flat_index % self.nx
        b = (flat_index // self.nx) % self.ny
        c = flat_index // (self.nx * self.ny)
        return np.column_stack([self.x0 + a * self.dx, self.y0 + b * self.dy, self.z0 + c * self.dz])

    def as_tuple(self):
        return (self.x0, self.y0, self.z0, self.dx, self.dy, self.dz, self.nx, self.ny, self.nz)


@dataclasses.dataclass
class Scene:
    name: str
    traj: np.ndarray        # float64[n_pos][3], metres
    freqs: np.ndarray       # float64[n_f], Hz, equidistant
    scat_pos: np.ndarray    # float64[n_s][3]
    scat_amp: np.ndarray    # complex128[n_s]
    grid: Grid
    snr_db: float | None
    noise_seed: int


def centred_grid(nx, ny, nz, dx, dy, dz, z0):
    return Grid(-(nx - 1) * dx / 2, -(ny - 1) * dy / 2, z0, dx, dy, dz, nx, ny, nz)


def freq_list(f_lo, f_hi, n_f):
    """n_f equidistant frequencies from f_lo to f_hi inclusive (Hz)."""
    return np.linspace(f_lo, f_hi, n_f)


def serpentine(n_lines, n_per_line, width, height):
    """Lines along x stepping in y, alternate lines reversed; endpoints included."""
    xs = np.linspace(-width / 2, width / 2, n_per_line)
    ys = np.linspace(-height / 2, height / 2, n_lines)
    rows = []
    for line in range(n_lines):
        row = xs if line % 2 == 0 else xs[::-1]
        rows.append(np.column_stack([row, np.full(n_per_line, ys[line])]))
    return np.concatenate(rows)


def random_walk_raster(rng, n_lines, n_per_line, width, height, step_sigma, clip, z_halfwidth):
    """Serpentine raster plus a clipped Gaussian random walk in x,y and uniform z jitter."""
    xy = serpentine(n_lines, n_per_line, width, height)
    walk = np.clip(np.cumsum(rng.normal(0.0, step_sigma, size=xy.shape), axis=0), -clip, clip)
    z = rng.uniform(-z_halfwidth, z_halfwidth, size=len(xy))
    return np.column_stack([xy + walk, z])


def jittered_zigzag(rng, n_lines, n_per_line, width, height, sigma):
    """Serpentine (zig-zag) raster with i.i.d. Gaussian jitter of std sigma on x, y and z."""
    xy = serpentine(n_lines, n_per_line, width, height)
    jit = rng.normal(0.0, sigma, size=(len(xy), 3))
    return np.column_stack([xy, np.zeros(len(xy))]) + jit


def plate(rng, centre, n_side, pitch, amp, max_tilt_deg):
    """A square n_side x n_side point lattice (pitch in m), tilted by <= max_tilt_deg."""
    g = (np.arange(n_side) - (n_side - 1) / 2) * pitch
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.column_stack([X.ravel(), Y.ravel(), np.zeros(X.size)])
    tilt = math.radians(rng.uniform(0.0, max_tilt_deg))
    az = rng.uniform(0.0, 2 * math.pi)
    axis = np.array([math.cos(az), math.sin(az), 0.0])
    # Rodrigues rotation about an in-plane axis
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rm = np.eye(3) + math.sin(tilt) * K + (1 - math.cos(tilt)) * K @ K
    return pts @ Rm.T + np.asarray(centre), np.full(len(pts), amp, dtype=np.complex128)


def tiny():
    """2,048 positions, 128 freqs 76-81 GHz, 8 points, 64x64x16 grid."""
    rng = np.random.default_rng(1000)
    traj = random_walk_raster(rng, 32, 64, 0.2, 0.2, 0.5e-3, 5e-3, 5e-3)
    n_s = 8
    pos = np.column_stack([rng.uniform(-0.05, 0.05, n_s), rng.uniform(-0.05, 0.05, n_s),
                           rng.uniform(0.29, 0.31, n_s)])
    return Scene("tiny", traj, freq_list(76e9, 81e9, 128), pos, np.ones(n_s, np.complex128),
                 centred_grid(64, 64, 16, 2e-3, 2e-3, 1e-2, 0.225), None, 2000)


def mid():
    """16,384 positions, 256 freqs, 64 points + 4 plates, 256x256x64 grid, SNR 20 dB."""
    rng = np.random.default_rng(1001)
    traj = jittered_zigzag(rng, 128, 128, 0.4, 0.4, 3e-3)
    n_p = 64
    pos = [np.column_stack([rng.uniform(-0.15, 0.15, n_p), rng.uniform(-0.15, 0.15, n_p),
                            rng.uniform(0.25, 0.45, n_p)])]
    amp = [np.ones(n_p, np.complex128)]
    for _ in range(4):
        c = (rng.uniform(-0.12, 0.12), rng.uniform(-0.12, 0.12), rng.uniform(0.27, 0.43))
        p, a = plate(rng, c, 32, 1e-3, 1.0 / 32, 10.0)
        pos.append(p)
        amp.append(a)
    return Scene("mid", traj, freq_list(76e9, 81e9, 256), np.concatenate(pos), np.concatenate(amp),
                 centred_grid(256, 256, 64, 0.4 / 256, 0.4 / 256, 0.2 / 64, 0.25), 20.0, 2001)


def large():
    """65,536 positions, 512 freqs, 256 points, 512x512x128 grid."""
    rng = np.random.default_rng(1004)
    traj = random_walk_raster(rng, 256, 256, 0.5, 0.5, 0.5e-3, 5e-3, 5e-3)
    n_s = 256
    pos = np.column_stack([rng.uniform(-0.2, 0.2, n_s), rng.uniform(-0.2, 0.2, n_s),
                           rng.uniform(0.2, 0.4, n_s)])
    return Scene("large", traj, freq_list(76e9, 81e9, 512), pos, np.ones(n_s, np.complex128),
                 centred_grid(512, 512, 128, 0.5 / 512, 0.5 / 512, 0.2 / 128, 0.2), None, 2004)


def small(n_lines=16, n_per_line=16, n_f=32, nx=24, ny=20, nz=6, seed=1100):
    """A deliberately small scene (ragged sizes) for fast parity and edge-case tests."""
    rng = np.random.default_rng(seed)
    traj = random_walk_raster(rng, n_lines, n_per_line, 0.1, 0.1, 0.5e-3, 3e-3, 3e-3)
    n_s = 4
    pos = np.column_stack([rng.uniform(-0.03, 0.03, n_s), rng.uniform(-0.03, 0.03, n_s),
                           rng.uniform(0.18, 0.22, n_s)])
    return Scene("small", traj, freq_list(76e9, 81e9, n_f), pos, np.ones(n_s, np.complex128),
                 centred_grid(nx, ny, nz, 2.5e-3, 2.5e-3, 1e-2, 0.17), None, seed + 1000)


def diff():
    """Differentiation scene: 8,192 positions (nominal track), 128 freqs, 32 points,
    128x128x32 grid.  The echoes of this scene come from the true track, nominal +
    diff_offsets() (smooth, 1 mm rms per axis): see diff_echo()."""
    rng = np.random.default_rng(1003)
    traj = random_walk_raster(rng, 64, 128, 0.25, 0.25, 0.5e-3, 5e-3, 5e-3)
    n_s = 32
    pos = np.column_stack([rng.uniform(-0.1, 0.1, n_s), rng.uniform(-0.1, 0.1, n_s),
                           rng.uniform(0.22, 0.38, n_s)])
    return Scene("diff", traj, freq_list(76e9, 81e9, 128), pos, np.ones(n_s, np.complex128),
                 centred_grid(128, 128, 32, 2e-3, 2e-3, 6.25e-3, 0.2), None, 2003)


def diff_offsets(n_pos, seed=3003, sigma_t=128.0, rms=1e-3):
    """Smooth position offsets: white Gaussian noise per axis, filtered along the track by a
    Gaussian of sigma_t samples, scaled to `rms` metres rms per axis."""
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(n_pos, 3))
    half = int(4 * sigma_t)
    ker = np.exp(-0.5 * (np.arange(-half, half + 1) / sigma_t) ** 2)
    out = np.column_stack([np.convolve(w[:, a], ker, mode="same") for a in range(3)])
    out -= out.mean(axis=0)
    return out * (rms / np.sqrt((out ** 2).mean(axis=0)))


def diff_echo(scene, offsets, device="cpu"):
    """complex64 echoes of the scene recorded along the true track traj + offsets."""
    import torch

    e = echoes(np.asarray(scene.traj) + offsets, scene.freqs, scene.scat_pos, scene.scat_amp, device=device)
    return e.to(torch.complex64)


def _smooth(rng, n, sigma, amp):
    """n samples of white Gaussian noise filtered by a Gaussian of sigma samples, scaled so
    that its largest magnitude is amp."""
    half = int(4 * sigma)
    ker = np.exp(-0.5 * (np.arange(-half, half + 1) / sigma) ** 2)
    x = np.convolve(rng.normal(size=n + 2 * half), ker, mode="same")[half:half + n]
    x -= x.mean()
    return x * (amp / np.abs(x).max())


def sim1():
    """Stand-in for the paper's point-scatterer simulation (Sec. V-A): a 101-element linear
    array (along y, 4.5 mm pitch) scanned over 101 positions along x (0.45 x 0.45 m), with
    smooth seeded fluctuations of the scan position (x +/- 5 mm), array height (+/- 1.5 cm),
    roll about the scan axis (+/- 6.5 deg) and yaw (+/- 2 deg): element depths within 8 cm;
    24 frequencies 12-15 GHz; a 3x3x3 lattice of unit point scatterers at 0.175 m pitch centred
    0.4 m in front of the aperture; a 101x101x51 grid over 0.5 m^3 centred at that depth."""
    rng = np.random.default_rng(1005)
    n_scan, n_el = 101, 101
    xs = np.linspace(-0.225, 0.225, n_scan)
    ys = np.linspace(-0.225, 0.225, n_el)
    dx = _smooth(rng, n_scan, 6.0, 5e-3)
    dz = _smooth(rng, n_scan, 6.0, 1.5e-2)
    roll = np.deg2rad(_smooth(rng, n_scan, 6.0, 6.5))
    yaw = np.deg2rad(_smooth(rng, n_scan, 6.0, 2.0))
    pts = []
    for i in range(n_scan):
        # element y rotated by yaw (about z) and roll (about x), then shifted
        ex = xs[i] + dx[i] - ys * np.sin(yaw[i])
        ey = ys * np.cos(yaw[i]) * np.cos(roll[i])
        ez = dz[i] + ys * np.cos(yaw[i]) * np.sin(roll[i])
        pts.append(np.column_stack([ex, ey, ez]))
    traj = np.concatenate(pts)
    g = np.array([-0.175, 0.0, 0.175])
    pos = np.stack(np.meshgrid(g, g, g + 0.4, indexing="ij"), -1).reshape(-1, 3)
    return Scene("sim1", traj, freq_list(12e9, 15e9, 24), pos, np.ones(len(pos), np.complex128),
                 centred_grid(101, 101, 51, 5e-3, 5e-3, 1e-2, 0.15), None, 2005)


def batch_scene(index, seed=3000):
    """Scan `index` of the batching workload: 4,096-32,768 positions (128 per raster line) of a
    random-walk raster over 0.2-0.4 m (growing with the length), 128-256 frequencies
    76-81 GHz, 16-64 unit points at z 0.22-0.38 m, a grid of 128-384 squared x 32-64 voxels
    over the aperture and 0.2 m of depth from z = 0.2 m."""
    rng = np.random.default_rng(seed + index)
    n_lines = int(rng.integers(32, 257))
    n_pos = 128 * n_lines
    width = 0.2 + 0.2 * math.sqrt((n_pos - 4096) / (32768 - 4096))
    traj = random_walk_raster(rng, n_lines, 128, width, width, 0.5e-3, 5e-3, 5e-3)
    n_f = 128 + 32 * int(rng.integers(0, 5))
    n_s = int(rng.integers(16, 65))
    pos = np.column_stack([rng.uniform(-0.4 * width, 0.4 * width, n_s), rng.uniform(-0.4 * width, 0.4 * width, n_s),
                           rng.uniform(0.22, 0.38, n_s)])
    nxy = 128 + 32 * int(rng.integers(0, 9))
    nz = 32 + 8 * int(rng.integers(0, 5))
    d = (width + 0.05) / nxy
    return Scene(f"batch{index}", traj, freq_list(76e9, 81e9, n_f), pos, np.ones(n_s, np.complex128),
                 centred_grid(nxy, nxy, nz, d, d, 0.2 / nz, 0.2), None, seed + 1000 + index)


CONFIGS = {"tiny": tiny, "mid": mid, "large": large, "small": small, "diff": diff, "sim1": sim1}


def echoes(traj, freqs, scat_pos, scat_amp, device="cpu", max_elems=1 << 25):
    """Monostatic Born-model echoes s[i, n] = sum_s a_s exp(-j 2 k_n ||p_s - p'_i||), Eq. (1).

    Computed in float64 with torch on ``device``; returns complex128[n_pos][n_f].
    """
    import torch

    t = torch.as_tensor(np.asarray(traj, np.float64), device=device)
    P = torch.as_tensor(np.asarray(scat_pos, np.float64), device=device)
    a = torch.as_tensor(np.asarray(scat_amp, np.complex128), device=device)
    k = torch.as_tensor(2 * np.pi * np.asarray(freqs, np.float64) / C_LIGHT, device=device)
    n_pos, n_s, n_f = t.shape[0], P.shape[0], k.shape[0]
    out = torch.empty((n_pos, n_f), dtype=torch.complex128, device=device)
    chunk = max(1, max_elems // max(1, n_s * n_f))
    for i0 in range(0, n_pos, chunk):
        i1 = min(n_pos, i0 + chunk)
        d = t[i0:i1, None, :] - P[None, :, :]
        R = torch.sqrt((d * d).sum(-1))                       # [c, S]
        ph = -2.0 * R[:, :, None] * k[None, None, :]         # [c, S, F]
        out[i0:i1] = (a[None, :, None] * torch.polar(torch.ones_like(ph), ph)).sum(1)
    return out


def add_noise(echo, snr_db, seed):
    """Additive circular complex Gaussian noise with mean|s|^2 / sigma^2 = 10^(snr/10)."""
    import torch

    if snr_db is None:
        return echo
    rng = np.random.default_rng(seed)
    p_sig = float((echo.abs() ** 2).mean())
    sigma = math.sqrt(p_sig / 10 ** (snr_db / 10) / 2)
    nz = rng.standard_normal((echo.shape[0], echo.shape[1], 2)) * sigma
    noise = torch.as_tensor(nz[..., 0] + 1j * nz[..., 1], device=echo.device)
    return echo + noise


def scene_echo(scene: Scene, device="cpu"):
    """Echoes of a scene as complex64 (the library's input type), noise included."""
    import torch

    e = echoes(scene.traj, scene.freqs, scene.scat_pos, scene.scat_amp, device=device)
    e = add_noise(e, scene.snr_db, scene.noise_seed)
    return e.to(torch.complex64)
