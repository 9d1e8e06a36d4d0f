"""Seeded synthetic space-time fields.

These stand in for the paper's LES dataset of flow past a cylinder (float64,
three fluctuating velocity components, 695x396x149 grid, 1024 snapshots; Sec. 3),
which is not available here.  They mimic its structure: smooth advecting
vortical structures, a multiscale band of modes with a -5/3 amplitude slope,
and a small noise floor, stored as fluctuation fields.

This module holds none of the compression arithmetic.  It only draws seeded
parameters (numpy Philox) and evaluates the fields with torch on any device, so
the same bytes can be handed to both the CUDA library and the CPU oracle.

Layout of every returned tensor: (nvars, nt, nz, ny, nx), x fastest.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _periodic(d: torch.Tensor) -> torch.Tensor:
    return torch.remainder(d + 0.5, 1.0) - 0.5


def _wavevectors(rng, count, kmax):
    ks = []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=3)
        r = math.sqrt(float((k * k).sum()))
        if 1.0 <= r <= kmax:
            ks.append(k)
    return np.array(ks, dtype=np.int64)


def _modes(rng, dims, count, kmax, period, device, window=None):
    """sum_k a_k sin(2 pi k.x + omega_k t + phi_k), a_k ~ |k|^(-5/3), unit RMS.

    Evaluated per timestep as a complex separable product (one small matmul).
    `window` = ((x0, y0, z0, t0), (wx, wy, wz, wt)) evaluates a sub-box of the
    same field."""
    nx, ny, nz, nt = dims
    (x0, y0, z0, t0), (wx, wy, wz, wt) = window if window else ((0, 0, 0, 0), dims)
    ks = _wavevectors(rng, count, kmax)
    kn = np.sqrt((ks * ks).sum(1)).astype(np.float64)
    amp = kn ** (-5.0 / 3.0)
    amp /= math.sqrt(float((amp * amp).sum()) / 2.0)          # unit RMS
    phase = rng.uniform(0.0, 2.0 * math.pi, size=count)
    freq = rng.uniform(0.0, 2.0, size=count)                   # cycles per `period` steps
    omega = 2.0 * math.pi * freq / period
    cd = torch.complex128
    kx = torch.tensor(ks[:, 0], dtype=torch.float64, device=device)
    ky = torch.tensor(ks[:, 1], dtype=torch.float64, device=device)
    kz = torch.tensor(ks[:, 2], dtype=torch.float64, device=device)
    ix = torch.arange(x0, x0 + wx, dtype=torch.float64, device=device)
    iy = torch.arange(y0, y0 + wy, dtype=torch.float64, device=device)
    iz = torch.arange(z0, z0 + wz, dtype=torch.float64, device=device)
    EX = torch.polar(torch.ones(count, wx, dtype=torch.float64, device=device), 2 * math.pi * kx[:, None] * ix[None] / nx)
    EY = torch.polar(torch.ones(count, wy, dtype=torch.float64, device=device), 2 * math.pi * ky[:, None] * iy[None] / ny)
    EZ = torch.polar(torch.ones(count, wz, dtype=torch.float64, device=device), 2 * math.pi * kz[:, None] * iz[None] / nz)
    B = (EZ[:, :, None] * EY[:, None, :]).reshape(count, wz * wy)      # (K, wz*wy)
    a = torch.tensor(amp, dtype=torch.float64, device=device)
    ph = torch.tensor(phase, dtype=torch.float64, device=device)
    om = torch.tensor(omega, dtype=torch.float64, device=device)
    for t in range(wt):
        w = torch.polar(a, om * (t0 + t) + ph).to(cd)                  # (K,)
        U = (B * w[:, None]).transpose(0, 1) @ EX                      # (wz*wy, wx)
        yield t, U.imag.reshape(wz, wy, wx)


def _vortices(rng, dims, count, wrange, vrange, arange, dt, device, three_d=True):
    """sum_i A_i exp(-|x - c_i - v_i t|^2_periodic / (2 w_i^2)), separable per axis."""
    nx, ny, nz, nt = dims
    c = rng.uniform(0.0, 1.0, size=(count, 3))
    w = rng.uniform(wrange[0], wrange[1], size=count)
    v = rng.uniform(vrange[0], vrange[1], size=(count, 3))
    A = rng.uniform(arange[0], arange[1], size=count) * rng.choice([-1.0, 1.0], size=count)
    if not three_d:
        c[:, 2] = 0.0
        v[:, 2] = 0.0
    xs = torch.arange(nx, dtype=torch.float64, device=device) / nx
    ys = torch.arange(ny, dtype=torch.float64, device=device) / ny
    zs = torch.arange(nz, dtype=torch.float64, device=device) / max(nz, 1)
    wt = torch.tensor(w, dtype=torch.float64, device=device)
    At = torch.tensor(A, dtype=torch.float64, device=device)
    for t in range(nt):
        pos = torch.tensor(c + v * (t * dt), dtype=torch.float64, device=device)
        gx = torch.exp(-_periodic(xs[None] - pos[:, 0:1]) ** 2 / (2 * wt[:, None] ** 2))   # (V, nx)
        gy = torch.exp(-_periodic(ys[None] - pos[:, 1:2]) ** 2 / (2 * wt[:, None] ** 2))
        if three_d:
            gz = torch.exp(-_periodic(zs[None] - pos[:, 2:3]) ** 2 / (2 * wt[:, None] ** 2))
        else:
            gz = torch.ones(count, nz, dtype=torch.float64, device=device)
        B = (At[:, None, None] * gz[:, :, None] * gy[:, None, :]).reshape(count, nz * ny)
        yield t, (B.transpose(0, 1) @ gx).reshape(nz, ny, nx)


def vortex2d(nx=64, ny=64, nt=32, seed=1, count=6, noise=1e-4, device="cpu", dtype=torch.float64):
    """2-D time-dependent field: six advecting Gaussian vortices on [0,1)^2
    (periodic), dt = 1/nt, centres U[0,1)^2, widths U[0.03,0.10], velocities
    U[-0.5,0.5]^2, amplitudes +-U[0.5,1.5], plus noise * range * U[-1,1]."""
    rng = _rng(seed)
    out = torch.empty((1, nt, 1, ny, nx), dtype=torch.float64, device=device)
    for t, f in _vortices(rng, (nx, ny, 1, nt), count, (0.03, 0.10), (-0.5, 0.5), (0.5, 1.5),
                          1.0 / nt, device, three_d=False):
        out[0, t] = f
    rngt = torch.Generator(device=device)
    rngt.manual_seed(int(seed) * 7919 + 1)
    rngv = float(out.max() - out.min())
    out += noise * rngv * (2 * torch.rand(out.shape, generator=rngt, dtype=torch.float64, device=device) - 1)
    return out.to(dtype)


def modes3d(nx=256, ny=256, nz=256, nt=64, seed=2, count=64, kmax=8, period=64, noise=1e-3,
            device="cpu", dtype=torch.float32, window=None):
    """3-D field: `count` integer wavevectors with 1 <= |k| <= kmax, amplitudes
    ~ |k|^(-5/3), random phases, temporal frequencies U[0,2] cycles per 64
    steps, normalised to unit RMS, plus N(0, noise^2).  With `window` =
    ((x0, y0, z0, t0), (wx, wy, wz, wt)) only that sub-box is evaluated (same
    modes; its noise is drawn for the window alone)."""
    rng = _rng(seed)
    wx, wy, wz, wt = window[1] if window else (nx, ny, nz, nt)
    out = torch.empty((1, wt, wz, wy, wx), dtype=dtype, device=device)
    rngt = torch.Generator(device=device)
    rngt.manual_seed(int(seed) * 7919 + 2 + (0 if window is None else 1 + hash(tuple(window[0])) % 1000003))
    for t, f in _modes(rng, (nx, ny, nz, nt), count, kmax, period, device, window):
        nz_ = torch.randn((wz, wy, wx), generator=rngt, dtype=torch.float64, device=device)
        out[0, t] = (f + noise * nz_).to(dtype)
    return out


# Per-variable affine maps for the five-variable field: u, v, w, p, T.
_MULTIVAR = [(0.0, 1.0), (0.0, 1.0), (0.0, 0.6), (1.0, 0.3), (300.0, 5.0)]


def multivar(nx=250, ny=190, nz=130, nt=50, seeds=(40, 41, 42, 43, 44), device="cpu",
             dtype=torch.float32, noise=1e-3):
    """Five variables (three velocity components, pressure, temperature).  Each
    is 8 advecting 3-D Gaussian vortices + 32 modes (|k| <= 8) at half unit RMS +
    N(0, noise^2), then offset/scaled per variable."""
    out = torch.empty((len(seeds), nt, nz, ny, nx), dtype=dtype, device=device)
    for vi, seed in enumerate(seeds):
        rng = _rng(seed)
        off, sc = _MULTIVAR[vi % len(_MULTIVAR)]
        vg = _vortices(rng, (nx, ny, nz, nt), 8, (0.05, 0.15), (-0.5, 0.5), (0.5, 1.5), 1.0 / nt, device)
        mg = _modes(rng, (nx, ny, nz, nt), 32, 8, 64, device)
        rngt = torch.Generator(device=device)
        rngt.manual_seed(int(seed) * 7919 + 3)
        for (t, fv), (_, fm) in zip(vg, mg):
            nzs = torch.randn((nz, ny, nx), generator=rngt, dtype=torch.float64, device=device)
            out[vi, t] = (off + sc * (fv + 0.5 * fm + noise * nzs)).to(dtype)
    return out


def lowrank(L, n, rank, seed, scale=1.0, noise=0.0, dtype=np.float64):
    """Block matrix A = P Q^T (L x n) of exact rank `rank` (Eckart-Young pin)."""
    rng = _rng(seed)
    P = rng.standard_normal((L, rank))
    Q = rng.standard_normal((n, rank))
    A = scale * (P @ Q.T)
    if noise:
        A = A + noise * rng.standard_normal((L, n))
    return A.astype(dtype)


def field_lowrank(nx, ny, nz, nt, rank, seed, dtype=torch.float64):
    """Field whose every block has temporal rank <= `rank`: sum of `rank`
    separable products f_i(x,y,z) g_i(t) with smooth random profiles."""
    rng = _rng(seed)
    out = torch.zeros((1, nt, nz, ny, nx), dtype=torch.float64)
    for _ in range(rank):
        fx = torch.tensor(rng.standard_normal(nx))
        fy = torch.tensor(rng.standard_normal(ny))
        fz = torch.tensor(rng.standard_normal(nz))
        g = torch.tensor(rng.standard_normal(nt))
        out[0] += g[:, None, None, None] * (fz[:, None, None] * fy[None, :, None] * fx[None, None, :])
    return out.to(dtype)


# ---------------------------------------------------------------- fixed bases
# The two non-adaptive bases of the basis comparison (Sec. 4), as inputs: an
# n x n matrix whose column k is mode k (orthonormal columns).


def dct_basis(n: int) -> np.ndarray:
    """Orthonormal DCT-II modes in frequency order: column k, component a =
    s_k cos(pi (a + 1/2) k / n), s_0 = sqrt(1/n), s_k = sqrt(2/n) for k > 0."""
    a = np.arange(n, dtype=np.float64)[:, None]
    k = np.arange(n, dtype=np.float64)[None, :]
    B = np.cos(np.pi * (a + 0.5) * k / n) * math.sqrt(2.0 / n)
    B[:, 0] = math.sqrt(1.0 / n)
    return np.ascontiguousarray(B)


def random_basis(n: int, seed: int) -> np.ndarray:
    """Seeded random orthonormal modes: Q of the QR factorisation of an n x n
    standard-normal matrix (numpy Philox), columns signed so that R has a
    positive diagonal (a Haar-distributed orthogonal matrix); then one
    Gram-Schmidt pass in FP64 so the columns are orthonormal to rounding."""
    G = _rng(seed).standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    for k in range(n):
        v = Q[:, k].copy()
        for j in range(k):
            v -= (Q[:, j] @ v) * Q[:, j]
        Q[:, k] = v / np.linalg.norm(v)
    return np.ascontiguousarray(Q)


def patch_origins(dims, patch, count: int, seed: int) -> np.ndarray:
    """Seeded origins (x, y, z) of `count` patches of shape `patch` (px, py, pz)
    inside a snapshot of dims (nx, ny, nz), uniform over every position where
    the patch fits (numpy Philox): the random sample of Algorithm 1 step 1,
    drawn here so that every implementation receives the same patches."""
    rng = _rng(seed)
    hi = [int(d) - int(p) + 1 for d, p in zip(dims[:3], patch)]
    if min(hi) < 1:
        raise ValueError("patch larger than the snapshot")
    return np.stack([rng.integers(0, h, size=count) for h in hi], axis=1).astype(np.int64)
