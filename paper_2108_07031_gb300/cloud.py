"""Seeded synthetic NACA 0012 O-type point clouds (input generator).

The paper benchmarks inviscid flow past a NACA 0012 aerofoil on seven point
distributions of 0.625M to 40M points (Section 4, opening paragraph of the
RDP study). Those distributions are not published, so this module builds
stand-ins of the same shape: an O-type cloud around the aerofoil, stretched
out to a far-field circle, with seeded jitter so the cloud is genuinely
unstructured, and radius-based stencils N(P0) = {P : d(P, P0) < eps} as in
Section 2 (definition of the stencil of P0).

This module only produces inputs: coordinates, normals, point flags and
neighbour lists. It holds none of the solver's arithmetic and is shared by the
CUDA path and by the CPU oracle tests.

Recipe
------
* Wall: closed-trailing-edge NACA 0012 half-thickness
  ``y_t = 0.6 (0.2969 sqrt(x) - 0.1260 x - 0.3516 x^2 + 0.2843 x^3 - 0.1036 x^4)``
  at ``x = 1 - sin(psi)``, ``psi = (pi - |pi - theta|) / 2``,
  ``theta_k = 2 pi k / n_c`` (half-cosine clustering: fine at the leading
  edge, near-uniform at the trailing edge), upper surface for ``sin theta > 0``. The wall loop runs
  counter-clockwise starting at the trailing edge.
* Far field: circle of radius 20 chords centred at (0.5, 0), matched angle.
* Layers: linear blend between the wall point and the far-field point of the
  same angle, blend parameter ``s_l = (r^l - 1) / (r^(n_r-1) - 1)`` with
  ``r = 1.1^(39/(n_r-1))`` (geometric ratio 1.1 at 40 layers; the same
  continuous distribution for finer clouds).
* Jitter: interior layers only, the (k, l) parameters perturbed by
  U(-0.1, 0.1) each (10 % of the local spacing), numpy PCG64 seeded.
* Stencils: candidates from the +-2 index window in both directions, kept if
  closer than ``1.6 max(h_c, h_r)`` (local spacings of the unjittered grid),
  nearest first, ties by index, at most 20. A tied group is never split by the
  cap, so mirror-symmetric clouds keep mirror-symmetric stencils.
* Flags: 0 interior, 1 wall, 2 outer (far field). Normals: wall normals point
  into the fluid (right-hand normal of the counter-clockwise loop, from the
  central difference of the loop), outer normals point out of the domain
  (radial), interior normals are (0, 1).
* Ordering: wall points first in loop order (0..n_c-1); with ``shuffle=True``
  every other point is placed by a seeded permutation, which is how an
  unstructured point distribution arrives.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

FLAG_INTERIOR = 0
FLAG_WALL = 1
FLAG_OUTER = 2

MAX_NEIGHBOURS = 20
FAR_FIELD_RADIUS = 20.0
FAR_FIELD_CENTRE = (0.5, 0.0)


@dataclasses.dataclass
class Cloud:
    """A point cloud ready for ``lskum_create`` / the oracle.

    Arrays are in user order. ``nbr_offsets``/``nbr_idx`` are CSR (int32).
    ``wall_loop`` lists the wall points in loop order (the first ``n_c``
    points). ``k``/``l`` are the circumferential / radial generator indices of
    every point (diagnostics and mirror tests only).
    """

    xy: np.ndarray
    normals: np.ndarray
    flags: np.ndarray
    nbr_offsets: np.ndarray
    nbr_idx: np.ndarray
    n_c: int
    n_r: int
    k: np.ndarray
    l: np.ndarray

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    @property
    def wall_loop(self) -> np.ndarray:
        return np.arange(self.n_c, dtype=np.int64)

    def neighbours(self, i: int) -> np.ndarray:
        return self.nbr_idx[self.nbr_offsets[i]:self.nbr_offsets[i + 1]]


def naca0012_half_thickness(x):
    x = np.clip(x, 0.0, 1.0)
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2
                  + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def _wall(theta):
    # half-cosine clustering: fine at the leading edge (theta = pi), near-uniform
    # at the trailing edge (theta = 0, 2 pi)
    psi = 0.5 * (np.pi - np.abs(np.pi - np.mod(theta, 2.0 * np.pi)))
    x = 1.0 - np.sin(psi)
    yt = naca0012_half_thickness(x)
    y = np.where(np.sin(theta) > 0.0, yt, -yt)
    return x, y


def _outer(theta):
    cx, cy = FAR_FIELD_CENTRE
    return cx + FAR_FIELD_RADIUS * np.cos(theta), cy + FAR_FIELD_RADIUS * np.sin(theta)


def _blend(n_r, lf):
    ratio = 1.1 ** (39.0 / (n_r - 1))
    return (ratio ** lf - 1.0) / (ratio ** (n_r - 1) - 1.0)


def _points(kf, lf, n_c, n_r):
    """Coordinates at (possibly fractional) generator parameters."""
    theta = 2.0 * np.pi * kf / n_c
    wx, wy = _wall(theta)
    ox, oy = _outer(theta)
    s = _blend(n_r, lf)
    return (1.0 - s) * wx + s * ox, (1.0 - s) * wy + s * oy


def cloud_dims(n_points: int) -> tuple[int, int]:
    """(n_c, n_r) for a target size, keeping the 128 x 40 aspect of the base cloud."""
    if n_points <= 0:
        raise ValueError("n_points must be positive")
    scale = math.sqrt(n_points / (128 * 40))
    n_c = max(8, int(round(128 * scale)))
    n_c += n_c % 2  # even, so the cloud can be mirror symmetric
    n_r = max(5, int(round(40 * scale)))
    return n_c, n_r


def naca0012_cloud(n_c: int = 128, n_r: int = 40, seed: int = 12345, jitter: float = 0.1,
                   shuffle: bool = False, symmetric: bool = False,
                   radius_factor: float = 1.6) -> Cloud:
    """Build the O-type NACA 0012 cloud with ``n_c * n_r`` points.

    ``symmetric=True`` mirrors the jitter of the lower half onto the upper half
    (about y = 0), so the cloud, its stencils and its normals are exactly
    mirror symmetric; used by the alpha = 0 symmetry test.
    """
    if n_c < 8 or n_r < 5:
        raise ValueError("need n_c >= 8 and n_r >= 5")
    if symmetric and n_c % 2:
        raise ValueError("a symmetric cloud needs an even n_c")
    rng = np.random.Generator(np.random.PCG64(seed))
    kk, ll = np.meshgrid(np.arange(n_c), np.arange(n_r), indexing="xy")  # [l, k]
    dk = rng.uniform(-jitter, jitter, size=(n_r, n_c))
    dl = rng.uniform(-jitter, jitter, size=(n_r, n_c))
    dk[0, :] = dk[-1, :] = 0.0
    dl[0, :] = dl[-1, :] = 0.0
    if symmetric:
        # point k mirrors point (n_c - k) mod n_c; points 0 and n_c/2 lie on the axis
        mirror = (n_c - np.arange(n_c)) % n_c
        upper = np.arange(1, n_c // 2)
        dk[:, mirror[upper]] = -dk[:, upper]
        dl[:, mirror[upper]] = dl[:, upper]
        dk[:, 0] = 0.0
        dk[:, n_c // 2] = 0.0
    x, y = _points(kk + dk, ll + dl, n_c, n_r)
    if symmetric:
        # make the mirror exact in floating point
        mirror = (n_c - np.arange(n_c)) % n_c
        upper = np.arange(1, n_c // 2)
        x[:, mirror[upper]] = x[:, upper]
        y[:, mirror[upper]] = -y[:, upper]
        y[:, 0] = 0.0
        y[:, n_c // 2] = 0.0
    x = x.reshape(-1)
    y = y.reshape(-1)
    n = n_c * n_r

    # local spacing of the unjittered grid
    gx, gy = _points(kk.astype(np.float64), ll.astype(np.float64), n_c, n_r)
    hc = 0.5 * np.hypot(np.roll(gx, -1, axis=1) - np.roll(gx, 1, axis=1),
                        np.roll(gy, -1, axis=1) - np.roll(gy, 1, axis=1))
    lp = np.minimum(np.arange(n_r) + 1, n_r - 1)
    lm = np.maximum(np.arange(n_r) - 1, 0)
    hr = np.hypot(gx[lp, :] - gx[lm, :], gy[lp, :] - gy[lm, :]) / (lp - lm)[:, None]
    eps = (radius_factor * np.maximum(hc, hr)).reshape(-1)
    if symmetric:
        e2 = eps.reshape(n_r, n_c)
        mirror = (n_c - np.arange(n_c)) % n_c
        upper = np.arange(1, n_c // 2)
        e2[:, mirror[upper]] = e2[:, upper]

    flags = np.zeros(n, dtype=np.int8)
    flags[:n_c] = FLAG_WALL
    flags[n - n_c:] = FLAG_OUTER

    normals = np.zeros((n, 2), dtype=np.float64)
    normals[:, 1] = 1.0
    # wall: right-hand normal of the counter-clockwise loop (points into the fluid)
    wxl, wyl = x[:n_c], y[:n_c]
    tx = np.roll(wxl, -1) - np.roll(wxl, 1)
    ty = np.roll(wyl, -1) - np.roll(wyl, 1)
    tn = np.hypot(tx, ty)
    normals[:n_c, 0] = ty / tn
    normals[:n_c, 1] = -tx / tn
    if symmetric:
        mirror = (n_c - np.arange(n_c)) % n_c
        upper = np.arange(1, n_c // 2)
        normals[mirror[upper], 0] = normals[upper, 0]
        normals[mirror[upper], 1] = -normals[upper, 1]
        normals[0, :] = (1.0, 0.0)
        normals[n_c // 2, :] = (-1.0, 0.0)
    theta = 2.0 * np.pi * np.arange(n_c) / n_c
    normals[n - n_c:, 0] = np.cos(theta)
    normals[n - n_c:, 1] = np.sin(theta)
    if symmetric:
        normals[n - n_c:, 0][mirror[upper]] = normals[n - n_c:, 0][upper]
        normals[n - n_c:, 1][mirror[upper]] = -normals[n - n_c:, 1][upper]
        normals[n - n_c, :] = (1.0, 0.0)
        normals[n - n_c + n_c // 2, :] = (-1.0, 0.0)

    offsets, idx = _stencils(x, y, eps, n_c, n_r)

    xy = np.stack([x, y], axis=1)
    k_of = np.tile(np.arange(n_c), n_r)
    l_of = np.repeat(np.arange(n_r), n_c)
    cloud = Cloud(xy=xy, normals=normals, flags=flags, nbr_offsets=offsets, nbr_idx=idx,
                  n_c=n_c, n_r=n_r, k=k_of, l=l_of)
    if shuffle:
        cloud = _shuffle(cloud, seed)
    return cloud


def _stencils(x, y, eps, n_c, n_r, chunk_rows=256):
    """CSR neighbour lists from the +-2 index window, nearest first, <= 20."""
    n = n_c * n_r
    window = [(dk, dl) for dl in range(-2, 3) for dk in range(-2, 3) if (dk, dl) != (0, 0)]
    counts = np.zeros(n, dtype=np.int64)
    lists = []
    for r0 in range(0, n_r, chunk_rows):
        r1 = min(n_r, r0 + chunk_rows)
        kk, ll = np.meshgrid(np.arange(n_c), np.arange(r0, r1), indexing="xy")
        kk = kk.reshape(-1)
        ll = ll.reshape(-1)
        me = ll * n_c + kk
        cand = np.empty((me.size, len(window)), dtype=np.int64)
        valid = np.empty((me.size, len(window)), dtype=bool)
        for c, (dk, dl) in enumerate(window):
            lj = ll + dl
            kj = (kk + dk) % n_c
            ok = (lj >= 0) & (lj < n_r)
            cand[:, c] = np.where(ok, lj * n_c + kj, 0)
            valid[:, c] = ok
        dx = x[cand] - x[me][:, None]
        dy = y[cand] - y[me][:, None]
        d2 = dx * dx + dy * dy
        e = eps[me][:, None]
        valid &= d2 < e * e
        d2 = np.where(valid, d2, np.inf)
        # sort by (distance, index) per row
        key_idx = np.argsort(cand, axis=1, kind="stable")
        d2_s = np.take_along_axis(d2, key_idx, axis=1)
        cand_s = np.take_along_axis(cand, key_idx, axis=1)
        valid_s = np.take_along_axis(valid, key_idx, axis=1)
        o2 = np.argsort(d2_s, axis=1, kind="stable")
        d2_s = np.take_along_axis(d2_s, o2, axis=1)
        cand_s = np.take_along_axis(cand_s, o2, axis=1)
        valid_s = np.take_along_axis(valid_s, o2, axis=1)
        nvalid = valid_s.sum(axis=1)
        keep = np.minimum(nvalid, MAX_NEIGHBOURS)
        # never split a tied group at the cap
        over = nvalid > MAX_NEIGHBOURS
        if np.any(over):
            rows = np.nonzero(over)[0]
            for r in rows:
                kc = MAX_NEIGHBOURS
                while kc > 0 and d2_s[r, kc - 1] == d2_s[r, kc]:
                    kc -= 1
                keep[r] = kc
        mask = np.arange(len(window))[None, :] < keep[:, None]
        counts[me] = keep
        lists.append((me, cand_s, mask))
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    idx = np.empty(int(offsets[-1]), dtype=np.int32)
    for me, cand_s, mask in lists:
        rows, cols = np.nonzero(mask)
        # rows are sorted, cols ascending within a row
        pos = offsets[me[rows]] + (cols)
        idx[pos] = cand_s[rows, cols]
    if offsets[-1] > np.iinfo(np.int32).max:
        raise ValueError("too many neighbour entries for int32 offsets")
    return offsets.astype(np.int32), idx


def _shuffle(cloud: Cloud, seed: int) -> Cloud:
    """Seeded permutation of all non-wall points (wall loop stays first, in order)."""
    n, n_c = cloud.n, cloud.n_c
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    perm = np.arange(n)  # new position -> old id
    perm[n_c:] = n_c + rng.permutation(n - n_c)
    inv = np.empty(n, dtype=np.int64)  # old id -> new position
    inv[perm] = np.arange(n)
    counts = np.diff(cloud.nbr_offsets.astype(np.int64))[perm]
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    starts = cloud.nbr_offsets[:-1].astype(np.int64)[perm]
    # gather old lists in new order
    rep = np.repeat(starts - offsets[:-1], counts)
    src = np.arange(offsets[-1]) + rep
    idx = inv[cloud.nbr_idx[src]].astype(np.int32)
    return Cloud(xy=cloud.xy[perm].copy(), normals=cloud.normals[perm].copy(),
                 flags=cloud.flags[perm].copy(), nbr_offsets=offsets.astype(np.int32),
                 nbr_idx=idx, n_c=cloud.n_c, n_r=cloud.n_r, k=cloud.k[perm].copy(),
                 l=cloud.l[perm].copy())


def pack(clouds) -> tuple[Cloud, np.ndarray]:
    """Concatenate clouds into one (disconnected) cloud for a ragged batch.

    Returns the packed cloud and the point offset of every member (length
    len(clouds) + 1). Each member's wall loop stays contiguous and first in
    its block, so the loops stay separate; neighbour lists keep their order.
    """
    clouds = list(clouds)
    offs = np.zeros(len(clouds) + 1, dtype=np.int64)
    for i, c in enumerate(clouds):
        offs[i + 1] = offs[i] + c.n
    nnz = [int(c.nbr_offsets[-1]) for c in clouds]
    if sum(nnz) > np.iinfo(np.int32).max or offs[-1] > np.iinfo(np.int32).max:
        raise ValueError("packed cloud too large for int32 connectivity")
    nbr_off = [np.zeros(1, dtype=np.int64)]
    base = 0
    for c in clouds:
        nbr_off.append(c.nbr_offsets[1:].astype(np.int64) + base)
        base += int(c.nbr_offsets[-1])
    idx = np.concatenate([c.nbr_idx.astype(np.int64) + o for c, o in zip(clouds, offs[:-1])])
    packed = Cloud(xy=np.concatenate([c.xy for c in clouds]),
                   normals=np.concatenate([c.normals for c in clouds]),
                   flags=np.concatenate([c.flags for c in clouds]),
                   nbr_offsets=np.concatenate(nbr_off).astype(np.int32),
                   nbr_idx=idx.astype(np.int32), n_c=clouds[0].n_c, n_r=clouds[0].n_r,
                   k=np.concatenate([c.k for c in clouds]), l=np.concatenate([c.l for c in clouds]))
    return packed, offs


def ragged_sizes(n_clouds: int = 16, lo: int = 100_000, hi: int = 1_000_000, seed: int = 2021):
    """Seeded cloud sizes ~ U[lo, hi] for a ragged batch."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    return [int(v) for v in rng.uniform(lo, hi, n_clouds)]


def cloud_for_points(n_points: int, seed: int = 12345, shuffle: bool = True) -> Cloud:
    """The cloud whose size is closest to ``n_points`` (same continuous distribution)."""
    n_c, n_r = cloud_dims(n_points)
    return naca0012_cloud(n_c, n_r, seed=seed, shuffle=shuffle)


def conditions(n_cond: int, seed: int = 2021):
    """Seeded (Mach, alpha_deg) pairs: M ~ U[0.3, 0.8], alpha ~ U[-4, 6] deg."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.3, 0.8, n_cond), rng.uniform(-4.0, 6.0, n_cond)


def perturbed_state(cloud: Cloud, mach: float, alpha_deg: float, amplitude: float = 0.05,
                    seed: int = 7):
    """Smooth, seeded non-uniform primitive state (rho, u1, u2, p) per point.

    Free stream (rho = 1, p = 1/1.4, |u| = M) modulated by a few seeded
    low-frequency sine modes of the coordinates; used to test one residual
    evaluation away from the trivially uniform state.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y = cloud.xy[:, 0], cloud.xy[:, 1]
    a = np.deg2rad(alpha_deg)
    w = np.empty((cloud.n, 4), dtype=np.float64)
    base = [1.0, mach * math.cos(a), mach * math.sin(a), 1.0 / 1.4]
    for c in range(4):
        kx, ky = rng.uniform(0.5, 3.0, 2)
        ph = rng.uniform(0, 2 * np.pi, 2)
        amp = amplitude * (1.0 if c in (0, 3) else max(mach, 0.1))
        w[:, c] = base[c] + amp * np.sin(kx * x + ph[0]) * np.cos(ky * y + ph[1])
    return w
