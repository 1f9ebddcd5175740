"""Seeded synthetic initial states for the KFVM-WENO workloads.

This module is the ONE place both the CUDA path's tests/bench and the oracle
take their inputs from.  It holds none of the method's arithmetic: it only
draws random numbers (SplitMix64), evaluates the initial-condition functions
and averages them over each cell with a tensor Gauss-Legendre rule of R points
per dimension (the paper's initial-condition stage, Sec. 5.2, which precedes
the hot path).

Workloads (state arrays are float64 [nv, ny, nx] or [nv, nz, ny, nx], the
conserved variables rho, rho*u, rho*v[, rho*w], E, gamma = 1.4):

* ``sine_2d(n)``        rho = 1 + 0.2 sin(2 pi (x + y)), u = v = 1, p = 1 on
                         [0,1]^2, periodic.  The exact solution is a
                         translation with velocity (1, 1).
* ``voronoi_2d(n, k, seed)``  piecewise-constant over k Voronoi regions whose
                         sites are uniform in [0,1]^2; per region, drawn in site
                         order, rho, p ~ U[0.1, 1] and u, v ~ U[-1, 1]; outflow.
* ``half_sine_voronoi_3d(n, k, seed)``  x < 1/2: rho = 1 + 0.2 sin(2 pi (x+y+z)),
                         u = v = w = 1, p = 1; x >= 1/2: k Voronoi regions with
                         sites uniform in [1/2,1] x [0,1]^2 and the constants above.
* ``isentropic_vortex(n, R, t)``  the isentropic vortex of Sec. 6.1 on the
                         periodic square [-10, 10]^2, advected by (1, 1): an
                         exact smooth solution of the Euler equations.
* ``mixed_voronoi(dim, n, k, seed)``  k regions over the whole box; per region a
                         coin (probability 1/2) picks the smooth sine state, else a
                         random constant state as above.

Voronoi regions: nearest site in Euclidean distance, ties to the lowest index.
Cells whose 3^d neighbouring cell centres all lie in one region lie wholly in
it (Voronoi regions are convex and the cell lies in the hull of those
centres), so only the remaining cells are evaluated at their Gauss points.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GAMMA = 1.4
MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """(x >> 11) * 2^-53 mapped to [lo, hi)."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


def _gl(R: int):
    """Gauss-Legendre nodes on [-1/2, 1/2] and weights summing to one."""
    x, w = np.polynomial.legendre.leggauss(R)
    return 0.5 * x, 0.5 * w


def _prim_to_cons(rho, vel, p, gamma=GAMMA):
    ke = 0.5 * rho * sum(v * v for v in vel)
    return [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke]


def _sine_prim(coords, dim):
    """Smooth advected state: rho = 1 + 0.2 sin(2 pi sum x), velocity 1, p = 1."""
    s = coords[0]
    for c in coords[1:dim]:
        s = s + c
    rho = 1.0 + 0.2 * torch.sin(2.0 * math.pi * s)
    one = torch.ones_like(rho)
    return rho, [one] * dim, one


def _cell_average(fn_prim, dim, n, lo, dx, R, device, zslab=None):
    """Tensor-GL cell averages of the conserved variables of fn_prim(coords) -> (rho, vel, p)."""
    xg, wg = _gl(R)
    nv = dim + 2
    shape = tuple(reversed(n[:dim]))
    out = torch.zeros((nv,) + shape, dtype=torch.float64, device=device)
    axes = [lo[a] + (torch.arange(n[a], dtype=torch.float64, device=device) + 0.5) * dx[a] for a in range(dim)]
    for idx in np.ndindex(*([R] * dim)):
        w = float(np.prod([wg[i] for i in idx]))
        pts = [axes[a] + xg[idx[a]] * dx[a] for a in range(dim)]
        if dim == 2:
            Y, X = torch.meshgrid(pts[1], pts[0], indexing="ij")
            coords = [X, Y]
        else:
            Z, Y, X = torch.meshgrid(pts[2], pts[1], pts[0], indexing="ij")
            coords = [X, Y, Z]
        rho, vel, p = fn_prim(coords)
        U = _prim_to_cons(rho, vel, p)
        for v in range(nv):
            out[v] += w * U[v]
    return out


def sine_2d(n: int, R: int = 2, device="cpu") -> torch.Tensor:
    """C1 family: smooth translation on the periodic unit square (exact solution known)."""
    return _cell_average(lambda c: _sine_prim(c, 2), 2, [n, n], [0.0, 0.0], [1.0 / n, 1.0 / n], R, device)


def sine_2d_exact_density(n: int, t: float) -> np.ndarray:
    """Exact cell averages of rho at time t for ``sine_2d``: the sine is translated by (t, t),
    and its cell average is the point value times (sin(pi h)/(pi h))^2."""
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    damp = (math.sin(math.pi * h) / (math.pi * h)) ** 2
    return 1.0 + 0.2 * np.sin(2 * math.pi * (X + Y - 2 * t)) * damp


def sine_3d(n: int, R: int = 3, device="cpu") -> torch.Tensor:
    """The C3 smooth state on the periodic unit cube: rho = 1 + 0.2 sin(2 pi (x + y + z)), velocity 1, p = 1."""
    h = 1.0 / n
    return _cell_average(lambda c: _sine_prim(c, 3), 3, [n, n, n], [0.0] * 3, [h] * 3, R, device)


def sine_3d_exact_density(n: int, t: float) -> np.ndarray:
    """Exact cell averages of rho at time t for ``sine_3d`` ([z][y][x]): translation by (t, t, t),
    cell average = point value times (sin(pi h)/(pi h))^3."""
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    damp = (math.sin(math.pi * h) / (math.pi * h)) ** 3
    return 1.0 + 0.2 * np.sin(2 * math.pi * (X + Y + Z - 3 * t)) * damp


def _vortex_prim(coords, t, gamma=GAMMA):
    """Isentropic vortex of radius 1 on [-10, 10]^2 (Sec. 6.1), advected by (1, 1) for a time t:
    omega = 5 sqrt(2e)/(4 pi) exp(-r^2/2) about the centre (t, t) (periodic images are below 1e-21),
    rho = (1 + (1-gamma)/2 omega^2)^(1/(gamma-1)), u = 1 - y omega, v = 1 + x omega,
    p = (1/gamma) (1 + (1-gamma)/2 omega^2)^(gamma/(gamma-1))."""
    x = torch.remainder(coords[0] - t + 10.0, 20.0) - 10.0
    y = torch.remainder(coords[1] - t + 10.0, 20.0) - 10.0
    om = 5.0 * math.sqrt(2.0 * math.e) / (4.0 * math.pi) * torch.exp(-0.5 * (x * x + y * y))
    base = 1.0 + 0.5 * (1.0 - gamma) * om * om
    rho = base ** (1.0 / (gamma - 1.0))
    p = base ** (gamma / (gamma - 1.0)) / gamma
    return rho, [1.0 - y * om, 1.0 + x * om], p


def isentropic_vortex(n: int, R: int = 2, t: float = 0.0, device="cpu") -> torch.Tensor:
    """The isentropic vortex (Sec. 6.1) on the periodic square [-10, 10]^2 with n x n cells; at
    t > 0 the exact solution (the initial state translated by (t, t)); t = 20 is the initial state."""
    h = 20.0 / n
    return _cell_average(lambda c: _vortex_prim(c, t), 2, [n, n], [-10.0, -10.0], [h, h], R, device)


def _draw_regions(rng: SplitMix64, k: int, dim: int, site_lo, site_hi, with_coin: bool):
    sites = np.array([[rng.uniform(site_lo[a], site_hi[a]) for a in range(dim)] for _ in range(k)])
    states = []
    for _ in range(k):
        smooth = (rng.uniform() < 0.5) if with_coin else False
        rho = rng.uniform(0.1, 1.0)
        p = rng.uniform(0.1, 1.0)
        vel = [rng.uniform(-1.0, 1.0) for _ in range(dim)]
        states.append((smooth, rho, vel, p))
    return sites, states


def _nearest_site_exact(pts, sites_t):
    """float64 Euclidean distances to every site, first minimum (ties: lowest index)."""
    d2 = torch.cdist(pts, sites_t, compute_mode="donot_use_mm_for_euclid_dist")
    return torch.argmin(d2, dim=1)


def _nearest_site(coords, sites_t):
    """Index of the nearest site for each point (ties: lowest index), chunked.

    A float32 screen (|x|^2 + |s|^2 - 2 x.s, error below 1e-6 on the unit box) picks the nearest
    site where the second nearest is more than 1e-5 farther in squared distance; every other point
    (near a bisector, or a tie) is decided by the exact float64 comparison, so the result is that
    of the float64 search everywhere."""
    flat = torch.stack([c.reshape(-1) for c in coords], dim=1)
    out = torch.empty(flat.shape[0], dtype=torch.long, device=flat.device)
    k = sites_t.shape[0]
    if k < 2:
        out.zero_()
        return out.reshape(coords[0].shape)
    s32 = sites_t.to(torch.float32)
    s2 = (s32 * s32).sum(dim=1)
    chunk = max(1, (1 << 25) // k)
    for s in range(0, flat.shape[0], chunk):
        p = flat[s:s + chunk]
        p32 = p.to(torch.float32)
        d2 = (p32 * p32).sum(dim=1, keepdim=True) + s2[None, :] - 2.0 * (p32 @ s32.T)
        top = torch.topk(d2, 2, dim=1, largest=False)
        idx = top.indices[:, 0].clone()
        unsure = (top.values[:, 1] - top.values[:, 0]) <= 1e-5
        if bool(unsure.any()):
            sel = torch.nonzero(unsure).squeeze(1)
            idx[sel] = _nearest_site_exact(p[sel], sites_t)
        out[s:s + chunk] = idx
    return out.reshape(coords[0].shape)


def _voronoi_state(dim, n, lo, hi, sites, states, R, device, smooth_mask_fn=None, crop=None):
    """Cell averages of the piecewise state.

    A cell whose 3^d neighbouring centres share one region (and one side of the
    x = 1/2 plane, when a mask is given) lies wholly in that region, so it takes
    the region's constant, or the Gauss-Legendre average of the sine state.
    Only the remaining cells are averaged point by point with a region lookup.
    ``crop`` (cells per axis) generates only the corner block [0, crop)^d of the
    n^d grid: the same values as the corner of the full state.
    """
    nv = dim + 2
    dx = [(hi[a] - lo[a]) / n[a] for a in range(dim)]
    if crop is not None:
        n = [min(int(crop), n[a]) for a in range(dim)]
    sites_t = torch.tensor(sites, dtype=torch.float64, device=device)
    table = torch.zeros((len(states), nv), dtype=torch.float64, device=device)
    smooth = torch.zeros(len(states), dtype=torch.bool, device=device)
    for r, (sm, rho, vel, p) in enumerate(states):
        table[r] = torch.tensor(_prim_to_cons(rho, vel, p), dtype=torch.float64)
        smooth[r] = bool(sm)

    ext = [lo[a] + (torch.arange(-1, n[a] + 1, dtype=torch.float64, device=device) + 0.5) * dx[a] for a in range(dim)]
    grids = torch.meshgrid(*reversed(ext), indexing="ij")
    ecoords = list(reversed(grids))
    creg = _nearest_site(ecoords, sites_t)
    csm = smooth[creg]
    if smooth_mask_fn is not None:
        csm = csm | smooth_mask_fn(ecoords)
    inner = tuple(slice(1, -1) for _ in range(dim))
    c0 = creg[inner]
    s0 = csm[inner]
    uniform = torch.ones_like(c0, dtype=torch.bool)
    for off in np.ndindex(*([3] * dim)):
        sl = tuple(slice(o, o + c0.shape[i]) for i, o in enumerate(off))
        uniform &= (creg[sl] == c0) & (csm[sl] == s0)
    del creg, csm, ecoords, grids

    out = table[c0].permute(*([dim] + list(range(dim)))).contiguous()
    smooth_cells = uniform & s0
    if bool(smooth_cells.any()):
        sine = _cell_average(lambda c: _sine_prim(c, dim), dim, n, lo, dx, R, device)
        out = torch.where(smooth_cells.unsqueeze(0), sine, out)
        del sine
    todo = torch.nonzero(~uniform.reshape(-1)).squeeze(1)
    if todo.numel():
        # coordinates of the cell centres that need a point-by-point average
        idx = todo
        cidx = []
        for a in range(dim):
            cidx.append(idx % n[a])
            idx = idx // n[a]
        centres = [lo[a] + (cidx[a].to(torch.float64) + 0.5) * dx[a] for a in range(dim)]
        xg, wg = _gl(R)
        acc = torch.zeros((nv, todo.numel()), dtype=torch.float64, device=device)
        for gi in np.ndindex(*([R] * dim)):
            w = float(np.prod([wg[i] for i in gi]))
            coords = [centres[a] + xg[gi[a]] * dx[a] for a in range(dim)]
            reg = _nearest_site(coords, sites_t)
            U = [table[reg, v] for v in range(nv)]
            use_sine = smooth[reg]
            if smooth_mask_fn is not None:
                use_sine = use_sine | smooth_mask_fn(coords)
            rho, vel, p = _sine_prim(coords, dim)
            Us = _prim_to_cons(rho, vel, p)
            for v in range(nv):
                acc[v] += w * torch.where(use_sine, Us[v], U[v])
        flat = out.reshape(nv, -1)
        flat[:, todo] = acc
    return out


def voronoi_2d(n: int, k: int = 64, seed: int = 2, R: int = 2, device="cpu", crop=None) -> torch.Tensor:
    """C2 family: k constant Voronoi regions on [0,1]^2 (outflow boundaries)."""
    rng = SplitMix64(seed)
    sites, states = _draw_regions(rng, k, 2, [0.0, 0.0], [1.0, 1.0], with_coin=False)
    return _voronoi_state(2, [n, n], [0.0, 0.0], [1.0, 1.0], sites, states, R, device, crop=crop)


def half_sine_voronoi_3d(n: int, k: int = 128, seed: int = 3, R: int = 2, device="cpu", crop=None) -> torch.Tensor:
    """C3 family: smooth sine for x < 1/2, k constant Voronoi regions in x >= 1/2."""
    rng = SplitMix64(seed)
    sites, states = _draw_regions(rng, k, 3, [0.5, 0.0, 0.0], [1.0, 1.0, 1.0], with_coin=False)
    return _voronoi_state(3, [n, n, n], [0.0] * 3, [1.0] * 3, sites, states, R, device,
                          smooth_mask_fn=lambda c: c[0] < 0.5, crop=crop)


def mixed_voronoi(dim: int, n: int, k: int, seed: int, R: int = 2, device="cpu", crop=None) -> torch.Tensor:
    """C4/C5 family: k regions, each the smooth sine state (coin 1/2) or a random constant."""
    rng = SplitMix64(seed)
    sites, states = _draw_regions(rng, k, dim, [0.0] * dim, [1.0] * dim, with_coin=True)
    return _voronoi_state(dim, [n] * dim, [0.0] * dim, [1.0] * dim, sites, states, R, device, crop=crop)


def constant_state(dim: int, n, rho=1.0, vel=None, p=1.0) -> torch.Tensor:
    """A uniform state (free-stream tests)."""
    vel = vel if vel is not None else [0.3] * dim
    U = _prim_to_cons(rho, vel, p)
    shape = tuple(reversed(list(n)[:dim]))
    return torch.stack([torch.full(shape, float(u), dtype=torch.float64) for u in U])
