"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input recipes only: it draws random numbers and lays the
drawn problems out in memory.  It contains none of the integration method's
arithmetic, so the CPU oracle and the CUDA path can both be fed from it
without sharing any numerical code.

Random numbers come from SplitMix64 used as a counter-based generator: the
``k``-th draw of stream ``key`` is ``mix64(key + (k + 1) * 0x9E3779B97F4A7C15)``
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014).  Every cell (or grid point) owns one stream, keyed from the
global seed and its index, so any draw of any cell can be produced directly
and the recipe is independent of vectorisation or chunking.

Workloads (the problem statements follow the paper's two use cases, Sec. 2:
many small independent systems, one per grid cell, and one large coupled
system; the Brusselator reaction terms are the demonstration problem of
Sec. 7):

* ``robertson``  - Robertson kinetics, 3 species per cell, rate constants
  scaled per cell by independent log-uniform factors in [0.5, 2].
* ``mass_action`` - random mass-action networks: ``2 n`` reactions per cell,
  each with m in {2, 3, 4} distinct reactant species and m distinct product
  species (all stoichiometric coefficients 1, so the total concentration is
  conserved), rate constants log-uniform in [1e-2, 1e8], initial
  concentrations Dirichlet(1, ..., 1).
* ``mass_action_shared`` - one random network shared by all cells, initial
  states drawn per cell.
* ``brusselator3d`` - u, v, w on a periodic n^3 grid, initial state the
  reaction steady state times (1 + 0.01 U[-1, 1]).
* ``brusselator1d`` - the demonstration problem itself: u, v, w advected on a
  periodic line, the paper's Gaussian-bump initial state (no random draws).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 20111298

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CELLMUL = np.uint64(0xD1B54A32D192ED03)
_NONE = 255  # empty slot in a reactant / product list


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_keys(seed: int, index: np.ndarray) -> np.ndarray:
    """One stream key per cell / grid point: mix64(seed XOR (index+1)*C)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ ((idx + np.uint64(1)) * _CELLMUL))


def uniform(keys: np.ndarray, draw: np.ndarray | int) -> np.ndarray:
    """Draw number ``draw`` (0-based) of each stream, as a double in [0, 1).

    ``keys`` and ``draw`` broadcast against each other.
    """
    d = np.asarray(draw, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = keys + (d + np.uint64(1)) * _GOLDEN
    return (_mix64(s) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_vectors(length: int, count: int = 1, seed: int = DEFAULT_SEED,
                    lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """``count`` vectors of ``length`` doubles, U[lo, hi) (the isolated
    vector-operation study of Sec. 4.2 uses random doubles)."""
    out = np.empty((count, length), dtype=np.float64)
    chunk = 1 << 22
    for p0 in range(0, length, chunk):
        keys = stream_keys(seed, np.arange(p0, min(length, p0 + chunk), dtype=np.uint64))
        for j in range(count):
            out[j, p0:p0 + len(keys)] = lo + (hi - lo) * uniform(keys, j)
    return out


# --------------------------------------------------------------------------
# Robertson kinetics
# --------------------------------------------------------------------------
ROBERTSON_K = (0.04, 3.0e7, 1.0e4)


@dataclass
class RobertsonProblem:
    """``k[c] = (k1, k2, k3)`` for cell c; y' as in Robertson (1966):
    y1' = -k1 y1 + k3 y2 y3, y2' = k1 y1 - k3 y2 y3 - k2 y2^2, y3' = k2 y2^2."""
    k: np.ndarray          # [ncell, 3] float64
    y0: np.ndarray         # [ncell * 3] float64 (cell-contiguous)
    kind: str = "robertson"

    @property
    def ncell(self) -> int:
        return self.k.shape[0]

    @property
    def n(self) -> np.ndarray:
        return np.full(self.ncell, 3, dtype=np.int32)

    @property
    def y_off(self) -> np.ndarray:
        return (np.arange(self.ncell + 1, dtype=np.int64) * 3)

    def subset(self, cells) -> "RobertsonProblem":
        cells = np.asarray(cells, dtype=np.int64)
        return RobertsonProblem(k=self.k[cells].copy(),
                                y0=self.y0.reshape(-1, 3)[cells].reshape(-1).copy())


def robertson(ncell: int, seed: int = DEFAULT_SEED, lo: float = 0.5,
              hi: float = 2.0) -> RobertsonProblem:
    keys = stream_keys(seed, np.arange(ncell, dtype=np.uint64))
    u = uniform(keys[:, None], np.arange(3)[None, :])
    fac = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    k = np.asarray(ROBERTSON_K)[None, :] * fac
    y0 = np.tile(np.array([1.0, 0.0, 0.0]), ncell)
    return RobertsonProblem(k=np.ascontiguousarray(k), y0=y0)


# --------------------------------------------------------------------------
# Random mass-action networks
# --------------------------------------------------------------------------
MAXM = 4            # at most 4 reactants and 4 products per reaction
DRAWS_PER_RXN = 10  # u_m, 4 reactant picks, 4 product picks, u_k


@dataclass
class MassActionProblem:
    """Packed description of ``ncell`` independent mass-action networks.

    Cell c has ``n[c]`` species stored at ``y0[y_off[c]:y_off[c+1]]`` and
    reactions ``rxn_off[c]:rxn_off[c+1]``.  Reaction r consumes the species
    listed in ``reactants[r]`` and produces those in ``products[r]`` (local
    species indices, 255 = empty slot) at rate ``k[r] * prod(y[reactants])``.
    """
    n: np.ndarray          # [ncell] int32
    y_off: np.ndarray      # [ncell+1] int64
    rxn_off: np.ndarray    # [ncell+1] int64
    reactants: np.ndarray  # [nrxn, 4] uint8
    products: np.ndarray   # [nrxn, 4] uint8
    k: np.ndarray          # [nrxn] float64
    y0: np.ndarray         # [sum n] float64
    kind: str = "massaction"
    shared: bool = False   # every cell carries the network of cell 0

    @property
    def ncell(self) -> int:
        return int(self.n.shape[0])

    def subset(self, cells) -> "MassActionProblem":
        """The listed cells as a problem of their own (same data, repacked)."""
        cells = np.asarray(cells, dtype=np.int64)
        n = self.n[cells]
        y_off = np.zeros(len(cells) + 1, np.int64)
        y_off[1:] = np.cumsum(n)
        nr = (self.rxn_off[cells + 1] - self.rxn_off[cells])
        rxn_off = np.zeros(len(cells) + 1, np.int64)
        rxn_off[1:] = np.cumsum(nr)
        yi = np.concatenate([np.arange(self.y_off[c], self.y_off[c + 1]) for c in cells]) \
            if len(cells) else np.zeros(0, np.int64)
        ri = np.concatenate([np.arange(self.rxn_off[c], self.rxn_off[c + 1]) for c in cells]) \
            if len(cells) else np.zeros(0, np.int64)
        return MassActionProblem(n=n.copy(), y_off=y_off, rxn_off=rxn_off,
                                 reactants=self.reactants[ri].copy(),
                                 products=self.products[ri].copy(),
                                 k=self.k[ri].copy(), y0=self.y0[yi].copy(), shared=self.shared)


def _pick_distinct(u: np.ndarray, n: int) -> np.ndarray:
    """Partial Fisher-Yates: MAXM distinct indices in [0, n) from MAXM draws.

    ``u`` has shape [..., MAXM]; returns int16 [..., MAXM] (the first m of
    them are used for a reaction with m species)."""
    shape = u.shape[:-1]
    perm = np.broadcast_to(np.arange(n, dtype=np.int16), shape + (n,)).copy()
    flat = perm.reshape(-1, n)
    uf = u.reshape(-1, MAXM)
    rows = np.arange(flat.shape[0])
    for j in range(min(MAXM, n)):
        pick = j + np.minimum((uf[:, j] * (n - j)).astype(np.int64), n - j - 1)
        a = flat[rows, j].copy()
        flat[rows, j] = flat[rows, pick]
        flat[rows, pick] = a
    out = np.full(shape + (MAXM,), -1, dtype=np.int16)
    out.reshape(-1, MAXM)[:, :min(MAXM, n)] = flat[:, :min(MAXM, n)]
    return out


def mass_action(ncell: int, sizes=(3, 10, 32, 54), seed: int = DEFAULT_SEED,
                rxn_per_species: int = 2, mvals=(2, 3, 4),
                log10k=(-2.0, 8.0), chunk: int = 2048) -> MassActionProblem:
    """Random mass-action cells; sizes drawn uniformly from ``sizes``.

    Draw layout of cell c's stream: draw 0 picks the size; reaction r uses
    draws 1 + 10 r ... 10 + 10 r (m, reactant picks, product picks, rate);
    species i of the initial state uses draw 1 + 10 R + i.
    """
    sizes = np.asarray(sizes, dtype=np.int32)
    keys = stream_keys(seed, np.arange(ncell, dtype=np.uint64))
    u0 = uniform(keys, 0)
    n = sizes[np.minimum((u0 * len(sizes)).astype(np.int64), len(sizes) - 1)]
    R = rxn_per_species * n.astype(np.int64)
    y_off = np.zeros(ncell + 1, np.int64)
    y_off[1:] = np.cumsum(n)
    rxn_off = np.zeros(ncell + 1, np.int64)
    rxn_off[1:] = np.cumsum(R)
    nr = int(rxn_off[-1])
    reactants = np.full((nr, MAXM), _NONE, np.uint8)
    products = np.full((nr, MAXM), _NONE, np.uint8)
    k = np.empty(nr, np.float64)
    y0 = np.empty(int(y_off[-1]), np.float64)

    for ns in np.unique(n):
        ns = int(ns)
        cells_all = np.nonzero(n == ns)[0]
        Rn = rxn_per_species * ns
        mv = np.asarray([m for m in mvals if m <= ns], dtype=np.int64)
        for c0 in range(0, len(cells_all), chunk):
            cells = cells_all[c0:c0 + chunk]
            kc = keys[cells][:, None, None]
            d = 1 + DRAWS_PER_RXN * np.arange(Rn)[None, :, None] + np.arange(DRAWS_PER_RXN)[None, None, :]
            u = uniform(kc, d)                      # [C, Rn, 10]
            m = mv[np.minimum((u[..., 0] * len(mv)).astype(np.int64), len(mv) - 1)]  # [C, Rn]
            ra = _pick_distinct(u[..., 1:5], ns)
            pa = _pick_distinct(u[..., 5:9], ns)
            slot = np.arange(MAXM)[None, None, :]
            keep = slot < m[..., None]
            ra = np.where(keep, ra, _NONE).astype(np.uint8)
            pa = np.where(keep, pa, _NONE).astype(np.uint8)
            lk = log10k[0] + u[..., 9] * (log10k[1] - log10k[0])
            rows = (rxn_off[cells][:, None] + np.arange(Rn)[None, :]).reshape(-1)
            reactants[rows] = ra.reshape(-1, MAXM)
            products[rows] = pa.reshape(-1, MAXM)
            k[rows] = np.power(10.0, lk).reshape(-1)
            uy = uniform(kc[:, :, 0], 1 + DRAWS_PER_RXN * Rn + np.arange(ns)[None, :])
            e = -np.log1p(-uy)                      # Exp(1) samples
            yrows = (y_off[cells][:, None] + np.arange(ns)[None, :]).reshape(-1)
            y0[yrows] = (e / e.sum(axis=1, keepdims=True)).reshape(-1)
    return MassActionProblem(n=n.astype(np.int32), y_off=y_off, rxn_off=rxn_off,
                             reactants=reactants, products=products, k=k, y0=y0)


def mass_action_shared(ncell: int, n: int = 10, seed: int = DEFAULT_SEED, network: int = 0,
                       **kw) -> MassActionProblem:
    """``ncell`` cells that all carry one random ``n``-species network (the
    network of cell ``network`` of ``mass_action(.., sizes=(n,), seed + 1)``)
    and differ in their initial states: cell c's Dirichlet(1, ..., 1) state
    uses draws 1 + 10 R + i of its stream under ``seed`` (the draws an
    unshared cell of this size would use for it)."""
    base = mass_action(network + 1, sizes=(n,), seed=seed + 1, **kw).subset([network])
    R = int(base.rxn_off[1])
    keys = stream_keys(seed, np.arange(ncell, dtype=np.uint64))
    y0 = np.empty((ncell, n), np.float64)
    for c0 in range(0, ncell, 65536):
        kc = keys[c0:c0 + 65536][:, None]
        e = -np.log1p(-uniform(kc, 1 + DRAWS_PER_RXN * R + np.arange(n)[None, :]))
        y0[c0:c0 + 65536] = e / e.sum(axis=1, keepdims=True)
    return MassActionProblem(n=np.full(ncell, n, np.int32),
                             y_off=np.arange(ncell + 1, dtype=np.int64) * n,
                             rxn_off=np.arange(ncell + 1, dtype=np.int64) * R,
                             reactants=np.tile(base.reactants, (ncell, 1)),
                             products=np.tile(base.products, (ncell, 1)),
                             k=np.tile(base.k, ncell), y0=y0.reshape(-1), shared=True)


def mass_action_banded(ncell: int, n: int = 128, window: int = 6, seed: int = DEFAULT_SEED,
                       rxn_per_species: int = 2, mvals=(2, 3),
                       log10k=(-2.0, 8.0)) -> MassActionProblem:
    """``ncell`` cells that share one sparse ``n``-species network (a larger
    mechanism whose reactions couple nearby species, as chains of reactions
    do) and differ in their initial states.

    Reaction r of the network (stream ``seed + 2``, key 0) uses draws
    1 + 11 r ... 11 + 11 r: m from ``mvals``, a window start b uniform in
    [0, n - window], m distinct reactants and m distinct products among
    species b .. b + window - 1 (partial Fisher-Yates), log10 k uniform in
    ``log10k``.  The Jacobian of every cell then has one banded pattern
    (|i - j| < window).  Cell c's Dirichlet(1, ..., 1) state uses draws
    1 .. n of its stream under ``seed``.  The problem is expanded per cell
    (the layout of the other generators); ``shared`` marks it."""
    if not (2 <= window <= n <= 255):
        raise ValueError("need 2 <= window <= n <= 255")
    R = rxn_per_species * n
    key = stream_keys(seed + 2, np.zeros(1, dtype=np.uint64))
    d = 1 + 11 * np.arange(R)[:, None] + np.arange(11)[None, :]
    u = uniform(key[:, None], d)                              # [R, 11]
    mv = np.asarray([m for m in mvals if m <= window], dtype=np.int64)
    m = mv[np.minimum((u[:, 0] * len(mv)).astype(np.int64), len(mv) - 1)]
    base = np.minimum((u[:, 1] * (n - window + 1)).astype(np.int64), n - window)
    ra = _pick_distinct(u[:, 2:6], window).astype(np.int64) + base[:, None]
    pa = _pick_distinct(u[:, 6:10], window).astype(np.int64) + base[:, None]
    keep = np.arange(MAXM)[None, :] < m[:, None]
    reac = np.where(keep, ra, _NONE).astype(np.uint8)
    prod = np.where(keep, pa, _NONE).astype(np.uint8)
    k = np.power(10.0, log10k[0] + u[:, 10] * (log10k[1] - log10k[0]))
    keys = stream_keys(seed, np.arange(ncell, dtype=np.uint64))
    y0 = np.empty((ncell, n), np.float64)
    for c0 in range(0, ncell, 65536):
        kc = keys[c0:c0 + 65536][:, None]
        e = -np.log1p(-uniform(kc, 1 + np.arange(n)[None, :]))
        y0[c0:c0 + 65536] = e / e.sum(axis=1, keepdims=True)
    return MassActionProblem(n=np.full(ncell, n, np.int32),
                             y_off=np.arange(ncell + 1, dtype=np.int64) * n,
                             rxn_off=np.arange(ncell + 1, dtype=np.int64) * R,
                             reactants=np.tile(reac, (ncell, 1)), products=np.tile(prod, (ncell, 1)),
                             k=np.tile(k, ncell), y0=y0.reshape(-1), shared=True)


# --------------------------------------------------------------------------
# Brusselator reaction-diffusion on a periodic 3-D grid
# --------------------------------------------------------------------------
@dataclass
class Brusselator3D:
    """u, v, w on an ``nx^3`` periodic grid over [0, 1)^3, stored species-major
    (``y0[s * nx^3 + (i * nx + j) * nx + k]``)."""
    nx: int
    A: float
    B: float
    eps: float
    D: float
    y0: np.ndarray = field(repr=False)
    kind: str = "brusselator3d"

    @property
    def npts(self) -> int:
        return self.nx ** 3

    @property
    def dx(self) -> float:
        return 1.0 / self.nx


def brusselator_steady_state(A: float, B: float, eps: float):
    """Reaction steady state of the Sec. 7 Brusselator terms:
    u* = A, w* = B / (1 + eps A), v* = w* / A."""
    w = B / (1.0 + eps * A)
    return A, w / A, w


def brusselator3d(nx: int, seed: int = DEFAULT_SEED, A: float = 1.0, B: float = 3.0,
                  eps: float = 5.0e-6, D: float = 1.0e-2, noise: float = 0.01,
                  chunk: int = 1 << 22) -> Brusselator3D:
    npts = nx ** 3
    ss = brusselator_steady_state(A, B, eps)
    y0 = np.empty(3 * npts, np.float64)
    for p0 in range(0, npts, chunk):
        p = np.arange(p0, min(npts, p0 + chunk), dtype=np.uint64)
        keys = stream_keys(seed, p)
        for s in range(3):
            y0[s * npts + p0: s * npts + p0 + len(p)] = ss[s] * (1.0 + noise * (2.0 * uniform(keys, s) - 1.0))
    return Brusselator3D(nx=nx, A=A, B=B, eps=eps, D=D, y0=y0)


@dataclass
class Brusselator1D:
    """The paper's demonstration problem (Sec. 7): u, v, w advected with speed
    ``c`` on a periodic line of ``nx`` points over [0, length), stored
    species-major (``y0[s * nx + i]``, point i at x = i length / nx)."""
    nx: int
    A: float
    B: float
    eps: float
    c: float
    length: float
    y0: np.ndarray = field(repr=False)
    kind: str = "brusselator1d"

    @property
    def npts(self) -> int:
        return self.nx


def brusselator1d(nx: int, length: float = 10.0, A: float = 1.0, B: float = 3.5, eps: float = 5.0e-6,
                  c: float = 0.01, alpha: float = 0.1) -> Brusselator1D:
    """The demo's initial state (Sec. 7): u = A + p, v = B / A + p, w = 3 + p
    with the Gaussian bump p(x) = alpha exp(-(x - mu)^2 / (2 sigma^2)),
    mu = length / 2, sigma = length / 4 (no random draws)."""
    x = np.arange(nx, dtype=np.float64) * (length / nx)
    mu, sigma = 0.5 * length, 0.25 * length
    p = alpha * np.exp(-((x - mu) ** 2) / (2.0 * sigma * sigma))
    y0 = np.concatenate([A + p, B / A + p, 3.0 + p])
    return Brusselator1D(nx=nx, A=A, B=B, eps=eps, c=c, length=length, y0=y0)
