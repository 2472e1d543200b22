"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module produces *inputs only*: tight-binding lattices in the paper's input
form (neighbour list, hoppings, on-site potentials, bond x-displacements, system
length and volume -- the data the paper's neighbour/hopping/potential/position
files carry, Sec. 4.2, Eqs. 32-34), random-phase vectors for the stochastic
trace (Sec. 3.1, Eq. 13), time-step lists and energy grids.  It contains none of
the method's arithmetic (no Chebyshev recursion, no Bessel coefficients, no
kernel-polynomial reconstruction); both the oracle and the GPU library consume
what it returns.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th output of a SplitMix64 stream seeded with s is ``mix(s + (i+1)*G)`` with
``G = 0x9E3779B97F4A7C15`` and ``mix`` the published 64-bit finaliser.  A stream
is keyed as ``key(seed, stream) = mix(seed + (stream+1)*G)`` and draw i of it is
``mix(key + (i+1)*G)``; a uniform double in [0,1) is the top 53 bits / 2**53.
The GPU library implements the same definition on its own for its on-device
random-phase generator and native lattice builders.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers.  Phase vectors use PHASE + r for vector r; realisation q
# of a ragged batch offsets every stream by REALISATION_STRIDE * (q + 1).
STREAM_ONSITE = 1
STREAM_VACANCY = 2
STREAM_RAGGED = 3
STREAM_PHASE = 1 << 20
REALISATION_STRIDE = 1 << 24

BASE_SEED = 1705013870

KIND_CHAIN, KIND_SQUARE, KIND_HONEYCOMB, KIND_CUBIC = 1, 2, 3, 4


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed % (1 << 64)) + np.uint64(stream + 1) * GOLDEN
    return _mix(np.array([s], dtype=np.uint64))[0]


def draws_u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Raw 64-bit draws start..start+count-1 of stream ``stream``."""
    key = stream_key(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + i * GOLDEN)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of each draw times 2**-53."""
    return (draws_u64(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Lattice:
    """A tight-binding model in the paper's input form (Sec. 4.2).

    Row ``i`` of the neighbour list holds ``nb_count[i]`` neighbours
    ``nb_idx[i, :nb_count[i]]``; ``hop[i, k]`` is H_{i, nb_idx[i,k]} (Eq. 32),
    ``onsite[i]`` is U_i and ``dx[i, k] = X_{nb} - X_i`` is the bond's
    displacement along the transport direction taken as the minimum image
    under periodic boundaries (Eq. 34).  ``volume`` is Omega (Eqs. 25-27).
    Slots at or beyond ``nb_count[i]`` hold index i, hopping 0 and dx 0.
    ``dy`` (optional) is the displacement along the second in-plane direction
    (Hall responses); it is None for models that do not define it.
    """

    name: str
    n: int
    max_nb: int
    nb_count: np.ndarray  # int32 [N]
    nb_idx: np.ndarray  # int32 [N, K]
    hop: np.ndarray  # complex128 [N, K]
    onsite: np.ndarray  # float64 [N]
    dx: np.ndarray  # float64 [N, K]
    length_x: float
    volume: float
    kind: int = 0
    dims: tuple = ()
    seg_offsets: np.ndarray | None = None  # int64 [nseg+1] for block-diagonal batches
    dy: np.ndarray | None = None  # float64 [N, K], Y_nb - Y_i (minimum image)

    def hop_is_real(self) -> bool:
        return bool(np.all(self.hop.imag == 0.0))


def _onsite(n: int, W: float, seed: int, stream_offset: int = 0) -> np.ndarray:
    if W == 0.0:
        return np.zeros(n, dtype=np.float64)
    return W * (uniform(seed, STREAM_ONSITE + stream_offset, n) - 0.5)


def vacancy_sites(n: int, frac: float, seed: int, stream_offset: int = 0) -> np.ndarray:
    """Exactly round(frac*n) distinct sites: those with the smallest draws of
    the vacancy stream (ties broken by site index)."""
    nv = int(round(frac * n))
    if nv == 0:
        return np.zeros(0, dtype=np.int64)
    keys = draws_u64(seed, STREAM_VACANCY + stream_offset, n)
    order = np.argsort(keys, kind="stable")
    return np.sort(order[:nv])


def _apply_vacancies(lat: Lattice, sites: np.ndarray) -> None:
    if sites.size == 0:
        return
    vac = np.zeros(lat.n, dtype=bool)
    vac[sites] = True
    kill = vac[:, None] | vac[lat.nb_idx]
    lat.hop[kill] = 0.0


def chain(L: int, t: float = -1.0, W: float = 0.0, seed: int = BASE_SEED, stream_offset: int = 0) -> Lattice:
    """Periodic 1D chain, lattice constant 1 (the localized example, Sec. 5.2)."""
    if L < 3:
        raise ValueError("chain needs L >= 3")
    i = np.arange(L, dtype=np.int64)
    idx = np.stack([(i + 1) % L, (i - 1) % L], axis=1).astype(np.int32)
    dx = np.tile(np.array([1.0, -1.0]), (L, 1))
    hop = np.full((L, 2), complex(t), dtype=np.complex128)
    return Lattice("chain", L, 2, np.full(L, 2, np.int32), idx, hop, _onsite(L, W, seed, stream_offset), dx,
                   float(L), float(L), KIND_CHAIN, (L,), dy=np.zeros((L, 2)))


def square(Lx: int, Ly: int, t: float = -1.0, W: float = 0.0, seed: int = BASE_SEED, stream_offset: int = 0) -> Lattice:
    """Periodic square lattice, site (ix, iy) -> ix + Lx*iy; slots +x, -x, +y, -y
    (the diffusive example, Sec. 5.1, Eq. 35)."""
    if Lx < 3 or Ly < 3:
        raise ValueError("square needs Lx, Ly >= 3")
    n = Lx * Ly
    s = np.arange(n, dtype=np.int64)
    ix, iy = s % Lx, s // Lx
    idx = np.stack([((ix + 1) % Lx) + Lx * iy, ((ix - 1) % Lx) + Lx * iy,
                    ix + Lx * ((iy + 1) % Ly), ix + Lx * ((iy - 1) % Ly)], axis=1).astype(np.int32)
    dx = np.tile(np.array([1.0, -1.0, 0.0, 0.0]), (n, 1))
    dy = np.tile(np.array([0.0, 0.0, 1.0, -1.0]), (n, 1))
    hop = np.full((n, 4), complex(t), dtype=np.complex128)
    return Lattice("square", n, 4, np.full(n, 4, np.int32), idx, hop, _onsite(n, W, seed, stream_offset), dx,
                   float(Lx), float(n), KIND_SQUARE, (Lx, Ly), dy=dy)


def cubic(L: int, t: float = -1.0, W: float = 0.0, seed: int = BASE_SEED, stream_offset: int = 0) -> Lattice:
    """Periodic simple-cubic lattice, site (x,y,z) -> x + L*y + L*L*z; slots
    +x, -x, +y, -y, +z, -z."""
    if L < 3:
        raise ValueError("cubic needs L >= 3")
    n = L ** 3
    s = np.arange(n, dtype=np.int64)
    x, y, z = s % L, (s // L) % L, s // (L * L)
    idx = np.stack([((x + 1) % L) + L * y + L * L * z, ((x - 1) % L) + L * y + L * L * z,
                    x + L * ((y + 1) % L) + L * L * z, x + L * ((y - 1) % L) + L * L * z,
                    x + L * y + L * L * ((z + 1) % L), x + L * y + L * L * ((z - 1) % L)], axis=1).astype(np.int32)
    dx = np.tile(np.array([1.0, -1.0, 0.0, 0.0, 0.0, 0.0]), (n, 1))
    dy = np.tile(np.array([0.0, 0.0, 1.0, -1.0, 0.0, 0.0]), (n, 1))
    hop = np.full((n, 6), complex(t), dtype=np.complex128)
    return Lattice("cubic", n, 6, np.full(n, 6, np.int32), idx, hop, _onsite(n, W, seed, stream_offset), dx,
                   float(L), float(n), KIND_CUBIC, (L,), dy=dy)


SQRT3 = math.sqrt(3.0)


def honeycomb(L1: int, L2: int, t: float = -2.7, W: float = 0.0, seed: int = BASE_SEED,
              vacancy_frac: float = 0.0, stream_offset: int = 0) -> Lattice:
    """Periodic honeycomb (graphene) lattice of L1 x L2 two-site unit cells,
    carbon-carbon distance 1.  Cell (c1, c2) sits at c1*a1 + c2*a2 with
    a1 = (sqrt3, 0), a2 = (sqrt3/2, 3/2); its B site is 1 above its A site.
    Site index 2*(c1 + L1*c2) + s (s = 0 for A, 1 for B); x runs along a1.
    A(c1,c2) bonds to B(c1,c2) (dx 0), B(c1+1,c2-1) (dx +sqrt3/2) and
    B(c1,c2-1) (dx -sqrt3/2); B rows list the reverse bonds in the same order.
    Omega = L1*L2*3*sqrt3/2."""
    if L1 < 2 or L2 < 2:
        raise ValueError("honeycomb needs L1, L2 >= 2")
    ncell = L1 * L2
    n = 2 * ncell
    c = np.arange(ncell, dtype=np.int64)
    c1, c2 = c % L1, c // L1

    def cell(a, b):
        return (a % L1) + L1 * (b % L2)

    idx = np.empty((n, 3), dtype=np.int64)
    idx[0::2, 0] = 2 * cell(c1, c2) + 1
    idx[0::2, 1] = 2 * cell(c1 + 1, c2 - 1) + 1
    idx[0::2, 2] = 2 * cell(c1, c2 - 1) + 1
    idx[1::2, 0] = 2 * cell(c1, c2)
    idx[1::2, 1] = 2 * cell(c1 - 1, c2 + 1)
    idx[1::2, 2] = 2 * cell(c1, c2 + 1)
    dx = np.empty((n, 3), dtype=np.float64)
    dx[0::2] = [0.0, SQRT3 / 2, -SQRT3 / 2]
    dx[1::2] = [0.0, -SQRT3 / 2, SQRT3 / 2]
    dy = np.empty((n, 3), dtype=np.float64)
    dy[0::2] = [1.0, -0.5, -0.5]
    dy[1::2] = [-1.0, 0.5, 0.5]
    hop = np.full((n, 3), complex(t), dtype=np.complex128)
    lat = Lattice("honeycomb", n, 3, np.full(n, 3, np.int32), idx.astype(np.int32), hop,
                  _onsite(n, W, seed, stream_offset), dx, L1 * SQRT3, ncell * 1.5 * SQRT3,
                  KIND_HONEYCOMB, (L1, L2), dy=dy)
    if vacancy_frac > 0.0:
        _apply_vacancies(lat, vacancy_sites(n, vacancy_frac, seed, stream_offset))
    return lat


def haldane(L1: int, L2: int, t1: float = -1.0, t2: float = 0.15, phi: float = math.pi / 2, mass: float = 0.0,
            W: float = 0.0, seed: int = BASE_SEED, stream_offset: int = 0) -> Lattice:
    """Haldane model on the periodic honeycomb lattice of ``honeycomb`` (same
    cells, site order and nearest-neighbour slots 0-2 with hopping t1), plus six
    next-nearest-neighbour slots per site with hopping t2*exp(+-i phi): for the
    vectors d in {a1, a2 - a1, -a2} an A site hops to A(c + d) with exp(+i phi)
    and to A(c - d) with exp(-i phi); B sites take the opposite signs.  On-site
    energy +mass on A, -mass on B, plus Anderson disorder W (stream 1).  A
    Chern insulator for |mass| < 3 sqrt3 |t2 sin phi| (zero net flux per cell).
    Slots 3-8: +a1, -a1, +(a2-a1), -(a2-a1), -a2, +a2."""
    if L1 < 3 or L2 < 3:
        raise ValueError("haldane needs L1, L2 >= 3")
    base = honeycomb(L1, L2, t1, 0.0)
    ncell = L1 * L2
    n = 2 * ncell
    c = np.arange(ncell, dtype=np.int64)
    c1, c2 = c % L1, c // L1

    def cell(a, b):
        return (a % L1) + L1 * (b % L2)

    a1 = np.array([SQRT3, 0.0])
    a2 = np.array([SQRT3 / 2, 1.5])
    steps = [((1, 0), +1), ((-1, 0), -1), ((-1, 1), +1), ((1, -1), -1), ((0, -1), +1), ((0, 1), -1)]
    K = 9
    idx = np.empty((n, K), np.int64)
    hop = np.empty((n, K), np.complex128)
    dx = np.empty((n, K), np.float64)
    dy = np.empty((n, K), np.float64)
    idx[:, :3], hop[:, :3], dx[:, :3], dy[:, :3] = base.nb_idx, base.hop, base.dx, base.dy
    for k, ((e1, e2), sgn) in enumerate(steps):
        d = e1 * a1 + e2 * a2
        for s in (0, 1):
            idx[s::2, 3 + k] = 2 * cell(c1 + e1, c2 + e2) + s
            hop[s::2, 3 + k] = t2 * np.exp(1j * phi * sgn * (1 if s == 0 else -1))
            dx[s::2, 3 + k] = d[0]
            dy[s::2, 3 + k] = d[1]
    onsite = _onsite(n, W, seed, stream_offset)
    onsite[0::2] += mass
    onsite[1::2] -= mass
    return Lattice("haldane", n, K, np.full(n, K, np.int32), idx.astype(np.int32), hop, onsite, dx,
                   L1 * SQRT3, ncell * 1.5 * SQRT3, 0, (L1, L2), dy=dy)


def block_diagonal(parts: list[Lattice]) -> Lattice:
    """Concatenate independent lattices into one block-diagonal model with
    segment offsets (a ragged batch of disorder realisations)."""
    K = max(p.max_nb for p in parts)
    n = sum(p.n for p in parts)
    cnt = np.zeros(n, np.int32)
    idx = np.zeros((n, K), np.int32)
    hop = np.zeros((n, K), np.complex128)
    dx = np.zeros((n, K), np.float64)
    dy = np.zeros((n, K), np.float64) if all(p.dy is not None for p in parts) else None
    ons = np.zeros(n, np.float64)
    offs = [0]
    for p in parts:
        o = offs[-1]
        sl = slice(o, o + p.n)
        cnt[sl] = p.nb_count
        idx[sl] = np.arange(o, o + p.n, dtype=np.int32)[:, None]
        idx[sl, :p.max_nb] = p.nb_idx + o
        hop[sl, :p.max_nb] = p.hop
        dx[sl, :p.max_nb] = p.dx
        if dy is not None:
            dy[sl, :p.max_nb] = p.dy
        ons[sl] = p.onsite
        offs.append(o + p.n)
    return Lattice("block_diagonal", n, K, cnt, idx, hop, ons, dx, 0.0, float(sum(p.volume for p in parts)),
                   0, (), np.array(offs, dtype=np.int64), dy)


def ragged_cubic(count: int, lmin: int, lmax: int, t: float, W: float, seed: int) -> Lattice:
    """``count`` simple-cubic realisations with L drawn uniformly from
    lmin..lmax (stream STREAM_RAGGED), each with its own disorder stream."""
    u = uniform(seed, STREAM_RAGGED, count)
    Ls = lmin + np.minimum((u * (lmax - lmin + 1)).astype(np.int64), lmax - lmin)
    parts = [cubic(int(L), t, W, seed, stream_offset=REALISATION_STRIDE * (q + 1)) for q, L in enumerate(Ls)]
    return block_diagonal(parts)


def random_phase(n: int, R: int = 1, seed: int = BASE_SEED, first_vector: int = 0) -> np.ndarray:
    """Random-phase vectors phi_i = exp(i theta_i)/sqrt(n), theta = 2*pi*u with u
    from stream STREAM_PHASE + r (vector r); layout [n, R] (site-major, the R
    vectors of one site contiguous).  Unit norm: the paper's <phi|phi> = N
    convention (Eq. 13) differs by the factor N, restored in the
    reconstruction prefactor."""
    out = np.empty((n, R), dtype=np.complex128)
    for r in range(R):
        theta = 2.0 * math.pi * uniform(seed, STREAM_PHASE + first_vector + r, n)
        out[:, r] = (np.cos(theta) + 1j * np.sin(theta)) / math.sqrt(n)
    return out


def energy_scale_rule(z: int, t: float, W: float) -> float:
    """Delta E = 1.05 * (z|t| + W/2): the Gershgorin bound of the Anderson model
    with a 5% margin (the spectrum of H/Delta E must lie in [-1, 1], Eq. 19)."""
    return 1.05 * (z * abs(t) + W / 2.0)


@dataclasses.dataclass
class Workload:
    name: str
    lattice_args: dict
    energy_scale: float
    R: int
    M: int
    dt: float
    n_steps: int
    energies: np.ndarray
    seed: int
    fp32: bool = False


def config(index: int, small: bool = False) -> Workload:
    """The five synthetic workloads, seed 1705013870 + index.  Units: eV for
    energies, hbar/eV for times (Delta t = x hbar/|t| is x/|t| in these units).
    ``small`` shrinks the lattice (not the method parameters) for tests."""
    seed = BASE_SEED + index
    if index == 0:
        return Workload("honeycomb32x32_fp64", dict(kind="honeycomb", L1=32, L2=32, t=-2.7, W=1.0),
                        energy_scale_rule(3, -2.7, 1.0), 1, 512, 1.0 / 2.7, 10, np.linspace(-8, 8, 1001), seed)
    if index == 1:
        L1, L2 = (64, 32) if small else (4096, 2048)
        return Workload("honeycomb4096x2048_fp64", dict(kind="honeycomb", L1=L1, L2=L2, t=-2.7, W=2.0),
                        energy_scale_rule(3, -2.7, 2.0), 1, 3000, 2.0 / 2.7, 100, np.linspace(-8, 8, 1001), seed)
    if index == 2:
        L = 16 if small else 256
        return Workload("cubic256_R32_fp32", dict(kind="cubic", L=L, t=-1.0, W=16.5),
                        energy_scale_rule(6, -1.0, 16.5), 32, 2048, 0.0, 0, np.linspace(-14, 14, 1001), seed, True)
    if index == 3:
        L1 = 64 if small else 2048
        return Workload("honeycomb2048x2048_vac1pct_R8_fp32",
                        dict(kind="honeycomb", L1=L1, L2=L1, t=-2.7, W=0.5, vacancy_frac=0.01),
                        energy_scale_rule(3, -2.7, 0.5), 8, 4000, 2.0 / 2.7, 200, np.linspace(-8, 8, 1001), seed, True)
    if index == 4:
        L1 = 16 if small else 256
        return Workload("honeycomb256x256_grad", dict(kind="honeycomb", L1=L1, L2=L1, t=-2.7, W=2.0),
                        energy_scale_rule(3, -2.7, 2.0), 1, 1024, 2.0 / 2.7, 51, np.linspace(-2, 2, 64), seed)
    raise ValueError(index)


def build_lattice(args: dict, seed: int) -> Lattice:
    a = dict(args)
    kind = a.pop("kind")
    if kind == "honeycomb":
        return honeycomb(a["L1"], a["L2"], a["t"], a["W"], seed, a.get("vacancy_frac", 0.0))
    if kind == "cubic":
        return cubic(a["L"], a["t"], a["W"], seed)
    if kind == "square":
        return square(a["Lx"], a["Ly"], a["t"], a["W"], seed)
    if kind == "chain":
        return chain(a["L"], a["t"], a["W"], seed)
    raise ValueError(kind)


def with_random_bond_phases(lat: Lattice, seed: int, stream: int = 5) -> Lattice:
    """Multiply every bond's hopping by a random phase exp(i theta_b), keeping H
    Hermitian: slot (i,k) -> j gets exp(+i theta), its reverse slot (j,k') -> i
    gets exp(-i theta).  Gives a complex-hopping model for tests."""
    n, K = lat.n, lat.max_nb
    hop = lat.hop.copy()
    done = np.zeros((n, K), dtype=bool)
    u = uniform(seed, stream, n * K).reshape(n, K)
    for i in range(n):
        for k in range(lat.nb_count[i]):
            if done[i, k]:
                continue
            j = int(lat.nb_idx[i, k])
            rev = [kk for kk in range(lat.nb_count[j]) if lat.nb_idx[j, kk] == i and not done[j, kk]
                   and (j != i or kk != k)]
            if not rev:
                raise ValueError("neighbour list is not symmetric")
            kk = rev[0]
            ph = np.exp(2j * math.pi * u[i, k])
            hop[i, k] *= ph
            hop[j, kk] *= np.conj(ph)
            done[i, k] = done[j, kk] = True
    out = dataclasses.replace(lat, hop=hop, name=lat.name + "_phases")
    return out
