"""Seeded synthetic charge systems shaped like the paper's workloads.

This module only draws inputs (positions, charges, rotations, separation
vectors).  It holds none of the method's arithmetic, imports nothing from the
rest of the package, and serves both the CUDA path and the CPU oracle, so the
two always see identical inputs.

Shapes follow the paper: random charges in spheres (Section III-A: radius
proportional to N^(1/3), R0 = 1.5 (R_A + R_B)) and protein-sized systems
scanned over orientation and distance (Section IV).  The protein structure and
charges the paper uses are not available, so compact random-walk chains with
normal partial charges stand in for them.

All generators use numpy's PCG64 (``np.random.default_rng``).  Positions and
charges are returned as float64 arrays of shape (N, 4) holding (x, y, z, q).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------- primitives

def unit_vectors(rng, k):
    """k directions uniform on the unit sphere (normalised Gaussians)."""
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_rotations(rng, k):
    """k rotation matrices uniform on SO(3) (normalised Gaussian quaternions), shape (k, 3, 3)."""
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def uniform_ball(rng, n, radius):
    """n points uniform in a ball of the given radius about the origin."""
    d = unit_vectors(rng, n)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


def uniform_shell(rng, n, r_in, r_out):
    """n points uniform in volume in the shell r_in <= r <= r_out."""
    d = unit_vectors(rng, n)
    u = rng.random(n)
    r = (r_in ** 3 + u * (r_out ** 3 - r_in ** 3)) ** (1.0 / 3.0)
    return d * r[:, None]


def random_walk_chains(rng, ns, radii, bond=1.5):
    """Random-walk chains confined to spheres, advanced together.

    Chain c has ``ns[c]`` atoms and stays inside the sphere of radius
    ``radii[c]`` about its start (the origin): each step has length ``bond`` and
    a direction uniform on the sphere; a step that would leave the sphere is
    redrawn (only that step).  Each chain is then re-centred on its centroid.
    Returns a list of (n_c, 3) arrays.
    """
    ns = np.asarray(ns, dtype=np.int64)
    radii = np.asarray(radii, dtype=np.float64)
    nc = len(ns)
    nmax = int(ns.max()) if nc else 0
    offs = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(ns, out=offs[1:])
    flat = np.zeros((int(offs[-1]), 3))  # every chain starts at the origin
    pos = np.zeros((nc, 3))
    r2 = radii ** 2
    order = np.argsort(-ns, kind="stable")  # longest first: the active chains form a prefix
    neg_sorted = -ns[order]
    for s in range(1, nmax):
        nact = int(np.searchsorted(neg_sorted, -s, side="left"))  # chains with n > s
        act = order[:nact]
        todo = act
        slot = np.arange(nact)
        new = np.empty((nact, 3))
        while len(todo):
            prop = pos[todo] + bond * unit_vectors(rng, len(todo))
            ok = np.einsum("ij,ij->i", prop, prop) <= r2[todo]
            new[slot[ok]] = prop[ok]
            todo = todo[~ok]
            slot = slot[~ok]
        pos[act] = new
        flat[offs[act] + s] = new
    out = []
    for c in range(nc):
        p = flat[offs[c]:offs[c + 1]]
        if len(p):
            p -= p.mean(axis=0)
        out.append(p)
    return out


def random_walk(rng, n, radius, bond=1.5):
    """One confined random-walk chain (see ``random_walk_chains``)."""
    return random_walk_chains(rng, [n], [radius], bond)[0]


def charges_uniform_net_zero(rng, n):
    """q ~ U[-1, 1], shifted to a net charge of zero."""
    q = rng.uniform(-1.0, 1.0, n)
    return q - q.mean()


def charges_normal_net_zero(rng, n, sigma=0.3):
    """q ~ N(0, sigma), shifted to a net charge of zero."""
    q = rng.normal(0.0, sigma, n)
    return q - q.mean() if n else q


def charges_pm_one_excess(rng, n, excess=0.02):
    """Charges +-1 with n_plus - n_minus = round(excess * n), in random order."""
    d = int(round(excess * n))
    n_plus = (n + d) // 2
    q = -np.ones(n)
    q[:n_plus] = 1.0
    rng.shuffle(q)
    return q


def pack(pos, q):
    """(N, 3) positions and (N,) charges -> (N, 4) float64 records (x, y, z, q)."""
    out = np.empty((len(q), 4))
    out[:, :3] = pos
    out[:, 3] = q
    return out


def centroid_and_radius(xyzq):
    """Centroid of positions (unit masses) and max distance from it (generator-side helper)."""
    c = xyzq[:, :3].mean(axis=0)
    return c, float(np.sqrt(((xyzq[:, :3] - c) ** 2).sum(axis=1)).max())


# ----------------------------------------------------------------------------- workloads

@dataclass
class PairScan:
    """Two systems and a list of orientations of B (rotation about B's centre plus R0)."""
    A: np.ndarray
    B: np.ndarray
    rotB: np.ndarray  # (k, 3, 3)
    R0: np.ndarray  # (k, 3), vector from centre of A to centre of B
    L: int
    name: str = ""


@dataclass
class Batch:
    """Many pairs of uneven systems, each pair with its own L, rotation and R0."""
    systems: list
    pair_a: np.ndarray  # (P,) index into systems
    pair_b: np.ndarray
    rotB: np.ndarray  # (P, 3, 3)
    R0: np.ndarray  # (P, 3)
    L: np.ndarray  # (P,)
    name: str = ""


@dataclass
class ServeStream:
    """A pool of resident systems and a Poisson stream of scan requests."""
    systems: list
    arrivals: np.ndarray  # (Q,) seconds
    pair_a: np.ndarray
    pair_b: np.ndarray
    n_orient: np.ndarray
    L: np.ndarray
    rot_seed: np.ndarray  # per-request seed for its rotations and R0
    name: str = ""
    extra: dict = field(default_factory=dict)


def single_pair_sphere(seed=1, n=200, radius=10.0, dist=40.0, L=10):
    """Two n-charge systems uniform in spheres, U[-1,1] net-zero charges, R0 = dist along a seeded direction."""
    rng = np.random.default_rng(seed)
    A = pack(uniform_ball(rng, n, radius), charges_uniform_net_zero(rng, n))
    B = pack(uniform_ball(rng, n, radius), charges_uniform_net_zero(rng, n))
    R0 = dist * unit_vectors(rng, 1)
    return PairScan(A, B, np.eye(3)[None], R0, L, name=f"single pair, 2x{n} charges in r={radius} A spheres, R0={dist} A, L={L}")


def protein_pes_scan(seed=2, n=20000, radius=30.0, n_orient=256, r_lo=70.0, r_hi=150.0, L=20):
    """Protein-like pair: random-walk chains (bond 1.5 A) in r=radius spheres, N(0,0.3) net-zero
    charges, n_orient rotations of B at |R0| uniform in [r_lo, r_hi] along uniform directions."""
    rng = np.random.default_rng(seed)
    pa, pb = random_walk_chains(rng, [n, n], [radius, radius])
    A = pack(pa, charges_normal_net_zero(rng, n))
    B = pack(pb, charges_normal_net_zero(rng, n))
    rot = random_rotations(rng, n_orient)
    R0 = unit_vectors(rng, n_orient) * rng.uniform(r_lo, r_hi, n_orient)[:, None]
    return PairScan(A, B, rot, R0, L,
                    name=f"protein-like PES scan, 2x{n} random-walk atoms (r={radius} A), {n_orient} orientations, R0 in [{r_lo},{r_hi}] A, L={L}")


def uneven_batch(seed=3, n_pairs=4096, n_lo=100, n_hi=100000, Ls=(8, 12, 16, 24), r_lo=1.2, r_hi=3.0):
    """Uneven pairs: N log-uniform, random-walk radius 1.9 N^(1/3), L per pair, R0 = U[r_lo,r_hi] (a_A + a_B)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), 2 * n_pairs)).astype(np.int64)
    radii = 1.9 * ns ** (1.0 / 3.0)
    pos = random_walk_chains(rng, ns, radii)
    systems = [pack(p, charges_normal_net_zero(rng, len(p))) for p in pos]
    a_rad = np.array([centroid_and_radius(s)[1] for s in systems])
    pa = np.arange(0, 2 * n_pairs, 2)
    pb = np.arange(1, 2 * n_pairs, 2)
    rot = random_rotations(rng, n_pairs)
    dist = rng.uniform(r_lo, r_hi, n_pairs) * (a_rad[pa] + a_rad[pb])
    R0 = unit_vectors(rng, n_pairs) * dist[:, None]
    L = rng.choice(np.asarray(Ls), n_pairs)
    return Batch(systems, pa, pb, rot, R0, L, name=f"{n_pairs} uneven pairs, N log-uniform [{n_lo},{n_hi}], L in {tuple(Ls)}")


def large_assembly(seed=4, n_shell=1_000_000, r_in=80.0, r_out=100.0, n_lig=50000, n_orient=10000,
                   r_lo=150.0, r_hi=300.0, L=24):
    """A: +-1 charges (2% excess) in a shell; B: random-walk ligand (radius 1.9 N^(1/3)).
    |R0| is uniform in [max(r_lo, 1.05 (a_A + a_B)), r_hi] so that every orientation converges."""
    rng = np.random.default_rng(seed)
    A = pack(uniform_shell(rng, n_shell, r_in, r_out), charges_pm_one_excess(rng, n_shell))
    B = pack(random_walk(rng, n_lig, 1.9 * n_lig ** (1.0 / 3.0)), charges_normal_net_zero(rng, n_lig))
    aA = centroid_and_radius(A)[1]
    aB = centroid_and_radius(B)[1]
    lo = max(r_lo, 1.05 * (aA + aB))
    rot = random_rotations(rng, n_orient)
    R0 = unit_vectors(rng, n_orient) * rng.uniform(lo, r_hi, n_orient)[:, None]
    return PairScan(A, B, rot, R0, L, name=f"large assembly, {n_shell}-charge shell + {n_lig}-atom ligand, {n_orient} orientations, L={L}")


def serve_stream(seed=5, n_pool=512, n_lo=500, n_hi=200000, rate=2000.0, seconds=60.0,
                 orient_lo=1, orient_hi=64, L_lo=8, L_hi=24):
    """Pool of resident random-walk systems and Poisson scan requests over pairs from it."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), n_pool)).astype(np.int64)
    pos = random_walk_chains(rng, ns, 1.9 * ns ** (1.0 / 3.0))
    systems = [pack(p, charges_normal_net_zero(rng, len(p))) for p in pos]
    n_req = int(rng.poisson(rate * seconds))
    arrivals = np.sort(rng.uniform(0.0, seconds, n_req))
    pa = rng.integers(0, n_pool, n_req)
    pb = (pa + rng.integers(1, n_pool, n_req)) % n_pool
    n_or = rng.integers(orient_lo, orient_hi + 1, n_req)
    L = rng.integers(L_lo, L_hi + 1, n_req)
    seeds = rng.integers(0, 2 ** 62, n_req)
    return ServeStream(systems, arrivals, pa, pb, n_or, L, seeds,
                       name=f"serving stream, {n_pool} resident systems, Poisson {rate}/s for {seconds} s")


def request_orientations(seed, k, a_sum, r_lo=1.2, r_hi=3.0):
    """Rotations and R0 vectors for one scan request: |R0| = U[r_lo, r_hi] * a_sum."""
    rng = np.random.default_rng(int(seed))
    rot = random_rotations(rng, k)
    R0 = unit_vectors(rng, k) * (rng.uniform(r_lo, r_hi, k) * a_sum)[:, None]
    return rot, R0


@dataclass
class PesGrid:
    """Two fixed systems and a grid of separations in the xy-plane: R0 = R (cos T, sin T, 0)."""
    A: np.ndarray
    B: np.ndarray
    R: np.ndarray       # (nR,) centre distances
    theta: np.ndarray   # (nT,) angles from the x axis, degrees
    lmax: tuple
    name: str = ""

    def R0(self):
        """(nR * nT, 3) separations, R-major."""
        t = np.radians(self.theta)
        RR, TT = np.meshgrid(self.R, t, indexing="ij")
        return np.stack([RR * np.cos(TT), RR * np.sin(TT), np.zeros_like(RR)], axis=-1).reshape(-1, 3)


def pes_grid_pair(seed=6, n_a=3260, n_b=2587, r_lo=58.0, r_hi=100.0, dr=1.0, dtheta=1.0,
                  lmax=(1, 2, 3, 4, 6, 8, 10)):
    """The shape of the protein-protein surface scan of Section IV: two protein-sized systems
    (5,847 atoms together, split as 223 : 177 residues) fixed in space, the centre of B moved
    over R0 in [r_lo, r_hi] A and Theta in [0, 360) degrees in the xy-plane, energies at several
    Lmax.  Synthetic stand-ins: compact random-walk chains (bond 1.5 A) confined to spheres of
    radius 1.75 N^(1/3) A, N(0, 0.3) net-zero charges."""
    rng = np.random.default_rng(seed)
    pa, pb = random_walk_chains(rng, [n_a, n_b], [1.75 * n_a ** (1 / 3), 1.75 * n_b ** (1 / 3)])
    A = pack(pa, charges_normal_net_zero(rng, n_a))
    B = pack(pb, charges_normal_net_zero(rng, n_b))
    R = np.arange(r_lo, r_hi + 0.5 * dr, dr)
    theta = np.arange(0.0, 360.0, dtheta)
    return PesGrid(A, B, R, theta, tuple(lmax),
                   name=f"surface scan, {n_a} + {n_b} random-walk atoms, R0 in [{r_lo},{r_hi}] A x {len(theta)} angles "
                        f"in the xy-plane, Lmax in {tuple(lmax)}")

