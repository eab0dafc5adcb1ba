"""The domain-decomposition driver (paper_1107_5463_gb300/shard.py) on CPU
ranks with the gloo backend: world sizes 1 to 4, each rank holding one slab
of the lattice.  The slab here is the CPU oracle behind the library's plane
layout (per colour Lz + 2 planes of L^(d-1)/2 bytes, halo planes first and
last, colour index inside a plane = plane-local natural index // 2, 0 = up),
its sites updated by the oracle's single-site update from the configuration
their colour's pass sees.  The split run must equal the oracle's unsplit
sweeps bit for bit: every spin and the whole E and |m| series.  This checks
the exchange plan (which plane goes to which neighbour's which halo, after
which pass), the global indexing of the random numbers and the all-reduce of
the measured shares."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleSlab:
    """Planes z0 .. z0 + Lz - 1 of an Ising lattice, updated by the oracle."""

    def __init__(self, d, L, z0, Lz, seed, J=1.0):
        import torch
        import oracle
        self.d, self.L, self.z0, self.Lz, self.J = d, L, z0, Lz, J
        self.Lp = L ** (d - 1)          # sites per plane
        self.P = self.Lp // 2           # sites of one colour per plane
        self.buf = torch.zeros(2 * (Lz + 2) * self.P, dtype=torch.uint8)
        self.t = 0
        self.k = 0
        self.E = self.M = None
        s = oracle.ising_init(d, L, seed)
        self._set_planes(s, range(z0, z0 + Lz))

    # plane p (-1 .. Lz) of colour c
    def _plane(self, c, p):
        base = c * (self.Lz + 2) * self.P
        return self.buf[base + (p + 1) * self.P: base + (p + 2) * self.P]

    def _colour(self, z, q):
        if self.d == 2:
            return (q + z) & 1
        return (q % self.L + q // self.L + z) & 1

    def _set_planes(self, s, zs):
        for z in zs:
            p = z - self.z0
            for q in range(self.Lp):
                v = 1 if s[z * self.Lp + q] < 0 else 0
                self._plane(self._colour(z, q), p)[q >> 1] = v

    def _conf(self):
        """Global natural-order configuration: own and halo planes filled."""
        s = np.zeros(self.L ** self.d, np.int8)
        order = [-1, self.Lz] + list(range(self.Lz))   # own planes written last
        for p in order:
            z = (self.z0 + p) % self.L
            for q in range(self.Lp):
                b = int(self._plane(self._colour(z, q), p)[q >> 1])
                s[z * self.Lp + q] = -1 if b else 1
        return s

    def own_spins(self):
        s = self._conf()
        return s[self.z0 * self.Lp:(self.z0 + self.Lz) * self.Lp].copy()

    def planes(self, colour):
        return [self._plane(colour, 0), self._plane(colour, self.Lz - 1),
                self._plane(colour, -1), self._plane(colour, self.Lz)]

    def series(self, E, M):
        self.E, self.M, self.k = E, M, 0

    def pass_(self, beta, seed, colour):
        import oracle
        s = self._conf()
        sites = [z * self.Lp + q for z in range(self.z0, self.z0 + self.Lz)
                 for q in range(self.Lp) if self._colour(z, q) == colour]
        new = oracle.ising_site_updates(self.d, self.L, s, sites, beta, seed, self.t, J=self.J)
        s[sites] = new
        self._set_planes(s, range(self.z0, self.z0 + self.Lz))
        if colour == 1:
            # the slab's share: bonds of its colour-1 sites, its own spins
            a = s.reshape((self.L,) * self.d).astype(np.int64)
            h = sum(np.roll(a, sh, axis=ax) for ax in range(self.d) for sh in (1, -1))
            own = slice(self.z0 * self.Lp, (self.z0 + self.Lz) * self.Lp)
            sa, ha = a.reshape(-1)[own], h.reshape(-1)[own]
            c1 = np.array([self._colour(z, q) == 1 for z in range(self.z0, self.z0 + self.Lz)
                           for q in range(self.Lp)])
            if self.E is not None:
                self.E[self.k] = -self.J * float((sa * ha)[c1].sum())
                self.M[self.k] = float(sa.sum())
            self.k += 1
            self.t += 1

    def reduce_series(self, EM, nsweeps, N):
        E = EM[:nsweeps].clone()
        m = EM[nsweeps:].abs() / N
        return E, m


def _rank(rank, world, port, d, L, seed, beta, sweep_seed, nsw, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1107_5463_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    z0, Lz = shard.slab_bounds(L, rank, world)
    local = OracleSlab(d, L, z0, Lz, seed)
    sh = shard.ShardedLattice(local, L, d)
    E, m = sh.sweep_series(beta, nsw, sweep_seed)
    out.put((rank, local.own_spins(), E.numpy(), m.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,d,L", [(2, 2, 16), (3, 2, 16), (4, 2, 8), (2, 3, 8), (1, 2, 8)])
def test_split_lattice_equals_unsplit_oracle(world, d, L):
    import oracle
    seed, beta, sweep_seed, nsw = 7, 0.44, 21, 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, d, L, seed, beta, sweep_seed, nsw, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s = oracle.ising_init(d, L, seed)
    E_ref, m_ref = oracle.ising_sweeps(d, L, s, beta, sweep_seed, 0, nsw)
    np.testing.assert_array_equal(np.concatenate([r[1] for r in res]), s)
    for _, _, E, m in res:
        np.testing.assert_array_equal(E, E_ref)
        np.testing.assert_array_equal(m, m_ref)


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_slab_bounds_tile_the_lattice(world):
    from paper_1107_5463_gb300 import shard
    for L in (8, 16, 64, 16384):
        z = 0
        for r in range(world):
            z0, Lz = shard.slab_bounds(L, r, world)
            assert z0 == z and Lz in (L // world, L // world + 1)
            z += Lz
        assert z == L
