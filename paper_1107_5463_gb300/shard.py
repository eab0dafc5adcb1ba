"""One lattice split across torch.distributed ranks (domain decomposition,
Weigel & Yavors'kii 2011, Section 2): rank r of W holds the slab of planes
[L r / W, L (r + 1) / W) along the slowest axis (y in 2D, z in 3D).

Per sweep every rank runs its colour-0 pass, exchanges the boundary planes
of colour 0 with its two neighbours (its first own plane to the rank below,
whose upper halo it is, and its last to the rank above), runs its colour-1
pass, which measures its share of E and M, and exchanges colour 1.  After
the run one all-reduce sums the per-sweep shares of all ranks.  The planes
are views of the slab's device buffer; the exchange is torch.distributed
point-to-point (NCCL between GPUs, gloo on CPU) and the arithmetic runs in
the library's kernels.  Random numbers are keyed by the global site, so the
result equals the unsplit lattice's bit for bit.

The driver talks to its slab through four methods, which the library's
``spinmc.Slab`` provides (a test may pass another implementation):
``planes(colour)`` -> (send_lo, send_hi, recv_lo, recv_hi) tensors,
``series(E, M)`` to direct the per-sweep shares, ``pass_(beta, seed,
colour)``, and ``reduce_series(EM, nsweeps, N)`` -> (E, |m|).
"""
import torch
import torch.distributed as dist


def slab_bounds(L, rank, world):
    """(z0, Lz) of rank `rank` of `world`: contiguous planes, sizes within one."""
    z0 = L * rank // world
    return z0, L * (rank + 1) // world - z0


class ShardedLattice:
    """The rank's slab of an L^d lattice and the exchanges with its neighbours."""

    def __init__(self, local, L, d, group=None):
        self.local, self.L, self.d, self.group = local, L, d, group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self._peer = (lambda r: dist.get_global_rank(group, r)) if group is not None else (
            lambda r: r)

    def exchange(self, colour):
        """Boundary planes of `colour` into the neighbours' halos (periodic)."""
        send_lo, send_hi, recv_lo, recv_hi = self.local.planes(colour)
        if self.world == 1:
            # a single slab is its own neighbour on both sides
            recv_hi.copy_(send_lo)
            recv_lo.copy_(send_hi)
            return
        lo = self._peer((self.rank - 1) % self.world)
        hi = self._peer((self.rank + 1) % self.world)
        # per neighbour, sends and receives pair up in posting order: with two
        # ranks (lo == hi) send_lo meets the peer's recv_hi, send_hi its recv_lo
        ops = [dist.P2POp(dist.isend, send_lo, lo, self.group),
               dist.P2POp(dist.irecv, recv_hi, hi, self.group),
               dist.P2POp(dist.isend, send_hi, hi, self.group),
               dist.P2POp(dist.irecv, recv_lo, lo, self.group)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def sweep_series(self, beta, nsweeps, seed):
        """nsweeps sweeps; returns (E, |m|) of the whole lattice on every rank."""
        dev = self.local.planes(0)[0].device
        EM = torch.zeros(2 * nsweeps, dtype=torch.float64, device=dev)
        self.local.series(EM[:nsweeps], EM[nsweeps:])
        self.exchange(0)
        self.exchange(1)
        for _ in range(nsweeps):
            for c in (0, 1):
                self.local.pass_(beta, seed, c)
                self.exchange(c)
        if self.world > 1:
            dist.all_reduce(EM, group=self.group)
        return self.local.reduce_series(EM, nsweeps, float(self.L ** self.d))
