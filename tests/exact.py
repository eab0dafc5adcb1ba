"""Exact results used to pin the oracle (no Monte Carlo, no oracle code).

- Brute-force enumeration of small Ising lattices (Eq. 1 summed over all
  2^N states) and of their exact checkerboard transition matrices (Eq. 2
  applied to one colour at a time, Section 2).
- Kaufman's closed-form partition function of the L x L periodic Ising model
  (the finite-lattice solution behind the exact density of states the paper
  compares its Wang-Landau runs with, Section 4).
- Two-spin O(n) bond distributions p(x) ~ exp(beta J x) (1 - x^2)^((n-3)/2).
- Binning error bars.

Energies here are computed with numpy rolls of the whole configuration: a
different formulation of Eq. (1) from the oracle's site loop.
"""
import itertools
import math

import numpy as np
from scipy import integrate, special


def roll_energy(s, d, L, J=1.0, Jb=None):
    """E = -J sum_i sum_mu Jb[mu][i] s_i s_{i+e_mu} for natural-order arrays.

    s has shape (..., N) (Ising) or (..., N, n) (vector spins)."""
    vec = s.ndim >= 2 and s.shape[-1] in (2, 3) and s.shape[-2] == L ** d
    shape = (L,) * d
    lead = s.shape[:-2] if vec else s.shape[:-1]
    if vec:
        a = s.reshape(lead + shape[::-1] + (s.shape[-1],))
    else:
        a = s.reshape(lead + shape[::-1])
    nlead = len(lead)
    e = 0.0
    for mu in range(d):
        axis = nlead + (d - 1 - mu)          # natural order: x fastest
        nb = np.roll(a, -1, axis=axis)
        prod = (a * nb).sum(axis=-1) if vec else a.astype(np.int64) * nb
        if Jb is not None:
            jb = np.asarray(Jb[mu]).reshape(shape[::-1])
            prod = prod * jb
        e = e + prod.reshape(lead + (-1,)).sum(axis=-1)
    return -J * e


def chunked_energy(s, d, L, rows=512):
    """roll_energy for uniform J = 1 on lattices too large for whole-array
    temporaries: slabs of `rows` rows (2D) or planes (3D) with their wrapped
    successor, int64 sums."""
    a = s.reshape((L,) * d)
    e = 0
    for y0 in range(0, L, rows):
        y1 = min(y0 + rows, L)
        blk = a[y0:y1]
        nxt = np.concatenate([a[y0 + 1:y1], a[(y1) % L][None]], axis=0)
        e += int((blk * nxt).sum(dtype=np.int64))                          # +e along the slow axis
        for ax in range(1, d):
            e += int((blk * np.roll(blk, -1, axis=ax)).sum(dtype=np.int64))
    return -e


def all_states(N):
    """All 2^N Ising configurations, shape (2^N, N), int8."""
    idx = np.arange(2 ** N, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(N)) & 1
    return (1 - 2 * bits).astype(np.int8)


def enumerate_ising(d, L, beta, J=1.0, Jb=None):
    """Exact <E>, <E^2>, <|m|> and ln Z by summing over all states."""
    N = L ** d
    S = all_states(N)
    E = roll_energy(S, d, L, J, Jb).astype(np.float64)
    absm = np.abs(S.astype(np.int64).sum(axis=1)) / N
    w = -beta * E
    wmax = w.max()
    p = np.exp(w - wmax)
    Z = p.sum()
    p /= Z
    return dict(E=(p * E).sum(), E2=(p * E * E).sum(), absm=(p * absm).sum(),
                lnZ=math.log(Z) + wmax, energies=E, probs=p, states=S)


def neighbour(d, L, i, k):
    """Natural index of neighbour k = 2 mu + (0 for -e_mu, 1 for +e_mu) of site i."""
    x = [i % L, (i // L) % L, i // (L * L)][:d]
    mu = k >> 1
    x[mu] = (x[mu] + (1 if k & 1 else -1)) % L
    return sum(c * L ** a for a, c in enumerate(x))


def colour_of_site(d, L):
    N = L ** d
    i = np.arange(N)
    c = i % L + (i // L) % L
    if d == 3:
        c = c + i // (L * L)
    return c & 1


def exact_sweep_matrix(d, L, beta, J=1.0, Jb=None, heatbath=False):
    """Exact transition matrix of one checkerboard sweep (colour 0 then 1).

    Within a half-sweep the sites of one colour are updated independently:
    Metropolis flips each with probability min(1, exp(-beta dE)); heat-bath
    sets each to its flipped value with probability
    exp(-beta E') / (exp(-beta E) + exp(-beta E')), energies E (current) and
    E' (flipped) taken from the full Hamiltonian."""
    N = L ** d
    S = all_states(N)
    E = roll_energy(S, d, L, J, Jb).astype(np.float64)
    colour = colour_of_site(d, L)
    index = {tuple(s): k for k, s in enumerate(S)}
    mats = []
    for c in (0, 1):
        sites = np.nonzero(colour == c)[0]
        T = np.zeros((len(S), len(S)))
        for a in range(len(S)):
            # per-site flip probabilities given the (fixed) other colour
            pflip = []
            for i in sites:
                s2 = S[a].copy()
                s2[i] = -s2[i]
                dE = E[index[tuple(s2)]] - E[a]
                if heatbath:
                    pflip.append(1.0 / (1.0 + math.exp(beta * dE)))
                else:
                    pflip.append(1.0 if dE <= 0 else math.exp(-beta * dE))
            for flips in itertools.product((0, 1), repeat=len(sites)):
                s2 = S[a].copy()
                prob = 1.0
                for f, i, pf in zip(flips, sites, pflip):
                    if f:
                        s2[i] = -s2[i]
                        prob *= pf
                    else:
                        prob *= 1.0 - pf
                T[a, index[tuple(s2)]] += prob
        mats.append(T)
    return mats[0], mats[1], S, E


def multihit_sweep_distribution(d, L, T, k, beta, start, J=1.0):
    """Exact distribution over all 2^N states after one k-fold multi-hit
    sweep from `start`: for tile colour 0 then 1, k times, site colour 0 then
    1, every site of that tile colour and site colour flips independently
    with min(1, exp(-beta dE)), dE from the full Eq. (1).  States are encoded
    with bit i set for s_i = -1."""
    N = L ** d
    S = all_states(N)
    E = roll_energy(S, d, L, J).astype(np.float64)
    colour = colour_of_site(d, L)
    i = np.arange(N)
    tcol = (i % L) // T + ((i // L) % L) // T
    if d == 3:
        tcol = tcol + (i // (L * L)) // T
    tcol &= 1
    states = np.arange(2 ** N, dtype=np.int64)
    p = np.zeros(2 ** N)
    p[int(sum(1 << q for q in range(N) if start[q] < 0))] = 1.0
    for tc in (0, 1):
        for _ in range(k):
            for c in (0, 1):
                sites = np.nonzero((colour == c) & (tcol == tc))[0]
                pf = [np.minimum(1.0, np.exp(-beta * (E[states ^ (1 << q)] - E))) for q in sites]
                new = np.zeros_like(p)
                for flips in itertools.product((0, 1), repeat=len(sites)):
                    mask = sum(1 << q for f, q in zip(flips, sites) if f)
                    w = p.copy()
                    for f, pq in zip(flips, pf):
                        w *= pq if f else 1.0 - pq
                    np.add.at(new, states ^ mask, w)
                p = new
    return p


def forward_bonds(d, L):
    """The d N forward bonds (i, i + e_mu) of the periodic lattice as two
    arrays of site indices (a multigraph for L = 2)."""
    N = L ** d
    i = np.arange(N)
    coords = [(i // L ** mu) % L for mu in range(d)]
    a, b = [], []
    for mu in range(d):
        nb = i + (((coords[mu] + 1) % L) - coords[mu]) * L ** mu
        a.append(i)
        b.append(nb)
    return np.concatenate(a), np.concatenate(b)


def exact_sw_matrix(d, L, beta, J=1.0):
    """Exact transition matrix of one Swendsen-Wang update (Section 3): every
    satisfied bond (J s_a s_b > 0) is activated independently with
    p = 1 - exp(-2 beta |J|), the clusters are the connected components of the
    active bonds (scipy's connected_components), and every cluster flips
    independently with probability 1/2.  Summed over all bond subsets."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    N = L ** d
    S = all_states(N)
    E = roll_energy(S, d, L, J).astype(np.float64)
    A, B = forward_bonds(d, L)
    p = 1.0 - math.exp(-2.0 * beta * abs(J))
    codes = ((S < 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    row_of = {int(c): k for k, c in enumerate(codes)}
    T = np.zeros((len(S), len(S)))
    for a_state, s in enumerate(S):
        sat = np.nonzero(J * s[A].astype(np.int64) * s[B] > 0)[0]
        for mask in range(1 << len(sat)):
            on = [sat[q] for q in range(len(sat)) if (mask >> q) & 1]
            w = p ** len(on) * (1.0 - p) ** (len(sat) - len(on))
            if w == 0.0:
                continue
            g = coo_matrix((np.ones(len(on)), (A[on], B[on])), shape=(N, N))
            ncl, comp = connected_components(g, directed=False)
            for flips in range(1 << ncl):
                f = (flips >> comp) & 1
                code = int(codes[a_state] ^ (f << np.arange(N)).sum())
                T[a_state, row_of[code]] += w / (1 << ncl)
    return T, S, E


def ising_dos_enumerated(L):
    """Density of states g[k] of the L x L torus by enumeration, levels
    k = (E + 2N) / 4 (E from Eq. 1 with J = 1)."""
    N = L * L
    E = roll_energy(all_states(N), 2, L).astype(np.int64)
    return np.bincount((E + 2 * N) // 4, minlength=N + 1).astype(np.float64)


def ising_dos_transfer(L):
    """Density of states g[k] of the L x L torus from the row transfer
    matrix: T(r, r') = y^(unlike bonds inside row r' + unlike bonds between
    rows r and r'), Z(y) = Tr T^L = sum over configurations of y^(unlike
    bonds) = sum_k g[k] y^(2k); Z is evaluated at the 2N+1 complex roots of
    unity and its coefficients recovered by an inverse DFT.  For L <= 6 the
    counts are below 2^53 and round to the exact integers; beyond, the
    rounding error of the largest coefficients swamps the smallest, so larger
    L is refused."""
    if L > 6:
        raise ValueError("exact only for L <= 6")
    N = L * L
    R = np.arange(2 ** L)
    bits = (R[:, None] >> np.arange(L)) & 1
    within = (bits != np.roll(bits, -1, axis=1)).sum(axis=1)          # periodic row
    between = np.array([[bin(a ^ b).count("1") for b in R] for a in R])
    expo = between + within[None, :]
    M = 2 * N + 1
    Z = np.empty(M, complex)
    for j in range(M):
        y = np.exp(2j * np.pi * j / M)
        T = y ** expo
        Z[j] = np.trace(np.linalg.matrix_power(T, L))
    coef = np.real(np.fft.fft(Z)) / M   # Z[j] = sum_m c_m w^(jm), w = e^(2 pi i / M)
    return np.round(coef[0::2][: N + 1])


# ------------------------------------------------------- Kaufman 1949 ----

def _ln2cosh(x):
    ax = abs(x)
    return ax + math.log1p(math.exp(-2.0 * ax))


def _ln2sinh_signed(x):
    ax = abs(x)
    return ax + math.log1p(-math.exp(-2.0 * ax)), (1.0 if x >= 0 else -1.0)


def kaufman_lnZ(K, L):
    """ln Z of the L x L periodic Ising model at coupling K = beta J.

    Z = 1/2 (2 sinh 2K)^(L^2/2) (Z1 + Z2 + Z3 + Z4) with
    Z1,2 = prod_{r<L} 2 cosh|sinh (L gamma_{2r+1} / 2),
    Z3,4 = prod_{r<L} 2 cosh|sinh (L gamma_{2r} / 2),
    cosh gamma_l = cosh 2K coth 2K - cos(pi l / L), gamma_0 = 2K + ln tanh K."""
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def gamma(l):
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(c - math.cos(math.pi * l / L))

    terms = []          # (log|Z_i|, sign)
    for parity in (1, 0):
        g = [gamma(2 * r + parity) for r in range(L)]
        terms.append((sum(_ln2cosh(L * x / 2) for x in g), 1.0))
        lsum, sgn = 0.0, 1.0
        for x in g:
            v, s = _ln2sinh_signed(L * x / 2)
            lsum += v
            sgn *= s
        terms.append((lsum, sgn))
    m = max(t[0] for t in terms)
    acc = sum(s * math.exp(v - m) for v, s in terms)
    return math.log(0.5) + (L * L / 2) * math.log(2 * math.sinh(2 * K)) + m + math.log(acc)


def kaufman_energy_per_site(beta, L, J=1.0, h=1e-5):
    """<E>/N = -(1/N) d ln Z / d beta by a central difference."""
    f = lambda b: kaufman_lnZ(b * J, L)
    return -(f(beta + h) - f(beta - h)) / (2 * h) / (L * L)


# ------------------------------------------------- two-spin O(n) laws ----

def two_spin_mean(n, beta):
    """<s_a . s_b> for one bond of strength 1 between two O(n) spins."""
    if n == 1:
        return math.tanh(beta)
    if n == 2:
        return special.i1(beta) / special.i0(beta)
    if n == 3:
        return 1.0 / math.tanh(beta) - 1.0 / beta
    raise ValueError(n)


def two_spin_cdf(n, beta):
    """CDF of x = s_a . s_b (n = 2, 3) under p(x) ~ e^{beta x} (1-x^2)^((n-3)/2)."""
    if n == 3:
        return lambda x: (np.exp(beta * x) - math.exp(-beta)) / (math.exp(beta) - math.exp(-beta))
    if n == 2:
        dens = lambda x: math.exp(beta * x) / math.sqrt(1 - x * x)
        Z = integrate.quad(dens, -1, 1, limit=200)[0]

        def cdf(xs):
            xs = np.atleast_1d(xs)
            # substitute x = cos(theta): F(x) = int_{arccos x}^{pi} e^{beta cos t} dt / Z
            return np.array([integrate.quad(lambda t: math.exp(beta * math.cos(t)),
                                            math.acos(min(1.0, max(-1.0, x))), math.pi)[0]
                             for x in xs]) / Z
        return cdf
    raise ValueError(n)


# ------------------------------------------------------------ errors ----

def binned_mean(x, nbins=20):
    """Mean and its standard error from nbins equal bins (autocorrelation-safe
    when each bin is much longer than the autocorrelation time)."""
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins)
