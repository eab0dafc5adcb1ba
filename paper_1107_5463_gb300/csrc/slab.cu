// Domain decomposition of one lattice into slabs (Weigel & Yavors'kii 2011,
// Section 2: the lattice is decomposed into tiles that different processors
// update in parallel; here the pieces are slabs along the slowest axis, y in
// 2D and z in 3D, one per GPU or per rank).
//
// A slab owns planes z0 .. z0 + Lz - 1 of an L^d Ising lattice and keeps one
// halo plane of each colour before and after them.  A checkerboard sweep is
// the colour-0 pass of every slab, the exchange of the just-updated colour's
// boundary planes into the neighbours' halos, the colour-1 pass (which also
// measures the slab's share of E and M) and the exchange of colour 1.  Every
// random number is keyed by the global site, so any split reproduces the
// whole lattice's trajectory bit for bit, and the slab sums of E and M add up
// to the lattice's.
//
// The exchange is the caller's (NCCL send / receive between ranks, for
// instance, on the planes sl_slab_planes reports) or the library's for slabs
// held by one process (sl_slabs_exchange: device-to-device or peer copies
// ordered by events between the slabs' streams).
#include <cmath>
#include <cstring>

#include "internal.h"

namespace spinmc {
namespace {

constexpr int kMaxParts = 64;

struct SeriesParts {
    const double* p[kMaxParts];
};

__global__ void slab_series_kernel(Ctrl* c, long long base, double* E, double* M)
{
    c->series_base = base;
    c->series_E = E;
    c->series_absm = M;
}

// E[k] = sum of the parts' E, |m|[k] = |sum of the parts' M| / N; each part
// holds nsweeps energies followed by nsweeps magnetisations.  Parts are added
// in order, so the result does not depend on the launch.
__global__ void series_reduce_kernel(SeriesParts parts, int nparts, long long nsweeps, double N,
                                     double* E, double* absm)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nsweeps;
         k += (long long)gridDim.x * blockDim.x) {
        double e = 0.0, m = 0.0;
        for (int q = 0; q < nparts; ++q) {
            e += parts.p[q][k];
            m += parts.p[q][nsweeps + k];
        }
        if (E) E[k] = e;
        if (absm) absm[k] = fabs(m) / N;
    }
}

size_t plane_bytes(const sl_lattice* h)
{
    return h->storage == SL_STORE_I8 ? (size_t)h->P : (size_t)h->P / 8;
}

int check_slab_config(int d, int L, int storage, int z0, int Lz)
{
    if (d != 2 && d != 3) return fail(SL_EINVAL, "d must be 2 or 3 (got %d)", d);
    if (storage != SL_STORE_I8 && storage != SL_STORE_BITS)
        return fail(SL_EINVAL, "slabs hold Ising spins (SL_STORE_I8 or SL_STORE_BITS)");
    if (L < 8 || L % 8)
        return fail(SL_EINVAL, "a slab needs L %% 8 == 0 (got %d): random-number groups of four "
                               "sites must not straddle a plane", L);
    if (storage == SL_STORE_BITS && L % 64)
        return fail(SL_EINVAL, "SL_STORE_BITS needs L %% 64 == 0 (got %d)", L);
    if (z0 < 0 || Lz < 1 || (long long)z0 + Lz > L)
        return fail(SL_EINVAL, "slab planes [%d, %d) outside [0, %d)", z0, z0 + Lz, L);
    const double N = std::pow((double)L, d - 1) * Lz;
    if (N > 4.0e9) return fail(SL_EINVAL, "slab too large: %.0f sites > 4e9", N);
    return SL_OK;
}

bool is_slab(const sl_lattice* h) { return h && h->slab; }

// The slabs must tile the lattice in order: slab 0 starts at plane 0, each
// ends where the next begins, the last ends at L; same shape and sweep count.
int check_ring(sl_lattice* const* slabs, int n)
{
    if (!slabs || n < 1) return fail(SL_EINVAL, "need at least one slab");
    if (n > kMaxParts) return fail(SL_EINVAL, "at most %d slabs", kMaxParts);
    const sl_lattice* a = slabs[0];
    if (!is_slab(a)) return fail(SL_EINVAL, "slab 0 is not a slab handle");
    int z = 0;
    for (int i = 0; i < n; ++i) {
        const sl_lattice* h = slabs[i];
        if (!is_slab(h)) return fail(SL_EINVAL, "slab %d is not a slab handle", i);
        if (h->d != a->d || h->L != a->L || h->storage != a->storage || h->J != a->J ||
            h->replica != a->replica)
            return fail(SL_EINVAL, "slab %d differs from slab 0 in d, L, storage, J or replica", i);
        if (h->z0 != z) return fail(SL_EINVAL, "slab %d starts at plane %d, not %d", i, h->z0, z);
        if (h->sweeps_done != a->sweeps_done || h->next_colour != a->next_colour)
            return fail(SL_EINVAL, "slab %d is at another point of the sweep", i);
        z += h->Lz;
    }
    if (z != a->L) return fail(SL_EINVAL, "the slabs end at plane %d, not %d", z, a->L);
    return SL_OK;
}

void planes(const sl_lattice* h, int c, char** send_lo, char** send_hi, char** recv_lo,
            char** recv_hi)
{
    const size_t pb = plane_bytes(h);
    char* own = (char*)h->spins[c];
    *send_lo = own;
    *send_hi = own + (size_t)(h->Lz - 1) * pb;
    *recv_lo = own - pb;
    *recv_hi = own + (size_t)h->Lz * pb;
}

struct DeviceGuard {
    int saved = -1;
    explicit DeviceGuard() { cudaGetDevice(&saved); }
    ~DeviceGuard()
    {
        if (saved >= 0) cudaSetDevice(saved);
    }
};

int pass(sl_lattice* h, double beta, uint64_t seed, int c)
{
    if (!is_slab(h)) return fail(SL_EINVAL, "not a slab handle");
    if (c != h->next_colour)
        return fail(SL_EINVAL, "colour %d passed out of turn (colour %d is next)", c,
                    h->next_colour);
    if (!(beta >= 0.0) || !std::isfinite(beta))
        return fail(SL_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
    if (h->sweeps_done >= 4294967296LL) return fail(SL_EINVAL, "sweep index would exceed 2^32");
    SweepParams p;
    std::memset(&p, 0, sizeof p);
    p.beta = beta;
    p.seed = seed;
    p.rk = make_round_keys(seed);
    p.beta_f = (float)beta;
    int st = ising_table(h, beta, &p.tab);
    if (st != SL_OK) return st;
    const cudaError_t e = h->storage == SL_STORE_I8 ? ising_i8_pass(h, p, c, h->stream)
                                                    : ising_bits_pass(h, p, c, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab pass");
    h->next_colour = 1 - c;
    if (c == 1) ++h->sweeps_done;
    return SL_OK;
}

int exchange(sl_lattice* const* slabs, int n, int c)
{
    DeviceGuard guard;
    // every slab marks the end of its last pass on its stream ...
    for (int i = 0; i < n; ++i) {
        sl_lattice* h = slabs[i];
        cudaError_t e = cudaSetDevice(h->device);
        if (e == cudaSuccess && !h->ev) e = cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "slab exchange: event");
    }
    // ... and each slab's stream waits for both neighbours' marks, then copies
    // their boundary planes of colour c into its halos
    const size_t pb = plane_bytes(slabs[0]);
    for (int i = 0; i < n; ++i) {
        sl_lattice* h = slabs[i];
        const sl_lattice* lo = slabs[(i + n - 1) % n];
        const sl_lattice* hi = slabs[(i + 1) % n];
        char *slo, *shi, *rlo, *rhi, *a_lo, *a_hi, *b_lo, *b_hi, *x, *y;
        planes(h, c, &slo, &shi, &rlo, &rhi);
        planes(lo, c, &a_lo, &a_hi, &x, &y);
        planes(hi, c, &b_lo, &b_hi, &x, &y);
        cudaError_t e = cudaSetDevice(h->device);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, lo->ev, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, hi->ev, 0);
        if (e == cudaSuccess)
            e = lo->device == h->device
                    ? cudaMemcpyAsync(rlo, a_hi, pb, cudaMemcpyDeviceToDevice, h->stream)
                    : cudaMemcpyPeerAsync(rlo, h->device, a_hi, lo->device, pb, h->stream);
        if (e == cudaSuccess)
            e = hi->device == h->device
                    ? cudaMemcpyAsync(rhi, b_lo, pb, cudaMemcpyDeviceToDevice, h->stream)
                    : cudaMemcpyPeerAsync(rhi, h->device, b_lo, hi->device, pb, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "slab exchange: copy");
    }
    return SL_OK;
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

extern "C" {

int sl_slab_required_bytes(int d, int L, int storage, int z0, int Lz, size_t* bytes)
{
    if (!bytes) return fail(SL_EINVAL, "bytes is NULL");
    const int st = check_slab_config(d, L, storage, z0, Lz);
    if (st != SL_OK) return st;
    *bytes = slab_required_bytes(d, L, storage, Lz);
    return SL_OK;
}

int sl_slab_create(int d, int L, int storage, double J, uint64_t seed, uint32_t replica, int z0,
                   int Lz, void* dev_buf, size_t dev_buf_bytes, void* stream, sl_lattice** out)
{
    if (out) *out = nullptr;
    const int st = check_slab_config(d, L, storage, z0, Lz);
    if (st != SL_OK) return st;
    return create_lattice(d, L, 1, SL_J_UNIFORM, storage, J, nullptr, seed, replica, true, z0, Lz,
                          dev_buf, dev_buf_bytes, stream, out);
}

int sl_slab_planes(const sl_lattice* lat, int colour, void** send_lo, void** send_hi,
                   void** recv_lo, void** recv_hi, size_t* bytes)
{
    if (!is_slab(lat)) return fail(SL_EINVAL, "not a slab handle");
    if (colour != 0 && colour != 1) return fail(SL_EINVAL, "colour must be 0 or 1");
    char *a, *b, *c, *e;
    planes(lat, colour, &a, &b, &c, &e);
    if (send_lo) *send_lo = a;
    if (send_hi) *send_hi = b;
    if (recv_lo) *recv_lo = c;
    if (recv_hi) *recv_hi = e;
    if (bytes) *bytes = plane_bytes(lat);
    return SL_OK;
}

int sl_slab_series(sl_lattice* lat, double* dev_E, double* dev_M)
{
    if (!is_slab(lat)) return fail(SL_EINVAL, "not a slab handle");
    slab_series_kernel<<<1, 1, 0, lat->stream>>>(lat->ctrl, (long long)lat->sweeps_done, dev_E,
                                                 dev_M);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SL_OK : cuda_fail(e, "sl_slab_series");
}

int sl_slab_pass(sl_lattice* lat, double beta, uint64_t seed, int colour)
{
    return pass(lat, beta, seed, colour);
}

int sl_slabs_exchange(sl_lattice* const* slabs, int nslabs, int colour)
{
    if (colour != 0 && colour != 1) return fail(SL_EINVAL, "colour must be 0 or 1");
    const int st = check_ring(slabs, nslabs);
    if (st != SL_OK) return st;
    return exchange(slabs, nslabs, colour);
}

int sl_slabs_sweep(sl_lattice* const* slabs, int nslabs, double beta, int64_t nsweeps,
                   uint64_t seed, double* const* dev_EM)
{
    int st = check_ring(slabs, nslabs);
    if (st != SL_OK) return st;
    if (nsweeps < 0) return fail(SL_EINVAL, "nsweeps must be >= 0");
    if (slabs[0]->next_colour != 0) return fail(SL_EINVAL, "the slabs are inside a sweep");
    if (slabs[0]->sweeps_done + nsweeps > 4294967296LL)
        return fail(SL_EINVAL, "sweep index would exceed 2^32");
    if (nsweeps == 0) return SL_OK;
    DeviceGuard guard;
    for (int i = 0; i < nslabs; ++i) {
        cudaError_t e = cudaSetDevice(slabs[i]->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
        double* part = dev_EM ? dev_EM[i] : nullptr;
        st = sl_slab_series(slabs[i], part, part ? part + nsweeps : nullptr);
        if (st != SL_OK) return st;
    }
    // halos of both colours current before the first pass
    for (int c = 0; c < 2 && st == SL_OK; ++c) st = exchange(slabs, nslabs, c);
    for (int64_t k = 0; k < nsweeps && st == SL_OK; ++k)
        for (int c = 0; c < 2 && st == SL_OK; ++c) {
            for (int i = 0; i < nslabs && st == SL_OK; ++i) {
                const cudaError_t e = cudaSetDevice(slabs[i]->device);
                if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
                st = pass(slabs[i], beta, seed, c);
            }
            if (st == SL_OK) st = exchange(slabs, nslabs, c);
        }
    return st;
}

int sl_series_reduce(const double* const* parts, int nparts, int64_t nsweeps, double N,
                     double* dev_E, double* dev_absm, void* stream)
{
    if (!parts || nparts < 1 || nparts > kMaxParts)
        return fail(SL_EINVAL, "need 1 to %d parts", kMaxParts);
    if (nsweeps < 0 || !(N > 0.0)) return fail(SL_EINVAL, "bad nsweeps or N");
    if (nsweeps == 0) return SL_OK;
    SeriesParts sp;
    std::memset(&sp, 0, sizeof sp);
    for (int q = 0; q < nparts; ++q) {
        if (!parts[q]) return fail(SL_EINVAL, "part %d is NULL", q);
        sp.p[q] = parts[q];
    }
    long long g = (nsweeps + 255) / 256;
    if (g > 1024) g = 1024;
    series_reduce_kernel<<<(int)g, 256, 0, (cudaStream_t)stream>>>(sp, nparts, nsweeps, N, dev_E,
                                                                   dev_absm);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SL_OK : cuda_fail(e, "sl_series_reduce");
}

}  // extern "C"
