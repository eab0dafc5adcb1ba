// Energy and magnetisation of an Ising configuration without any device
// allocation: the per-block partial sums and the arrival counter that the
// fixed-order reduction needs live in one file-scope static device array
// instead of a caller or library allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's device-memory pool (where a raw allocation would bypass the
// pool's accounting or exceed its budget), or a latency-critical loop that
// must not pay for an allocation and its implicit synchronisation.  They pass
// only their input configuration and a two-double output.
//
// The array is StaticScratch below (about 192 KiB); every GPU that loads this
// library holds it until the process exits.  All calls share it, so calls
// that overlap on the GPU (on different streams, or from different threads)
// race; calls issued one after another on a stream are safe.  The arrival
// counter is cleared at the start of every call.
//
// The host needs the array's device address, which it looks up with the
// device current on the first call there.  The address belongs to the
// device's context: after cudaDeviceReset a new context loads the module
// again, possibly elsewhere, so the cache keys each address by the context's
// unique id and looks the address up again when the id changes.
#include <cmath>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"

namespace spinmc {
namespace {

constexpr int kStaticBlocks = 4096;                    // largest grid the scratch serves
constexpr long long kStaticSitesPerBlock = 65536;      // sites one block reduces
constexpr long long kStaticMaxSites = kStaticBlocks * kStaticSitesPerBlock;  // 2^28

struct StaticScratch {
    Ctrl ctrl;  // only the arrival counter `done` is used
    Partial partials[kStaticBlocks];
};

static __device__ __align__(256) StaticScratch g_static_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticScratch* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];  // context id the address belongs to

// E = -J sum_i sum_mu s_i s_{i+e_mu} (nearest-neighbour pairs, each once) and M = sum_i s_i of a
// natural-order +-1 configuration; block b reduces sites
// [b * kStaticSitesPerBlock, (b + 1) * kStaticSitesPerBlock).
__global__ void __launch_bounds__(256) static_measure_kernel(const int8_t* s, long long N, int L,
                                                             int d, double J, double* out,
                                                             StaticScratch* scr)
{
    __shared__ long long red[32];
    const long long lo = (long long)blockIdx.x * kStaticSitesPerBlock;
    const long long hi = lo + kStaticSitesPerBlock < N ? lo + kStaticSitesPerBlock : N;
    long long bond = 0, down = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int x = (int)(i % L);
        const long long r = i / L;
        const int y = (int)(r % L);
        const int z = (int)(r / L);
        const int si = s[i];
        const long long xp = i - x + (x == L - 1 ? 0 : x + 1);
        const long long yp = i + (long long)L * ((y == L - 1 ? 0 : y + 1) - y);
        int h = s[xp] + s[yp];
        if (d == 3) h += s[i + (long long)L * L * ((z == L - 1 ? 0 : z + 1) - z)];
        bond += si * h;
        down += si < 0;
    }
    Partial mine;
    mine.i0 = block_sum(bond, red);
    mine.i1 = block_sum(down, red);
    mine.f[0] = mine.f[1] = mine.f[2] = mine.f[3] = 0.0;
    finish_pass(&scr->ctrl, scr->partials, mine, [&](const Partial& tot) {
        out[0] = -J * (double)tot.i0;
        out[1] = (double)(N - 2 * tot.i1);
    });
}

// The driver's cuCtxGetId, fetched through the runtime (no link against the
// driver library), or null where the driver does not offer it.
PFN_cuCtxGetId_v12000 ctx_get_id_fn()
{
    static PFN_cuCtxGetId_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuCtxGetId_v12000)p;
    }();
    return fn;
}

// Unique id of the current context, or 0 if there is none yet (or no way to ask).
unsigned long long current_ctx_id()
{
    unsigned long long id = 0;
    const PFN_cuCtxGetId_v12000 fn = ctx_get_id_fn();
    if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the static scratch on the current device.  It is looked
// up (cudaGetSymbolAddress, with the device current) on the first call on a
// device and again only when the device's context has changed since, as
// after cudaDeviceReset.
int scratch_for_current_device(StaticScratch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SL_EINVAL, "device %d out of range", dev);
    unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        if (ctx == 0) ctx = current_ctx_id();  // the lookup made the primary context current
        g_scratch_addr[dev] = (StaticScratch*)p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return SL_OK;
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

extern "C" int sl_ising_measure_static(int d, int L, double J, const int8_t* dev_spins,
                                       double* dev_out, void* stream)
{
    if (d != 2 && d != 3) return fail(SL_EINVAL, "d must be 2 or 3 (got %d)", d);
    if (L < 2 || (L & 1)) return fail(SL_EINVAL, "L must be even and >= 2 (got %d)", L);
    if (!dev_spins || !dev_out) return fail(SL_EINVAL, "NULL device pointer");
    if (!std::isfinite(J)) return fail(SL_EINVAL, "J must be finite");
    // the site count in FP64 first: L^3 overflows 64-bit integers for L near 2^21
    const double Nd = std::pow((double)L, d);
    if (Nd > (double)kStaticMaxSites)
        return fail(SL_EINVAL,
                    "%.0f sites exceed the %lld this entry point's static scratch serves",
                    Nd, kStaticMaxSites);
    const long long N = (long long)L * L * (d == 3 ? L : 1);
    StaticScratch* scr = nullptr;
    const int st = scratch_for_current_device(&scr);
    if (st != SL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(&scr->ctrl.done, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "clear arrival counter");
    const int grid = (int)((N + kStaticSitesPerBlock - 1) / kStaticSitesPerBlock);
    static_measure_kernel<<<grid, 256, 0, s>>>(dev_spins, N, L, d, J, dev_out, scr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "static measure launch");
    return SL_OK;
}
