// The C ABI of libspinmc (include/spinmc.h): argument checking, the layout
// of the caller's device buffer, the exact Ising acceptance thresholds,
// sweep scheduling (plain launches or replays of a captured CUDA graph), and
// measurement / state transfer.  Every compute step runs in the kernels of
// the per-model .cu files.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace spinmc {

static thread_local char g_msg[512];

int fail(int status, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(SL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {

constexpr int kGraphSweeps = 32;  // sweeps in the long graph; a one-sweep graph takes the rest

struct Layout {
    size_t spin_colour;   // bytes of one colour's spins
    size_t bond_array;    // bytes of one (colour, direction) bond array
    size_t staging;
    size_t off_spins[2];
    size_t off_bonds[2][3];
    size_t off_staging, off_ctrl, off_partials, total;
};

int check_config(int d, int L, int n, int j_layout, int storage)
{
    if (d != 2 && d != 3) return fail(SL_EINVAL, "d must be 2 or 3 (got %d)", d);
    if (L < 2 || (L & 1)) return fail(SL_EINVAL, "L must be even and >= 2 (got %d)", L);
    if (j_layout != SL_J_UNIFORM && j_layout != SL_J_BONDS)
        return fail(SL_EINVAL, "unknown coupling layout %d", j_layout);
    const double N = std::pow((double)L, d);
    if (N > 4.0e9) return fail(SL_EINVAL, "lattice too large: L^d = %.0f > 4e9", N);
    switch (storage) {
    case SL_STORE_I8:
        if (n != 1) return fail(SL_EINVAL, "SL_STORE_I8 needs n = 1");
        break;
    case SL_STORE_BITS:
        if (n != 1) return fail(SL_EINVAL, "SL_STORE_BITS needs n = 1");
        if (L % 64) return fail(SL_EINVAL, "SL_STORE_BITS needs L %% 64 == 0 (got %d)", L);
        if (j_layout != SL_J_UNIFORM) return fail(SL_EINVAL, "SL_STORE_BITS needs SL_J_UNIFORM");
        break;
    case SL_STORE_F32_ANGLE:
        if (n != 2) return fail(SL_EINVAL, "SL_STORE_F32_ANGLE needs n = 2");
        break;
    case SL_STORE_F32_VEC:
        if (n != 3) return fail(SL_EINVAL, "SL_STORE_F32_VEC needs n = 3");
        break;
    default:
        return fail(SL_EINVAL, "unknown storage %d", storage);
    }
    return SL_OK;
}

// Lz planes along the slowest axis (L for a whole lattice); a slab stores Lz + 2
// planes per colour (halo planes before and after its own).
Layout make_layout(int d, int L, int n, int j_layout, int storage, int Lz = 0, bool slab = false)
{
    Layout y;
    if (Lz <= 0) Lz = L;
    const size_t P = (size_t)L * (d == 3 ? L : 1) / 2;  // sites of one colour per plane
    const size_t H = P * Lz, N = 2 * H;
    const size_t Hs = P * (Lz + (slab ? 2 : 0));          // stored entries per colour
    switch (storage) {
    case SL_STORE_I8: y.spin_colour = Hs; break;
    case SL_STORE_BITS: y.spin_colour = Hs / 8; break;
    case SL_STORE_F32_ANGLE: y.spin_colour = 4 * Hs; break;
    default: y.spin_colour = 12 * Hs; break;
    }
    const size_t bond_elem = n == 1 ? 1 : 4;
    y.bond_array = j_layout == SL_J_BONDS ? H * bond_elem : 0;  // slabs have uniform J
    const size_t nat_elem = n == 1 ? 1 : (n == 2 ? 4 : 12);
    y.staging = N * nat_elem;
    if (j_layout == SL_J_BONDS && d * N * bond_elem > y.staging) y.staging = d * N * bond_elem;
    size_t off = 0;
    for (int c = 0; c < 2; ++c) {
        y.off_spins[c] = off;
        off += align_up(y.spin_colour);
    }
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < 3; ++mu) {
            y.off_bonds[c][mu] = off;
            if (j_layout == SL_J_BONDS && mu < d) off += align_up(y.bond_array);
        }
    y.off_staging = off;
    off += align_up(y.staging);
    y.off_ctrl = off;
    off += align_up(sizeof(Ctrl));
    y.off_partials = off;
    off += align_up(sizeof(Partial) * (kMaxBlocks + 1));
    y.total = off;
    return y;
}

__global__ void set_series_kernel(Ctrl* c, long long base, double* E, double* m)
{
    c->series_base = base;
    c->series_E = E;
    c->series_absm = m;
}

__global__ void set_t_kernel(Ctrl* c, unsigned long long t) { c->t = t; }

}  // namespace

size_t slab_required_bytes(int d, int L, int storage, int Lz)
{
    return make_layout(d, L, 1, SL_J_UNIFORM, storage, Lz, true).total;
}

// Exact integer thresholds for the Ising classes (see ising_i8.cu).  Class k
// has s_i h_i sign(J) = 2d - 2k (+-1 couplings) or 2d - k (couplings that may
// be zero) and dE = 2 J s_i h_i evaluated exactly as the definition does;
// u < exp(-beta dE) 2^32 is the same test as u <= ceil(exp(-beta dE) 2^32) - 1
// for integer u.
int ising_table(const sl_lattice* h, double beta, IsingTable* tab)
{
    const int d = h->d;
    tab->sigma_neg = h->J < 0.0;
    tab->scheme = h->bonds_have_zero ? 1 : 0;
    tab->ncmp = tab->scheme ? 2 * d : d;
    tab->heatbath = h->update == SL_UPDATE_HEATBATH;
    for (int k = 0; k < 6; ++k) tab->thr[k] = 0xFFFFFFFFu;
    for (int k = 0; k < 13; ++k) tab->hb[k] = 0u;
    tab->sw_thr = 0u;
    tab->sw_never = 1;
    if (h->update == SL_UPDATE_SW) {
        // Swendsen-Wang: a satisfied bond is active iff u < (1 - exp(-2 beta |J|)) 2^32,
        // the same test as u <= ceil(x) - 1 for integer u
        const double x = (1.0 - std::exp(-2.0 * beta * std::fabs(h->J))) * 4294967296.0;
        if (x > 0.0) {
            double T = std::ceil(x) - 1.0;
            if (T > 4294967295.0) T = 4294967295.0;
            tab->sw_thr = (uint32_t)T;
            tab->sw_never = 0;
        }
        return SL_OK;
    }
    if (h->update == SL_UPDATE_HEATBATH) {
        // heat-bath: s_i = +1 iff u < 2^32 / (1 + exp(-beta a)), a = 2 J h,
        // h = sum_k Jb_k s_k in [-2d, 2d]; u <= ceil(x) - 1 is the same test
        for (int hs = -2 * d; hs <= 2 * d; ++hs) {
            const double a = 2.0 * h->J * (double)hs;
            const double x = 4294967296.0 / (1.0 + std::exp(-beta * a));
            if (!(x > 0.0))
                return fail(SL_EINVAL, "beta = %g too large for the heat-bath table", beta);
            double T = std::ceil(x) - 1.0;
            if (T > 4294967295.0) T = 4294967295.0;
            tab->hb[hs + 2 * d] = (uint32_t)T;
        }
        return SL_OK;
    }
    for (int k = 0; k < tab->ncmp; ++k) {
        const int e = tab->scheme ? 2 * d - k : 2 * d - 2 * k;
        const int sh = tab->sigma_neg ? -e : e;
        const double dE = 2.0 * h->J * (double)sh;
        if (dE <= 0.0) continue;
        const double x = std::exp(-beta * dE) * 4294967296.0;
        if (!(x > 0.0))
            return fail(SL_EINVAL, "beta = %g too large: exp(-beta dE) underflows", beta);
        double T = std::ceil(x) - 1.0;
        if (T > 4294967295.0) T = 4294967295.0;
        tab->thr[k] = (uint32_t)T;
    }
    return SL_OK;
}

namespace {

int model_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count, cudaStream_t s)
{
    cudaError_t e = cudaErrorInvalidValue;
    if (h->storage == SL_STORE_I8) e = ising_i8_sweeps(h, p, count, s);
    else if (h->storage == SL_STORE_BITS) e = ising_bits_sweeps(h, p, count, s);
    else if (h->n > 1) e = on_sweeps(h, p, count, s);
    return e == cudaSuccess ? SL_OK : cuda_fail(e, "sweep launch");
}

// Capture `count` sweeps into an executable graph on the private capture stream.
int capture_sweeps(sl_lattice* h, const SweepParams& p, int count, cudaGraphExec_t* out)
{
    *out = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const int st = model_sweeps(h, p, count, h->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (st != SL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    return SL_OK;
}

void drop_graphs(sl_lattice* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph1) cudaGraphExecDestroy(h->graph1);
    h->graph = h->graph1 = nullptr;
}

// The two graphs of the sweep parameters p (kGraphSweeps sweeps and one
// sweep), captured again only when p or an option that shapes the launches
// has changed.  The kernels read the sweep index and the series pointers
// from the device control block, so one capture serves every later call.
int ensure_graph(sl_lattice* h, const SweepParams& p)
{
    uint64_t key[4];
    std::memcpy(&key[0], &p.beta, 8);
    key[1] = p.seed;
    key[2] = ((uint64_t)h->kernel << 48) ^ ((uint64_t)h->rows << 32) ^
             ((uint64_t)h->fast_math << 24) ^ ((uint64_t)h->update << 40) ^
             (uint64_t)h->renorm_every;
    key[3] = ((uint64_t)h->multihit << 16) ^ (uint64_t)h->tile ^
             ((uint64_t)h->blocks_per_sm << 40);
    if (h->graph && h->graph1 && std::memcmp(key, h->graph_key, sizeof key) == 0) return SL_OK;
    drop_graphs(h);
    int st = capture_sweeps(h, p, kGraphSweeps, &h->graph);
    if (st == SL_OK) st = capture_sweeps(h, p, 1, &h->graph1);
    if (st != SL_OK) {
        drop_graphs(h);
        return st;
    }
    h->graph_sweeps = kGraphSweeps;
    std::memcpy(h->graph_key, key, sizeof key);
    return SL_OK;
}

int sync_and_check(sl_lattice* h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned err = 0;
    e = cudaMemcpy(&err, &h->ctrl->error, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read error word");
    if (err & 1u)
        return fail(SL_ETIMEOUT, "a kernel's bounded wait for its staged copies ran out; the "
                                 "configuration is not valid");
    return SL_OK;
}

size_t nat_bytes(const sl_lattice* h)
{
    return (size_t)h->N * (h->n == 1 ? 1 : (h->n == 2 ? 4 : 12));
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

extern "C" {

int sl_required_bytes(int d, int L, int n, int j_layout, int storage, size_t* bytes)
{
    if (!bytes) return fail(SL_EINVAL, "bytes is NULL");
    const int st = check_config(d, L, n, j_layout, storage);
    if (st != SL_OK) return st;
    *bytes = make_layout(d, L, n, j_layout, storage).total;
    return SL_OK;
}

int sl_create(int d, int L, int n, int j_layout, int storage, double J, const void* J_bonds,
              uint64_t seed, uint32_t replica, void* dev_buf, size_t dev_buf_bytes, void* stream,
              sl_lattice** out)
{
    return create_lattice(d, L, n, j_layout, storage, J, J_bonds, seed, replica, false, 0, L,
                          dev_buf, dev_buf_bytes, stream, out);
}

}  // extern "C"

namespace spinmc {

int create_lattice(int d, int L, int n, int j_layout, int storage, double J, const void* J_bonds,
                   uint64_t seed, uint32_t replica, bool slab, int z0, int Lz, void* dev_buf,
                   size_t dev_buf_bytes, void* stream, sl_lattice** out)
{
    if (!out) return fail(SL_EINVAL, "out is NULL");
    *out = nullptr;
    int st = check_config(d, L, n, j_layout, storage);
    if (st != SL_OK) return st;
    if (!std::isfinite(J)) return fail(SL_EINVAL, "J must be finite");
    if (j_layout == SL_J_BONDS && !J_bonds) return fail(SL_EINVAL, "SL_J_BONDS needs J_bonds");
    const Layout y = make_layout(d, L, n, j_layout, storage, Lz, slab);
    void* owned = nullptr;
    if (!dev_buf) {
        const cudaError_t e = cudaMalloc(&owned, y.total);
        if (e != cudaSuccess) return fail(SL_ENOMEM, "cudaMalloc(%zu): %s", y.total,
                                          cudaGetErrorString(e));
        dev_buf = owned;
        dev_buf_bytes = y.total;
    }
    if ((uintptr_t)dev_buf % kAlign) {
        return fail(SL_EINVAL, "dev_buf must be %zu-byte aligned", kAlign);
    }
    if (dev_buf_bytes < y.total) {
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "dev_buf holds %zu bytes, %zu needed", dev_buf_bytes, y.total);
    }
    sl_lattice* h = new (std::nothrow) sl_lattice();
    if (!h) {
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "host allocation failed");
    }
    char* base = (char*)dev_buf;
    h->d = d;
    h->L = L;
    h->n = n;
    h->j_layout = j_layout;
    h->storage = storage;
    h->P = (int64_t)L * (d == 3 ? L : 1) / 2;
    h->slab = slab ? 1 : 0;
    h->z0 = z0;
    h->Lz = Lz;
    h->N = 2 * h->P * Lz;
    h->H = h->N / 2;
    h->W = L / 2;
    h->J = J;
    h->init_seed = seed;
    h->replica = replica;
    h->sweeps_done = 0;
    h->stream = (cudaStream_t)stream;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1)
            sms = 1;
        h->sms = sms;
        h->device = dev;
    }
    // a slab's colour arrays start with a halo plane: spins[c] points at its
    // first own plane, the halos sit at planes -1 and Lz
    const size_t halo_bytes =
        !slab ? 0 : (storage == SL_STORE_I8 ? (size_t)h->P : (size_t)h->P / 8);
    for (int c = 0; c < 2; ++c) {
        h->spins[c] = base + y.off_spins[c] + halo_bytes;
        for (int mu = 0; mu < 3; ++mu)
            h->bonds[c][mu] =
                (j_layout == SL_J_BONDS && mu < d) ? (void*)(base + y.off_bonds[c][mu]) : nullptr;
    }
    h->staging = base + y.off_staging;
    h->staging_bytes = y.staging;
    h->ctrl = (Ctrl*)(base + y.off_ctrl);
    h->partials = (Partial*)(base + y.off_partials);
    h->bonds_have_zero = false;
    h->renorm_every = 16;
    h->fast_math = 0;
    h->kernel = 0;
    h->rows = 0;
    h->blocks_per_sm = 0;
    h->use_graph = 1;
    h->update = 0;
    h->multihit = 0;
    h->tile = 16;
    h->graph = nullptr;
    h->graph1 = nullptr;
    h->graph_sweeps = 0;
    h->next_colour = 0;
    h->ev = nullptr;
    h->owned_buf = owned;
    h->ws = nullptr;
    h->ws_bytes = 0;
    h->ws_owned = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "cudaStreamCreate");
        if (owned) cudaFree(owned);
        delete h;
        return st;
    }
    e = cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->partials + kMaxBlocks, 0, sizeof(Partial), h->stream);
    if (e == cudaSuccess && storage == SL_STORE_I8) e = ising_i8_init(h, h->stream);
    if (e == cudaSuccess && storage == SL_STORE_BITS) e = ising_bits_init(h, h->stream);
    if (e == cudaSuccess && n > 1) e = on_init(h, h->stream);
    if (e == cudaSuccess && j_layout == SL_J_BONDS) {
        unsigned* flags = (unsigned*)h->partials;
        e = cudaMemsetAsync(flags, 0, sizeof(unsigned), h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->staging, J_bonds, (size_t)d * h->N * (n == 1 ? 1 : 4),
                                cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess && n == 1)
            e = ising_bonds_scatter(h, (const int8_t*)h->staging, flags, h->stream);
        if (e == cudaSuccess && n > 1)
            e = float_bonds_scatter(h, (const float*)h->staging, h->stream);
        unsigned f = 0;
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaMemcpy(&f, flags, sizeof f, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && (f & 2u)) {
            sl_destroy(h);
            return fail(SL_EINVAL, "Ising couplings must be -1, 0 or +1");
        }
        h->bonds_have_zero = (f & 1u) != 0;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "sl_create");
        sl_destroy(h);
        return st;
    }
    *out = h;
    return SL_OK;
}

int sweep_plain(const sl_lattice* h, const SweepParams& p, int64_t count, cudaStream_t s)
{
    return model_sweeps(h, p, count, s);
}

int sweep_params(const sl_lattice* h, double beta, uint64_t seed, SweepParams* p)
{
    std::memset(p, 0, sizeof *p);
    p->beta = beta;
    p->seed = seed;
    p->rk = make_round_keys(seed);
    p->beta_f = (float)beta;
    return h->n == 1 ? ising_table(h, beta, &p->tab) : SL_OK;
}

cudaError_t set_sweep_index(const sl_lattice* h, int64_t t, cudaStream_t s)
{
    set_t_kernel<<<1, 1, 0, s>>>(h->ctrl, (unsigned long long)t);
    return cudaGetLastError();
}

cudaError_t clear_series(const sl_lattice* h, cudaStream_t s)
{
    set_series_kernel<<<1, 1, 0, s>>>(h->ctrl, (long long)h->sweeps_done, nullptr, nullptr);
    return cudaGetLastError();
}

void forget_graphs(sl_lattice* h) { drop_graphs(h); }

}  // namespace spinmc

extern "C" {

int sl_sweep_series(sl_lattice* h, double beta, int64_t nsweeps, uint64_t seed, double* dev_E,
                    double* dev_absm)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    if (h->slab)
        return fail(SL_EINVAL, "a slab sweeps by sl_slab_pass between halo exchanges "
                               "(or sl_slabs_sweep)");
    if (nsweeps < 0) return fail(SL_EINVAL, "nsweeps must be >= 0");
    if (!(beta >= 0.0) || !std::isfinite(beta))
        return fail(SL_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
    if (h->sweeps_done + nsweeps > 4294967296LL)
        return fail(SL_EINVAL, "sweep index would exceed 2^32");
    if (h->multihit > 0 && (h->sweeps_done + nsweeps) * (int64_t)h->multihit > 4294967296LL)
        return fail(SL_EINVAL, "multi-hit index t*k would exceed 2^32");
    if (nsweeps == 0) return SL_OK;
    SweepParams p;
    std::memset(&p, 0, sizeof p);
    p.beta = beta;
    p.seed = seed;
    p.rk = make_round_keys(seed);
    p.beta_f = (float)beta;
    if (h->n == 1) {
        const int st = ising_table(h, beta, &p.tab);
        if (st != SL_OK) return st;
    }
    set_series_kernel<<<1, 1, 0, h->stream>>>(h->ctrl, (long long)h->sweeps_done, dev_E, dev_absm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "series setup");
    int64_t left = nsweeps;
    if (h->use_graph && nsweeps >= 2) {
        // whole runs of kGraphSweeps sweeps, then single-sweep replays
        const int st = ensure_graph(h, p);
        if (st != SL_OK) return st;
        while (left > 0) {
            const bool big = left >= h->graph_sweeps;
            e = cudaGraphLaunch(big ? h->graph : h->graph1, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            left -= big ? h->graph_sweeps : 1;
        }
    }
    if (left > 0) {
        const int st = model_sweeps(h, p, left, h->stream);
        if (st != SL_OK) return st;
    }
    h->sweeps_done += nsweeps;
    return SL_OK;
}

int sl_sweep(sl_lattice* h, double beta, int64_t nsweeps, uint64_t seed)
{
    return sl_sweep_series(h, beta, nsweeps, seed, nullptr, nullptr);
}

int sl_measure(sl_lattice* h, double* energy, double* magnetisation)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    cudaError_t e = cudaErrorInvalidValue;
    if (h->storage == SL_STORE_I8) e = ising_i8_measure(h, h->stream);
    else if (h->storage == SL_STORE_BITS) e = ising_bits_measure(h, h->stream);
    else if (h->n > 1) e = on_measure(h, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "measure launch");
    int st = sync_and_check(h);
    if (st != SL_OK) return st;
    double obs[4];
    e = cudaMemcpy(obs, h->ctrl->obs, sizeof obs, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read observables");
    if (energy) *energy = obs[0];
    if (magnetisation) {
        double m2 = 0.0;
        for (int a = 0; a < h->n; ++a) {
            magnetisation[a] = obs[1 + a];
            m2 += obs[1 + a] * obs[1 + a];
        }
        magnetisation[h->n] = std::sqrt(m2) / (double)h->N;
    }
    return SL_OK;
}

int sl_get_spins(sl_lattice* h, void* dst)
{
    if (!h || !dst) return fail(SL_EINVAL, "NULL argument");
    cudaError_t e = cudaErrorInvalidValue;
    if (h->storage == SL_STORE_I8) e = ising_i8_gather(h, (int8_t*)h->staging, h->stream);
    else if (h->storage == SL_STORE_BITS) e = ising_bits_gather(h, (int8_t*)h->staging, h->stream);
    else if (h->n > 1) e = on_layout(h, (float*)h->staging, 1, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst, h->staging, nat_bytes(h), cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_get_spins");
    return sync_and_check(h);
}

int sl_set_spins(sl_lattice* h, const void* src)
{
    if (!h || !src) return fail(SL_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(h->staging, src, nat_bytes(h), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) {
        if (h->storage == SL_STORE_I8) e = ising_i8_scatter(h, (const int8_t*)h->staging, h->stream);
        else if (h->storage == SL_STORE_BITS)
            e = ising_bits_scatter(h, (const int8_t*)h->staging, h->stream);
        else if (h->n > 1) e = on_layout(h, (float*)h->staging, 0, h->stream);
        else e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(e, "sl_set_spins");
    return sync_and_check(h);
}

int sl_get_state(sl_lattice* h, uint64_t* init_seed, int64_t* sweeps_done)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    if (init_seed) *init_seed = h->init_seed;
    if (sweeps_done) *sweeps_done = h->sweeps_done;
    return SL_OK;
}

int sl_set_state(sl_lattice* h, int64_t sweeps_done)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    if (sweeps_done < 0 || sweeps_done > 4294967296LL)
        return fail(SL_EINVAL, "sweeps_done out of range");
    set_t_kernel<<<1, 1, 0, h->stream>>>(h->ctrl, (unsigned long long)sweeps_done);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sl_set_state");
    h->sweeps_done = sweeps_done;
    h->next_colour = 0;
    return SL_OK;
}

int sl_set_option(sl_lattice* h, int option, int64_t value)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    switch (option) {
    case SL_OPT_RENORM_EVERY:
        if (value < 0 || value > (1 << 30)) return fail(SL_EINVAL, "renorm_every out of range");
        h->renorm_every = (int)value;
        return SL_OK;
    case SL_OPT_FAST_MATH:
        if (value != 0 && value != 1) return fail(SL_EINVAL, "fast_math must be 0 or 1");
        h->fast_math = (int)value;
        return SL_OK;
    case SL_OPT_KERNEL:
        if (value < 0 || value > 4) return fail(SL_EINVAL, "kernel must be 0, 1, 2, 3 or 4");
        if (value == 4) {
            const int kept = h->kernel;
            h->kernel = 4;
            const bool ok = on_tile_ok(h);
            h->kernel = kept;
            if (!ok)
                return fail(SL_EINVAL, "kernel 4 (staged tiles) is for 3D Heisenberg spins with "
                                       "uniform J, L in {64, 128, 256, 512}, Metropolis and "
                                       "accurate functions");
        }
        if (value == 3 && (h->n != 3 || h->j_layout != SL_J_UNIFORM || h->W % 32 != 0))
            return fail(SL_EINVAL, "kernel 3 (single-column streaming) is for Heisenberg spins "
                                   "with uniform J and L %% 64 == 0");
        if (value == 1 && h->storage == SL_STORE_BITS)
            return fail(SL_EINVAL, "bit storage has only the streaming kernel");
        if (value == 2 && h->n == 1 && (h->W % 16 != 0 || h->bonds_have_zero))
            return fail(SL_EINVAL, "the streaming kernel needs L %% 32 == 0 and +-1 couplings");
        if (value == 2 && h->n > 1 &&
            (h->j_layout != SL_J_UNIFORM || (h->n == 3 && h->W % 32 != 0) ||
             (h->n == 2 && (h->d != 2 || h->W % 64 != 0))))
            return fail(SL_EINVAL, "the streaming kernel needs uniform J and L %% 64 == 0 "
                                   "(Heisenberg) or a 2D lattice with L %% 128 == 0 (XY)");
        h->kernel = (int)value;
        return SL_OK;
    case SL_OPT_ROWS:
        if (value < 0 || (value > 0 && (h->Lz % value != 0)))
            return fail(SL_EINVAL, "rows must be 0 (automatic) or divide the planes held");
        h->rows = (int)value;
        return SL_OK;
    case SL_OPT_BLOCKS_PER_SM:
        if (value < 0 || value > 64) return fail(SL_EINVAL, "blocks_per_sm must be in [0, 64]");
        h->blocks_per_sm = (int)value;
        return SL_OK;
    case SL_OPT_GRAPH:
        if (value != 0 && value != 1) return fail(SL_EINVAL, "graph must be 0 or 1");
        h->use_graph = (int)value;
        return SL_OK;
    case SL_OPT_UPDATE:
        if (value != SL_UPDATE_METROPOLIS && value != SL_UPDATE_HEATBATH && value != SL_UPDATE_SW)
            return fail(SL_EINVAL, "update must be 0 (Metropolis), 1 (heat-bath) or 2 "
                                   "(Swendsen-Wang)");
        if (value == SL_UPDATE_HEATBATH && h->storage == SL_STORE_BITS)
            return fail(SL_EINVAL, "the heat-bath rule needs byte (Ising) or FP32 storage");
        if (value == SL_UPDATE_SW && h->storage != SL_STORE_I8)
            return fail(SL_EINVAL, "Swendsen-Wang updates need Ising byte storage");
        if (value == SL_UPDATE_SW && h->slab)
            return fail(SL_EINVAL, "Swendsen-Wang updates need the whole lattice, not a slab");
        if (value != SL_UPDATE_METROPOLIS && h->multihit > 0)
            return fail(SL_EINVAL, "multi-hit sweeps use the Metropolis rule");
        if (value == SL_UPDATE_SW) {
            if (h->j_layout != SL_J_UNIFORM)
                return fail(SL_EINVAL, "Swendsen-Wang updates need a uniform coupling J");
            if (h->N > 1073741824LL)
                return fail(SL_EINVAL, "Swendsen-Wang updates need N <= 2^30");
            const size_t need = sw_workspace_bytes(h->d, h->L);
            if (h->ws_bytes < need) {
                if (!h->owned_buf)
                    return fail(SL_EINVAL, "Swendsen-Wang updates need a workspace of %zu bytes "
                                           "(sl_attach_workspace)", need);
                void* p = nullptr;
                const cudaError_t e = cudaMalloc(&p, need);
                if (e != cudaSuccess)
                    return fail(SL_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
                if (h->ws_owned) cudaFree(h->ws_owned);
                h->ws_owned = p;
                h->ws = p;
                h->ws_bytes = need;
            }
        }
        h->update = (int)value;
        return SL_OK;
    case SL_OPT_MULTIHIT:
        if (value < 0 || value > 65536) return fail(SL_EINVAL, "multihit must be in [0, 65536]");
        if (value > 0 && (h->storage != SL_STORE_I8 || h->j_layout != SL_J_UNIFORM ||
                          h->update != 0 || h->slab))
            return fail(SL_EINVAL, "multi-hit sweeps need a whole lattice of Ising bytes, "
                                   "uniform J and Metropolis");
        if (value > 0 && !tile_size_ok(h->d, h->L, h->tile))
            return fail(SL_EINVAL, "tile side %d does not fit L = %d (L %% 2T == 0)", h->tile,
                        h->L);
        h->multihit = (int)value;
        return SL_OK;
    case SL_OPT_TILE:
        if (!tile_size_ok(h->d, h->L, (int)value))
            return fail(SL_EINVAL, "tile side must be 8, 16, 32, 64 (2D) or 8, 16 (3D) with "
                                   "L %% 2T == 0");
        h->tile = (int)value;
        return SL_OK;
    default:
        return fail(SL_EINVAL, "unknown option %d", option);
    }
}

void sl_destroy(sl_lattice* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->owned_buf) cudaFree(h->owned_buf);
    if (h->ws_owned) cudaFree(h->ws_owned);
    delete h;
}

int sl_workspace_bytes(const sl_lattice* h, int update, size_t* bytes)
{
    if (!h || !bytes) return fail(SL_EINVAL, "NULL argument");
    if (update != SL_UPDATE_METROPOLIS && update != SL_UPDATE_HEATBATH && update != SL_UPDATE_SW)
        return fail(SL_EINVAL, "unknown update rule %d", update);
    *bytes = update == SL_UPDATE_SW ? sw_workspace_bytes(h->d, h->L) : 0;
    return SL_OK;
}

int sl_attach_workspace(sl_lattice* h, void* dev_buf, size_t bytes)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    if (dev_buf && (uintptr_t)dev_buf % kAlign)
        return fail(SL_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    if (h->update == SL_UPDATE_SW && bytes < sw_workspace_bytes(h->d, h->L))
        return fail(SL_ENOMEM, "workspace holds %zu bytes, %zu needed", bytes,
                    sw_workspace_bytes(h->d, h->L));
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (h->ws_owned) {
        cudaFree(h->ws_owned);
        h->ws_owned = nullptr;
    }
    h->ws = dev_buf;
    h->ws_bytes = dev_buf ? bytes : 0;
    drop_graphs(h);
    return SL_OK;
}

const char* sl_strerror(int status)
{
    switch (status) {
    case SL_OK: return "ok";
    case SL_EINVAL: return "invalid argument";
    case SL_ENOMEM: return "out of memory or buffer too small";
    case SL_ECUDA: return "CUDA runtime error";
    case SL_ETIMEOUT: return "device wait timed out";
    case SL_EDEVICE: return "a kernel reported a failure";
    default: return "unknown status";
    }
}

int sl_last_error(char* msg, size_t cap)
{
    const size_t len = std::strlen(g_msg);
    if (msg && cap) {
        const size_t k = len < cap - 1 ? len : cap - 1;
        std::memcpy(msg, g_msg, k);
        msg[k] = 0;
    }
    return (int)len;
}

}  // extern "C"
