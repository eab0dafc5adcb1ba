// The launch-shape autotuner of the single-lattice sweeps.
//
// The row-streaming kernels give each thread a column chunk and R rows to
// march through, and cover the lattice with a grid of blocks; R and the grid
// change only the launch shape, never a decision (every random number is
// keyed by its site), so any choice gives the same chain.  sl_autotune times
// trial sweeps of every shape in a small set (R dividing the planes, grids
// capped at 0, 2, 4, 8 or 16 blocks per SM, and for Heisenberg spins the
// column-pair, single-column or staged-tile kernel where each applies) on the
// lattice itself, restores its spins and sweep counter, and keeps the
// fastest.  Choices can be cached
// in a file of JSON lines, one per (device, d, L, n, storage, couplings,
// update rule, fast math), read before timing and appended after.
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

namespace spinmc {
namespace {

constexpr int kRows[] = {1, 2, 4, 8, 16, 32};
constexpr int kCaps[] = {0, 2, 4, 8, 16};

struct TuneKey {
    std::string device;
    int sms, d, L, n, storage, j_layout, update, fast;
};

TuneKey key_of(const sl_lattice* h)
{
    TuneKey k;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) k.device = prop.name;
    else k.device = "unknown";
    k.sms = h->sms;
    k.d = h->d;
    k.L = h->L;
    k.n = h->n;
    k.storage = h->storage;
    k.j_layout = h->j_layout;
    k.update = h->update;
    k.fast = h->fast_math;
    return k;
}

// The value of "name": in a JSON line (a string without escapes, or a number).
bool field(const char* line, const char* name, std::string* out)
{
    std::string pat = std::string("\"") + name + "\":";
    const char* p = std::strstr(line, pat.c_str());
    if (!p) return false;
    p += pat.size();
    while (*p == ' ') ++p;
    if (*p == '"') {
        const char* e = std::strchr(p + 1, '"');
        if (!e) return false;
        out->assign(p + 1, e);
        return true;
    }
    const char* e = p;
    while (*e && *e != ',' && *e != '}' && *e != '\n') ++e;
    out->assign(p, e);
    return true;
}

bool int_field(const char* line, const char* name, int* v)
{
    std::string s;
    if (!field(line, name, &s)) return false;
    char* end = nullptr;
    const long x = std::strtol(s.c_str(), &end, 10);
    if (end == s.c_str()) return false;
    *v = (int)x;
    return true;
}

bool cache_lookup(const char* path, const TuneKey& k, int* rows, int* caps, int* kernel)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        std::string dev;
        int v[9];
        const char* names[] = {"sms", "d", "L", "n", "storage", "j_layout", "update", "fast",
                               "rows"};
        bool ok = field(line, "device", &dev) && dev == k.device;
        for (int q = 0; q < 9 && ok; ++q) ok = int_field(line, names[q], &v[q]);
        int cap = 0, kern = 0;
        ok = ok && int_field(line, "blocks_per_sm", &cap) && int_field(line, "kernel", &kern);
        if (ok && v[0] == k.sms && v[1] == k.d && v[2] == k.L && v[3] == k.n &&
            v[4] == k.storage && v[5] == k.j_layout && v[6] == k.update && v[7] == k.fast) {
            *rows = v[8];
            *caps = cap;
            *kernel = kern;
            found = true;  // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

void cache_append(const char* path, const TuneKey& k, int rows, int caps, int kernel, double ms)
{
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"device\": \"%s\", \"sms\": %d, \"d\": %d, \"L\": %d, \"n\": %d, "
                 "\"storage\": %d, \"j_layout\": %d, \"update\": %d, \"fast\": %d, "
                 "\"rows\": %d, \"blocks_per_sm\": %d, \"kernel\": %d, "
                 "\"ms_per_sweep\": %.6f}\n",
                 k.device.c_str(), k.sms, k.d, k.L, k.n, k.storage, k.j_layout, k.update, k.fast,
                 rows, caps, kernel, ms);
    std::fclose(f);
}

bool tunable(const sl_lattice* h)
{
    if (h->slab || h->multihit > 0 || h->update == SL_UPDATE_SW) return false;
    if (h->storage == SL_STORE_BITS) return true;
    if (h->storage == SL_STORE_I8) return i8_streams(h);
    return on_streams(h);
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

extern "C" int sl_autotune(sl_lattice* h, double beta, int trial_sweeps, const char* cache_path,
                           int* rows, int* blocks_per_sm)
{
    if (!h) return fail(SL_EINVAL, "lattice is NULL");
    if (trial_sweeps < 1 || trial_sweeps > 1000)
        return fail(SL_EINVAL, "trial_sweeps must be in [1, 1000]");
    auto report = [&]() {
        if (rows) *rows = h->rows;
        if (blocks_per_sm) *blocks_per_sm = h->blocks_per_sm;
        return SL_OK;
    };
    if (!tunable(h)) return report();
    const TuneKey key = key_of(h);
    int r = 0, c = 0, kc = 0;
    if (cache_path && cache_lookup(cache_path, key, &r, &c, &kc) && r > 0 && h->Lz % r == 0 &&
        (kc == 0 || kc == 2 || (kc == 3 && h->n == 3) || (kc == 4 && h->n == 3 && h->d == 3))) {
        h->rows = r;
        h->blocks_per_sm = c;
        if (kc) h->kernel = kc;
        forget_graphs(h);
        return report();
    }
    SweepParams p;
    int st = sweep_params(h, beta, 0x7E57ull, &p);
    if (st != SL_OK) return st;
    // keep the spins (both colour arrays) in the staging area meanwhile
    const size_t H = (size_t)h->H;
    const size_t colour_bytes = h->storage == SL_STORE_I8     ? H
                                : h->storage == SL_STORE_BITS ? H / 8
                                : h->n == 2                   ? 4 * H
                                                              : 12 * H;
    if (2 * colour_bytes > h->staging_bytes)
        return fail(SL_EINVAL, "no room to keep the spins while tuning");
    cudaStream_t s = h->stream;
    char* keep = (char*)h->staging;
    cudaError_t e = cudaMemcpyAsync(keep, h->spins[0], colour_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(keep + colour_bytes, h->spins[1], colour_bytes,
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = clear_series(h, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int saved_rows = h->rows, saved_caps = h->blocks_per_sm, saved_kernel = h->kernel;
    int best_r = saved_rows, best_c = saved_caps, best_k = saved_kernel;
    float best = -1.f;
    // Heisenberg: the kernel as set, single columns (3) where pairs are the
    // default, and the staged 3D tiles (4) where they apply
    int kernels[3] = {saved_kernel, -1, -1};
    if (h->n == 3 && h->W % 64 == 0 && saved_kernel != 3) kernels[1] = 3;
    h->kernel = 4;
    if (on_tile_ok(h)) kernels[2] = 4;
    h->kernel = saved_kernel;
    for (int kern : kernels)
    for (int R : kRows) {
        if (kern < 0 || h->Lz % R) continue;
        if (kern == 4 && R != kRows[0]) continue;  // the staged tiles take no rows per thread
        for (int cap : kCaps) {
            if (e != cudaSuccess || st != SL_OK) break;
            if (kern == 4 && cap > 2) continue;     // at most four resident blocks per SM
            h->kernel = kern;
            h->rows = R;
            h->blocks_per_sm = cap;
            st = sweep_plain(h, p, 1, s);  // warm-up
            if (st == SL_OK) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess && st == SL_OK) st = sweep_plain(h, p, trial_sweeps, s);
            if (e == cudaSuccess && st == SL_OK) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && st == SL_OK) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess && st == SL_OK) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && st == SL_OK && (best < 0.f || ms < best)) {
                best = ms;
                best_r = R;
                best_c = cap;
                best_k = h->kernel;
            }
        }
    }
    // put the state back whatever happened
    h->rows = best_r;
    h->blocks_per_sm = best_c;
    h->kernel = best_k;
    cudaError_t e2 = cudaMemcpyAsync(h->spins[0], keep, colour_bytes, cudaMemcpyDeviceToDevice, s);
    if (e2 == cudaSuccess)
        e2 = cudaMemcpyAsync(h->spins[1], keep + colour_bytes, colour_bytes,
                             cudaMemcpyDeviceToDevice, s);
    if (e2 == cudaSuccess) e2 = set_sweep_index(h, h->sweeps_done, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    forget_graphs(h);
    if (st != SL_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "sl_autotune");
    if (e2 != cudaSuccess) return cuda_fail(e2, "sl_autotune: restore");
    if (cache_path && best >= 0.f)
        cache_append(cache_path, key, best_r, best_c, best_k, best / trial_sweeps);
    return report();
}
