// Host-side internals of libspinmc shared between translation units: the
// lattice handle, the layout of the caller's device buffer, and the kernel
// launchers each model's .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "spinmc.h"
#include "common.cuh"

namespace spinmc {

constexpr int kMaxBlocks = 4096;     // upper bound on any measuring grid
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Acceptance thresholds for the Ising classes (see ising_thresholds()).
struct IsingTable {
    uint32_t thr[6];
    int ncmp;      // number of classes with dE > 0 (d, or 2d when bonds may be zero)
    int scheme;    // 0: class = unsatisfied bonds (couplings +-1); 1: class = 2d - e
    int sigma_neg; // the scalar J is negative
    int heatbath;  // 1: heat-bath rule with the thresholds hb[h + 2d], h = sum_k Jb_k s_k
    uint32_t hb[13];
    uint32_t sw_thr;  // Swendsen-Wang: a satisfied bond is active iff u <= sw_thr
    int sw_never;     // Swendsen-Wang: no bond can be active (beta = 0)
};

// Per-sweep parameters common to every model.
struct SweepParams {
    double beta;
    uint64_t seed;
    RoundKeys rk;
    IsingTable tab;   // Ising only
    float beta_f;     // continuous spins
};

}  // namespace spinmc

struct sl_lattice {
    int d, L, n, j_layout, storage;
    int64_t N, H;            // sites, sites per colour
    int W;                   // sites of one colour in one row (L / 2)
    int sms;                 // multiprocessors of the device the handle was created on
    // A slab of a larger lattice split along its slowest axis (y in 2D, z in
    // 3D): it owns global planes z0 .. z0 + Lz - 1, stores one halo plane on
    // each side of each colour array, and keys its random numbers by global
    // site.  A whole lattice has slab = 0, z0 = 0, Lz = L.
    int slab, z0, Lz;
    int64_t P;               // sites of one colour in one plane (L/2 in 2D, L*L/2 in 3D)
    int next_colour;         // slab passes: the colour the next pass updates
    int device;              // the CUDA device the handle was created on
    cudaEvent_t ev;          // slab exchanges: marks the end of this slab's last pass
    double J;
    uint64_t init_seed;
    uint32_t replica;
    int64_t sweeps_done;
    cudaStream_t stream;     // the caller's stream
    cudaStream_t cap_stream; // private stream used only to capture graphs
    // views into the device buffer
    void* spins[2];          // per colour
    void* bonds[2][3];       // per colour, per direction (null for uniform J)
    void* staging;           // natural-order staging area
    size_t staging_bytes;
    spinmc::Ctrl* ctrl;
    spinmc::Partial* partials;  // kMaxBlocks block partials, then the integer
                                // totals a deferred byte pass accumulates
    bool bonds_have_zero;
    // options
    int renorm_every, fast_math, kernel, rows, use_graph;
    int blocks_per_sm;       // cap of the streaming kernels' grids per SM (0 = none)
    int update;              // SL_UPDATE_METROPOLIS, _HEATBATH or _SW
    int multihit, tile;      // k-fold multi-hit sweeps in tiles of side `tile` (0 = off)
    // cached graphs of kGraphSweeps sweeps and of one sweep
    cudaGraphExec_t graph, graph1;
    int graph_sweeps;
    uint64_t graph_key[4];
    void* owned_buf;
    // update workspace (Swendsen-Wang labels), caller-owned unless ws_owned
    void* ws;
    size_t ws_bytes;
    void* ws_owned;
};

namespace spinmc {

// error reporting (thread-local message, see sl_last_error)
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// the lattice constructor behind sl_create and sl_slab_create (lattice.cu)
int create_lattice(int d, int L, int n, int j_layout, int storage, double J, const void* J_bonds,
                   uint64_t seed, uint32_t replica, bool slab, int z0, int Lz, void* dev_buf,
                   size_t dev_buf_bytes, void* stream, sl_lattice** out);
size_t slab_required_bytes(int d, int L, int storage, int Lz);
int ising_table(const sl_lattice* h, double beta, IsingTable* tab);
// plain (uncaptured) sweeps, their parameters, and control-block setters (lattice.cu)
int sweep_plain(const sl_lattice* h, const SweepParams& p, int64_t count, cudaStream_t s);
int sweep_params(const sl_lattice* h, double beta, uint64_t seed, SweepParams* p);
cudaError_t set_sweep_index(const sl_lattice* h, int64_t t, cudaStream_t s);
cudaError_t clear_series(const sl_lattice* h, cudaStream_t s);
void forget_graphs(sl_lattice* h);
// whether a lattice's sweeps run the row-streaming kernels (ising_i8.cu, on_f32.cu)
bool i8_streams(const sl_lattice* h);
bool on_streams(const sl_lattice* h);
bool on_tile_ok(const sl_lattice* h);  // the staged 3D Heisenberg kernel applies

// ---- Ising int8 (ising_i8.cu) ----
cudaError_t ising_i8_init(const sl_lattice* h, cudaStream_t s);
cudaError_t ising_i8_scatter(const sl_lattice* h, const int8_t* nat, cudaStream_t s);
cudaError_t ising_i8_gather(const sl_lattice* h, int8_t* nat, cudaStream_t s);
cudaError_t ising_bonds_scatter(const sl_lattice* h, const int8_t* nat, unsigned* flags,
                                cudaStream_t s);
cudaError_t ising_i8_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                            cudaStream_t s);
// one colour pass (c = 1 measures and advances the sweep counter)
cudaError_t ising_i8_pass(const sl_lattice* h, const SweepParams& p, int c, cudaStream_t s);
cudaError_t ising_i8_measure(const sl_lattice* h, cudaStream_t s);
// measurement that also closes a sweep (series entry, sweep counter + 1)
cudaError_t ising_i8_measure_advance(const sl_lattice* h, cudaStream_t s);

// ---- Ising multi-hit sweeps in big tiles (ising_tile.cu) ----
bool tile_size_ok(int d, int L, int T);
cudaError_t ising_tile_sweep(const sl_lattice* h, const SweepParams& p, cudaStream_t s);

// ---- Ising Swendsen-Wang updates (ising_sw.cu) ----
size_t sw_workspace_bytes(int d, int L);
cudaError_t ising_sw_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                            cudaStream_t s);

// ---- Ising bit-packed (ising_bits.cu) ----
cudaError_t ising_bits_init(const sl_lattice* h, cudaStream_t s);
cudaError_t ising_bits_scatter(const sl_lattice* h, const int8_t* nat, cudaStream_t s);
cudaError_t ising_bits_gather(const sl_lattice* h, int8_t* nat, cudaStream_t s);
cudaError_t ising_bits_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                              cudaStream_t s);
cudaError_t ising_bits_pass(const sl_lattice* h, const SweepParams& p, int c, cudaStream_t s);
cudaError_t ising_bits_measure(const sl_lattice* h, cudaStream_t s);

// ---- XY / Heisenberg FP32 (on_f32.cu) ----
cudaError_t on_init(const sl_lattice* h, cudaStream_t s);
cudaError_t on_layout(const sl_lattice* h, float* nat, int dir, cudaStream_t s);
cudaError_t float_bonds_scatter(const sl_lattice* h, const float* nat, cudaStream_t s);
cudaError_t on_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count, cudaStream_t s);
cudaError_t on_measure(const sl_lattice* h, cudaStream_t s);

}  // namespace spinmc
