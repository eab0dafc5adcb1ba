/*
 * spinmc — checkerboard single-spin-flip Metropolis for classical O(n) lattice
 * spin models on one GB300 (sm_103a).  C ABI.
 *
 * Method: Weigel & Yavors'kii, "GPU accelerated Monte Carlo simulations of
 * lattice spin models", Physics Procedia 15 (2011), Section 2:
 *   Eq. (1)  H = - sum_<ij> J_ij s_i . s_j, nearest neighbours on a periodic
 *            square (d = 2) or simple-cubic (d = 3) lattice, n = 1 (Ising),
 *            2 (XY) or 3 (Heisenberg);
 *   Eq. (2)  a single-spin move s_i -> s_i' is accepted with probability
 *            min[1, exp(-beta dE)];
 *   the lattice is split into two checkerboard colours; all sites of one
 *   colour are updated in parallel, then all sites of the other (one sweep).
 * The Edwards-Anderson +-J spin glass (Section 2, last paragraph) runs as a
 * batch of disorder samples with replica exchange between temperatures.
 *
 * Conventions shared by every call:
 *   - L must be even (the checkerboard must close under the periodic wrap);
 *     N = L^d sites; natural index i = x + L*y (+ L*L*z); colour
 *     c = (x+y(+z)) & 1; colour index j = i >> 1.
 *   - Random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     64-bit seed (key = (seed_lo, seed_hi)) with counter
 *     (group, sweep index t, replica, purpose << 1 | colour), purpose 0 for a
 *     sweep, 1 for the initial state, 2 for couplings, 3 for replica
 *     exchange, 4 for multi-hit sweeps, 5 and 6 for Swendsen-Wang bonds and
 *     cluster flips; group = j >> 2 (Ising, site uses output j & 3), j >> 1 (XY,
 *     outputs 2(j&1) accept and 2(j&1)+1 proposal), j (Heisenberg, outputs 0
 *     accept, 1 and 2 proposal).  A run is therefore a pure function of
 *     (seed, sweep indices, start state).
 *   - Ising moves with dE > 0 are accepted iff u < exp(-beta dE) * 2^32 for
 *     the site's raw 32-bit output u (exact integer thresholds built on the
 *     host in FP64); dE <= 0 is always accepted.  Continuous spins propose a
 *     fresh uniform angle (XY) or direction (Heisenberg), compute dE and the
 *     acceptance in FP32 against u24 = (u >> 8) 2^-24, and accumulate the
 *     observables in FP64.
 *   - Every call returns SL_OK or a negative status and never throws.  Calls
 *     that take a stream pointer enqueue work on it and return before the
 *     GPU finishes, except where a call says it synchronises.
 *   - Ownership: device memory is owned by the caller.  sl_create takes a
 *     caller-allocated device buffer of sl_required_bytes bytes, 256-byte
 *     aligned, which must outlive the handle; passing NULL makes the library
 *     allocate (and free in sl_destroy) its own.  Host pointers passed in are
 *     only read during the call.
 */
#ifndef SPINMC_H
#define SPINMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SL_OK 0
#define SL_EINVAL (-1)    /* invalid argument (message in sl_last_error) */
#define SL_ENOMEM (-2)    /* buffer too small or allocation failed */
#define SL_ECUDA (-3)     /* a CUDA runtime call failed */
#define SL_ETIMEOUT (-4)  /* a kernel's bounded wait for its own asynchronous copies ran
                             out (reported by the next synchronising call; sticky) */
#define SL_EDEVICE (-5)   /* a kernel reported a failure it detected (a walker that did
                             not reach its window) */

/* coupling layouts */
#define SL_J_UNIFORM 0    /* every bond has J_ij = J */
#define SL_J_BONDS 1      /* J_ij = J * Jb[mu][i] per forward bond (i, i+e_mu) */

/* spin storage */
#define SL_STORE_I8 0         /* Ising, one int8 (+1 / -1) per site */
#define SL_STORE_BITS 1       /* Ising, one bit per site (1 = spin down) */
#define SL_STORE_F32_ANGLE 2  /* XY, FP32 angle in [0, 2 pi) */
#define SL_STORE_F32_VEC 3    /* Heisenberg, FP32 unit vector (3 components) */

/* options for sl_set_option */
#define SL_OPT_RENORM_EVERY 1  /* Heisenberg: renormalise every k sweeps (default 16, 0 = never) */
#define SL_OPT_FAST_MATH 2     /* continuous spins: 1 = hardware sin/cos/exp intrinsics */
#define SL_OPT_KERNEL 3        /* 0 = automatic, 1 = generic per-site kernel, 2 = row-streaming
                                  kernel, 3 = row-streaming kernel on single columns
                                  (Heisenberg; 2 takes column pairs where L % 128 == 0),
                                  4 = staged tiles (3D Heisenberg, uniform J, L in {64, 128,
                                  256, 512}, Metropolis, accurate functions: planes stream
                                  into shared memory by bulk asynchronous copies) */
#define SL_OPT_ROWS 4          /* rows each thread marches through in the streaming kernel */
#define SL_OPT_GRAPH 5         /* 1 = replay sweeps through CUDA graphs (default), 0 = plain launches */
#define SL_OPT_UPDATE 6        /* one of SL_UPDATE_* below (default SL_UPDATE_METROPOLIS) */
#define SL_OPT_MULTIHIT 7      /* k > 0: k-fold multi-hit sweeps in big tiles (Ising bytes,
                                  uniform J, Metropolis); 0 = plain sweeps (default) */
#define SL_OPT_TILE 8          /* big-tile side T for multi-hit sweeps: 8, 16 (default), 32 or
                                  64 in 2D, 8 or 16 in 3D; L % 2T == 0 */
#define SL_OPT_BLOCKS_PER_SM 9 /* cap of a streaming kernel's grid, in blocks per SM (each
                                  thread then takes several row segments); 0 = no cap
                                  (default): one segment per thread up to 4096 blocks */

/* update rules for SL_OPT_UPDATE */
#define SL_UPDATE_METROPOLIS 0 /* Eq. 2 */
#define SL_UPDATE_HEATBATH 1   /* heat-bath (Section 2): each spin drawn from its conditional
                                  law given its neighbours.  Ising bytes: s_i = +1 iff
                                  u < 2^32 / (1 + exp(-2 beta J h_i)).  XY: the offset from the
                                  angle of h by the von Mises rejection method of Best and
                                  Fisher, attempt a of a site using Philox counter word 3 =
                                  a << 16 | colour (at most 32 attempts, else the angle is
                                  kept).  Heisenberg: c = s'.h/|h| by inverting its exponential
                                  law at u24(output 0), azimuth 2 pi u24(output 1) in the
                                  orthonormal basis of Duff et al. (2017) around h.  Not for
                                  bit storage or multi-hit sweeps */
#define SL_UPDATE_SW 2         /* Ising bytes, uniform J, N <= 2^30: Swendsen-Wang cluster
                                  updates (Section 3), one per sweep index; needs a workspace
                                  (sl_workspace_bytes / sl_attach_workspace) */

typedef struct sl_lattice sl_lattice;

/*
 * sl_required_bytes — device bytes sl_create needs for this lattice.
 * d in {2,3}; L even, >= 2; n = 1 with storage SL_STORE_I8 or SL_STORE_BITS
 * (bits need L % 64 == 0), n = 2 with SL_STORE_F32_ANGLE, n = 3 with
 * SL_STORE_F32_VEC.  Returns SL_EINVAL for other combinations.
 */
int sl_required_bytes(int d, int L, int n, int j_layout, int storage, size_t* bytes);

/*
 * sl_create — build a lattice (Eq. 1) on the caller's stream and draw its
 * start configuration from Philox purpose 1 keyed by `seed`: Ising s = +1 iff
 * the top bit of the site's output is set; XY theta = 2 pi u24 (output
 * 2(j&1)+1); Heisenberg z = 2 u24(out 1) - 1, phi = 2 pi u24(out 2).
 *   J         the scalar coupling.
 *   J_bonds   SL_J_BONDS only: natural-order forward-bond couplings [d][N],
 *             int8 in {-1, 0, +1} for n = 1, float for n > 1; host or device
 *             pointer; J_ij = J * J_bonds.  Ignored for SL_J_UNIFORM.
 *   replica   the counter word 2 used for this lattice's random streams.
 *   dev_buf   device buffer of dev_buf_bytes >= sl_required_bytes bytes,
 *             256-byte aligned, owned by the caller; NULL = library-owned.
 *   stream    cudaStream_t (NULL = legacy default stream).
 * On success *out receives the handle.
 */
int sl_create(int d, int L, int n, int j_layout, int storage, double J, const void* J_bonds,
              uint64_t seed, uint32_t replica, void* dev_buf, size_t dev_buf_bytes,
              void* stream, sl_lattice** out);

/*
 * sl_sweep — nsweeps checkerboard Metropolis sweeps (Section 2, Eq. 2) at
 * inverse temperature beta >= 0, random stream keyed by `seed`, sweep indices
 * continuing from the handle's sweeps_done (so sweep(a) then sweep(b) equals
 * sweep(a+b)).  Asynchronous on the handle's stream.  SL_EINVAL if beta is
 * negative or so large that exp(-beta dE) underflows to zero.
 */
int sl_sweep(sl_lattice* lat, double beta, int64_t nsweeps, uint64_t seed);

/*
 * sl_sweep_series — as sl_sweep, and after sweep k writes the energy (Eq. 1)
 * to dev_E[k] and |m| = |M|/N to dev_absm[k] (device pointers to nsweeps
 * doubles; either may be NULL).  Ising values are exact (integer sums);
 * continuous-spin values are FP64 sums of FP32 per-thread partials.
 */
int sl_sweep_series(sl_lattice* lat, double beta, int64_t nsweeps, uint64_t seed,
                    double* dev_E, double* dev_absm);

/*
 * sl_measure — energy (Eq. 1) and magnetisation of the current state.
 * magnetisation receives n components of M = sum_i s_i followed by |M|/N
 * (n + 1 doubles).  Synchronises the handle's stream.
 */
int sl_measure(sl_lattice* lat, double* energy, double* magnetisation);

/*
 * sl_get_spins / sl_set_spins — copy the configuration out of / into the
 * lattice in natural order: int8 +-1 per site (n = 1), float angle (n = 2),
 * float[3] per site (n = 3).  dst / src may be host or device memory.  Both
 * synchronise the handle's stream.
 */
int sl_get_spins(sl_lattice* lat, void* dst);
int sl_set_spins(sl_lattice* lat, const void* src);

/*
 * sl_get_state / sl_set_state — checkpoint support: the start seed and the
 * number of sweeps done (the next sweep index).  With the spins saved by
 * sl_get_spins, restoring both resumes the run exactly.
 */
int sl_get_state(sl_lattice* lat, uint64_t* init_seed, int64_t* sweeps_done);
int sl_set_state(sl_lattice* lat, int64_t sweeps_done);

/* sl_set_option — set one SL_OPT_* value; SL_EINVAL for unknown options or
 * values out of range. */
int sl_set_option(sl_lattice* lat, int option, int64_t value);

/*
 * sl_autotune — pick the launch shape of the row-streaming sweep kernels for
 * this lattice: rows per thread R (SL_OPT_ROWS, every R in {1, 2, 4, 8, 16,
 * 32} dividing L), the grid cap (SL_OPT_BLOCKS_PER_SM in {0, 2, 4, 8, 16})
 * and, for Heisenberg spins, the kernel (SL_OPT_KERNEL 2, 3 or 4 where each
 * applies), by timing trial_sweeps sweeps at inverse
 * temperature beta of each shape (CUDA events on the lattice's stream, after
 * one warm-up sweep).  The
 * spins and the sweep counter are restored afterwards and the shape never
 * changes a decision, so the run continues as if the call had not happened.
 * cache_path (or NULL): a file of JSON lines keyed by the device name, its
 * SM count and (d, L, n, storage, couplings, update rule, fast math); a
 * matching line is used without timing, and a new choice is appended.  The
 * chosen values are returned in *rows and *blocks_per_sm (either may be
 * NULL).  Lattices whose sweeps do not use the streaming kernels (slabs,
 * multi-hit, Swendsen-Wang, short rows, zero couplings) keep their options.
 * Synchronises.
 */
int sl_autotune(sl_lattice* lat, double beta, int trial_sweeps, const char* cache_path,
                int* rows, int* blocks_per_sm);

/*
 * sl_workspace_bytes — device bytes of workspace an update rule needs on this
 * lattice: 0 for SL_UPDATE_METROPOLIS and SL_UPDATE_HEATBATH; for
 * SL_UPDATE_SW, 4 N bytes of cluster labels, one bit per tile-face bond and
 * a list of up to N tile roots (4 N bytes) (Section 3: clusters are labelled
 * in tiles, then the tiles are joined).
 * SL_EINVAL for a NULL argument or an unknown rule.
 */
int sl_workspace_bytes(const sl_lattice* lat, int update, size_t* bytes);

/*
 * sl_attach_workspace — hand the lattice a caller-owned device workspace,
 * 256-byte aligned, of at least sl_workspace_bytes bytes for the update rule
 * it will use; it must outlive the handle or the next attach.  NULL detaches.
 * Synchronises the handle's stream first.  Selecting SL_UPDATE_SW without a
 * large enough workspace fails with SL_EINVAL, except on a lattice whose
 * buffer the library allocated (sl_create with dev_buf = NULL), where the
 * library allocates the workspace too.  SL_ENOMEM if the workspace is too
 * small for the rule in use.
 *
 * Swendsen-Wang update t (SL_UPDATE_SW): the forward bond (i, i + e_mu) is
 * active iff J s_i s_j > 0 and u < (1 - exp(-2 beta |J|)) 2^32, u = output
 * 2 (i & 1) + mu of Philox(i >> 1, t, replica, 5 << 1) in 2D, output mu of
 * Philox(i, t, replica, 5 << 1) in 3D; the cluster whose smallest site is r
 * flips iff the top bit of output 0 of Philox(r, t, replica, 6 << 1) is set.
 * E and |m| are measured after every update, as after a sweep.
 */
int sl_attach_workspace(sl_lattice* lat, void* dev_buf, size_t bytes);

/* sl_destroy — release host metadata (and the buffer if library-owned).
 * Synchronises the handle's stream first. */
void sl_destroy(sl_lattice* lat);

/* ---- Domain decomposition: one lattice split into slabs ------------------
 *
 * Section 2 of the paper decomposes the lattice so that different processors
 * update different parts of it in parallel.  Here an Ising lattice (Eq. 1
 * with a uniform J) is split along its slowest axis (y in 2D, z in 3D) into
 * slabs, one per GPU or per rank.  A slab owns the global planes
 * z0 .. z0 + Lz - 1 and keeps one halo plane of each colour on either side
 * of them (the last plane of the slab below and the first of the slab
 * above, periodically).  A sweep is: every slab's colour-0 pass; the
 * exchange of colour 0 (each slab's first own plane of that colour into the
 * lower neighbour's upper halo, its last into the upper neighbour's lower
 * halo); every slab's colour-1 pass, which also measures the slab's part of
 * E and M; the exchange of colour 1.  Random numbers are keyed by the global
 * site, so the slabs reproduce the whole lattice's trajectory bit for bit
 * and their E and M add up to the lattice's.  A slab handle works with
 * sl_get_spins / sl_set_spins (its own sites, local natural order
 * i = x + L*(y - z0) in 2D, x + L*y + L*L*(z - z0) in 3D), sl_measure (its
 * share; the halos must be current), sl_get_state / sl_set_state,
 * sl_set_option (Metropolis or heat-bath, kernel and rows) and sl_destroy;
 * sl_sweep and sl_sweep_series refuse it. */

/* Device bytes of a slab: d in {2,3}; L % 8 == 0 (% 64 for bits);
 * storage SL_STORE_I8 or SL_STORE_BITS; 0 <= z0, 1 <= Lz, z0 + Lz <= L. */
int sl_slab_required_bytes(int d, int L, int storage, int z0, int Lz, size_t* bytes);

/* Create a slab (uniform coupling J) and draw its sites' start spins exactly
 * as sl_create draws those sites of the whole lattice.  The halos are filled
 * by the first exchange.  dev_buf and stream as for sl_create. */
int sl_slab_create(int d, int L, int storage, double J, uint64_t seed, uint32_t replica, int z0,
                   int Lz, void* dev_buf, size_t dev_buf_bytes, void* stream, sl_lattice** out);

/* Device addresses of a slab's planes of one colour: send_lo / send_hi its
 * first / last own plane, recv_lo / recv_hi the halo planes below / above
 * them; *bytes the size of one plane (L^(d-1) / 2 bytes, or / 16 for bits).
 * An exchange copies send_lo into the lower neighbour's recv_hi and send_hi
 * into the upper neighbour's recv_lo (NCCL send / receive, a peer copy ...),
 * on an order with the passes that both sides see. */
int sl_slab_planes(const sl_lattice* lat, int colour, void** send_lo, void** send_hi,
                   void** recv_lo, void** recv_hi, size_t* bytes);

/* From the next sweep on, the colour-1 pass of sweep k (counted from 0 at
 * this call) writes the slab's share of the energy to dev_E[k] and of
 * M = sum_i s_i to dev_M[k] (device pointers, either may be NULL).
 * Asynchronous on the slab's stream. */
int sl_slab_series(sl_lattice* lat, double* dev_E, double* dev_M);

/* One colour pass of a slab (asynchronous).  Colours alternate, 0 first;
 * the colour-1 pass ends the sweep.  The halos of the other colour must
 * hold the neighbours' current boundary planes. */
int sl_slab_pass(sl_lattice* lat, double beta, uint64_t seed, int colour);

/* For slabs held by one process (on one or several devices): the exchange
 * of one colour between slabs[0..nslabs-1], which must tile the lattice in
 * order (slab 0 from plane 0, each starting where the previous ends, the
 * last ending at L).  Each slab's stream waits for its neighbours' last
 * passes (events) and then copies their planes into its halos
 * (cudaMemcpyAsync, or cudaMemcpyPeerAsync across devices). */
int sl_slabs_exchange(sl_lattice* const* slabs, int nslabs, int colour);

/* nsweeps sweeps of slabs held by one process: both exchanges first (the
 * halos need not be current), then per sweep the colour-0 passes, the
 * colour-0 exchange, the colour-1 passes and the colour-1 exchange.
 * dev_EM[i] (device, on slab i's device, or NULL for every slab) receives
 * slab i's energy shares in [0, nsweeps) and M shares in
 * [nsweeps, 2 nsweeps).  Asynchronous. */
int sl_slabs_sweep(sl_lattice* const* slabs, int nslabs, double beta, int64_t nsweeps,
                   uint64_t seed, double* const* dev_EM);

/* Sum 1 to 64 parts laid out as sl_slabs_sweep writes them (nsweeps
 * energies, then nsweeps magnetisations; device memory readable from the
 * stream's device) in order: dev_E[k] = sum of the energies, dev_absm[k] =
 * |sum of the M| / N for the whole lattice's N sites.  After an all-reduce
 * across ranks, nparts = 1.  Asynchronous. */
int sl_series_reduce(const double* const* parts, int nparts, int64_t nsweeps, double N,
                     double* dev_E, double* dev_absm, void* stream);

/* ---- Edwards-Anderson +-J spin glass, batched, with replica exchange ----
 *
 * Section 2 of the paper: for quenched disorder, independent disorder samples
 * are a trivially parallel layer on top of the lattice decomposition.  A batch
 * holds nsamples Edwards-Anderson samples with the global indices
 * s = first_sample .. first_sample + nsamples - 1 (couplings J_ij = +-1 with
 * p = 1/2, J_ij = +1 iff the top bit of output 0 of Philox(i, mu, s, 2 << 1)
 * under the create seed is set), each with ntemps <= 32 replicas ("slots") at
 * the inverse temperatures betas[0..ntemps-1].  Slot r of sample s starts from
 * the Ising start state of replica id s * ntemps + r and always draws its
 * moves with that replica id.  Every random number is keyed by the global
 * index, so batches that split a sample range (one per GPU, say) together
 * hold exactly the samples of one batch over the whole range.  Calls that
 * take a `sample` argument count it from the batch's first sample (0 ..
 * nsamples - 1).  After every sweep the energies of all slots
 * are measured and temperature pairs (k, k+1), k = t mod 2, t mod 2 + 2, ...
 * attempt an exchange accepted iff Delta >= 0 or U < exp(Delta) 2^32,
 * Delta = (b_k - b_{k+1}) (E_{r(k)} - E_{r(k+1)}), U = output 0 of
 * Philox(k, t, s, 3 << 1) under the sweep seed (s the global index); accepted pairs swap which
 * slot holds which temperature.  The replica exchange is not in the paper:
 * it is the standard Metropolis swap between neighbouring temperatures. */

typedef struct sl_batch sl_batch;

/* Device bytes for a batch: d in {2,3}; L_per_sample[s] a multiple of 4 in
 * [4, 32]; 2 <= ntemps <= 32; betas (host, ntemps finite values >= 0) size
 * the exchange tables. */
int sl_batch_required_bytes(int d, const int* L_per_sample, int nsamples, int ntemps,
                            const double* betas, size_t* bytes);

/* Create the batch on `stream` and draw its couplings and start states from
 * `seed`.  L_per_sample[q] is the side of global sample first_sample + q.
 * betas: ntemps finite values >= 0 (host).  (first_sample + nsamples) *
 * ntemps must not exceed 2^32.  dev_buf as for sl_create (caller-owned,
 * 256-byte aligned, NULL = library-owned). */
int sl_batch_create(int d, const int* L_per_sample, int nsamples, int ntemps,
                    const double* betas, uint64_t seed, uint32_t first_sample, void* dev_buf,
                    size_t dev_buf_bytes, void* stream, sl_batch** out);

/* nsweeps sweeps of every slot of every sample, each followed by the energy
 * measurement and the exchange step, in one graph-captured launch per sample
 * size.  Sweep indices continue from the batch's sweeps done.  dev_E (device,
 * or NULL) receives nsamples * nsweeps * ntemps doubles: the energy at
 * temperature k of sample s after sweep i (before its exchange step) at
 * [(s * nsweeps + i) * ntemps + k].  Asynchronous. */
int sl_batch_run(sl_batch* b, int64_t nsweeps, uint64_t seed, double* dev_E);

/*
 * sl_batch_set_option — SL_BOPT_AUTOTUNE: 1 (default) times, before the first
 * run, 2-sweep trials of every pack size k in {1, 2, 4, 8} that fits a CTA's
 * shared memory for each sample size (on a copy of the state, which is then
 * restored) and keeps the combination whose largest-first schedule over the
 * GPU's CTAs finishes first; 0 packs as many samples per CTA as fit.
 * SL_BOPT_PACK: 0 (default) uses the tuned or fitted pack sizes, 1/2/4/8
 * forces that pack size (capped by what fits).  Results never depend on
 * either option.  Both take effect at the next sl_batch_run.
 */
#define SL_BOPT_AUTOTUNE 1
#define SL_BOPT_PACK 2
int sl_batch_set_option(sl_batch* b, int option, int64_t value);

/* sl_batch_tuning — the pack size (samples per CTA) and the measured time of
 * one sweep of a pack divided by its samples, in ms (0 if untimed), of size
 * class cls (classes are the distinct sides, largest first); returns the
 * number of classes or a negative status. */
int sl_batch_tuning(sl_batch* b, int cls, int* L, int* pack, double* ms_per_sample_sweep);

/* Copy slot `slot` of sample `sample` out in natural order (int8 +-1, host or
 * device dst) and report the temperature index it holds.  Synchronises. */
int sl_batch_get(sl_batch* b, int sample, int slot, int8_t* dst, int* temp_index);

/* Copy the couplings of a sample out as natural-order int8 [d][N] (+-1,
 * forward bond of site i along mu).  Synchronises. */
int sl_batch_get_bonds(sl_batch* b, int sample, int8_t* dst);

/* Sweeps done by the batch (the next sweep index). */
int sl_batch_sweeps_done(sl_batch* b, int64_t* sweeps_done);

/* Checkpoint load: the spins of every slot of a sample (ntemps x N int8 +-1,
 * slot after slot, each in natural order; host or device memory) and the
 * slot holding each temperature (ntemps int32 on the host, a permutation of
 * 0 .. ntemps-1, as sl_batch_get reports it).  With sl_batch_set_sweeps_done
 * and the create seed, a batch saved by sl_batch_get after n sweeps resumes
 * exactly: its next sweeps equal those of an uninterrupted run.  SL_EINVAL
 * if slot_of_temp is not a permutation.  Synchronises. */
int sl_batch_set(sl_batch* b, int sample, const int8_t* spins, const int32_t* slot_of_temp);

/* Set the sweeps done (the next sweep index) for resuming a checkpoint. */
int sl_batch_set_sweeps_done(sl_batch* b, int64_t sweeps_done);

/* Release host metadata (and the buffer if library-owned); synchronises. */
void sl_batch_destroy(sl_batch* b);

/*
 * sl_ising_measure_static — energy E = -J sum over nearest-neighbour pairs of
 * s_i s_j (each pair once, periodic lattice) and magnetisation of an Ising
 * configuration, without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as code running under another framework's device-memory
 * pool (a raw allocation would bypass its accounting or budget) or a
 * latency-critical loop that must not pay for an allocation.
 *   dev_spins  device pointer, N = L^d int8 values +1 / -1 in natural order
 *              (the layout sl_get_spins writes);
 *   dev_out    device pointer to two doubles: E, then M = sum_i s_i;
 *   stream     cudaStream_t (NULL = legacy default stream); asynchronous.
 * Its reduction scratch is one static device array of about 192 KiB, held by
 * every GPU that loads the library until the process exits; it serves at
 * most 2^28 sites (2D L <= 16384, 3D L <= 644; larger lattices return
 * SL_EINVAL).  The first call on a device (and the first after the device's
 * context was replaced, as by cudaDeviceReset) looks up that array's device
 * address with the device current, so make the first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race,
 * calls in order on one stream do not.
 */
int sl_ising_measure_static(int d, int L, double J, const int8_t* dev_spins, double* dev_out,
                            void* stream);

/* ---- Windowed multicanonical and Wang-Landau walkers (2D Ising) ---------
 *
 * Section 4 of the paper: every thread runs its own copy of the L x L Ising
 * torus (J = 1) inside a fixed energy window, the walkers of a window share a
 * block, histograms and ln g estimates sit in shared memory, and the window
 * estimates are glued into S(E) afterwards.  Energies are counted in levels
 * k = (E + 2N) / 4, 0 <= k <= N; window w spans the levels klo[w] .. khi[w]
 * (at least 3, at most 64) and a walker's arrays are indexed by k - klo.
 * L is a power of two in [4, 128]; walkers_per_window is a multiple of 32;
 * walker j lives in window j / walkers_per_window.
 *
 * Random numbers (Philox4x32-10 keyed by the seed of each call): every sweep
 * visits each site once, all walkers in the same order, step q of sweep t at
 * site (a q + b) mod N with a = (x mod N) | 1, b = y mod N, (x, y) = outputs
 * 0, 1 of Philox(0, t, 0, 11 << 1); step q draws output q & 3 of
 * Philox(q >> 2, t, walker, 9 << 1) (Wang-Landau) or (..., 10 << 1)
 * (multicanonical).  A move that leaves the window is rejected.  The sweep
 * index t continues across calls on one walker set.
 */
typedef struct sl_walkers sl_walkers;

/* sl_walkers_required_bytes — device bytes of a walker set (spins bit-packed
 * 32 walkers per word, levels, stages, visited masks, ln g and histograms). */
int sl_walkers_required_bytes(int L, int nwin, const int* klo, const int* khi,
                              int walkers_per_window, size_t* bytes);

/* sl_walkers_create — place every walker in its window: a nearest ground
 * state (ferromagnetic if the window's middle level is <= N/2, else Neel;
 * the copy with spin 0 down iff the top bit of output 0 of
 * Philox(0, 1, walker, 8 << 1) under `seed` is set), then attempt a flips
 * site (u N) >> 32, u = output 0 of Philox(a, 0, walker, 8 << 1), iff that
 * moves the energy towards the window without passing its far edge.
 * Synchronises; SL_EDEVICE if a walker did not arrive within 1000 N
 * attempts.  dev_buf as for sl_create (NULL: library-owned). */
int sl_walkers_create(int L, int nwin, const int* klo, const int* khi, int walkers_per_window,
                      uint64_t seed, void* dev_buf, size_t dev_buf_bytes, void* stream,
                      sl_walkers** out);

/* sl_wl_run — nsweeps Wang-Landau sweeps of every walker (asynchronous).
 * ln g is kept per walker in fixed point (units of 2^-32, ln f = 2^-stage):
 * a move k -> k' is accepted iff D >= 0 or u < exp(D 2^-32) 2^32,
 * D = S(k) - S(k'); after every attempt S(k) += 2^(32 - stage), H(k) += 1.
 * After every sweep a walker whose visited levels all hold
 * H(k) nvisited 100 >= flat_percent sum(H) advances a stage (H = 0, S lowered
 * by its minimum over the visited levels); walkers past final_stage (<= 32)
 * stop moving. */
int sl_wl_run(sl_walkers* w, int64_t nsweeps, int final_stage, int flat_percent, uint64_t seed);

/* sl_muca_run — nsweeps multicanonical sweeps with fixed weights lnW (host,
 * [nwin][kmax] doubles, kmax from sl_walkers_info, entry q of row w the
 * level klo[w] + q): a move k -> k' is accepted iff
 * u < exp(lnW(k) - lnW(k')) 2^32 (exact integer thresholds built on the
 * host in FP64).  The histograms restart at 0 and count the level after every
 * attempt.  Synchronises to upload the thresholds; the sweeps are
 * asynchronous.  SL_EINVAL for non-finite weights. */
int sl_muca_run(sl_walkers* w, const double* lnW, int64_t nsweeps, uint64_t seed);

/* sl_walkers_read — synchronise and copy to host: S ([walker][kmax] int64,
 * ln g in units of 2^-32), H ([walker][kmax]), level, stage, visited-level
 * masks ([walker]); any pointer may be NULL. */
int sl_walkers_read(sl_walkers* w, int64_t* S, uint32_t* H, int32_t* level, int32_t* stage,
                    uint64_t* visited);

/* sl_walkers_get_spins — one walker's spins in natural order as int8 +-1
 * (host or device pointer, N entries).  Synchronises. */
int sl_walkers_get_spins(sl_walkers* w, int walker, int8_t* dst);

/* Checkpoint load.  sl_walkers_set_spins writes one walker's configuration
 * (natural order int8 +-1, host or device, N entries) and sets the walker's
 * level to that of the configuration (k = (E + 2N) / 4); SL_EINVAL if the
 * level lies outside the walker's window.  sl_walkers_write sets S, H (host,
 * [walker][kmax], as sl_walkers_read returns them), stages and visited-level
 * masks; any pointer may be NULL to keep that array.
 * sl_walkers_set_sweeps_done sets the next sweep index.  Restoring all of
 * them from what sl_walkers_read, sl_walkers_get_spins and sl_walkers_info
 * returned after n sweeps resumes the run exactly.  Each synchronises. */
int sl_walkers_set_spins(sl_walkers* w, int walker, const int8_t* src);
int sl_walkers_write(sl_walkers* w, const int64_t* S, const uint32_t* H, const int32_t* stage,
                     const uint64_t* visited);
int sl_walkers_set_sweeps_done(sl_walkers* w, int64_t sweeps_done);

/* sl_walkers_set_option — SL_WOPT_SPINS_SMEM: 1 keeps each warp's 32
 * lattices in shared memory for the length of a run, 0 (default) reads and
 * writes them in place in global memory (L2).  The results do not depend on
 * it.
 * SL_EINVAL for unknown options or values. */
#define SL_WOPT_SPINS_SMEM 1
int sl_walkers_set_option(sl_walkers* w, int option, int64_t value);

/* sl_walkers_info — number of walkers, levels per walker array (kmax) and
 * sweeps done. */
int sl_walkers_info(const sl_walkers* w, int* nwalk, int* kmax, int64_t* sweeps_done);

/* sl_walkers_destroy — release host metadata (and the buffer if
 * library-owned); synchronises first. */
void sl_walkers_destroy(sl_walkers* w);

/* sl_dos_glue — glue per-window estimates (row w of S, `stride` doubles
 * apart, level klo[w] + q in entry q) into S over the levels 0..N of the
 * L x L torus (host only): window 0 as it is, window w + 1 shifted so that
 * its first level, which must be window w's last, matches; levels no window
 * visited (visited[w] bit q) are NaN.  SL_EINVAL if consecutive windows do
 * not share their edge level or it was not visited in both. */
int sl_dos_glue(int L, int nwin, const int* klo, const int* khi, const double* S, int stride,
                const uint64_t* visited, double* out);

/* sl_strerror — static text for a status code. */
const char* sl_strerror(int status);

/* sl_last_error — copy the calling thread's last error message (or "") into
 * msg (cap bytes, NUL-terminated); returns its full length. */
int sl_last_error(char* msg, size_t cap);

/*
 * Microbenchmarks — throughput of the units the sweeps lean on, so that a
 * measured compute ceiling can stand beside the one from unit counts and the
 * clock (the paper's speed-ups are bounded by the same units).  One call
 * launches, asynchronously on `stream`, a full-occupancy grid of
 * sl_microbench_threads() threads, each running independent chains:
 *   SL_MB_PHILOX  Philox4x32-10 with key 1: thread g makes `iterations` calls
 *                 with counters (g * iterations + i, 7, 0, 0) and writes the
 *                 xor of all their outputs to dev_out[g] (uint32; checkable
 *                 against any Philox implementation);
 *   SL_MB_IMAD    32-bit integer multiplies (mulhi and mullo chains);
 *   SL_MB_FFMA    FP32 fused multiply-adds;
 *   SL_MB_MUFU    hardware exp2 of the special-function unit.
 * dev_out holds 4 bytes per thread (device memory, caller-owned); *ops
 * receives the operations the launch performs (calls for SL_MB_PHILOX,
 * lane operations otherwise).  The caller times the launch (CUDA events on
 * the same stream).  SL_EINVAL for an unknown kind, iterations < 1, a short
 * buffer, or Philox counters beyond 32 bits; SL_ECUDA if the launch fails.
 */
/* sl_wait_selftest — check the bounded wait of the staged kernels: a
 * one-block kernel arms an mbarrier for 16 bytes that no copy ever delivers
 * and polls it with the same limit the staged kernels use (a few seconds);
 * *timed_out = 1 if the poll gave up and the kernel returned, as it must.  No
 * copy is issued.  Synchronises the stream. */
int sl_wait_selftest(void* stream, int* timed_out);

#define SL_MB_PHILOX 0
#define SL_MB_IMAD 1
#define SL_MB_FFMA 2
#define SL_MB_MUFU 3
int sl_microbench_threads(int* threads);
int sl_microbench(int kind, int iterations, void* dev_out, size_t out_bytes, void* stream,
                  double* ops);

#ifdef __cplusplus
}
#endif

#endif /* SPINMC_H */
