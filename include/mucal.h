/*
 * mucal: parallel multicanonical simulation of a fixed-N lattice gas on one GPU.
 *
 * C ABI of libmucal.so.  Every function returns an int status (MUCAL_OK = 0,
 * negative on error; see the MUCAL_ERR_* codes) unless stated otherwise, and
 * never throws.  Host buffers passed in are owned by the caller and only read
 * or written during the call; every device buffer is owned by the library and
 * freed by mucal_destroy.  A context is bound to the CUDA device that is
 * current when mucal_init_systems is called and to one CUDA stream; calls on
 * one context must not run concurrently from several host threads.
 * There is no CPU fallback: without a usable CUDA device mucal_init_systems
 * fails with MUCAL_ERR_NO_DEVICE.
 *
 * The method (Zierenberg, Wiedenmann, Janke, "Application of the parallel
 * multicanonical method to lattice gas condensation"):
 *   - model, Sec. 3 / Eq. 5: sites of a periodic L^d lattice (d = 2 square,
 *     d = 3 simple cubic) hold n_i in {0,1} with sum n_i = N fixed, and
 *     E = -J * #{occupied nearest-neighbour pairs}, J = 1;
 *   - Sec. 2: p independent walkers run equilibrium Metropolis updates with
 *     the same weights W(E), accepting with min(1, W(E_n)/W(E_o)); their
 *     histograms are summed, H^i(E) = sum_j H^i_j(E) (Eq. 2), and the next
 *     weights follow from W^i and H^i (W^{i+1} = W^i / H^i, or a recursion).
 *
 * Conventions fixed by this library where the paper is silent:
 *   - site s = x_0 + L x_1 (+ L^2 x_2), periodic neighbours x_k +- 1 mod L;
 *   - move: a uniformly chosen particle jumps to a uniformly chosen empty
 *     site.  Particle and empty-site lists are kept in one array S per walker,
 *     S[0..N) = particle sites, S[N..V) = empty sites; an accepted move of
 *     particle index k to empty index m swaps S[k] and S[N+m];
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit seed
 *     of walker w = seed_base + w (low word first), counter =
 *     (t low, t high, iteration, 0) for attempt t of an iteration;
 *     r0 -> k = floor(r0 N / 2^32), r1 -> m = floor(r1 (V-N) / 2^32),
 *     r2 -> acceptance variate, r3 unused.  The initial placement is a partial
 *     Fisher-Yates shuffle drawing output j from counter (j/4 low, j/4 high,
 *     0, 1), word j%4: for j < N, swap S[j] with S[j + floor(r (V-j) / 2^32)];
 *   - acceptance: per window bin b = E_o - e_lo and dE in [-2d, 2d] a uint32
 *     threshold T, built in double precision on the host from lnW:
 *     0 if E_o + dE leaves the window, 0xFFFFFFFF if lnW(E_o+dE) >= lnW(E_o),
 *     else min(floor(2^32 exp(lnW(E_o+dE) - lnW(E_o))), 0xFFFFFFFE);
 *     a move is accepted iff T == 0xFFFFFFFF or r2 < T;
 *   - every attempt, accepted or not, records the energy after the attempt.
 *   - Walker states carry over from one iteration to the next.
 */
#ifndef MUCAL_H
#define MUCAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MUCAL_OK                 0
#define MUCAL_ERR_INVALID_ARG   -1  /* bad pointer, size, index or parameter */
#define MUCAL_ERR_CUDA          -2  /* a CUDA runtime call failed */
#define MUCAL_ERR_OOM           -3  /* device or pinned host allocation failed */
#define MUCAL_ERR_NO_DEVICE     -4  /* no usable CUDA device */
#define MUCAL_ERR_NOT_READY     -5  /* call order violated (e.g. no histogram yet) */
#define MUCAL_ERR_STATE         -6  /* a device-side consistency check failed */

/* ---- flags of mucal_init_systems ---------------------------------------- */
/* Keep the per-walker histograms H_j(E) of the last iteration readable via
 * mucal_get_histogram (they always exist on the device; without the flag the
 * library may skip keeping them). */
#define MUCAL_FLAG_PER_WALKER_HIST 0x1u

/* ---- weight-update schemes of mucal_update_weights ---------------------- */
/* W^{i+1}(E) = W^i(E) / H^i(E) where H^i(E) > 0, unchanged elsewhere (Sec. 2). */
#define MUCAL_SCHEME_SIMPLE     0
/* The accumulated-statistics recursion cited in Sec. 2, on consecutive
 * visited energies E_prev < E of the cumulative visited set:
 * g = H(E_prev) H(E) / (H(E_prev) + H(E)), p(E) += g, kappa = g / p(E),
 * ln(W(E)/W(E_prev)) += kappa (ln H(E_prev) - ln H(E)); unvisited bins keep
 * their log-weight offset to the nearest visited bin above them (below if
 * none is above).  Its first step equals MUCAL_SCHEME_SIMPLE on the visited
 * bins. */
#define MUCAL_SCHEME_RECURSIVE  1
/* Flag, or-ed with either scheme: after the update, bins below the lowest
 * visited energy and above the highest take lnW continued linearly with the
 * slope between that end and the 8th visited bin counted inwards from it
 * (canonical weights at the microcanonical temperature of the sampled edge;
 * without the flag they keep the edge's weight).  The walkers then keep
 * moving into the energies not sampled yet instead of being held back by the
 * entropy there, which is how the range of Sec. 2's iteration grows.  Not
 * stated in the paper (its recursion is cited, not printed). */
#define MUCAL_SCHEME_EXTRAPOLATE 0x10

/* ---- walker-update kernels (mucal_launch_config.kernel) ------------------ */
/* One thread advances one walker, attempt after attempt; the random numbers
 * and list reads of the next attempts are in flight while one is evaluated. */
#define MUCAL_KERNEL_THREAD     0
/* A group of lanes advances one walker: the lanes evaluate consecutive
 * attempts against the same state in parallel and commit them in order,
 * re-evaluating after every accepted move, so the chain is identical to the
 * one-thread chain. */
#define MUCAL_KERNEL_GROUP      1
/* The group kernel with a local field: each walker of a block keeps the
 * number of occupied neighbours of every site (one byte per site) in shared
 * memory, so an attempt reads two counts instead of 2*2d occupation bits and
 * a commit updates the 2*2d counts around the two sites.  Same chain as the
 * other two; needs V bytes (rounded up to 16) of shared memory per walker of
 * a block, so it suits lattices up to a few thousand sites. */
#define MUCAL_KERNEL_FIELD      2

typedef struct mucal_system_desc {
    int32_t d;          /* lattice dimension, 2 or 3 */
    int32_t L;          /* linear size, 3 <= L, L^d <= 2^24 */
    int32_t N;          /* particles, 0 < N < L^d */
    int32_t n_walkers;  /* independent walkers (the p processes of Sec. 2), >= 1 */
    int32_t e_lo;       /* energy window [e_lo, e_hi]; e_lo = e_hi = 0 selects */
    int32_t e_hi;       /*   the full range [-dN, 0]; otherwise -dN <= e_lo < e_hi <= 0 */
    uint64_t seed_base; /* walker w uses Philox key seed_base + w */
} mucal_system_desc;

typedef struct mucal_launch_config {
    int32_t kernel;            /* MUCAL_KERNEL_THREAD, _GROUP or _FIELD */
    int32_t lanes_per_walker;  /* 1 for THREAD; 2, 4, 8, 16 or 32 for GROUP and FIELD */
    int32_t walkers_per_block; /* threads per block = walkers_per_block * lanes: <= 512;
                                  a multiple of 32 for GROUP and FIELD */
    int32_t bits_in_smem;      /* 1: stage each walker's occupation bitset in shared
                                  memory for the launch; 0: use it in global memory.
                                  FIELD keeps its counts in shared memory and needs 1 */
    int32_t persistent;        /* 1: launch only the blocks that fit on the device at
                                  once; each pulls the next block of walkers from a
                                  counter when it finishes one.  0: one block per block
                                  of walkers, scheduled by the hardware */
    int32_t thr_window;        /* GROUP and FIELD kernels, when some system's threshold
                                  table does not fit in shared memory next to the
                                  block's bitsets or fields: 1 = every walker keeps the
                                  32 rows around its current energy in shared memory
                                  (refilled by asynchronous bulk copies as the energy
                                  moves), 0 = thresholds are read from global memory;
                                  2 = the row windows even when the table would fit.
                                  If the windows do not fit next to the block's
                                  walkers, thresholds are read from global memory
                                  (mucal_get_launch_config then reports 0, as it does
                                  when the whole table is staged in shared memory).
                                  Ignored by THREAD.  Default 1 */
    int32_t multi_commit;      /* GROUP and FIELD kernels with 4 or more lanes and the
                                  thresholds in global or shared memory (no row
                                  windows): 1 = one round of G proposals may commit
                                  several accepted moves in order, each lane re-deciding
                                  against the energy its predecessors left while its
                                  move stays independent of theirs; 0 = one commit per
                                  round.  Both give the same chain (Sec. 2's Metropolis
                                  sequence, bit-identical).  With tunnelling events
                                  recorded the one-commit rounds run.  Reported as 0
                                  where it does not apply.  Default 0 */
} mucal_launch_config;

typedef struct mucal_system_info {
    int32_t d, L, N, n_walkers, e_lo, e_hi;
    int32_t V;          /* L^d */
    int32_t n_bins;     /* e_hi - e_lo + 1 */
    int32_t width;      /* 4d + 1 thresholds per bin */
    int32_t index_bytes;/* 2 if V <= 65536 else 4: bytes per entry of S */
    uint64_t seed_base;
} mucal_system_info;

typedef struct mucal_stats {
    uint64_t attempts;      /* attempts of the last mucal_run_iteration, all walkers */
    uint64_t accepts;       /* accepted moves of the last iteration, all walkers */
    double   kernel_ms;     /* device time of the last walker-update launch (CUDA events) */
    double   iteration_ms;  /* device time of the last whole mucal_run_iteration */
    uint64_t walker_launches; /* walker-update kernel launches so far */
} mucal_stats;

/* Create a context holding n_sys systems (Sec. 2 walkers of Sec. 3 lattice
 * gases) and place every walker's N particles at random (initial placement
 * above).  sys: host array of n_sys descriptors (copied).  cuda_stream: a
 * cudaStream_t to run on, or NULL for a stream owned by the context.  The
 * weights start at lnW = 0 (all moves inside the window accepted).
 * Errors: INVALID_ARG (bad descriptor; an initial energy outside a
 * user-given window), NO_DEVICE, OOM, CUDA.  *out is NULL on error. */
int mucal_init_systems(void **out, const mucal_system_desc *sys, int32_t n_sys,
                       void *cuda_stream, uint32_t flags);

/* Release every device and host resource of the context (NULL is allowed). */
void mucal_destroy(void *ctx);

/* Text of the last error on this context (or of the last failed
 * mucal_init_systems if ctx is NULL); valid until the next call. */
const char *mucal_last_error(void *ctx);

/* Set lnW(E) of system sys for E = e_lo .. e_hi (host float64 array of
 * n_bins finite values, copied).  Builds the acceptance thresholds in double
 * precision (min(1, W(E_n)/W(E_o)), Sec. 2) and uploads them.  Resets the
 * recursion memory (cumulative visited set and accumulated weights).
 * Errors: INVALID_ARG (index, size, non-finite value), CUDA. */
int mucal_set_weights(void *ctx, int32_t sys, const double *lnW, int32_t n_bins);

/* Read back the current lnW of system sys into lnW_out[n_bins] (host). */
int mucal_get_weights(void *ctx, int32_t sys, double *lnW_out, int32_t n_bins);

/* Read back the uint32 threshold table of system sys into T[n_bins*width]
 * (host), laid out T[b*width + dE + 2d]. */
int mucal_get_thresholds(void *ctx, int32_t sys, uint32_t *T, int64_t n);

/* Choose the walker-update kernel and its launch shape for later
 * iterations.  Errors: INVALID_ARG (unsupported combination, or more shared
 * memory than a block can have for some system). */
int mucal_set_launch_config(void *ctx, const mucal_launch_config *cfg);
int mucal_get_launch_config(void *ctx, mucal_launch_config *cfg);

/* CUDA-graph mode (enable = 1): mucal_run_iteration then launches its device
 * work (histogram clears, walker update, histogram sums, timing events) as
 * one CUDA graph, captured on the context's stream the first time and again
 * whenever sweeps, the launch shape or the kernel flavour changes; between
 * launches only the iteration number of the walker-update node is updated.
 * Results are identical to the direct launches; mucal_stats.kernel_ms then
 * times the whole graph (clears and sums included).  Waits for the stream.
 * Errors: INVALID_ARG, CUDA. */
int mucal_set_graph_mode(void *ctx, int32_t enable);

/* One iteration of Sec. 2 for every system of the context, asynchronous on
 * the context's stream: zero the histograms, let every walker perform
 * sweeps * N attempted moves with the current weights (iteration enters the
 * Philox counter), record H_j(E) per walker, and sum them into H(E) (Eq. 2)
 * on the device.  sweeps >= 1; sweeps * N must be below 2^40.
 * Errors: INVALID_ARG, CUDA. */
int mucal_run_iteration(void *ctx, int64_t sweeps, uint32_t iteration);

/* Wait for the context's stream and copy the summed histogram H(E) of system
 * sys into H[n_bins] (host int64).  per_walker: NULL, or host int64
 * [n_walkers * n_bins] that receives H_j(E), walker-major (needs
 * MUCAL_FLAG_PER_WALKER_HIST).  Errors: INVALID_ARG, NOT_READY (no
 * iteration run yet), CUDA. */
int mucal_get_histogram(void *ctx, int32_t sys, int64_t *H, int32_t n_bins, int64_t *per_walker);

/* Weight update from the last histogram of system sys (Sec. 2):
 * scheme MUCAL_SCHEME_SIMPLE or MUCAL_SCHEME_RECURSIVE, optionally or-ed with
 * MUCAL_SCHEME_EXTRAPOLATE, in double precision on
 * the host, then lnW is shifted to max 0, the thresholds are rebuilt and
 * uploaded (the redistribution of the weights to all walkers).  lnW_out
 * (nullable, host float64[n_bins]) receives the new lnW; flatness_out
 * (nullable) receives min/max of H over the cumulative visited set inside the
 * target window, or -1 while an end of that window is unvisited.
 * Errors: INVALID_ARG, NOT_READY, CUDA. */
int mucal_update_weights(void *ctx, int32_t sys, int32_t scheme, double *lnW_out,
                         double *flatness_out);

/* Target window of the flatness measure of system sys (default: from the
 * lowest visited energy to the highest).  t_lo = t_hi = 0 restores it. */
int mucal_set_target_window(void *ctx, int32_t sys, int32_t t_lo, int32_t t_hi);

/* Replace the summed histogram that the next mucal_update_weights of system
 * sys uses by H (host int64[n_bins], copied).  This is how several processes
 * that each run part of the walkers with identical weights combine their
 * histograms (Eq. 2: H^i = sum over processes of H^i_j): every process sums
 * its local histograms with the others' (for example by an all-reduce) and
 * hands the total to its own context, so that every process computes the same
 * next weights (Sec. 2, the redistribution of the weights needs no further
 * message).  Waits for the context's stream.  Errors: INVALID_ARG (index,
 * size, a negative count), NOT_READY (no iteration run yet), CUDA. */
int mucal_set_histogram(void *ctx, int32_t sys, const int64_t *H, int32_t n_bins);

/* Resident blocks per SM of the current walker-update launch shape (the
 * CUDA occupancy of that kernel at its block size and shared memory) and the
 * device's SM count.  Not part of the paper; used to state how many walkers'
 * chains run at once.  Errors: INVALID_ARG, CUDA. */
int mucal_get_launch_occupancy(void *ctx, int32_t *blocks_per_sm, int32_t *sm_count);

/* One weight update of Sec. 2 on caller-owned host arrays, without a
 * context: the same double-precision code mucal_update_weights runs.
 *   scheme     MUCAL_SCHEME_SIMPLE or MUCAL_SCHEME_RECURSIVE, optionally or-ed
 *              with MUCAL_SCHEME_EXTRAPOLATE
 *   H          int64[n_bins], the summed histogram of the iteration (in)
 *   lnW        float64[n_bins], the weights H was sampled with (in), the next
 *              weights shifted to maximum 0 (out)
 *   visited    uint8[n_bins] cumulative visited set (in/out; start with zeros)
 *   pacc       float64[n_bins] accumulated pair weights of the recursion
 *              (in/out; start with zeros; unused and nullable for SIMPLE)
 *   t_lo, t_hi flatness target window in bins (t_lo < 0: the visited range)
 *   flatness_out (nullable) min/max of H over the visited bins of the target
 *              window, -1 while an end of it is unvisited.
 * Errors: INVALID_ARG (unknown scheme, NULL arrays, n_bins < 1, a negative
 * H, a non-finite lnW, a target window outside the bins).  Message:
 * mucal_last_error(NULL). */
int mucal_weight_update(int32_t scheme, int32_t n_bins, const int64_t *H, double *lnW,
                        uint8_t *visited, double *pacc, int32_t t_lo, int32_t t_hi,
                        double *flatness_out);

/* Copy walker w's state of system sys to host buffers (any may be NULL):
 * occ uint8[V] (n_i), S int32[V] (particle then empty sites), E (energy). */
int mucal_get_walker_state(void *ctx, int32_t sys, int32_t walker, uint8_t *occ, int32_t *S,
                           int32_t *E);

/* Sizes and parameters of system sys. */
int mucal_get_system_info(void *ctx, int32_t sys, mucal_system_info *info);

/* Counters and timings of the last iteration of system sys (kernel_ms and
 * iteration_ms cover the whole launch, all systems). */
int mucal_get_stats(void *ctx, int32_t sys, mucal_stats *stats);

/* Device pointer of the summed histogram H(E) of system sys (int64[n_bins],
 * library-owned, valid until mucal_destroy; contents valid once the
 * context's stream has finished the last mucal_run_iteration). */
int mucal_histogram_device_ptr(void *ctx, int32_t sys, void **dptr);

/* Library version string. */
const char *mucal_version(void);

/* ---- checkpoint / resume ---------------------------------------------------
 * A checkpoint of system sys holds every walker's state (bitset, particle and
 * empty-site lists, energy), the weights and the recursion memory (visited
 * set, accumulated pair weights) and the flatness target.  The random
 * numbers depend only on (seed, iteration, attempt), so a system restored
 * into a context with the same descriptor continues bit-for-bit when the
 * caller passes the same iteration numbers.  Layout (host byte order): a
 * header (magic "MUCALCK1", d, L, N, n_walkers, e_lo, e_hi, seed_base, list
 * entry bytes, bitset words, n_bins, target), then bits, lists, energies,
 * lnW (float64), visited (uint8), accumulated weights (float64).
 * mucal_checkpoint_size: bytes of the checkpoint of sys.
 * mucal_checkpoint_save: write it into the caller's host buffer of exactly
 *   that size (waits for the context's stream).
 * mucal_checkpoint_load: restore from such a buffer; it must come from a
 *   system with the same descriptor.  Energies outside the window, list
 *   entries off the lattice and non-finite weights are rejected with
 *   MUCAL_ERR_INVALID_ARG before anything is changed.  The thresholds are
 *   rebuilt from the restored weights. */
int mucal_checkpoint_size(void *ctx, int32_t sys, int64_t *bytes);
int mucal_checkpoint_save(void *ctx, int32_t sys, void *buf, int64_t bytes);
int mucal_checkpoint_load(void *ctx, int32_t sys, const void *buf, int64_t bytes);

/* ---- reweighting to canonical temperatures (Sec. 3) -----------------------
 * Multicanonical data are taken with the weights W(E) and reweighted to the
 * temperatures of interest afterwards.  A histogram H(E) sampled with
 * lnW(E) = ln W(E) estimates Omega(E), up to a constant factor, by
 * H(E) / W(E), so the canonical distribution at inverse temperature beta is
 *     P_beta(E) = H(E) exp(-beta E - lnW(E)) / Z_beta        (Eq. 1)
 * over the visited bins (H > 0).  Bin b holds energy e_lo + b.  For each
 * beta[i], i < n_beta:
 *   mean_E[i]  = sum_E P_beta(E) E,   mean_E2[i] = sum_E P_beta(E) E^2
 *   (both nullable, host float64[n_beta]);
 *   obs_out[i * n_obs + k] = sum_b P_beta(b) obs[k * n_bins + b] /
 *                            sum_b P_beta(b), both sums over the bins with
 *   H > 0 and a finite obs value (obs holds n_obs microcanonical means, for
 *   example the mean largest droplet at each energy, NaN where nothing was
 *   measured); NaN if no bin qualifies.  obs may be NULL with n_obs = 0.
 * Double precision on the host: exponents shifted by their maximum, bins
 * summed in ascending order.  Errors: INVALID_ARG (NULL H, lnW or beta with
 * n_beta > 0; n_bins < 1; n_beta or n_obs < 0; a negative H; no visited bin;
 * a non-finite lnW or beta).  Message: mucal_last_error(NULL). */
int mucal_reweight(const int64_t *H, const double *lnW, int32_t n_bins, int32_t e_lo,
                   const double *beta, int32_t n_beta, const double *obs, int32_t n_obs,
                   double *mean_E, double *mean_E2, double *obs_out);

/* Multi-histogram estimate of ln Omega(E) from K histograms H[k][n_bins]
 * sampled with log-weights lnW[k][n_bins] (for instance several iterations of
 * Sec. 2, or several production runs): the self-consistent combination
 *   Omega(E) = sum_k H_k(E) / sum_k N_k exp(lnW_k(E) - f_k),
 *   exp(f_k) = sum_E Omega(E) exp(lnW_k(E)),   N_k = sum_E H_k(E),
 * iterated from f_k = 0 (f_0 fixed to 0) until max_k |f_k change| < tol or
 * max_iter passes.  ln_omega (host float64[n_bins]) receives ln Omega shifted
 * to maximum 0, NaN where no histogram visited; iterations (nullable) the
 * passes made (max_iter means the tolerance was not reached).  With K = 1 it
 * is ln H(E) - lnW(E).  A run restricted to an energy window has weight 0
 * outside it: pass lnW = -inf there.  Errors: INVALID_ARG (NULL arrays, sizes < 1,
 * max_iter < 1, tol <= 0, a negative H, non-finite lnW where H > 0, all
 * histograms empty).  Message: mucal_last_error(NULL). */
int mucal_multi_histogram(const int64_t *H, const double *lnW, int32_t K, int32_t n_bins,
                          int32_t max_iter, double tol, double *ln_omega, int32_t *iterations);

/* The constant of Eq. 5: with s_i = 2 n_i - 1 the lattice-gas energy is
 * H_gas = H_Ising / 4 + c(N), c(N) = J d (V/4 - N), so an energy E of the
 * gas is E_Ising = 4 (E - c(N)) at fixed magnetisation M = 2N - V, and the
 * Ising temperature is 4T.  Errors: INVALID_ARG (d outside {2,3}, V < 1,
 * N outside [0, V], NULL c_N). */
/* Estimate of ln Omega(E) from one histogram and the weights it was
 * sampled with: the ideal weights W = 1/Omega give a flat histogram (Sec. 2),
 * so Omega(E) is proportional to H(E) / W(E).  ln_omega (host
 * float64[n_bins]) receives ln H(E) - lnW(E) on the bins with H > 0, NaN
 * elsewhere, shifted so that the visited bins together hold all C(V, N)
 * configurations of N particles on V sites.  Errors: INVALID_ARG (NULL
 * arrays, n_bins < 1, a negative H, no visited bin, a non-finite lnW where
 * H > 0, V < 1 or N outside [0, V]).  Message: mucal_last_error(NULL). */
int mucal_ln_omega(const int64_t *H, const double *lnW, int32_t n_bins, int64_t V, int64_t N,
                   double *ln_omega);

/* Shift the finite entries of ln_omega[n_bins] in place so that their
 * exponentials sum to C(V, N) (every configuration has some energy); NaN
 * entries (unvisited energies) stay NaN.  For the output of
 * mucal_multi_histogram.  Errors: INVALID_ARG (NULL, n_bins < 1, no finite
 * entry, V < 1 or N outside [0, V]). */
int mucal_ln_omega_normalise(double *ln_omega, int32_t n_bins, int64_t V, int64_t N);

int mucal_ising_constant(int32_t d, int64_t V, int64_t N, double J, double *c_N);

/* mucal_reweight of system sys's last summed histogram with the weights it
 * was sampled with (those in force at the last mucal_run_iteration, not the
 * ones a later mucal_update_weights or mucal_set_weights installed).  Waits
 * for the context's stream.  Errors: as mucal_reweight, NOT_READY, CUDA. */
int mucal_reweight_system(void *ctx, int32_t sys, const double *beta, int32_t n_beta,
                          const double *obs, int32_t n_obs, double *mean_E, double *mean_E2,
                          double *obs_out);

/* ---- tunnelling events (Sec. 4) ------------------------------------------
 * The paper stops its weight iteration once the walkers together have
 * travelled 30 times from the maximal to the minimal energy or back
 * ("tunnelling events").  Every walker keeps, across iterations, which end
 * of [e_min, e_max] it reached last and how many end-to-end travels it has
 * made: every energy the walker takes (its energy at the start of each
 * iteration and after every accepted move) is checked, E <= e_min being the
 * low end and E >= e_max the high end; reaching one end when the other was
 * the last one reached counts one event (the first end reached counts none).
 * The ends default to the window ends.  The bookkeeping runs in a separate
 * flavour of the walker kernels (it costs about a tenth of the throughput),
 * switched on for every system of the context by the first
 * mucal_set_tunnel_window call; before that nothing is counted.
 * mucal_set_tunnel_window: set the ends of system sys (e_min = e_max = 0
 *   takes the window ends), zero its states and counts, and switch the
 *   bookkeeping on.
 * mucal_get_tunnel_counts: events of system sys so far: total (nullable) and
 *   per walker (nullable, host uint32[n_walkers]); state (nullable, host
 *   uint8[n_walkers]: 0 = no end reached yet, 1 = low end last, 2 = high end
 *   last).  Waits for the stream.
 * mucal_reset_tunnel_counts: zero the states and counts of every system.
 * A checkpoint restore zeroes them for the restored system; the replica
 * exchange leaves them with the walker slot, not the configuration.
 * Errors: INVALID_ARG, CUDA. */
int mucal_set_tunnel_window(void *ctx, int32_t sys, int32_t e_min, int32_t e_max);
int mucal_get_tunnel_counts(void *ctx, int32_t sys, int64_t *total, uint32_t *per_walker,
                            uint8_t *state);
int mucal_reset_tunnel_counts(void *ctx);

/* ---- replica exchange (parallel tempering, Sec. 3) ------------------------
 * The energy ranges of the multicanonical runs come from short parallel-
 * tempering runs.  A context whose n_sys systems are copies of one lattice
 * (same d, L, N, walker count and window), system k set to the canonical
 * weights lnW_k(E) = -beta[k] E with mucal_set_weights, is a tempering
 * ladder: walker w of system k is replica w at inverse temperature beta[k],
 * and mucal_run_iteration is its canonical Metropolis update.
 * mucal_replica_exchange proposes, for every walker w and every pair of
 * systems (k, k+1) with k = parity, parity + 2, ... (k + 1 < n_sys), to
 * exchange the configurations of walker w of the two systems, accepted with
 * probability min(1, exp((beta[k] - beta[k+1]) (E_k - E_k+1))): per pair
 * and energy difference the host builds in double precision a uint32
 * threshold T (0xFFFFFFFF if the exponent is >= 0, else
 * min(floor(2^32 exp(exponent)), 0xFFFFFFFE)) and the device accepts iff
 * T == 0xFFFFFFFF or r < T, r = word 0 of Philox4x32-10 with walker w's key
 * of system k (seed_base_k + w) and counter (round, 0, 0, 2).  Asynchronous
 * on the context's stream; accepted (nullable, host int64[n_sys - 1])
 * receives the accepted exchanges per pair (pairs not of this parity get 0),
 * in which case the call waits for the stream.  Histograms and weights are
 * not touched.
 * Errors: INVALID_ARG (NULL beta, n_sys not the context's system count or
 * < 2, parity not 0/1, systems that differ, non-finite beta), OOM, CUDA. */
int mucal_replica_exchange(void *ctx, const double *beta, int32_t n_sys, uint32_t round,
                           int32_t parity, int64_t *accepted);

/* ---- largest droplet (Sec. 3) ---------------------------------------------
 * A droplet is a cluster of occupied sites connected through nearest-
 * neighbour bonds of the periodic lattice; its size is its number of
 * particles, and V_D below is the size of the largest one (0 for N = 0).
 * mucal_measure_droplets labels the clusters of every walker's current
 * configuration of every system on the device (asynchronous on the
 * context's stream), stores each walker's V_D, and adds to per-system
 * accumulators indexed by the walker's energy bin: count[b] += 1,
 * sum[b] += V_D, sum2[b] += V_D^2 (exact 64-bit integers).  Call it between
 * iterations as often as measurements are wanted; sum/count is the
 * microcanonical mean that mucal_reweight takes as an observable.
 * mucal_get_droplet_stats: copy the accumulators of sys (each host
 *   int64[n_bins], any may be NULL); waits for the stream.
 * mucal_get_largest_droplets: V_D of each walker of sys at the last
 *   measurement (host int32[n_walkers]); waits for the stream.
 * mucal_reset_droplet_stats: zero the accumulators of every system.
 * Errors: INVALID_ARG, NOT_READY (no measurement yet), CUDA, OOM; an
 * internal consistency failure of the labelling reports MUCAL_ERR_CUDA. */
int mucal_measure_droplets(void *ctx);
int mucal_get_droplet_stats(void *ctx, int32_t sys, int64_t *count, int64_t *sum, int64_t *sum2,
                            int32_t n_bins);
int mucal_get_largest_droplets(void *ctx, int32_t sys, int32_t *V_D, int32_t n_walkers);
int mucal_reset_droplet_stats(void *ctx);

/* ---- droplet theory (Sec. 3, Eqs. 8-10) -----------------------------------
 * mucal_droplet_delta: with the background density rho0, the reduced
 *   compressibility kappa_hat and the surface free energy tau_W, the excess
 *   volume V_L = (N - rho0 V) / (1 - 2 rho0) (Eq. 8) and the dimensionless
 *   Delta = (1 - 2 rho0)^2 / (2 kappa_hat tau_W) * V_L^((d+1)/d) / V
 *   (Eq. 10); Delta = 0 when V_L <= 0.  Either output may be NULL.
 * mucal_droplet_lambda: the infinite-volume fraction lambda in [0, 1) of the
 *   excess held by the largest droplet, the global minimiser over [0, 1] of
 *   lambda^((d-1)/d) + Delta (1 - lambda)^2 (the bracket of Eq. 9): 0 below
 *   the critical Delta_c, and the larger root of the stationarity condition
 *   above it (bisection to double precision).  Where both minima are equal
 *   (Delta = Delta_c) it returns 0.
 * Errors: INVALID_ARG for d outside {2, 3}, V < 1, N < 0, rho0 outside
 *   [0, 1/2), kappa_hat or tau_W <= 0, Delta < 0 or non-finite. */
int mucal_droplet_delta(int32_t d, int64_t V, int64_t N, double rho0, double kappa_hat,
                        double tau_W, double *Delta, double *V_L);
int mucal_droplet_lambda(int32_t d, double Delta, double *lambda);

/* ---- allocation-free walker update (no counterpart in the paper) ---------
 * For callers that cannot allocate device memory: code running where
 * cudaMalloc is not allowed or not wanted, such as inside a memory pool that
 * another framework owns, under a fixed device-memory budget, or between
 * set-up and teardown of a process whose allocator must stay untouched.  It
 * runs what mucal_run_iteration runs for one system (sweeps * N attempted
 * jump moves per walker with fixed thresholds, then H(E) = sum of the
 * walkers' histograms) on device buffers the caller owns, and allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *   sys        one system descriptor (as for mucal_init_systems)
 *   bits       device uint32[n_walkers][ceil(V/32)] occupation bitsets (in/out)
 *   S          device uint16 (V <= 65536) or uint32 [n_walkers][V] particle
 *              sites then empty sites (in/out)
 *   E          device int32[n_walkers] energies, inside the window (in/out)
 *   thr        device uint32[n_bins][4d+1] thresholds as built by
 *              mucal_set_weights (read with mucal_get_thresholds) (in)
 *   H          device uint64[n_bins], overwritten with H(E) (out)
 *   cuda_stream the stream to run on (NULL = legacy default stream); the call
 *              returns after that stream has finished the work.
 * Scratch (per-block histogram rows, accept counters, an input-check flag)
 * is a fixed array of 40 MiB in the library that every GPU which loads the
 * library holds until the process exits.  Limits: n_walkers <= 1048576 and
 * ceil(n_walkers / 32) * n_bins <= 4194304; larger sizes return
 * MUCAL_ERR_INVALID_ARG with a message.  Energies outside the window or list
 * entries outside the lattice are detected on the device and reported as
 * MUCAL_ERR_INVALID_ARG (bits, S and E are then left unchanged; H is
 * cleared).  The first call on a device looks up the scratch array's device
 * address and sets the kernels' shared-memory limit; make that first call
 * before any stream capture.  The look-up is repeated when the device's
 * context has been replaced (after cudaDeviceReset).  Every call reads the
 * input check's result back to the host, so it returns only after
 * cuda_stream has finished its work.  All calls share the one scratch
 * array, which keeps the last call's contents (the call clears what must
 * start at zero): calls that overlap on the GPU, from several streams or
 * threads, race and give wrong results.  mucal_run_walkers_noalloc_error()
 * returns the message of the calling thread's last failure. */
int mucal_run_walkers_noalloc(const mucal_system_desc *sys, int64_t sweeps, uint32_t iteration,
                              uint32_t *bits, void *S, int32_t *E, const uint32_t *thr, uint64_t *H,
                              void *cuda_stream);
const char *mucal_run_walkers_noalloc_error(void);

/* ---- weight-seeding network (not part of the paper) ---------------------
 * A 4-128-128-1 multilayer perceptron with GELU activations (gelu(z) =
 * z Phi(z)) that maps a caller-built feature vector of (d, L, rho, E/V) to a
 * prediction of ln Omega(E)/V.  Its only use is to propose starting weights
 * lnW = -V * prediction for the iteration of Sec. 2, which then runs
 * unchanged (the plain start lnW = 0 stays available).  Parameters:
 * fp32 master copy and Adam state; the forward and backward passes use the
 * bf16-rounded parameters, run the 128x128 layer on the tensor cores (bf16 x
 * bf16, fp32 accumulation; the layer-1 activations enter it as two bf16 terms,
 * hi + lo) and everything else in fp32.
 * Parameter vector (fp32, 17281 = mucal_mlp_param_count()): W1[128][4],
 * b1[128], W2[128][128] (row = output unit), b2[128], W3[128], b3.
 * Loss: mean over the batch of (y - t)^2.  All buffers are host buffers,
 * copied during the call; rows are 4 consecutive floats. */
int mucal_mlp_param_count(void);

/* Create a network with the given initial parameters (host fp32[n], n =
 * 17281) on the current device; cuda_stream NULL = own stream.  Errors:
 * INVALID_ARG, NO_DEVICE, OOM, CUDA. */
int mucal_mlp_create(void **out, const float *params, int64_t n, void *cuda_stream);
void mucal_mlp_destroy(void *mlp);
const char *mucal_mlp_last_error(void *mlp);

/* Copy the parameters to params[n]: the fp32 master copy (rounded = 0) or
 * the bf16-rounded values the kernels compute with, widened to fp32
 * (rounded = 1). */
int mucal_mlp_get_params(void *mlp, float *params, int64_t n, int32_t rounded);

/* y[B] = network(X[B][4]). */
int mucal_mlp_forward(void *mlp, const float *X, int64_t B, float *y);

/* y[B] = network(X[B][4]) with the 128x128 layer on the fifth-generation
 * tensor cores (tcgen05.mma, accumulator in tensor memory; 128 rows per CTA).
 * Same numerics as mucal_mlp_forward up to the order of fp32 sums.  Errors:
 * INVALID_ARG, OOM, CUDA, STATE (a tensor-core wait ran out). */
int mucal_mlp_forward_tcgen05(void *mlp, const float *X, int64_t B, float *y);

/* Select the tensor-core path of mucal_mlp_forward, mucal_mlp_gradients and
 * mucal_mlp_train: enable = 1 runs every 128x128 contraction (Z2 = H1 W2^T,
 * dH1 = dZ2 W2 and dW2 = dZ2^T H1 over each 128-row tile) with tcgen05.mma
 * on tensor memory (the default); 0 uses mma.sync.  The numerics are the
 * same (bf16 operands, fp32 accumulation) up to the order of fp32 sums.
 * The tensor-core path sums the gradients of its 128-row tiles in tile order
 * (run to run the same bits); the mma.sync path adds them with atomics, in
 * whatever order its blocks finish. */
int mucal_mlp_use_tcgen05(void *mlp, int32_t enable);

/* One forward and backward pass of the mean squared error against t[B]:
 * loss (nullable) and the gradient with respect to all 17281 parameters
 * (grad nullable, host fp32[17281]).  Parameters are not changed. */
int mucal_mlp_gradients(void *mlp, const float *X, const float *t, int64_t B, float *loss, float *grad);

/* steps full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) with
 * learning rate lr on (X, t), entirely on the device; loss_out (nullable)
 * receives the loss of the last step's forward pass. */
int mucal_mlp_train(void *mlp, const float *X, const float *t, int64_t B, int32_t steps, float lr,
                    float *loss_out);

#ifdef __cplusplus
}
#endif

#endif /* MUCAL_H */
