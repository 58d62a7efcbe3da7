/*
 * CPU oracle for the parallel multicanonical lattice gas.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
 * which the CUDA path is checked.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Model (Sec. 3, Eq. 5): sites i of a periodic L^d lattice carry n_i in {0,1};
 * E = -J * sum over nearest-neighbour pairs <i,j> of n_i n_j with J = 1 and a
 * fixed particle number N.
 *
 * Method (Sec. 2): every walker is an independent equilibrium Markov chain with
 * the same weights W(E); a proposed state is accepted with min(1, W(E_n)/W(E_o))
 * (the acceptance printed after Eq. 1).  Each walker fills its own histogram
 * H_j(E); the histograms are summed (Eq. 2).
 *
 * The readings of what the paper leaves open (the move set, the random-number
 * layout, the threshold quantisation, when a histogram entry is recorded) are:
 *   - move: a nonlocal jump of a uniformly chosen particle to a uniformly
 *     chosen empty site;
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key = 64-bit walker seed, counter = (t_lo, t_hi, iteration, stream tag),
 *     tag 0 for moves and 1 for the initial placement;
 *   - acceptance: a uint32 threshold T(E_o, dE) built in double precision;
 *     accept iff T == 0xFFFFFFFF or r < T;
 *   - every attempt, accepted or not, records the energy after the attempt.
 *
 * Occupation is stored as one byte per site here (the CUDA path bit-packs);
 * plain loops throughout.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon et al.,    */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of     */
/* two 32x32->64 multiplications on counter words 0 and 2, with the high    */
/* halves xor-ed into the other two words together with the round key; the  */
/* key is advanced by the two Weyl constants between rounds.                */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for the tests: n counters and keys in, n blocks of four out. */
void orc_philox_batch(int64_t n, const uint32_t *ctrs, const uint32_t *keys, uint32_t *outs)
{
    for (int64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctrs + 4 * i, keys + 2 * i, outs + 4 * i);
}

static void orc_key_of_seed(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
}

/* Multiply-high range reduction: floor(r * n / 2^32), in [0, n). */
static uint32_t orc_below(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 3): site s = sum_k x_k L^k with x_0 fastest; periodic.     */
/* ------------------------------------------------------------------------ */
int64_t orc_volume(int d, int L)
{
    int64_t v = 1;
    for (int k = 0; k < d; ++k) v *= L;
    return v;
}

/* The 2d nearest neighbours of s: for each axis k, x_k - 1 and x_k + 1 (mod L). */
void orc_neighbours(int d, int L, int64_t s, int64_t *nb)
{
    int64_t stride = 1;
    for (int k = 0; k < d; ++k) {
        int64_t xk = (s / stride) % L;
        int64_t base = s - xk * stride;
        int64_t down = (xk + L - 1) % L;
        int64_t up = (xk + 1) % L;
        nb[2 * k + 0] = base + down * stride;
        nb[2 * k + 1] = base + up * stride;
        stride *= L;
    }
}

/* E = -J * #{unordered nearest-neighbour pairs with both sites occupied} (Eq. 5,
 * J = 1).  Every pair is counted once by looking only in the +1 direction of
 * each axis; this needs L >= 3 so that +1 and -1 are different sites. */
int64_t orc_energy(int d, int L, const uint8_t *occ)
{
    int64_t V = orc_volume(d, L);
    int64_t pairs = 0;
    int64_t nb[6];
    for (int64_t s = 0; s < V; ++s) {
        if (!occ[s]) continue;
        orc_neighbours(d, L, s, nb);
        for (int k = 0; k < d; ++k)
            if (occ[nb[2 * k + 1]]) ++pairs;
    }
    return -pairs;
}

/* Energy change of moving the particle at a to the empty site b (a occupied,
 * b empty).  Bonds lost: occupied neighbours of a.  Bonds gained: occupied
 * neighbours of b other than a itself (a is emptied by the move). */
int orc_delta_e(int d, int L, const uint8_t *occ, int64_t a, int64_t b)
{
    int64_t nb[6];
    int n_a = 0, n_b = 0;
    orc_neighbours(d, L, a, nb);
    for (int k = 0; k < 2 * d; ++k) n_a += occ[nb[k]];
    orc_neighbours(d, L, b, nb);
    for (int k = 0; k < 2 * d; ++k)
        if (nb[k] != a) n_b += occ[nb[k]];
    /* E = -pairs: losing n_a pairs raises E by n_a, gaining n_b lowers it. */
    return n_a - n_b;
}

/* ------------------------------------------------------------------------ */
/* Initial placement: uniform random N-subset by a partial Fisher-Yates     */
/* shuffle of the site list, driven by the init stream (tag 1).  Output j  */
/* of the stream is word j%4 of Philox(counter=(j/4 lo, j/4 hi, 0, 1)).     */
/* S[0..N) are the particle sites, S[N..V) the empty sites, in array order. */
/* ------------------------------------------------------------------------ */
void orc_init_walker(int d, int L, int N, uint64_t seed, int32_t *S, uint8_t *occ, int64_t *E)
{
    int64_t V = orc_volume(d, L);
    uint32_t key[2], ctr[4], out[4];
    orc_key_of_seed(seed, key);
    for (int64_t i = 0; i < V; ++i) S[i] = (int32_t)i;
    for (int64_t j = 0; j < N; ++j) {
        uint64_t block = (uint64_t)j / 4;
        ctr[0] = (uint32_t)(block & 0xFFFFFFFFu);
        ctr[1] = (uint32_t)(block >> 32);
        ctr[2] = 0;
        ctr[3] = 1;
        orc_philox4x32_10(ctr, key, out);
        uint32_t r = out[j % 4];
        int64_t idx = j + (int64_t)orc_below(r, (uint32_t)(V - j));
        int32_t tmp = S[j];
        S[j] = S[idx];
        S[idx] = tmp;
    }
    memset(occ, 0, (size_t)V);
    for (int64_t j = 0; j < N; ++j) occ[S[j]] = 1;
    *E = orc_energy(d, L, occ);
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds.  The acceptance min(1, W(E_n)/W(E_o)) (Sec. 2)    */
/* becomes a 32-bit threshold per old-energy bin and energy change dE in    */
/* [-2d, 2d]: 0 when E_n leaves the window [e_lo, e_hi] (never accepted),   */
/* 0xFFFFFFFF when lnW(E_n) >= lnW(E_o) (always accepted), otherwise        */
/* min(floor(2^32 exp(lnW(E_n) - lnW(E_o))), 0xFFFFFFFE).                     */
/* Layout: T[bin * (4d+1) + (dE + 2d)], bin = E_o - e_lo.                    */
/* ------------------------------------------------------------------------ */
void orc_thresholds(int d, int e_lo, int e_hi, const double *lnW, uint32_t *T)
{
    int nb = e_hi - e_lo + 1;
    int width = 4 * d + 1;
    for (int bin = 0; bin < nb; ++bin) {
        for (int de = -2 * d; de <= 2 * d; ++de) {
            int to = bin + de;
            uint32_t t;
            if (to < 0 || to >= nb) {
                t = 0u;
            } else {
                double delta = lnW[to] - lnW[bin];
                if (delta >= 0.0) {
                    t = 0xFFFFFFFFu;
                } else {
                    double x = floor(ldexp(exp(delta), 32));
                    t = (x >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)x;
                }
            }
            T[bin * width + (de + 2 * d)] = t;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One walker, one iteration (Sec. 2): n_attempts Metropolis jump moves     */
/* with fixed weights.  Attempt t draws Philox(counter=(t lo, t hi,         */
/* iteration, 0), key=seed) -> (r0, r1, r2, r3): particle index             */
/* k = floor(r0 N / 2^32), empty-site index m = floor(r1 (V-N) / 2^32),     */
/* acceptance variate r2; r3 is unused.  After the attempt the current E    */
/* is recorded: hist[E - e_lo] += 1.  State (S, occ, E) carries over.       */
/* Returns 0, or -1 if E is outside the window (state left untouched).      */
/* ------------------------------------------------------------------------ */
/* Tunnelling events (Sec. 4): with tstate non-NULL every energy the walker
 * takes (the one it starts with, then the one after every attempt) is
 * compared with the ends: E <= t_min is the low end, E >= t_max the high
 * end.  *tstate records the end reached last (0 none, 1 low, 2 high);
 * reaching the other end adds one to *tcount. */
static void orc_tunnel_check(int64_t e, int t_min, int t_max, uint8_t *tstate, int64_t *tcount)
{
    if (!tstate) return;
    if (e <= t_min) {
        if (*tstate == 2) ++*tcount;
        *tstate = 1;
    } else if (e >= t_max) {
        if (*tstate == 1) ++*tcount;
        *tstate = 2;
    }
}

static int orc_chain(int d, int L, int N, uint64_t seed, uint32_t iteration,
                     int64_t n_attempts, int e_lo, int e_hi, const uint32_t *T,
                     int32_t *S, uint8_t *occ, int64_t *E, int64_t *hist,
                     int64_t *accepts, int t_min, int t_max, uint8_t *tstate,
                     int64_t *tcount)
{
    int64_t V = orc_volume(d, L);
    int width = 4 * d + 1;
    uint32_t key[2], ctr[4], r[4];
    int64_t e = *E;
    int64_t acc = 0;
    if (e < e_lo || e > e_hi) return -1;
    orc_key_of_seed(seed, key);
    orc_tunnel_check(e, t_min, t_max, tstate, tcount);
    for (int64_t t = 0; t < n_attempts; ++t) {
        ctr[0] = (uint32_t)((uint64_t)t & 0xFFFFFFFFu);
        ctr[1] = (uint32_t)((uint64_t)t >> 32);
        ctr[2] = iteration;
        ctr[3] = 0;
        orc_philox4x32_10(ctr, key, r);
        uint32_t k = orc_below(r[0], (uint32_t)N);
        uint32_t m = orc_below(r[1], (uint32_t)(V - N));
        int64_t a = S[k];
        int64_t b = S[N + m];
        int de = orc_delta_e(d, L, occ, a, b);
        uint32_t thr = T[(e - e_lo) * width + (de + 2 * d)];
        if (thr == 0xFFFFFFFFu || r[2] < thr) {
            occ[a] = 0;
            occ[b] = 1;
            S[k] = (int32_t)b;
            S[N + m] = (int32_t)a;
            e += de;
            ++acc;
        }
        hist[e - e_lo] += 1;
        orc_tunnel_check(e, t_min, t_max, tstate, tcount);
    }
    *E = e;
    if (accepts) *accepts += acc;
    return 0;
}

int orc_run_walker(int d, int L, int N, uint64_t seed, uint32_t iteration,
                   int64_t n_attempts, int e_lo, int e_hi, const uint32_t *T,
                   int32_t *S, uint8_t *occ, int64_t *E, int64_t *hist,
                   int64_t *accepts)
{
    return orc_chain(d, L, N, seed, iteration, n_attempts, e_lo, e_hi, T, S, occ, E, hist,
                     accepts, 0, 0, NULL, NULL);
}

/* Many walkers of one system (the p independent processes of Sec. 2),
 * walker w using seed seed_base + w.  States are stored walker-major:
 * S[w*V..], occ[w*V..], E[w], hist[w*n_bins..].  Walkers are independent, so
 * they are spread over the host threads.  Returns the number of walkers whose
 * energy was outside the window (those are left untouched). */
int64_t orc_run_walkers(int d, int L, int N, int64_t n_walkers, uint64_t seed_base,
                        uint32_t iteration, int64_t n_attempts, int e_lo, int e_hi,
                        const uint32_t *T, int32_t *S, uint8_t *occ, int64_t *E,
                        int64_t *hist, int64_t *accepts)
{
    int64_t V = orc_volume(d, L);
    int64_t nb = (int64_t)(e_hi - e_lo + 1);
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t w = 0; w < n_walkers; ++w) {
        int64_t acc = 0;
        int rc = orc_run_walker(d, L, N, seed_base + (uint64_t)w, iteration, n_attempts,
                                e_lo, e_hi, T, S + w * V, occ + w * V, E + w,
                                hist + w * nb, &acc);
        if (rc != 0) ++bad;
        if (accepts) accepts[w] += acc;
    }
    return bad;
}

/* orc_run_walkers with tunnelling bookkeeping per walker: tstate[w],
 * tcount[w] carry over between calls (see orc_tunnel_check). */
int64_t orc_run_walkers_tunnel(int d, int L, int N, int64_t n_walkers, uint64_t seed_base,
                               uint32_t iteration, int64_t n_attempts, int e_lo, int e_hi,
                               const uint32_t *T, int32_t *S, uint8_t *occ, int64_t *E,
                               int64_t *hist, int t_min, int t_max, uint8_t *tstate,
                               int64_t *tcount)
{
    int64_t V = orc_volume(d, L);
    int64_t nb = (int64_t)(e_hi - e_lo + 1);
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t w = 0; w < n_walkers; ++w) {
        int rc = orc_chain(d, L, N, seed_base + (uint64_t)w, iteration, n_attempts, e_lo, e_hi,
                           T, S + w * V, occ + w * V, E + w, hist + w * nb, NULL, t_min, t_max,
                           tstate + w, tcount + w);
        if (rc != 0) ++bad;
    }
    return bad;
}

void orc_init_walkers(int d, int L, int N, int64_t n_walkers, uint64_t seed_base,
                      int32_t *S, uint8_t *occ, int64_t *E)
{
    int64_t V = orc_volume(d, L);
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < n_walkers; ++w)
        orc_init_walker(d, L, N, seed_base + (uint64_t)w, S + w * V, occ + w * V, E + w);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Exact density of states by enumerating every N-subset of the V sites     */
/* (feasible for V <= 64 and small C(V,N)).  omega[-E] counts the           */
/* configurations of energy E, E in [-dN, 0].  Returns the number of        */
/* configurations visited, or -1 if V > 64.                                 */
/* ------------------------------------------------------------------------ */
static void orc_enum_rec(int d, int L, int64_t V, int N, int64_t start, int placed,
                         uint8_t *occ, int64_t *omega, int64_t *count)
{
    if (placed == N) {
        int64_t e = orc_energy(d, L, occ);
        omega[-e] += 1;
        *count += 1;
        return;
    }
    for (int64_t s = start; s <= V - (N - placed); ++s) {
        occ[s] = 1;
        orc_enum_rec(d, L, V, N, s + 1, placed + 1, occ, omega, count);
        occ[s] = 0;
    }
}

int64_t orc_enumerate(int d, int L, int N, int64_t *omega)
{
    int64_t V = orc_volume(d, L);
    if (V > 64) return -1;
    uint8_t occ[64];
    int64_t count = 0;
    memset(occ, 0, sizeof occ);
    memset(omega, 0, sizeof(int64_t) * (size_t)(d * N + 1));
    orc_enum_rec(d, L, V, N, 0, 0, occ, omega, &count);
    return count;
}

/* Energy of a configuration given as a bitmask of occupied sites (V <= 64). */
int64_t orc_energy_mask(int d, int L, uint64_t mask)
{
    int64_t V = orc_volume(d, L);
    uint8_t occ[64];
    for (int64_t s = 0; s < V; ++s) occ[s] = (uint8_t)((mask >> s) & 1u);
    return orc_energy(d, L, occ);
}

/* Energy change of moving site a to site b for a configuration bitmask. */
int orc_delta_e_mask(int d, int L, uint64_t mask, int64_t a, int64_t b)
{
    int64_t V = orc_volume(d, L);
    uint8_t occ[64];
    for (int64_t s = 0; s < V; ++s) occ[s] = (uint8_t)((mask >> s) & 1u);
    return orc_delta_e(d, L, occ, a, b);
}

/* ------------------------------------------------------------------------ */
/* Ising model at fixed magnetisation (the "micromagnetic" Metropolis       */
/* simulation of Sec. 4): spins s_i = 2 n_i - 1, H^I = -J sum_<ij> s_i s_j, */
/* canonical weight exp(-beta^I H^I).  A move exchanges a uniformly chosen  */
/* up spin with a uniformly chosen down spin (M fixed); accepted with       */
/* min(1, exp(-beta^I dH^I)) computed in double precision.  Random numbers: */
/* Philox with counter (t lo, t hi, 0, 2): r0 picks the up spin, r1 the     */
/* down spin, r2 / 2^32 is the uniform variate.  Records sum of H^I and of  */
/* (H^I)^2 after every attempt.  n_up plays the role of N.                  */
/* ------------------------------------------------------------------------ */
static int64_t orc_ising_energy(int d, int L, const int8_t *spin)
{
    int64_t V = orc_volume(d, L);
    int64_t sum = 0;
    int64_t nb[6];
    for (int64_t s = 0; s < V; ++s) {
        orc_neighbours(d, L, s, nb);
        for (int k = 0; k < d; ++k) sum += (int64_t)spin[s] * spin[nb[2 * k + 1]];
    }
    return -sum;
}

int orc_ising_fixed_m(int d, int L, int n_up, uint64_t seed, double beta_ising,
                      int64_t n_attempts, int64_t n_discard, double *mean_e, double *mean_e2)
{
    int64_t V = orc_volume(d, L);
    int8_t *spin = (int8_t *)malloc((size_t)V);
    int64_t *up = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    int64_t *down = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    if (!spin || !up || !down) { free(spin); free(up); free(down); return -1; }
    /* initial state: the first n_up sites up (a deterministic start; the
     * discarded attempts equilibrate it). */
    int64_t nu = 0, nd = 0;
    for (int64_t s = 0; s < V; ++s) {
        spin[s] = (s < n_up) ? 1 : -1;
        if (spin[s] > 0) up[nu++] = s; else down[nd++] = s;
    }
    int64_t h = orc_ising_energy(d, L, spin);
    uint32_t key[2], ctr[4], r[4];
    int64_t nb[6];
    orc_key_of_seed(seed, key);
    double se = 0.0, se2 = 0.0;
    int64_t nrec = 0;
    for (int64_t t = 0; t < n_attempts; ++t) {
        ctr[0] = (uint32_t)((uint64_t)t & 0xFFFFFFFFu);
        ctr[1] = (uint32_t)((uint64_t)t >> 32);
        ctr[2] = 0;
        ctr[3] = 2;
        orc_philox4x32_10(ctr, key, r);
        int64_t iu = orc_below(r[0], (uint32_t)nu);
        int64_t id = orc_below(r[1], (uint32_t)nd);
        int64_t a = up[iu], b = down[id];
        /* exchange: recompute the energy from scratch (plain, not local) */
        spin[a] = -1; spin[b] = 1;
        int64_t h_new = orc_ising_energy(d, L, spin);
        (void)nb;
        double dh = (double)(h_new - h);
        double u = (double)r[2] / 4294967296.0;
        if (dh <= 0.0 || u < exp(-beta_ising * dh)) {
            h = h_new;
            up[iu] = b;
            down[id] = a;
        } else {
            spin[a] = 1; spin[b] = -1;
        }
        if (t >= n_discard) {
            se += (double)h;
            se2 += (double)h * (double)h;
            ++nrec;
        }
    }
    *mean_e = nrec ? se / (double)nrec : 0.0;
    *mean_e2 = nrec ? se2 / (double)nrec : 0.0;
    free(spin); free(up); free(down);
    return 0;
}

/* Largest droplet (Sec. 3): the number of particles in the largest set of
 * occupied sites connected through nearest-neighbour bonds of the periodic
 * lattice; 0 for an empty lattice.  Breadth-first search from every
 * not-yet-seen particle, with an explicit queue. */
int64_t orc_largest_cluster(int d, int L, const uint8_t *occ)
{
    int64_t V = orc_volume(d, L);
    uint8_t *seen = (uint8_t *)calloc((size_t)V, 1);
    int64_t *queue = (int64_t *)malloc((size_t)V * sizeof(int64_t));
    int64_t best = 0;
    int64_t nb[6];
    for (int64_t start = 0; start < V; ++start) {
        if (!occ[start] || seen[start]) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = start;
        seen[start] = 1;
        while (head < tail) {
            int64_t s = queue[head++];
            orc_neighbours(d, L, s, nb);
            for (int k = 0; k < 2 * d; ++k) {
                int64_t t = nb[k];
                if (occ[t] && !seen[t]) {
                    seen[t] = 1;
                    queue[tail++] = t;
                }
            }
        }
        if (tail > best) best = tail;
    }
    free(seen);
    free(queue);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Replica exchange (parallel tempering; Sec. 3 takes its energy ranges     */
/* from short tempering runs).  K copies of one lattice at inverse          */
/* temperatures beta[k], n_walkers replicas each; arrays are               */
/* S[K][n_walkers][V], occ[K][n_walkers][V], E[K][n_walkers].  For each     */
/* pair (k, k+1) with k = parity, parity + 2, ... and each walker w, the    */
/* configurations of the two systems' walker w trade places with            */
/* probability min(1, exp((beta_k - beta_k+1) (E_k - E_k+1))), in the same */
/* uint32 form as the move acceptance (always if the exponent is >= 0,      */
/* else iff r < min(floor(2^32 e^x), 0xFFFFFFFE)) with r = word 0 of        */
/* Philox(counter = (round, 0, 0, 2), key = seeds[k] + w).  accepted[k]     */
/* counts the exchanges of pair k (the caller zeroes it).                    */
/* ------------------------------------------------------------------------ */
void orc_replica_exchange(int K, int64_t n_walkers, int64_t V, const uint64_t *seeds,
                          const double *beta, uint32_t round, int parity, int32_t *S,
                          uint8_t *occ, int64_t *E, int64_t *accepted)
{
    for (int k = parity; k + 1 < K; k += 2) {
        for (int64_t w = 0; w < n_walkers; ++w) {
            int64_t ia = (int64_t)k * n_walkers + w;
            int64_t ib = (int64_t)(k + 1) * n_walkers + w;
            uint32_t key[2], ctr[4] = {round, 0u, 0u, 2u}, r[4];
            orc_key_of_seed(seeds[k] + (uint64_t)w, key);
            orc_philox4x32_10(ctr, key, r);
            double x = (beta[k] - beta[k + 1]) * (double)(E[ia] - E[ib]);
            int take;
            if (x >= 0.0) {
                take = 1;
            } else {
                double q = floor(ldexp(exp(x), 32));
                uint32_t t = (q >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)q;
                take = r[0] < t;
            }
            if (!take) continue;
            ++accepted[k];
            for (int64_t i = 0; i < V; ++i) {
                int32_t ts = S[ia * V + i];
                S[ia * V + i] = S[ib * V + i];
                S[ib * V + i] = ts;
                uint8_t to = occ[ia * V + i];
                occ[ia * V + i] = occ[ib * V + i];
                occ[ib * V + i] = to;
            }
            int64_t te = E[ia];
            E[ia] = E[ib];
            E[ib] = te;
        }
    }
}
