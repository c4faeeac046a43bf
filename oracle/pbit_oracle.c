/*
 * pbit_oracle.c -- plain, slow CPU oracle for the graph-coloured parallel p-bit
 * annealer of "Probabilistic Computing Optimization of Complex Spin-Glass
 * Topologies" (arXiv 2510.23419).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline / reference arm of the benchmark may load this file.  The
 * CUDA library never links, calls or includes it, and it shares no code with
 * the library: its own Philox, its own instance generator, its own schedule,
 * its own threshold rule, its own energy.
 *
 * Everything floating is FP64.  Loops are plain and follow the paper's
 * definitions in order; there is no blocking, fusion or reordering.
 *
 * Readings of the paper that this file fixes (each is also listed in the
 * design notes of the repository):
 *   - Energy (Eq. 1 with the sign that makes Eq. 2/3 sample exp(-beta E)):
 *       E(m) = - sum_{edges (i,j)} J_ij m_i m_j - sum_i h_i m_i.
 *   - Local field (Eq. 3 with the field term): F_i = sum_j J_ij m_j + h_i,
 *     p-bit input I_i = beta F_i.
 *   - p-bit (Eq. 2, bipolar, tanh form of the sigmoid): m_i = +1 with
 *     probability 1/2 + tanh(I_i)/2.  One uint32 random word r decides:
 *       T = min(floor((0.5 + 0.5*tanh(beta*F)) * 2^32), 2^32 - 1),
 *       m_i = +1 iff r < T.
 *   - Update groups (Sec. 1.2.2): colour classes are updated one after the
 *     other, colour 0 first; a class has no internal edge, so the order inside
 *     a class does not matter.  One sweep = every class once.
 *   - beta is one value per sweep (classical annealing, Sec. 1.3.1).
 *   - Random words: Philox4x32-10, key = (seed lo, seed hi),
 *     counter = (k, s, r >> 2, (tag << 24) | c), word index r & 3, where k is
 *     the rank of spin i inside its colour class c (ascending index), s the
 *     sweep, r the replica; tag 0 = decisions, tag 1 = initial state.
 *   - Initial state: m_i = +1 iff word(tag 1, s = 0) < 2^31.
 *   - Running lowest energy (Fig. 1A): the best state starts as the initial
 *     state (best sweep -1); after every full sweep, if E < best (strictly)
 *     the best energy, sweep and state are replaced.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of the counter    */
/* words 0 and 2 with the published multipliers; the high halves are xored   */
/* with the other two counter words and the round key; the key is bumped by  */
/* the published Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
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

/* One 32-bit word of the stream: Philox(counter, key = seed) word idx. */
uint32_t orc_rand_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int idx)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[idx & 3];
}

/* Bulk helper for the tests: n counters/keys in, n x 4 words out. */
void orc_philox_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t t = 0; t < n; ++t)
        orc_philox4x32_10(ctr + 4 * t, key + 2 * t, out + 4 * t);
}

#define ORC_TAG_DECISION 0u
#define ORC_TAG_INIT 1u
#define ORC_TAG_INSTANCE 2u

/* ------------------------------------------------------------------------ */
/* Instance generation (random couplings, Sec. 2 cubic lattices and Sec. 3   */
/* bicliques with couplings drawn from [-1, 1]).  Coupling e draws from the  */
/* tag-2 stream:                                                             */
/*   dist 0 (+-1):   word(e>>2, 0, 0, 2<<24)[e&3] < 2^31 -> +1, else -1      */
/*   dist 1 (N(0,1)): Box-Muller on words 0,1 of (e, 1, 0, 2<<24),           */
/*                    u = (w + 0.5) / 2^32, z = sqrt(-2 ln u0) cos(2 pi u1), */
/*                    stored rounded to FP32                                 */
/*   dist 2 (U(-1,1)): word(e>>2, 2, 0, 2<<24)[e&3], u = (w+0.5)/2^32,       */
/*                    J = 2u - 1 rounded to FP32                             */
/* ------------------------------------------------------------------------ */
#define ORC_TWO_PI 6.283185307179586476925286766559
#define ORC_TWO_POW_32 4294967296.0

double orc_coupling(int dist, uint64_t seed, int64_t e)
{
    const uint32_t c3 = ORC_TAG_INSTANCE << 24;
    if (dist == 0) {
        uint32_t w = orc_rand_word(seed, (uint32_t)(e >> 2), 0u, 0u, c3, (int)(e & 3));
        return (w < 0x80000000u) ? 1.0 : -1.0;
    }
    if (dist == 1) {
        uint32_t w0 = orc_rand_word(seed, (uint32_t)e, 1u, 0u, c3, 0);
        uint32_t w1 = orc_rand_word(seed, (uint32_t)e, 1u, 0u, c3, 1);
        double u0 = ((double)w0 + 0.5) / ORC_TWO_POW_32;
        double u1 = ((double)w1 + 0.5) / ORC_TWO_POW_32;
        double z = sqrt(-2.0 * log(u0)) * cos(ORC_TWO_PI * u1);
        return (double)(float)z;
    }
    {
        uint32_t w = orc_rand_word(seed, (uint32_t)(e >> 2), 2u, 0u, c3, (int)(e & 3));
        double u = ((double)w + 0.5) / ORC_TWO_POW_32;
        return (double)(float)(2.0 * u - 1.0);
    }
}

/* EA cube of side L, periodic: bond e = d*N + i joins site i to its +x
 * (d=0), +y (d=1) or +z (d=2) neighbour; site i = x + L*(y + L*z). */
void orc_gen_ea(int32_t L, int32_t dist, uint64_t seed, double* J)
{
    int64_t N = (int64_t)L * L * L;
    for (int64_t e = 0; e < 3 * N; ++e) J[e] = orc_coupling(dist, seed, e);
}

/* Biclique K_{n,n}: bond e = i*n + j joins left spin i to right spin j. */
void orc_gen_biclique(int32_t n, int32_t dist, uint64_t seed, double* J)
{
    for (int64_t e = 0; e < (int64_t)n * n; ++e) J[e] = orc_coupling(dist, seed, e);
}

/* ------------------------------------------------------------------------ */
/* Topologies as explicit edge lists.                                        */
/* ------------------------------------------------------------------------ */
void orc_ea_edges(int32_t L, int32_t* eu, int32_t* ev)
{
    int64_t N = (int64_t)L * L * L;
    for (int32_t z = 0; z < L; ++z)
        for (int32_t y = 0; y < L; ++y)
            for (int32_t x = 0; x < L; ++x) {
                int64_t i = x + (int64_t)L * (y + (int64_t)L * z);
                int64_t nx = ((x + 1) % L) + (int64_t)L * (y + (int64_t)L * z);
                int64_t ny = x + (int64_t)L * (((y + 1) % L) + (int64_t)L * z);
                int64_t nz = x + (int64_t)L * (y + (int64_t)L * ((z + 1) % L));
                eu[0 * N + i] = (int32_t)i; ev[0 * N + i] = (int32_t)nx;
                eu[1 * N + i] = (int32_t)i; ev[1 * N + i] = (int32_t)ny;
                eu[2 * N + i] = (int32_t)i; ev[2 * N + i] = (int32_t)nz;
            }
}

/* Checkerboard colouring (Sec. 1.2.2: the cubic lattice is bipartite). */
void orc_ea_colour(int32_t L, int32_t* colour)
{
    for (int32_t z = 0; z < L; ++z)
        for (int32_t y = 0; y < L; ++y)
            for (int32_t x = 0; x < L; ++x)
                colour[x + L * (y + L * z)] = (x + y + z) & 1;
}

/* Left spins 0..n-1, right spins n..2n-1. */
void orc_biclique_edges(int32_t n, int32_t* eu, int32_t* ev)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            eu[(int64_t)i * n + j] = i;
            ev[(int64_t)i * n + j] = n + j;
        }
}

void orc_biclique_colour(int32_t n, int32_t* colour)
{
    for (int32_t i = 0; i < 2 * n; ++i) colour[i] = (i < n) ? 0 : 1;
}

/* Number of edges whose two ends share a colour (a proper colouring has 0). */
int64_t orc_count_monochrome(int64_t n_edges, const int32_t* eu, const int32_t* ev, const int32_t* colour)
{
    int64_t bad = 0;
    for (int64_t e = 0; e < n_edges; ++e)
        if (colour[eu[e]] == colour[ev[e]]) ++bad;
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Energy, Eq. 1 (sign reading above).                                       */
/* ------------------------------------------------------------------------ */
double orc_energy(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J,
                  const double* h, const int8_t* m)
{
    double E = 0.0;
    for (int64_t e = 0; e < n_edges; ++e) E -= J[e] * (double)m[eu[e]] * (double)m[ev[e]];
    if (h)
        for (int32_t i = 0; i < N; ++i) E -= h[i] * (double)m[i];
    return E;
}

/* Energies of all 2^N states; bit i of the state index set <=> m_i = +1. */
int orc_brute_force(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J,
                    const double* h, double* energies)
{
    if (N > 24) return -1;
    int8_t* m = (int8_t*)malloc((size_t)N);
    if (!m) return -2;
    for (int64_t st = 0; st < ((int64_t)1 << N); ++st) {
        for (int32_t i = 0; i < N; ++i) m[i] = ((st >> i) & 1) ? 1 : -1;
        energies[st] = orc_energy(N, n_edges, eu, ev, J, h, m);
    }
    free(m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Annealing schedule (Sec. 1.3.1 classical annealing; Algorithm 1 linear    */
/* beta step; optional step duration d).  Level l = floor(s / d) of          */
/* Lv = ceil(S / d) levels; both end points are included:                    */
/*   linear:    beta0 + (beta1 - beta0) * l / (Lv - 1)                       */
/*   geometric: beta0 * (beta1 / beta0)^(l / (Lv - 1))                       */
/*   explicit:  betas given per sweep                                        */
/* A single level uses beta0.                                                */
/* ------------------------------------------------------------------------ */
int orc_schedule(int32_t kind, double beta0, double beta1, int32_t S, int32_t d, const double* explicit_betas,
                 double* betas)
{
    if (S < 0 || d < 1) return -1;
    if (kind == 2) {
        for (int32_t s = 0; s < S; ++s) betas[s] = explicit_betas[s];
        return 0;
    }
    int32_t Lv = (S + d - 1) / d;
    for (int32_t s = 0; s < S; ++s) {
        int32_t l = s / d;
        double frac = (Lv > 1) ? (double)l / (double)(Lv - 1) : 0.0;
        if (kind == 0)
            betas[s] = beta0 + (beta1 - beta0) * frac;
        else if (kind == 1)
            betas[s] = beta0 * pow(beta1 / beta0, frac);
        else
            return -1;
    }
    return 0;
}

/* p-bit decision threshold (Eq. 2 with the uint32 reading above). */
uint32_t orc_threshold(double beta, double F)
{
    double P = 0.5 + 0.5 * tanh(beta * F);
    double T = floor(P * ORC_TWO_POW_32);
    if (T > 4294967295.0) T = 4294967295.0;
    if (T < 0.0) T = 0.0;
    return (uint32_t)T;
}

/* Local fields of one state (Eq. 3 with the field term): F_i = sum_j J_ij m_j + h_i. */
void orc_fields(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J,
                const double* h, const int8_t* m, double* F)
{
    for (int32_t i = 0; i < N; ++i) F[i] = h ? h[i] : 0.0;
    for (int64_t e = 0; e < n_edges; ++e) {
        F[eu[e]] += J[e] * (double)m[ev[e]];
        F[ev[e]] += J[e] * (double)m[eu[e]];
    }
}

/* ------------------------------------------------------------------------ */
/* Classical annealing of replicas r_first .. r_first+R-1 (independent; a    */
/* replica's trajectory depends only on its own index), with update groups.  */
/* Outputs are indexed 0..R-1.  Returns 0 on success, -1 on bad arguments, -2 if the colouring has an     */
/* internal edge, -3 on allocation failure.                                  */
/*   trace_E   optional [R][S] energy after each sweep                       */
/*   max_incr_err optional: largest |incremental E - recomputed E| seen      */
/* ------------------------------------------------------------------------ */
int orc_anneal(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J,
               const double* h, const int32_t* colour, int32_t n_colours, const double* betas, int32_t S,
               int32_t r_first, int32_t R, uint64_t seed, double* final_E, double* best_E, int32_t* best_sweep,
               int8_t* final_state, int8_t* best_state, double* trace_E, double* max_incr_err)
{
    if (N < 1 || R < 0 || r_first < 0 || S < 0 || n_colours < 1 || n_colours > 255) return -1;
    for (int32_t i = 0; i < N; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return -1;
    if (orc_count_monochrome(n_edges, eu, ev, colour) != 0) return -2;

    /* adjacency lists (each edge seen from both ends) */
    int64_t* deg = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc((size_t)(2 * n_edges + 1) * sizeof(int32_t));
    double* adjJ = (double*)malloc((size_t)(2 * n_edges + 1) * sizeof(double));
    int64_t* fill = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    uint32_t* rank = (uint32_t*)malloc((size_t)N * sizeof(uint32_t));
    int8_t* m = (int8_t*)malloc((size_t)N);
    if (!deg || !adj || !adjJ || !fill || !rank || !m) {
        free(deg); free(adj); free(adjJ); free(fill); free(rank); free(m);
        return -3;
    }
    for (int64_t e = 0; e < n_edges; ++e) {
        deg[eu[e] + 1]++;
        deg[ev[e] + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) deg[i + 1] += deg[i];
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t u = eu[e], v = ev[e];
        adj[deg[u] + fill[u]] = v; adjJ[deg[u] + fill[u]] = J[e]; fill[u]++;
        adj[deg[v] + fill[v]] = u; adjJ[deg[v] + fill[v]] = J[e]; fill[v]++;
    }
    /* rank of each spin inside its colour class, ascending index */
    for (int32_t c = 0; c < n_colours; ++c) {
        uint32_t k = 0;
        for (int32_t i = 0; i < N; ++i)
            if (colour[i] == c) rank[i] = k++;
    }

    double worst = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        const int32_t rg = r_first + r; /* global replica index */
        const uint32_t rq = (uint32_t)(rg >> 2);
        const int rw = rg & 3;
        /* initial state: tag 1, sweep 0 */
        for (int32_t i = 0; i < N; ++i) {
            uint32_t w = orc_rand_word(seed, rank[i], 0u, rq, (ORC_TAG_INIT << 24) | (uint32_t)colour[i], rw);
            m[i] = (w < 0x80000000u) ? 1 : -1;
        }
        double E = orc_energy(N, n_edges, eu, ev, J, h, m);
        double Einc = E;
        double best = E;
        int32_t bsweep = -1;
        if (best_state) memcpy(best_state + (int64_t)r * N, m, (size_t)N);

        for (int32_t s = 0; s < S; ++s) {
            const double beta = betas[s];
            for (int32_t c = 0; c < n_colours; ++c) {
                for (int32_t i = 0; i < N; ++i) {
                    if (colour[i] != c) continue;
                    double F = h ? h[i] : 0.0;
                    for (int64_t a = deg[i]; a < deg[i + 1]; ++a) F += adjJ[a] * (double)m[adj[a]];
                    uint32_t w = orc_rand_word(seed, rank[i], (uint32_t)s, rq,
                                               (ORC_TAG_DECISION << 24) | (uint32_t)c, rw);
                    int8_t mnew = (w < orc_threshold(beta, F)) ? 1 : -1;
                    /* Eq. 3: the energy change of spin i is fixed by its field */
                    Einc -= (double)(mnew - m[i]) * F;
                    m[i] = mnew;
                }
            }
            E = orc_energy(N, n_edges, eu, ev, J, h, m);
            double err = fabs(E - Einc);
            if (err > worst) worst = err;
            if (trace_E) trace_E[(int64_t)r * S + s] = E;
            if (E < best) {
                best = E;
                bsweep = s;
                if (best_state) memcpy(best_state + (int64_t)r * N, m, (size_t)N);
            }
        }
        if (final_E) final_E[r] = E;
        if (best_E) best_E[r] = best;
        if (best_sweep) best_sweep[r] = bsweep;
        if (final_state) memcpy(final_state + (int64_t)r * N, m, (size_t)N);
    }
    if (max_incr_err) *max_incr_err = worst;
    free(deg); free(adj); free(adjJ); free(fill); free(rank); free(m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One update-group step of the annealing loop above, from given states: the  */
/* spins of colour class c of replicas r_first .. r_first+R-1 take their      */
/* decisions of sweep s at inverse temperature beta (Eq. 3 field in FP64 from */
/* the given state, Eq. 2 decision with the tag-0 word of counter             */
/* (k, s, r >> 2, c), word r & 3); all other spins are left as they are.      */
/* m is [R][N] in/out.  Optional outputs per updated spin: P_out [R][N] the   */
/* FP64 probability 1/2 + tanh(beta F)/2 and w_out [R][N] the random word     */
/* (other entries untouched).  Returns 0, -1 on bad arguments, -2 if the      */
/* colouring has an internal edge, -3 on allocation failure.                  */
/* ------------------------------------------------------------------------ */
int orc_class_step(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J,
                   const double* h, const int32_t* colour, int32_t n_colours, int32_t c, double beta, int32_t s,
                   int32_t r_first, int32_t R, uint64_t seed, int8_t* m, double* P_out, uint32_t* w_out)
{
    if (N < 1 || R < 0 || r_first < 0 || s < 0 || n_colours < 1 || n_colours > 255 || c < 0 || c >= n_colours)
        return -1;
    for (int32_t i = 0; i < N; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return -1;
    if (orc_count_monochrome(n_edges, eu, ev, colour) != 0) return -2;
    uint32_t* rank = (uint32_t*)malloc((size_t)N * sizeof(uint32_t));
    double* F = (double*)malloc((size_t)N * sizeof(double));
    if (!rank || !F) {
        free(rank); free(F);
        return -3;
    }
    for (int32_t cc = 0; cc < n_colours; ++cc) {
        uint32_t k = 0;
        for (int32_t i = 0; i < N; ++i)
            if (colour[i] == cc) rank[i] = k++;
    }
    for (int32_t r = 0; r < R; ++r) {
        const int32_t rg = r_first + r;
        int8_t* mr = m + (int64_t)r * N;
        /* fields of the given state; class c has no internal edge, so they do not
           change while the class is updated */
        orc_fields(N, n_edges, eu, ev, J, h, mr, F);
        for (int32_t i = 0; i < N; ++i) {
            if (colour[i] != c) continue;
            uint32_t w = orc_rand_word(seed, rank[i], (uint32_t)s, (uint32_t)(rg >> 2),
                                       (ORC_TAG_DECISION << 24) | (uint32_t)c, rg & 3);
            mr[i] = (w < orc_threshold(beta, F[i])) ? 1 : -1;
            if (P_out) P_out[(int64_t)r * N + i] = 0.5 + 0.5 * tanh(beta * F[i]);
            if (w_out) w_out[(int64_t)r * N + i] = w;
        }
    }
    free(rank); free(F);
    return 0;
}

/* ------------------------------------------------------------------------
 * Parallel tempering (replica exchange; Hukushima & Nemoto, J. Phys. Soc. Jpn.
 * 65, 1604 (1996)), named by the paper as a better PC solving method
 * (Sec. 6.1).  Written from the standard definition:
 *   - M inverse temperatures ladder[0] < ... < ladder[M-1] and R independent
 *     chains; chain r has M slots g = k R + r (k = 0..M-1), slot g starts at
 *     temperature k with its own initial state (tag 1, replica index g).
 *   - Sweep s: every slot updates every colour class in order with the beta of
 *     its current temperature (decision words tag 0, replica index g).
 *   - After the sweep, energies are taken (and each slot's running best kept as
 *     in orc_anneal); then, for every chain r and every temperature pair
 *     (t, t+1) with t = s mod 2, t + 2, ..., the slots a (temperature t) and b
 *     (temperature t+1) exchange temperatures with probability
 *     min(1, exp((beta_{t+1} - beta_t) (E_b - E_a))): accepted iff that
 *     exponent x >= 0 or w < floor(exp(x) 2^32), w the word of counter
 *     (t, s, r >> 2, 3 << 24), index r & 3.
 * Outputs are per slot (arrays of M R) plus the final temperature of every
 * slot and the accepted exchanges per pair.
 * ------------------------------------------------------------------------ */
#define ORC_TAG_EXCHANGE 3u

int orc_pt(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, const double* J, const double* h,
           const int32_t* colour, int32_t n_colours, const double* ladder, int32_t M, int32_t S, int32_t R,
           uint64_t seed, double* final_E, double* best_E, int32_t* best_sweep, int8_t* final_state,
           int8_t* best_state, int32_t* slot_temp, int64_t* n_accept)
{
    if (N < 1 || M < 1 || R < 1 || S < 0 || n_colours < 1 || n_colours > 255) return -1;
    for (int32_t k = 0; k + 1 < M; ++k)
        if (!(ladder[k] < ladder[k + 1])) return -1;
    for (int32_t i = 0; i < N; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return -1;
    if (orc_count_monochrome(n_edges, eu, ev, colour) != 0) return -2;

    const int32_t G = M * R;
    int64_t* deg = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc((size_t)(2 * n_edges + 1) * sizeof(int32_t));
    double* adjJ = (double*)malloc((size_t)(2 * n_edges + 1) * sizeof(double));
    int64_t* fill = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    uint32_t* rank = (uint32_t*)malloc((size_t)N * sizeof(uint32_t));
    int8_t* m = (int8_t*)malloc((size_t)G * N);
    double* E = (double*)malloc((size_t)G * sizeof(double));
    int32_t* temp = (int32_t*)malloc((size_t)G * sizeof(int32_t));
    int32_t* slot_of = (int32_t*)malloc((size_t)G * sizeof(int32_t)); /* [t][r] -> slot */
    if (!deg || !adj || !adjJ || !fill || !rank || !m || !E || !temp || !slot_of) {
        free(deg); free(adj); free(adjJ); free(fill); free(rank); free(m); free(E); free(temp); free(slot_of);
        return -3;
    }
    for (int64_t e = 0; e < n_edges; ++e) {
        deg[eu[e] + 1]++;
        deg[ev[e] + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) deg[i + 1] += deg[i];
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t u = eu[e], v = ev[e];
        adj[deg[u] + fill[u]] = v; adjJ[deg[u] + fill[u]] = J[e]; fill[u]++;
        adj[deg[v] + fill[v]] = u; adjJ[deg[v] + fill[v]] = J[e]; fill[v]++;
    }
    for (int32_t c = 0; c < n_colours; ++c) {
        uint32_t k = 0;
        for (int32_t i = 0; i < N; ++i)
            if (colour[i] == c) rank[i] = k++;
    }
    if (n_accept)
        for (int32_t t = 0; t + 1 < M; ++t) n_accept[t] = 0;

    /* initial states, energies, bests */
    for (int32_t g = 0; g < G; ++g) {
        int8_t* mg = m + (int64_t)g * N;
        for (int32_t i = 0; i < N; ++i) {
            uint32_t w = orc_rand_word(seed, rank[i], 0u, (uint32_t)(g >> 2), (ORC_TAG_INIT << 24) | (uint32_t)colour[i],
                                       g & 3);
            mg[i] = (w < 0x80000000u) ? 1 : -1;
        }
        E[g] = orc_energy(N, n_edges, eu, ev, J, h, mg);
        temp[g] = g / R;
        slot_of[g] = g; /* temperature g / R of chain g % R sits in slot g */
        best_E[g] = E[g];
        best_sweep[g] = -1;
        if (best_state) memcpy(best_state + (int64_t)g * N, mg, (size_t)N);
    }
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t g = 0; g < G; ++g) {
            int8_t* mg = m + (int64_t)g * N;
            const double beta = ladder[temp[g]];
            for (int32_t c = 0; c < n_colours; ++c) {
                for (int32_t i = 0; i < N; ++i) {
                    if (colour[i] != c) continue;
                    double F = h ? h[i] : 0.0;
                    for (int64_t a = deg[i]; a < deg[i + 1]; ++a) F += adjJ[a] * (double)mg[adj[a]];
                    uint32_t w = orc_rand_word(seed, rank[i], (uint32_t)s, (uint32_t)(g >> 2),
                                               (ORC_TAG_DECISION << 24) | (uint32_t)c, g & 3);
                    mg[i] = (w < orc_threshold(beta, F)) ? 1 : -1;
                }
            }
            E[g] = orc_energy(N, n_edges, eu, ev, J, h, mg);
            if (E[g] < best_E[g]) {
                best_E[g] = E[g];
                best_sweep[g] = s;
                if (best_state) memcpy(best_state + (int64_t)g * N, mg, (size_t)N);
            }
        }
        for (int32_t r = 0; r < R; ++r) {
            for (int32_t t = s & 1; t + 1 < M; t += 2) {
                const int32_t a = slot_of[t * R + r], b = slot_of[(t + 1) * R + r];
                const double x = (ladder[t + 1] - ladder[t]) * (E[b] - E[a]);
                const uint32_t w = orc_rand_word(seed, (uint32_t)t, (uint32_t)s, (uint32_t)(r >> 2), ORC_TAG_EXCHANGE << 24,
                                                 r & 3);
                int accept = x >= 0.0;
                if (!accept) accept = (double)w < floor(exp(x) * ORC_TWO_POW_32);
                if (accept) {
                    temp[a] = t + 1;
                    temp[b] = t;
                    slot_of[t * R + r] = b;
                    slot_of[(t + 1) * R + r] = a;
                    if (n_accept) n_accept[t]++;
                }
            }
        }
    }
    for (int32_t g = 0; g < G; ++g) {
        if (final_E) final_E[g] = E[g];
        if (final_state) memcpy(final_state + (int64_t)g * N, m + (int64_t)g * N, (size_t)N);
        if (slot_temp) slot_temp[g] = temp[g];
    }
    free(deg); free(adj); free(adjJ); free(fill); free(rank); free(m); free(E); free(temp); free(slot_of);
    return 0;
}
