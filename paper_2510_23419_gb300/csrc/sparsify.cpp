// sparsify.cpp -- a bounded-degree copy graph of a biclique (arXiv 2510.23419,
// Sec. 5.3 outlook: dense instances turned into sparse ones whose vertices have
// at most six neighbours, with the update groups kept).  The paper describes
// the idea (copies of a vertex joined by ferromagnetic copy edges, a maximum
// number of neighbours per site); the construction here is this library's own:
//
//   * biclique edge (i, j) gets the parity pi = (i + j) mod 2;
//   * every vertex v becomes a path of copies v_0 - v_1 - ... - v_{c-1}; copy q
//     has slot q mod 2 and carries up to `per_copy` of v's edges of parity
//     slot (in increasing order of the other end), so c = 2 ceil(e_max /
//     per_copy) with e_max the larger of v's two parity counts;
//   * edge (i, j) of parity pi joins the copy of i and the copy of j that carry
//     it (both of slot pi), with the original coupling;
//   * consecutive copies are joined by a ferromagnetic copy edge of strength
//     copy_strength (for +-1 instances: that many unit edges, so fields stay
//     integers);
//   * colour of a left copy = its slot, of a right copy = 1 - its slot: every
//     edge joins the two colours, so the graph keeps two update groups.
// Interior copies have 2 copy-edge neighbours plus at most per_copy (<= 4)
// edge neighbours: at most six distinct neighbours.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pb_handles.h"

using namespace pb;

namespace {

struct Layout {
    int n, per;
    std::vector<int32_t> first;  // [2n + 1] id of copy 0 of each original vertex
};

// Copies of original vertex v (0..n-1 left, n..2n-1 right) and the number of
// its parity-0 / parity-1 edges.
int copies_of(int n, int v, int per)
{
    const int w = v < n ? v : v - n;
    const int e1 = (w % 2 == 0) ? n / 2 : (n + 1) / 2;  // other-side vertices u with (w + u) odd
    const int e0 = n - e1;
    const int emax = std::max(e0, e1);
    return 2 * std::max(1, (emax + per - 1) / per);
}

Layout layout(int n, int per)
{
    Layout L{n, per, std::vector<int32_t>((size_t)2 * n + 1, 0)};
    for (int v = 0; v < 2 * n; ++v) L.first[(size_t)v + 1] = L.first[(size_t)v] + copies_of(n, v, per);
    return L;
}

// Copy of vertex (side, w) that carries its edge to other-side vertex u.
int32_t carrier(const Layout& L, int side, int w, int u)
{
    const int pi = (w + u) & 1;
    // the other-side vertices of parity pi relative to w are u0, u0 + 2, ... with u0 = (w + pi) mod 2
    const int rank = (u - ((w + pi) & 1)) / 2;
    const int q = 2 * (rank / L.per) + pi;
    const int v = side == 0 ? w : L.n + w;
    return L.first[(size_t)v] + q;
}

}  // namespace

extern "C" {

int64_t pb_sparsify_biclique(int32_t n, int32_t jtype, const void* J, int32_t per_copy, int32_t copy_strength,
                             int32_t* N_out, int32_t* eu, int32_t* ev, void* J_out, int32_t* colour, int32_t* copy_of,
                             int64_t edge_capacity, int32_t vertex_capacity)
{
    if (n < 1 || per_copy < 1 || per_copy > 4 || copy_strength < 1 || !N_out) return -1;
    if (jtype != PB_J_PM1_I8 && jtype != PB_J_F32) return -1;
    const Layout L = layout(n, per_copy);
    const int32_t N = L.first[(size_t)2 * n];
    const int64_t chains = (int64_t)N - 2 * n;                          // copy-edge pairs
    const int64_t E = (int64_t)n * n + chains * (jtype == PB_J_PM1_I8 ? copy_strength : 1);
    *N_out = N;
    if (!eu || !ev || !J_out || !colour || !copy_of) return E;  // size query
    if (!J || edge_capacity < E || vertex_capacity < N) return -1;
    int64_t e = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            eu[e] = carrier(L, 0, i, j);
            ev[e] = carrier(L, 1, j, i);
            if (jtype == PB_J_PM1_I8)
                static_cast<int8_t*>(J_out)[e] = static_cast<const int8_t*>(J)[(size_t)i * n + j];
            else
                static_cast<float*>(J_out)[e] = static_cast<const float*>(J)[(size_t)i * n + j];
            ++e;
        }
    for (int v = 0; v < 2 * n; ++v) {
        for (int32_t id = L.first[(size_t)v]; id < L.first[(size_t)v + 1]; ++id) {
            const int q = id - L.first[(size_t)v];
            copy_of[id] = v;
            colour[id] = v < n ? (q & 1) : 1 - (q & 1);
            if (q == 0) continue;
            const int reps = jtype == PB_J_PM1_I8 ? copy_strength : 1;
            for (int k = 0; k < reps; ++k) {
                eu[e] = id - 1;
                ev[e] = id;
                if (jtype == PB_J_PM1_I8)
                    static_cast<int8_t*>(J_out)[e] = 1;
                else
                    static_cast<float*>(J_out)[e] = (float)copy_strength;
                ++e;
            }
        }
    }
    return e;
}

int32_t pb_sparse_project(int32_t N_sparse, const int32_t* copy_of, int32_t n_orig, int32_t R, const int8_t* states,
                          int8_t* out)
{
    if (N_sparse < 1 || n_orig < 1 || R < 1 || !copy_of || !states || !out) return -1;
    std::vector<int32_t> votes((size_t)n_orig), first((size_t)n_orig, -1);
    for (int32_t id = 0; id < N_sparse; ++id) {
        if (copy_of[id] < 0 || copy_of[id] >= n_orig) return -1;
        if (first[(size_t)copy_of[id]] < 0) first[(size_t)copy_of[id]] = id;
    }
    for (int32_t r = 0; r < R; ++r) {
        std::fill(votes.begin(), votes.end(), 0);
        const int8_t* m = states + (size_t)r * N_sparse;
        for (int32_t id = 0; id < N_sparse; ++id) votes[(size_t)copy_of[id]] += m[id];
        for (int32_t v = 0; v < n_orig; ++v) {
            const int s = votes[(size_t)v];
            // majority of the copies; a tie takes copy 0
            out[(size_t)r * n_orig + v] = s > 0 ? 1 : (s < 0 ? -1 : (first[(size_t)v] >= 0 ? m[first[(size_t)v]] : 1));
        }
    }
    return 0;
}

}  // extern "C"
