// Check schedule for the resident decoders (host, once per code).
//
// In the resident kernels the 32 lanes of a warp each update one check, and
// at step j every lane gathers the total LLR and the message of its check's
// j-th input from shared memory.  Messages and totals are stored in planes
// whose stride is a multiple of 32 words, so the bank of an access to bit v
// is v mod 32, and one step is free of bank conflicts when the 32 checks'
// j-th inputs lie in 32 distinct banks.
//
// The schedule makes that so:
//  1. Checks are partitioned into groups of at most 32 (one warp instruction
//     stream each; every group slot the launch offers is used, which leaves
//     some room) such that each group has at most d_c edges in every bank.  A greedy placement is refined
//     by targeted check swaps between groups (a little annealing included).
//  2. Within a group, the bipartite multigraph checks x banks has maximum
//     degree d_c and is edge-coloured with d_c colours (Konig's theorem) by
//     the alternating-path (Kempe chain) method; the colour of an edge is the
//     step at which its check processes it, so each step is a matching: 32
//     distinct banks.
// The colouring fixes each check's evaluation order (the order of its inputs
// in the prefix/suffix products); every decoder uses that order, so they
// produce identical bits.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <random>
#include <vector>

#include "ldpc_internal.h"

namespace ldpc {

namespace {

// Edge-colours one group: checks (left, < 32) x banks (right, 32), edges
// (u, b).  Returns colours in [0, delta).
std::vector<int> kempe_colour(const std::vector<std::pair<int, int>> &edges, int nleft, int delta) {
    const int E = (int)edges.size();
    std::vector<int> colour(E, -1);
    std::vector<int> at_l((size_t)nleft * delta, -1), at_r((size_t)32 * delta, -1);
    for (int e = 0; e < E; ++e) {
        const int u = edges[e].first, b = edges[e].second;
        int a = 0, c = 0;
        while (at_l[(size_t)u * delta + a] >= 0) ++a;   // free at the check
        while (at_r[(size_t)b * delta + c] >= 0) ++c;   // free at the bank
        if (at_r[(size_t)b * delta + a] >= 0) {
            // flip the a/c alternating path that starts at bank b with colour a
            std::vector<int> path;
            int side = 1, node = b, col = a;  // side 1 = bank, 0 = check
            for (;;) {
                const int ed = side ? at_r[(size_t)node * delta + col] : at_l[(size_t)node * delta + col];
                if (ed < 0) break;
                path.push_back(ed);
                node = side ? edges[ed].first : edges[ed].second;
                side ^= 1;
                col = (col == a) ? c : a;
            }
            for (int ed : path) {  // clear, then re-insert with swapped colours
                const int cu = edges[ed].first, cb = edges[ed].second, cc = colour[ed];
                at_l[(size_t)cu * delta + cc] = -1;
                at_r[(size_t)cb * delta + cc] = -1;
            }
            for (int ed : path) {
                const int nc = colour[ed] == a ? c : a;
                colour[ed] = nc;
                at_l[(size_t)edges[ed].first * delta + nc] = ed;
                at_r[(size_t)edges[ed].second * delta + nc] = ed;
            }
        }
        colour[e] = a;
        at_l[(size_t)u * delta + a] = e;
        at_r[(size_t)b * delta + a] = e;
    }
    return colour;
}

}  // namespace

int build_check_schedule(ldpc_code *c, int ngroups) {
    const int32_t m = c->m;
    const int cap = c->dc_max;
    ngroups = std::max<int>(ngroups, (int)ceil_div(m, 32));
    auto bank = [&](int32_t e) { return c->col_idx[e] & 31; };
    // 1. grouping: greedy, then improving swaps
    std::vector<int> group_of(m, -1), fill(ngroups, 0);
    std::vector<int16_t> hist((size_t)ngroups * 32, 0);
    std::vector<int32_t> perm(m);
    std::iota(perm.begin(), perm.end(), 0);
    std::mt19937_64 rng(0x5eedULL + (uint64_t)m * 131 + (uint64_t)c->n);
    std::shuffle(perm.begin(), perm.end(), rng);
    auto excess_add = [&](int g, int32_t chk, int sign) {  // change of excess when adding/removing chk
        int d = 0;
        int16_t *h = &hist[(size_t)g * 32];
        int16_t tmp[32];
        std::copy(h, h + 32, tmp);
        for (int32_t e = c->row_ptr[chk]; e < c->row_ptr[chk + 1]; ++e) {
            const int b = bank(e);
            if (sign > 0) {
                if (tmp[b] >= cap) ++d;
                ++tmp[b];
            } else {
                --tmp[b];
                if (tmp[b] >= cap) --d;
            }
        }
        return d;
    };
    auto apply = [&](int g, int32_t chk, int sign) {
        for (int32_t e = c->row_ptr[chk]; e < c->row_ptr[chk + 1]; ++e) hist[(size_t)g * 32 + bank(e)] += sign;
    };
    for (int32_t chk : perm) {
        int best = -1, bd = 1 << 30;
        for (int g = 0; g < ngroups; ++g) {
            if (fill[g] >= 32) continue;
            const int d = excess_add(g, chk, +1);
            if (d < bd) {
                bd = d;
                best = g;
                if (d == 0) break;
            }
        }
        group_of[chk] = best;
        ++fill[best];
        apply(best, chk, +1);
    }
    auto group_excess = [&](int g) {
        int x = 0;
        for (int b = 0; b < 32; ++b) x += std::max(0, (int)hist[(size_t)g * 32 + b] - cap);
        return x;
    };
    std::vector<std::vector<int32_t>> members(ngroups);
    for (int32_t chk = 0; chk < m; ++chk) members[group_of[chk]].push_back(chk);
    int64_t total = 0;
    for (int g = 0; g < ngroups; ++g) total += group_excess(g);
    // targeted swaps: take an over-full (group, bank), a check of that group
    // using the bank, and the best swap partner among the checks of groups
    // with room in that bank; ties and (rarely) worse moves are accepted to
    // leave plateaus.
    std::uniform_real_distribution<double> unif(0.0, 1.0);
    auto swap_delta = [&](int g1, int32_t c1, int g2, int32_t c2) {
        const int before = group_excess(g1) + group_excess(g2);
        apply(g1, c1, -1);
        apply(g2, c2, -1);
        apply(g1, c2, +1);
        apply(g2, c1, +1);
        const int after = group_excess(g1) + group_excess(g2);
        apply(g1, c2, -1);
        apply(g2, c1, -1);
        apply(g1, c1, +1);
        apply(g2, c2, +1);
        return after - before;
    };
    std::vector<int> bad;
    double temp = 0.6;
    for (int64_t it = 0; it < 400000 && total > 0; ++it) {
        if (it % 2000 == 0) temp *= 0.9;
        bad.clear();
        for (int g = 0; g < ngroups; ++g)
            if (group_excess(g) > 0) bad.push_back(g);
        if (bad.empty()) break;
        const int g1 = bad[rng() % bad.size()];
        int b1 = -1;
        for (int b = 0, seen = 0; b < 32; ++b)
            if (hist[(size_t)g1 * 32 + b] > cap && (int)(rng() % ++seen) == 0) b1 = b;
        // a check of g1 with an edge in bank b1
        std::vector<int> cand;
        for (int i = 0; i < (int)members[g1].size(); ++i)
            for (int32_t e = c->row_ptr[members[g1][i]]; e < c->row_ptr[members[g1][i] + 1]; ++e)
                if (bank(e) == b1) {
                    cand.push_back(i);
                    break;
                }
        const int i1 = cand[rng() % cand.size()];
        const int32_t c1 = members[g1][i1];
        int best_d = 1 << 30, bg = -1, bi = -1;
        for (int tries = 0; tries < 8; ++tries) {
            const int g2 = (int)(rng() % ngroups);
            if (g2 == g1 || hist[(size_t)g2 * 32 + b1] >= cap) continue;
            if (members[g2].size() < 32) {  // a free lane: move c1 there
                const int before = group_excess(g1) + group_excess(g2);
                apply(g1, c1, -1);
                apply(g2, c1, +1);
                const int d = group_excess(g1) + group_excess(g2) - before;
                apply(g2, c1, -1);
                apply(g1, c1, +1);
                if (d < best_d || (d == best_d && (rng() & 1))) {
                    best_d = d;
                    bg = g2;
                    bi = -1;
                }
            }
            for (int i2 = 0; i2 < (int)members[g2].size(); ++i2) {
                const int d = swap_delta(g1, c1, g2, members[g2][i2]);
                if (d < best_d || (d == best_d && (rng() & 1))) {
                    best_d = d;
                    bg = g2;
                    bi = i2;
                }
            }
        }
        if (bg < 0 && best_d == (1 << 30)) continue;
        if (best_d <= 0 || unif(rng) < std::exp(-best_d / temp)) {
            if (bi < 0) {  // move
                apply(g1, c1, -1);
                apply(bg, c1, +1);
                members[g1].erase(members[g1].begin() + i1);
                members[bg].push_back(c1);
                group_of[c1] = bg;
                total += best_d;
                continue;
            }
            const int32_t c2 = members[bg][bi];
            apply(g1, c1, -1);
            apply(bg, c2, -1);
            apply(g1, c2, +1);
            apply(bg, c1, +1);
            members[g1][i1] = c2;
            members[bg][bi] = c1;
            group_of[c1] = bg;
            group_of[c2] = g1;
            total += best_d;
        }
    }
    // 2. per group: colour edges by step, giving each check's evaluation order
    c->eval_edge.assign((size_t)c->nnz, -1);
    c->sched_groups.assign((size_t)ngroups * 32, -1);
    c->sched_excess = total;
    for (int g = 0; g < ngroups; ++g) {
        auto &mem = members[g];
        std::sort(mem.begin(), mem.end());
        int delta = cap;
        for (int b = 0; b < 32; ++b) delta = std::max(delta, (int)hist[(size_t)g * 32 + b]);
        std::vector<std::pair<int, int>> edges;
        std::vector<int32_t> eid;
        for (int u = 0; u < (int)mem.size(); ++u) {
            c->sched_groups[(size_t)g * 32 + u] = mem[u];
            for (int32_t e = c->row_ptr[mem[u]]; e < c->row_ptr[mem[u] + 1]; ++e) {
                edges.emplace_back(u, bank(e));
                eid.push_back(e);
            }
        }
        const std::vector<int> col = kempe_colour(edges, (int)mem.size(), delta);
        // evaluation order of a check: its edges by colour (ties cannot occur)
        size_t k = 0;
        for (int u = 0; u < (int)mem.size(); ++u) {
            const int32_t chk = mem[u], e0 = c->row_ptr[chk], d = c->row_ptr[chk + 1] - e0;
            std::vector<std::pair<int, int32_t>> byc;
            for (int j = 0; j < d; ++j, ++k) byc.emplace_back(col[k], eid[k]);
            std::sort(byc.begin(), byc.end());
            // step j of the check processes its evaluation position j; when the
            // group is balanced (delta = d_c) position j is colour j exactly
            for (int j = 0; j < d; ++j) c->eval_edge[e0 + j] = byc[j].second;
        }
    }
    return LDPC_OK;
}

}  // namespace ldpc
