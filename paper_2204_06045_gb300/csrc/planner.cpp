// Host planner: lightcone networks (§II-B), greedy min-fill elimination
// orders, bucket schedules with rank-sorted index bits, and the flat layout
// the kernels read.
#include "planner.hpp"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <queue>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>

#include "../../include/qt.h"

namespace qt {

namespace {

uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Rng {
    uint64_t s;
    uint64_t next() { return s = mix64(s); }
};

inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

int leaf_slots_per_graph(int p) { return 2 + 4 * p; }

int leaf_index(int kind, int layer) {
    if (kind == QT_LEAF_PLUS) return 0;
    if (kind == QT_LEAF_ZOBS) return 1;
    return 2 + 4 * layer + (kind - QT_LEAF_ZZ);
}

// ---------------------------------------------------------------------------
// Lightcone network of one edge (§II-B).
//
// For edge (j,k) let d(q) be the graph distance from {j,k}. Working outward
// from Z_j Z_k, the mixer of layer k (1-based) survives the cancellation of
// U^dagger (Z_j Z_k) U only on qubits with d(q) <= p - k, and the ZZ gate of
// layer k on edge (a,b) only when min(d(a), d(b)) <= p - k. Diagonal gates add
// no variable: a ZZ phase is a rank-2 tensor on the two current variables, a
// mixer is a rank-2 tensor from the current variable to a fresh one. The bra
// half mirrors the ket half with conjugated tensors.
// ---------------------------------------------------------------------------
// adj[v]: (neighbour, edge index) pairs of vertex v, in edge order
using Adjacency = std::vector<std::vector<std::pair<int, int>>>;

static Adjacency graph_adjacency(const GraphIn& g) {
    Adjacency adj(g.n);
    for (size_t i = 0; i < g.edges.size(); ++i) {
        adj[g.edges[i].first].emplace_back(g.edges[i].second, (int)i);
        adj[g.edges[i].second].emplace_back(g.edges[i].first, (int)i);
    }
    return adj;
}

static void build_network(const GraphIn& g, const Adjacency& adj, int p, int eidx, Network* net) {
    const int n = g.n;
    const int j = g.edges[eidx].first, k = g.edges[eidx].second;
    std::vector<int> dist(n, -1), cone;
    std::queue<int> bfs;
    dist[j] = dist[k] = 0;
    bfs.push(j);
    bfs.push(k);
    cone.push_back(j);
    cone.push_back(k);
    while (!bfs.empty()) {
        int a = bfs.front();
        bfs.pop();
        if (dist[a] == p) continue;
        for (const auto& nb : adj[a])
            if (dist[nb.first] < 0) {
                dist[nb.first] = dist[a] + 1;
                bfs.push(nb.first);
                cone.push_back(nb.first);
            }
    }
    // the qubits of the lightcone in vertex order, and the edges a ZZ gate may
    // sit on (an endpoint within distance p - 1, so both ends in the
    // lightcone) in edge order: the order of the gates below
    std::sort(cone.begin(), cone.end());
    std::vector<int> zz_edges;
    for (int v : cone)
        if (dist[v] <= p - 1)
            for (const auto& nb : adj[v]) zz_edges.push_back(nb.second);
    std::sort(zz_edges.begin(), zz_edges.end());
    zz_edges.erase(std::unique(zz_edges.begin(), zz_edges.end()), zz_edges.end());
    auto in_zz = [&](int a, int b, int layer1) { return std::min(dist[a], dist[b]) <= p - layer1; };
    auto has_mixer = [&](int q, int layer1) { return dist[q] <= p - layer1; };

    net->nvars = 0;
    net->leaves.clear();
    net->wire_vars.assign(n, 0);
    std::vector<int> cur(n, -1);
    auto add1 = [&](int kind, int v) { net->leaves.push_back(Leaf{kind, -1, 1, {v, -1}}); };
    auto add2 = [&](int kind, int layer, int a, int b) { net->leaves.push_back(Leaf{kind, layer, 2, {a, b}}); };

    for (int q : cone) {
        cur[q] = net->nvars++;
        net->wire_vars[q] = 1;
        add1(QT_LEAF_PLUS, cur[q]);
    }
    for (int l = 1; l <= p; ++l) {
        for (int ei : zz_edges) {
            const auto& e = g.edges[ei];
            if (in_zz(e.first, e.second, l)) add2(QT_LEAF_ZZ, l - 1, cur[e.first], cur[e.second]);
        }
        for (int q : cone)
            if (has_mixer(q, l)) {
                int nv = net->nvars++;
                net->wire_vars[q]++;
                add2(QT_LEAF_RX, l - 1, cur[q], nv);
                cur[q] = nv;
            }
    }
    add1(QT_LEAF_ZOBS, cur[j]);
    add1(QT_LEAF_ZOBS, cur[k]);
    for (int l = p; l >= 1; --l) {
        for (int q : cone)
            if (has_mixer(q, l)) {
                int nv = net->nvars++;
                net->wire_vars[q]++;
                add2(QT_LEAF_RX_CONJ, l - 1, cur[q], nv);
                cur[q] = nv;
            }
        for (int ei : zz_edges) {
            const auto& e = g.edges[ei];
            if (in_zz(e.first, e.second, l)) add2(QT_LEAF_ZZ_CONJ, l - 1, cur[e.first], cur[e.second]);
        }
    }
    for (int q : cone) add1(QT_LEAF_PLUS, cur[q]);
}

// ---------------------------------------------------------------------------
// Greedy min-fill elimination order (the paper's ordering algorithm is not
// specified, §II-D). The interaction graph joins variables that share a
// tensor; each step eliminates the variable whose neighbours need the fewest
// new edges to form a clique, ties going to the smaller degree and then to the
// lowest variable id (or to a random one for the randomised restarts). The
// bucket of a variable eliminated with degree d has width d + 1.
// ---------------------------------------------------------------------------
static void order_min_fill(const Network& net, bool randomized, uint64_t seed, std::vector<int>* order,
                           double* cost, int* maxw) {
    const int V = net.nvars, W = (V + 63) / 64;
    std::vector<uint64_t> adj((size_t)V * W, 0), alive(W, 0);
    auto row = [&](int v) { return &adj[(size_t)v * W]; };
    for (auto& L : net.leaves)
        if (L.rank == 2 && L.v[0] != L.v[1]) {
            row(L.v[0])[L.v[1] >> 6] |= 1ull << (L.v[1] & 63);
            row(L.v[1])[L.v[0] >> 6] |= 1ull << (L.v[0] & 63);
        }
    for (int v = 0; v < V; ++v) alive[v >> 6] |= 1ull << (v & 63);
    Rng rng{seed};
    order->clear();
    *cost = 0;
    *maxw = 0;
    for (int step = 0; step < V; ++step) {
        long best_fill = -1;
        int best_deg = 0, best = -1;
        uint64_t ties = 0;
        for (int v = 0; v < V; ++v) {
            if (!((alive[v >> 6] >> (v & 63)) & 1)) continue;
            const uint64_t* nv = row(v);
            int deg = 0;
            for (int w = 0; w < W; ++w) deg += popc64(nv[w]);
            if (best >= 0 && best_fill == 0 && deg > best_deg) continue;
            long fill = 0;
            for (int w = 0; w < W; ++w) {
                uint64_t bits = nv[w];
                while (bits) {
                    int a = (w << 6) | __builtin_ctzll(bits);
                    bits &= bits - 1;
                    const uint64_t* na = row(a);
                    for (int u = 0; u < W; ++u) {
                        uint64_t miss = nv[u] & ~na[u];
                        if (u == (a >> 6)) miss &= ~(1ull << (a & 63));
                        fill += popc64(miss);
                    }
                }
            }
            fill /= 2;
            bool better = best < 0 || fill < best_fill || (fill == best_fill && deg < best_deg);
            bool equal = !better && fill == best_fill && deg == best_deg;
            if (better) {
                best = v;
                best_fill = fill;
                best_deg = deg;
                ties = 1;
            } else if (equal && randomized) {
                ++ties;
                if (rng.next() % ties == 0) best = v;
            }
        }
        const int v = best;
        order->push_back(v);
        const int width = best_deg + 1;
        *cost += std::ldexp(1.0, width);
        *maxw = std::max(*maxw, width);
        std::vector<uint64_t> nv(row(v), row(v) + W);
        for (int w = 0; w < W; ++w) {
            uint64_t bits = nv[w];
            while (bits) {
                int a = (w << 6) | __builtin_ctzll(bits);
                bits &= bits - 1;
                uint64_t* ra = row(a);
                for (int u = 0; u < W; ++u) ra[u] |= nv[u];
                ra[a >> 6] &= ~(1ull << (a & 63));
                ra[v >> 6] &= ~(1ull << (v & 63));
            }
        }
        std::fill(row(v), row(v) + W, 0ull);
        alive[v >> 6] &= ~(1ull << (v & 63));
    }
}

// ---------------------------------------------------------------------------
// Lightcone deduplication. A network is fixed by its lightcone: the qubits
// within distance p of the edge, labelled by that distance, and the graph
// edges with an endpoint within distance p - 1 (the gates A1/A2 place). Two
// edges of one graph with isomorphic lightcones give the same network up to
// the names of its variables, so the same <Z_jZ_k> at the graph's angles.
// For a lightcone that is a tree the key is the AHU encoding of the tree
// hanging from the edge (each vertex: its children's encodings, sorted); for
// one with cycles, the smallest individualization-refinement certificate
// below. Both are canonical: equal keys exactly for isomorphic lightcones. A
// lightcone whose search gives up gets no key (its network is contracted).
// ---------------------------------------------------------------------------
// Canonical key of a lightcone with cycles: individualization-refinement on
// its core (the pendant trees stripped into the labels of the vertices that
// carry them). Colours start from those labels and are refined by each vertex's
// neighbour colours, renumbered by sorted signatures each round (so they do
// not depend on vertex ids). While a colour class holds several vertices,
// each of them is individualized in turn (split off above its class) and the
// search recurses; every discrete colouring orders the vertices, and the key
// is the smallest certificate (labels and edges in that order) over all
// leaves. Equal keys mean isomorphic lightcones, and isomorphic lightcones get
// equal keys. A search over kKeyLeaves leaves gives up: no key.
constexpr int kKeyLeaves = 256;

static void refine_colours(const std::vector<std::vector<int>>& adj, std::vector<int>* colour) {
    std::vector<int>& c = *colour;
    const int n = (int)adj.size();
    int classes = (int)std::set<int>(c.begin(), c.end()).size();
    for (;;) {
        std::vector<std::vector<int>> sig(n);
        for (int v = 0; v < n; ++v) {
            sig[v].push_back(c[v]);
            std::vector<int> nb;
            for (int u : adj[v]) nb.push_back(c[u]);
            std::sort(nb.begin(), nb.end());
            sig[v].insert(sig[v].end(), nb.begin(), nb.end());
        }
        std::vector<std::vector<int>> uniq(sig);
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        for (int v = 0; v < n; ++v) c[v] = (int)(std::lower_bound(uniq.begin(), uniq.end(), sig[v]) - uniq.begin());
        if ((int)uniq.size() == classes) return;
        classes = (int)uniq.size();
    }
}

static void search_key(const std::vector<std::vector<int>>& adj, const std::vector<std::string>& label,
                       std::vector<int> colour, std::string* best, int* leaves) {
    if (*leaves > kKeyLeaves) return;
    refine_colours(adj, &colour);
    const int n = (int)adj.size();
    std::vector<int> count(n + 1, 0);
    for (int v = 0; v < n; ++v) count[colour[v]]++;
    int cell = -1;
    for (int c = 0; c < n && cell < 0; ++c)
        if (count[c] > 1) cell = c;
    if (cell < 0) {  // discrete: certificate in colour order
        std::vector<int> at(n);
        for (int v = 0; v < n; ++v) at[colour[v]] = v;
        std::string cert;
        for (int i = 0; i < n; ++i) cert += label[at[i]] + ",";
        std::vector<std::pair<int, int>> ed;
        for (int v = 0; v < n; ++v)
            for (int u : adj[v])
                if (colour[v] < colour[u]) ed.emplace_back(colour[v], colour[u]);
        std::sort(ed.begin(), ed.end());
        for (auto& e : ed) cert += std::to_string(e.first) + "-" + std::to_string(e.second) + ";";
        if (best->empty() || cert < *best) *best = cert;
        ++*leaves;
        return;
    }
    for (int v = 0; v < n; ++v) {
        if (colour[v] != cell) continue;
        std::vector<int> c2(n);
        for (int w = 0; w < n; ++w) c2[w] = 2 * colour[w];
        c2[v] = 2 * colour[v] + 1;  // v alone, just above the rest of its class
        search_key(adj, label, c2, best, leaves);
        if (*leaves > kKeyLeaves) return;
    }
}

static std::string lightcone_key(const std::vector<std::vector<int>>& nbr, int p, int j, int k) {
    const int n = (int)nbr.size();
    std::vector<int> dist(n, -1), seen;
    std::queue<int> bfs;
    dist[j] = dist[k] = 0;
    bfs.push(j);
    bfs.push(k);
    seen.push_back(j);
    seen.push_back(k);
    while (!bfs.empty()) {
        const int a = bfs.front();
        bfs.pop();
        if (dist[a] == p) continue;
        for (int b : nbr[a])
            if (dist[b] < 0) {
                dist[b] = dist[a] + 1;
                bfs.push(b);
                seen.push_back(b);
            }
    }
    // the lightcone's edges: both ends within distance p, one within p - 1
    size_t n_edges = 0;
    for (int a : seen)
        for (int b : nbr[a])
            if (a < b && dist[b] >= 0 && std::min(dist[a], dist[b]) <= p - 1) ++n_edges;
    if (n_edges + 1 != seen.size()) {
        // cycles: strip the pendant trees (leaves inward), each vertex's label
        // gathering its distance and the sorted encodings of the trees it
        // carries; then search the labelled core
        const int nv = (int)seen.size();
        std::vector<int> local(n, -1);
        for (int i = 0; i < nv; ++i) local[seen[i]] = i;
        std::vector<std::vector<int>> nb(nv);
        for (int i = 0; i < nv; ++i)
            for (int b : nbr[seen[i]])
                if (dist[b] >= 0 && std::min(dist[seen[i]], dist[b]) <= p - 1) nb[i].push_back(local[b]);
        std::vector<int> deg(nv);
        std::vector<uint8_t> gone(nv, 0);
        std::vector<std::vector<std::string>> hang(nv);
        auto finish = [&](int v) {
            std::sort(hang[v].begin(), hang[v].end());
            std::string l = std::to_string(dist[seen[v]]) + "[";
            for (const std::string& h : hang[v]) l += h;
            return l + "]";
        };
        std::vector<int> leaf;
        for (int i = 0; i < nv; ++i) {
            deg[i] = (int)nb[i].size();
            if (deg[i] == 1) leaf.push_back(i);
        }
        while (!leaf.empty()) {
            std::vector<int> next;
            for (int u : leaf) {
                if (gone[u] || deg[u] != 1) continue;
                gone[u] = 1;
                for (int w : nb[u])
                    if (!gone[w]) {
                        hang[w].push_back("(" + finish(u) + ")");
                        if (--deg[w] == 1) next.push_back(w);
                    }
            }
            leaf.swap(next);
        }
        std::vector<int> core;
        std::vector<int> at(nv, -1);
        for (int i = 0; i < nv; ++i)
            if (!gone[i]) {
                at[i] = (int)core.size();
                core.push_back(i);
            }
        std::vector<std::vector<int>> adj(core.size());
        std::vector<std::string> label(core.size());
        for (size_t c = 0; c < core.size(); ++c) {
            label[c] = finish(core[c]);
            for (int w : nb[core[c]])
                if (!gone[w]) adj[c].push_back(at[w]);
        }
        std::vector<std::string> names(label);
        std::sort(names.begin(), names.end());
        names.erase(std::unique(names.begin(), names.end()), names.end());
        std::vector<int> colour(core.size());
        for (size_t c = 0; c < core.size(); ++c)
            colour[c] = (int)(std::lower_bound(names.begin(), names.end(), label[c]) - names.begin());
        std::string best;
        int leaves = 0;
        search_key(adj, label, colour, &best, &leaves);
        if (leaves > kKeyLeaves || best.empty()) return std::string();
        return "G" + best;
    }
    // encodings bottom-up: vertices in decreasing distance
    std::vector<std::string> enc(n);
    std::vector<int> order(seen.begin(), seen.end());
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dist[a] > dist[b]; });
    for (int v : order) {
        std::vector<const std::string*> kids;
        for (int u : nbr[v])
            if (dist[u] == dist[v] + 1 && dist[v] <= p - 1 && !(dist[v] == 0 && (u == j || u == k)))
                kids.push_back(&enc[u]);
        std::sort(kids.begin(), kids.end(), [](const std::string* a, const std::string* b) { return *a < *b; });
        std::string s = "(";
        for (const std::string* c : kids) s += *c;
        s += ")";
        enc[v] = std::move(s);
    }
    return "T" + std::min(enc[j], enc[k]) + "|" + std::max(enc[j], enc[k]);
}

// ---------------------------------------------------------------------------
// Index slicing. A network's value is a sum over every assignment of its
// variables (§II-B contraction), so fixing s of them splits it into 2^s
// networks of the remaining variables whose values add up to it, each with
// its own, possibly much narrower, buckets: the memory and the work of a
// bucket grow as 2^width (§II-B). A gate tensor left with one free variable
// becomes a rank-1 tensor: the gates here (ZZ, the mixer and their
// conjugates) are symmetric in their two variables, so its entries for the
// free variable x sit at x + 2 * (fixed value) in the gate's table. A gate
// whose variables are all fixed is a scalar per slice.
// Choice of variables: while the min-fill width exceeds the target, among the
// variables of the widest bucket (the kSliceCandidates of highest degree),
// fix the one whose removal gives the narrowest order (ties: the smaller sum
// of 2^width).
// ---------------------------------------------------------------------------
constexpr int kSliceCandidates = 12;

// Fix variable v of the network (the next slice bit) and renumber the others.
static void fix_variable(Network* net, int v, int orig_id) {
    const int k = (int)net->fixed_vars.size();
    net->fixed_vars.push_back(orig_id);
    std::vector<Leaf> kept;
    kept.reserve(net->leaves.size());
    for (const Leaf& L : net->leaves) {
        const bool has = L.v[0] == v || (L.rank == 2 && L.v[1] == v);
        if (!has) {
            kept.push_back(L);
        } else if (L.rank == 1) {
            // every variable fixed: a scalar per slice
            if (L.fix >= 0)
                net->fixed.push_back(FixedLeaf{L.kind, L.layer, 2, {k, L.fix}});
            else
                net->fixed.push_back(FixedLeaf{L.kind, L.layer, 1, {k, -1}});
        } else {
            Leaf R = L;
            R.rank = 1;
            R.v[0] = L.v[0] == v ? L.v[1] : L.v[0];
            R.v[1] = -1;
            R.fix = k;
            kept.push_back(R);
        }
    }
    for (Leaf& L : kept)
        for (int i = 0; i < L.rank; ++i)
            if (L.v[i] > v) L.v[i]--;
    net->leaves = std::move(kept);
    net->nvars--;
    net->slice_bits = k + 1;
}

// Variables of the widest bucket of an elimination order, by degree in the
// interaction graph (highest first).
static std::vector<int> widest_bucket(const Network& net, const std::vector<int>& order) {
    const int V = net.nvars, W = (V + 63) / 64;
    std::vector<uint64_t> adj((size_t)V * W, 0);
    auto row = [&](int v) { return &adj[(size_t)v * W]; };
    std::vector<int> deg(V, 0);
    for (auto& L : net.leaves)
        if (L.rank == 2 && L.v[0] != L.v[1]) {
            row(L.v[0])[L.v[1] >> 6] |= 1ull << (L.v[1] & 63);
            row(L.v[1])[L.v[0] >> 6] |= 1ull << (L.v[0] & 63);
        }
    for (int v = 0; v < V; ++v)
        for (int w = 0; w < W; ++w) deg[v] += popc64(row(v)[w]);
    std::vector<int> best;
    for (int v : order) {
        std::vector<int> nb;
        std::vector<uint64_t> nv(row(v), row(v) + W);
        for (int w = 0; w < W; ++w)
            for (uint64_t bits = nv[w]; bits; bits &= bits - 1) nb.push_back((w << 6) | __builtin_ctzll(bits));
        if (nb.size() + 1 > best.size()) {
            best = nb;
            best.push_back(v);
        }
        for (int a : nb) {
            uint64_t* ra = row(a);
            for (int u = 0; u < W; ++u) ra[u] |= nv[u];
            ra[a >> 6] &= ~(1ull << (a & 63));
            ra[v >> 6] &= ~(1ull << (v & 63));
        }
        std::fill(row(v), row(v) + W, 0ull);
    }
    std::stable_sort(best.begin(), best.end(), [&](int a, int b) { return deg[a] > deg[b]; });
    return best;
}

static void slice_network(Network* net, int target, int max_bits) {
    std::vector<int> orig(net->nvars);
    for (int i = 0; i < net->nvars; ++i) orig[i] = i;
    std::vector<int> ord;
    double cost = 0;
    int w = 0;
    order_min_fill(*net, false, 0, &ord, &cost, &w);
    while (w > target && net->slice_bits < max_bits && net->nvars > 1) {
        std::vector<int> cand = widest_bucket(*net, ord);
        if ((int)cand.size() > kSliceCandidates) cand.resize(kSliceCandidates);
        int best = -1, best_w = 1 << 30;
        double best_c = 0;
        for (int c : cand) {
            Network t = *net;
            fix_variable(&t, c, orig[c]);
            std::vector<int> o2;
            double c2 = 0;
            int w2 = 0;
            order_min_fill(t, false, 0, &o2, &c2, &w2);
            if (w2 < best_w || (w2 == best_w && c2 < best_c)) {
                best = c;
                best_w = w2;
                best_c = c2;
            }
        }
        if (best < 0) break;
        fix_variable(net, best, orig[best]);
        orig.erase(orig.begin() + best);
        order_min_fill(*net, false, 0, &ord, &cost, &w);
    }
}

// ---------------------------------------------------------------------------
// Bucket schedule for one order (§II-B). Every tensor goes to the bucket of
// its earliest variable. Bucket v multiplies its tensors and sums v out; the
// result's variables are the rest of the bucket's union, kept in rank order,
// and it joins the bucket of the earliest of them. Index bits of every tensor
// are its variables in rank order, earliest first, so v is bit 0 of each
// operand and each operand's other bits are a subset (mask) of the output's.
// ---------------------------------------------------------------------------
static int make_buckets(const Network& net, const std::vector<int>& order, int max_width, NetPlan* np) {
    const int V = net.nvars;
    std::vector<int> pos(V);
    for (int i = 0; i < V; ++i) pos[order[i]] = i;
    struct Tens {
        std::vector<int> vars;  // sorted by rank
        int src;                // producing bucket or -1
        int leaf;
    };
    std::vector<Tens> pool;
    std::vector<std::vector<int>> bucket_of(V);  // tensors waiting per variable
    pool.reserve(net.leaves.size() + V);
    for (size_t t = 0; t < net.leaves.size(); ++t) {
        const Leaf& L = net.leaves[t];
        Tens T;
        T.vars.assign(L.v, L.v + L.rank);
        std::sort(T.vars.begin(), T.vars.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        T.src = -1;
        T.leaf = (int)t;
        bucket_of[T.vars[0]].push_back((int)pool.size());
        pool.push_back(std::move(T));
    }
    np->buckets.clear();
    np->buckets.reserve(V);
    np->cost = 0;
    np->max_width = 0;
    std::vector<int> bucket_at(V, -1);  // bucket id by variable
    for (int step = 0; step < V; ++step) {
        const int v = order[step];
        auto& list = bucket_of[v];
        if (list.empty()) continue;  // cannot happen: every variable sits in a leaf
        std::vector<int> uni;
        for (int t : list)
            for (int x : pool[t].vars) uni.push_back(x);
        std::sort(uni.begin(), uni.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
        const int w = (int)uni.size();
        if (w > max_width) return QT_EWIDTH;
        if ((int)list.size() > kMaxOps) return QT_EWIDTH;
        HBucket B;
        B.var = v;
        B.width = w;
        B.parent = -1;
        B.n_deps = 0;
        B.level = 0;
        const int bid = (int)np->buckets.size();
        bucket_at[v] = bid;
        for (int t : list) {
            const Tens& T = pool[t];
            HOperand op;
            op.src = T.src;
            op.leaf = T.leaf;
            op.rank = (int)T.vars.size();
            op.mask = 0;
            for (size_t i = 1; i < T.vars.size(); ++i) {
                int at = (int)(std::find(uni.begin() + 1, uni.end(), T.vars[i]) - uni.begin()) - 1;
                op.mask |= 1u << at;
            }
            if (T.src >= 0) {
                B.n_deps++;
                np->buckets[T.src].parent = bid;
                B.level = std::max(B.level, np->buckets[T.src].level + 1);
            }
            B.ops.push_back(op);
        }
        np->cost += std::ldexp(1.0, w);
        np->max_width = std::max(np->max_width, w);
        list.clear();
        if (w > 1) {
            Tens R;
            R.vars.assign(uni.begin() + 1, uni.end());
            R.src = bid;
            R.leaf = -1;
            bucket_of[R.vars[0]].push_back((int)pool.size());
            pool.push_back(std::move(R));
        }
        np->buckets.push_back(std::move(B));
    }
    return QT_OK;
}

// Merged eliminations (the paper's merged-index contraction, §II-C): when a
// bucket's consumer only extends it (the consumer's one earlier result is
// this bucket's, and it adds no variable, so its width is one less), the two
// eliminations become one bucket that sums both variables. The consumer's
// summed variable is bit 0 of the bucket's output, so in the merged bucket
// the summed variables are the bucket's own and that bit; the output is the
// consumer's. The intermediate result is never written. Operands keep their
// index bits: the bucket's own operands move their output bit 0 into the
// summed mask, the consumer's gate tensors carry the second summed variable.
// A merged bucket may go on to absorb its own consumer on the same rule, up
// to kMaxSum eliminations. Chains are taken from the leaves up, for buckets
// of at least 2^kMergeMinOut outputs, so that a merged result (more than 2^8
// outputs) is never one a fused unit would have taken; the consumers' gate
// tensors must fit the merged bucket's gate table.
constexpr int kMergeMinOut = 10;
static void merge_chains(NetPlan* np) {
    auto& bs = np->buckets;
    const int nb = (int)bs.size();
    std::vector<uint8_t> gone(nb, 0);
    std::vector<int> into(nb);  // an absorbed consumer's results now come from this bucket
    for (int b = 0; b < nb; ++b) into[b] = b;
    for (int b = 0; b < nb; ++b) {
        // absorb consumers while the chain allows (a merged bucket may absorb its next consumer)
        while (!gone[b]) {
            HBucket& B = bs[b];
            const int p = B.parent;
            if (p < 0 || B.n_sum >= kMaxSum || B.width - B.n_sum < kMergeMinOut) break;
            HBucket& P = bs[p];
            // P's indices are exactly B's outputs
            if (P.n_sum != 1 || P.width != B.width - B.n_sum) break;
            int nonleaf = 0;
            bool from_b = false;
            for (const HOperand& op : P.ops)
                if (op.src >= 0) {
                    nonleaf++;
                    from_b = op.src == b;
                }
            if (nonleaf != 1 || !from_b || B.ops.size() + P.ops.size() - 1 > (size_t)kMaxOps) break;
            // the consumer's gate tensors go into the merged bucket's gate table,
            // with the bucket's own tensors of rank <= 2
            int small = 0;
            bool all_small = true;
            for (const HOperand& op : B.ops) small += op.rank <= 2;
            for (const HOperand& op : P.ops)
                if (op.src < 0) {
                    small++;
                    all_small = all_small && op.rank <= 2;
                }
            if (!all_small || small > kMaxFoldLeaves) break;
            const uint32_t sbit = 1u << B.n_sum;
            for (HOperand& op : B.ops) {
                if (op.mask & 1u) op.smask |= sbit;
                op.mask >>= 1;
            }
            for (const HOperand& op : P.ops) {
                if (op.src >= 0) continue;
                HOperand q = op;
                q.smask = sbit;  // the consumer's summed variable; its output bits are the merged output's
                B.ops.push_back(q);
            }
            (B.n_sum == 1 ? B.var2 : B.var3) = P.var;
            B.n_sum++;
            B.parent = P.parent;
            gone[p] = 1;
            into[p] = b;
            if (B.parent >= 0)  // P's consumer now reads B's result
                for (HOperand& op : bs[B.parent].ops)
                    if (op.src == p) op.src = b;
        }
    }
    // renumber the remaining buckets (elimination order kept)
    std::vector<int> id(nb, -1);
    int k = 0;
    for (int b = 0; b < nb; ++b)
        if (!gone[b]) id[b] = k++;
    for (int b = 0; b < nb; ++b)
        if (gone[b]) id[b] = id[into[b]];
    if (k == nb) return;
    std::vector<HBucket> out;
    out.reserve(k);
    for (int b = 0; b < nb; ++b) {
        if (gone[b]) continue;
        HBucket B = std::move(bs[b]);
        B.parent = B.parent >= 0 ? id[B.parent] : -1;
        B.n_deps = 0;
        B.level = 0;
        for (HOperand& op : B.ops)
            if (op.src >= 0) {
                op.src = id[op.src];
                B.n_deps++;
                B.level = std::max(B.level, out[op.src].level + 1);
            }
        out.push_back(std::move(B));
    }
    bs = std::move(out);
}

// Operands of rank <= 2 (gate tensors, and results of 4 entries or fewer) may
// be folded into the per-tile product table.
static bool foldable(const HOperand& op) { return op.rank <= 2; }

// Tile size of a bucket: the largest 2^cb outputs (cb <= cap) for which the
// footprints of the staged operands fit one shared-memory stage. Within an
// aligned tile an operand with mask M touches the contiguous block of
// 2^(popc(M & (2^cb - 1)) + 1) elements starting at 2 * pext(o0, M). Gate
// tensors are folded into one per-tile table when their tile bits number at
// most kLeafBits; otherwise they are staged like the others.
// Takes the device view of a bucket (device_view): operands with smask 0
// carry no summed variable and must be folded.
// A merged bucket's tiles hold whole groups of its summed outputs (min_cb
// bits: n_sum - 1).
static void pick_tile(const HBucket& B, const Network& net, int cap, int stage_elems, int min_cb, int* cb_out,
                      bool* fold_out) {
    (void)net;
    const int n_out = B.width - B.n_sum;
    bool must_fold = false;
    for (const HOperand& op : B.ops) must_fold = must_fold || op.smask == 0;
    for (int cb = std::max(std::min(n_out, cap), min_cb); cb >= min_cb; --cb) {
        const uint32_t low = cb >= 32 ? 0xffffffffu : ((1u << cb) - 1u);
        uint32_t U = 0;
        int nleaf = 0;
        for (const HOperand& op : B.ops)
            if (foldable(op)) {
                U |= op.mask & low;
                nleaf++;
            }
        // the gate table holds 2^n_sum entries per value of its tile bits
        const bool fold = nleaf > 0 && nleaf <= kMaxFoldLeaves && __builtin_popcount(U) + B.n_sum <= kLeafBits + 1;
        if (must_fold && !fold) continue;
        long foot = 0;
        for (const HOperand& op : B.ops)
            if (!(fold && foldable(op)))
                foot += (1l << __builtin_popcount(op.smask)) << __builtin_popcount(op.mask & low);
        if (foot <= stage_elems) {
            *cb_out = cb;
            *fold_out = fold;
            return;
        }
    }
    *cb_out = 0;
    *fold_out = false;
}

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// A bucket as the device contracts it. A merged bucket (summing s0, then s1,
// then s2) becomes the bucket of s0 alone with outputs (o, s1, s2), s1 as bit
// 0 and s2 as bit 1: operand masks gain those bits where they carry s1 or s2,
// and smask keeps only s0 (0 for the consumers' gate tensors). Other buckets
// are unchanged.
static HBucket device_view(const HBucket& B) {
    HBucket V = B;
    if (B.n_sum == 1) return V;
    const int m = B.n_sum - 1;
    V.n_sum = 1;
    for (HOperand& op : V.ops) {
        op.mask = (op.mask << m) | ((op.smask >> 1) & ((1u << m) - 1u));
        op.smask &= 1u;
    }
    return V;
}

// Fused units (§III-A and §III-C: small buckets dominate GPU time). A bucket
// whose subtree (it and every bucket producing, directly or not, one of its
// operands) holds only small buckets can run as one work group without waiting
// for any other: a warp contracts the subtree's buckets in elimination order,
// each intermediate in its shared-memory stage, and writes only the root's
// result. Units are the maximal such subtrees whose intermediates, placed
// first-fit by lifetime (a result is freed once its consumer is done), fit the
// stage; a subtree that does not fit is split at its root.
static void form_units(HostPlan* hp, int stage_elems) {
    hp->unit_prog.clear();
    hp->n_units = 0;
    hp->n_fused = 0;
    if (!hp->cfg.fuse) return;
    const uint32_t nb = (uint32_t)hp->buckets.size();
    std::vector<uint8_t> ok(nb, 0);  // the bucket's whole subtree is small
    // a bucket's producers, in operand order (read from its operands in place)
    auto each_kid = [hp](uint32_t u, auto&& f) {
        const DBucket& d = hp->buckets[u];
        for (uint32_t i = d.op_begin; i < d.op_begin + d.n_ops; ++i)
            if (hp->op_src[i] >= 0) f((uint32_t)hp->op_src[i]);
    };
    for (uint32_t b = 0; b < nb; ++b) {
        const DBucket& d = hp->buckets[b];
        bool good = d.n_out <= kFuseOutBits && bucket_n_sum(d.flags) == 1;  // units sum one variable per bucket
        each_kid(b, [&](uint32_t c) { good = good && ok[c]; });  // producers precede their consumer
        ok[b] = good;
    }
    // Steps: consecutive members that run together, one output per lane --
    // at most 4 mutually independent buckets of at most 16 outputs each, 32
    // lanes and 31 records (their headers and operands) in all, none the
    // root; any other member is a step of its own, over the whole warp.
    // step[k] = index of the first member of k's step.
    auto make_steps = [&](const std::vector<uint32_t>& order, uint32_t root, std::vector<uint32_t>& step) {
        step.assign(order.size(), 0);
        for (size_t k = 0; k < order.size();) {
            const uint32_t u = order[k];
            const DBucket& du = hp->buckets[u];
            size_t e = k + 1;
            if (u != root && du.n_out <= 4) {
                uint32_t lanes = 1u << du.n_out, recs = 1u + du.n_ops;
                while (e < order.size() && e - k < 4) {
                    const uint32_t v = order[e];
                    const DBucket& dv = hp->buckets[v];
                    if (v == root || dv.n_out > 4 || lanes + (1u << dv.n_out) > 32 || recs + 1u + dv.n_ops > 31) break;
                    bool indep = true;
                    each_kid(v, [&](uint32_t c) {
                        for (size_t j = k; j < e; ++j) indep = indep && c != order[j];
                    });
                    if (!indep) break;
                    lanes += 1u << dv.n_out;
                    recs += 1u + dv.n_ops;
                    ++e;
                }
            }
            for (size_t j = k; j < e; ++j) step[j] = (uint32_t)k;
            k = e;
        }
    };
    // first-fit placement of a subtree's intermediates in step order; false if
    // it overflows. A step's results are all placed before any of its
    // members' producers are freed (they run at the same time).
    auto place = [&](const std::vector<uint32_t>& order, uint32_t root, const std::vector<uint32_t>& step) {
        std::vector<std::pair<uint32_t, uint32_t>> used;  // (offset, size), sorted by offset
        auto alloc = [&](uint32_t u) {
            const uint32_t sz = 1u << hp->buckets[u].n_out;
            uint32_t at = 0;
            for (auto& iv : used) {
                if (at + sz <= iv.first) break;
                at = std::max(at, iv.first + iv.second);
            }
            if (at + sz > (uint32_t)stage_elems) return false;
            used.insert(std::upper_bound(used.begin(), used.end(), std::make_pair(at, 0u)), {at, sz});
            hp->buckets[u].scr_off = (uint16_t)at;
            return true;
        };
        auto release = [&](uint32_t u) {  // u's producers are consumed now: free their space
            each_kid(u, [&](uint32_t c) {
                const uint32_t co = hp->buckets[c].scr_off, cs = 1u << hp->buckets[c].n_out;
                auto it = std::find(used.begin(), used.end(), std::make_pair(co, cs));
                if (it != used.end()) used.erase(it);
            });
        };
        for (size_t k = 0; k < order.size();) {
            size_t e = k + 1;
            while (e < order.size() && step[e] == k) ++e;
            for (size_t j = k; j < e; ++j)
                if (order[j] != root && !alloc(order[j])) return false;
            for (size_t j = k; j < e; ++j) release(order[j]);
            k = e;
        }
        return true;
    };
    // Depth order: a member's depth is 0 without producers in the unit, else
    // one more than its deepest producer's; the members of one depth are
    // independent, so they pack into steps (elimination order within a depth).
    auto depth_order = [&](const std::vector<uint32_t>& members, std::vector<uint32_t>& order) {
        std::vector<std::pair<uint32_t, uint32_t>> keyed;
        std::unordered_map<uint32_t, uint32_t> depth;
        for (uint32_t u : members) {  // elimination order: producers first
            uint32_t dp = 0;
            each_kid(u, [&](uint32_t c) {
                auto it = depth.find(c);
                if (it != depth.end()) dp = std::max(dp, it->second + 1);
            });
            depth[u] = dp;
            keyed.push_back({dp, u});
        }
        std::sort(keyed.begin(), keyed.end());
        order.clear();
        for (auto& kv : keyed) order.push_back(kv.second);
    };
    std::vector<uint32_t> stack, members, todo, order, step;
    for (uint32_t r = nb; r-- > 0;) {  // parents before producers: maximal subtrees first
        const DBucket& d = hp->buckets[r];
        if (!ok[r] || (d.flags & kBucketInUnit)) continue;
        if (d.parent != kNone && ok[d.parent]) continue;  // part of a larger candidate
        stack.assign(1, r);
        while (!stack.empty()) {
            const uint32_t root = stack.back();
            stack.pop_back();
            members.clear();
            todo.assign(1, root);
            while (!todo.empty()) {
                const uint32_t u = todo.back();
                todo.pop_back();
                members.push_back(u);
                each_kid(u, [&](uint32_t c) { todo.push_back(c); });
            }
            std::sort(members.begin(), members.end());  // elimination order
            // depth order packs the most; it keeps more results alive at once,
            // so elimination order (consecutive independent members) is the
            // fallback when its placement overflows the stage
            depth_order(members, order);
            make_steps(order, root, step);
            bool placed = place(order, root, step);
            if (!placed) {
                order = members;
                make_steps(order, root, step);
                placed = place(order, root, step);
            }
            if (placed) {
                hp->buckets[root].flags |= kBucketUnitRoot;
                for (uint32_t u : members)
                    if (u != root) hp->buckets[u].flags |= kBucketInUnit;
                hp->buckets[root].unit_begin = (uint32_t)hp->unit_prog.size() + 1u;
                hp->buckets[root].unit_count = (uint32_t)members.size();
                for (size_t k = 0; k < order.size();) {
                    size_t e = k + 1;
                    while (e < order.size() && step[e] == k) ++e;
                    const size_t at = hp->unit_prog.size();
                    if (e - k > 1) {  // the step record, completed below
                        hp->unit_prog.push_back(URec{0, 0, 0});
                    }
                    uint32_t lane = 0, item_off = 0;
                    uint64_t map = 0;
                    for (size_t j = k; j < e; ++j) {
                        const uint32_t u = order[j];
                        const DBucket& m = hp->buckets[u];
                        const uint32_t rel = (uint32_t)(hp->unit_prog.size() - at);
                        if (j > k) item_off |= rel << (8 * (j - k - 1));
                        for (uint32_t l = lane; l < lane + (1u << m.n_out); ++l) map |= (uint64_t)(j - k) << (2 * l);
                        hp->unit_prog.push_back(URec{(uint32_t)m.n_out | ((uint32_t)m.n_ops << 8) | (u == root ? 1u << 16 : 0u),
                                                     u == root ? 0u : (uint32_t)m.scr_off, e - k > 1 ? (uint64_t)lane : 0});
                        lane += 1u << m.n_out;
                        for (uint32_t i = m.op_begin; i < m.op_begin + m.n_ops; ++i) {
                            const DOperand& o = hp->operands[i];
                            const bool leaf = (o.flags & kOpLeaf) != 0;
                            // a mask that is one run of bits extracts by a shift
                            const uint32_t sh = o.mask ? (uint32_t)__builtin_ctz(o.mask) : 0u;
                            const uint32_t run = o.mask >> sh;
                            const uint32_t flags = (leaf ? 0u : 1u) | ((run & (run + 1u)) == 0u ? 2u | (sh << 8) : 0u);
                            hp->unit_prog.push_back(
                                URec{o.mask, flags, leaf ? o.off : (uint64_t)hp->buckets[hp->op_src[i]].scr_off});
                        }
                    }
                    if (e - k > 1) {
                        const uint32_t recs = (uint32_t)(hp->unit_prog.size() - at);
                        hp->unit_prog[at] = URec{recs | kUnitStep | ((uint32_t)(e - k) << 20) | (lane << 24), item_off, map};
                    }
                    k = e;
                }
                hp->n_units++;
                hp->n_fused += members.size();
            } else {
                each_kid(root, [&](uint32_t c) { stack.push_back(c); });  // split at the root
            }
        }
    }
    // Units pay when they remove more work groups than the GPU has warps to
    // run them; otherwise (few small buckets, as in a single graph's networks)
    // the plan keeps every bucket on its own and the kernel without unit code.
    if (hp->n_fused - hp->n_units <= 2ull * (uint64_t)std::max(1, hp->cfg.sim_workers)) {
        for (uint32_t b = 0; b < nb; ++b) {
            DBucket& d = hp->buckets[b];
            d.flags &= (uint8_t)~(kBucketInUnit | kBucketUnitRoot);
            d.unit_begin = d.unit_count = 0;
            d.scr_off = 0;
        }
        hp->unit_prog.clear();
        hp->n_units = hp->n_fused = 0;
        return;
    }
    hp->unit_prog.resize(hp->unit_prog.size() + 2 * kURecWindow, URec{0, 0, 0});  // window reads past the last unit
    // a unit is one group; its members are never claimed on their own
    hp->n_groups = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        DBucket& d = hp->buckets[b];
        if (d.flags & kBucketInUnit) d.n_groups = 0;
        else if (d.flags & kBucketUnitRoot) d.n_groups = 1;
        hp->n_groups += d.n_groups;
    }
}

static DRun unit_run(const HostPlan& hp, uint32_t root) {
    const DBucket& d = hp.buckets[root];
    return DRun{root, 0, 1, d.op_begin, 0, d.unit_begin, d.unit_count, d.n_ops};  // one "tile": the whole unit
}

// Claim order by list scheduling on the host. Each of W simulated warps takes,
// whenever it is free, the ready group whose bucket has the longest remaining
// path to its network's result (the sum, along the path, of the time each
// bucket takes with the whole GPU); a bucket's groups become ready when its
// last producer finishes. A group's time is its bytes at one warp's share of
// the memory bandwidth plus fixed per-tile and per-group costs. The order in
// which the simulated warps start groups is the claim order used on the
// device: it is topological (a group starts after its producers finish), and
// it front-loads the critical path instead of serving buckets first come,
// first served.
static void simulate_order(HostPlan* hp) {
    const PlanConfig& cfg = hp->cfg;
    const size_t nb = hp->buckets.size();
    const double esize = cfg.dtype == 1 ? 16.0 : 8.0;
    const double W = std::max(1, cfg.sim_workers);
    const double bw = 6.5e12;                  // bytes per second, whole GPU
    const double t_tile = 0.3e-6, t_group = 1.5e-6;
    std::vector<double> tile_s(nb), whole_s(nb), prio(nb, 0.0);
    // one small bucket inside a fused unit: measured on GB300, 0.8 us gave the
    // complex64 64-graph batch 1.591 vs 1.675 ms at 0.15 us, while the complex128
    // N=30 p=4 plan (few units) ran best at 0.15 us (5.67 vs 5.79 ms)
    const double t_unit_bucket = cfg.dtype == 1 ? 0.15e-6 : 0.8e-6;
    for (size_t b = 0; b < nb; ++b) {
        const DBucket& d = hp->buckets[b];
        const double tile_bytes =
            ((double)d.total_foot + std::ldexp(1.0, d.chunk_bits - (bucket_n_sum(d.flags) - 1))) * esize;
        tile_s[b] = tile_bytes / (bw / W) + t_tile;
        if (d.flags & kBucketUnitRoot) {  // the whole unit, as one group of one "tile"
            tile_s[b] = t_unit_bucket * d.unit_count;
            whole_s[b] = tile_s[b] + t_group;
            continue;
        }
        const double groups_in_parallel = std::min<double>(W, std::max<uint32_t>(1, d.n_groups));
        whole_s[b] = std::max(tile_s[b] * d.n_tasks / groups_in_parallel, tile_s[b] * d.group_tiles) + t_group;
    }
    // buckets of a network are in elimination order, so parents come after children
    for (size_t i = nb; i-- > 0;) {
        const DBucket& d = hp->buckets[i];
        prio[i] = whole_s[i] + (d.parent != kNone ? prio[d.parent] : 0.0);
    }
    // event simulation
    std::vector<uint32_t> deps_left(nb);
    for (size_t b = 0; b < nb; ++b) {
        const DBucket& d = hp->buckets[b];
        // a fused unit waits for nothing; its members never run on their own
        deps_left[b] = (d.flags & kBucketUnitRoot) ? 0u : (d.flags & kBucketInUnit) ? 1u : d.n_deps;
    }
    std::vector<uint32_t> groups_left(nb), gsize(nb);
    for (size_t b = 0; b < nb; ++b) {
        groups_left[b] = hp->buckets[b].n_groups;
        gsize[b] = hp->buckets[b].group_tiles;
    }
    struct Ready {
        double prio;
        uint32_t bucket, next_tile;
        bool operator<(const Ready& o) const { return prio < o.prio || (prio == o.prio && bucket > o.bucket); }
    };
    std::priority_queue<Ready> ready;  // buckets with unstarted groups, highest priority first
    for (size_t b = 0; b < nb; ++b)
        if (deps_left[b] == 0) ready.push(Ready{prio[b], (uint32_t)b, 0});
    using Ev = std::pair<double, uint32_t>;  // (finish time, bucket)
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
    double now = 0.0;
    uint64_t free_workers = (uint64_t)W;
    hp->runs.clear();
    hp->runs.reserve(hp->n_groups);
    while (!ready.empty() || !running.empty()) {
        while (free_workers > 0 && !ready.empty()) {
            Ready r = ready.top();
            ready.pop();
            const DBucket& d = hp->buckets[r.bucket];
            if (d.flags & kBucketUnitRoot) {
                hp->runs.push_back(unit_run(*hp, r.bucket));
                running.push(Ev{now + tile_s[r.bucket] + t_group, r.bucket});
                --free_workers;
                continue;
            }
            if (r.next_tile == 0 && cfg.run_tiles == 0) {
                // Group size when the bucket starts: where the GPU is nearly
                // idle (kSplitShare free warps or more per ready bucket, as on
                // the chains that end every network), the bucket spreads over
                // its share of them, in groups of min_group tiles or more;
                // elsewhere group_tiles. Measured on GB300 (N=30 p=4): groups
                // of at least 4 tiles for complex64 (0.945 vs 0.969 ms at 8),
                // 8 for complex128 (5.65 vs 5.75 ms at 4); larger shares or
                // smaller ones did not help.
                constexpr double kSplitShare = 64.0;
                const double min_group = cfg.dtype == 1 ? 8.0 : 4.0;
                const double share = (double)free_workers / (double)(ready.size() + 1);
                if (share >= kSplitShare) {
                    const double want = std::ceil((double)d.n_tasks / share);
                    gsize[r.bucket] = (uint32_t)std::max<double>(std::min<double>(min_group, d.group_tiles),
                                                                 std::min<double>(d.group_tiles, want));
                }
                groups_left[r.bucket] = (d.n_tasks + gsize[r.bucket] - 1) / gsize[r.bucket];
            }
            const uint32_t c = r.next_tile;
            const uint32_t n = std::min(gsize[r.bucket], d.n_tasks - c);
            hp->runs.push_back(DRun{r.bucket, c, n, d.op_begin, d.n_deps, 0, 0, d.n_ops});
            running.push(Ev{now + tile_s[r.bucket] * n + t_group, r.bucket});
            --free_workers;
            r.next_tile = c + n;
            if (r.next_tile < d.n_tasks) ready.push(r);
        }
        if (running.empty()) break;  // cannot happen with a consistent plan
        const Ev e = running.top();
        running.pop();
        now = e.first;
        ++free_workers;
        if (--groups_left[e.second] == 0) {
            const uint32_t par = hp->buckets[e.second].parent;
            if (par != kNone && --deps_left[par] == 0) ready.push(Ready{prio[par], par, 0});
        }
    }
    while (!running.empty()) {
        now = std::max(now, running.top().first);
        running.pop();
    }
    hp->sim_seconds = now;
    hp->n_groups = hp->runs.size();  // the queue: every group, in claim order
}

int build_host_plan(const std::vector<GraphIn>& graphs, const PlanConfig& cfg, HostPlan* hp) {
    auto t0 = std::chrono::steady_clock::now();
    hp->cfg = cfg;
    hp->graphs = graphs;
    if (cfg.p < 1 || cfg.p > 64 || graphs.empty()) return QT_EINVAL;
    if (cfg.max_width < 2 || cfg.max_width > kMaxOutBits + 1) return QT_EINVAL;
    for (auto& g : graphs) {
        if (g.n < 1) return QT_EINVAL;  // a graph without edges has no networks and energy 0
        std::set<std::pair<int, int>> seen;
        for (auto& e : g.edges) {
            if (e.first < 0 || e.second < 0 || e.first >= g.n || e.second >= g.n || e.first == e.second)
                return QT_EINVAL;
            auto key = std::minmax(e.first, e.second);
            if (!seen.insert(key).second) return QT_EINVAL;
        }
        for (int e : g.sel)
            if (e < 0 || e >= (int)g.edges.size()) return QT_EINVAL;
    }
    // networks, one per edge of every graph
    hp->graph_first_net.assign(1, 0);
    for (size_t g = 0; g < graphs.size(); ++g)
        hp->graph_first_net.push_back(hp->graph_first_net.back() + (int)graphs[g].n_nets());
    const int n_nets = hp->graph_first_net.back();
    hp->nets.assign(n_nets, Network());
    hp->nplans.assign(n_nets, NetPlan());
    std::vector<int> status(n_nets, QT_OK);
    std::vector<int> rep(n_nets, -1);
    if (cfg.dedup) {
        // keys in parallel, then per graph the first network of each key is contracted
        std::vector<std::string> key(n_nets);
        std::vector<std::vector<std::vector<int>>> nbr(graphs.size());
        for (size_t g = 0; g < graphs.size(); ++g) {
            nbr[g].assign(graphs[g].n, {});
            for (auto& e : graphs[g].edges) {
                nbr[g][e.first].push_back(e.second);
                nbr[g][e.second].push_back(e.first);
            }
        }
        std::atomic<int> nk{0};
        auto keyer = [&]() {
            for (;;) {
                const int i = nk.fetch_add(1);
                if (i >= n_nets) break;
                const int g = (int)(std::upper_bound(hp->graph_first_net.begin(), hp->graph_first_net.end(), i) -
                                    hp->graph_first_net.begin()) - 1;
                const auto& ed = graphs[g].edges[graphs[g].edge_of((size_t)(i - hp->graph_first_net[g]))];
                key[i] = lightcone_key(nbr[g], cfg.p, ed.first, ed.second);
            }
        };
        const unsigned nt = std::max(1u, std::min({std::thread::hardware_concurrency(), 64u, (unsigned)n_nets}));
        std::vector<std::thread> kp;
        for (unsigned t = 0; t + 1 < nt; ++t) kp.emplace_back(keyer);
        keyer();
        for (auto& th : kp) th.join();
        for (size_t g = 0; g < graphs.size(); ++g) {
            std::unordered_map<std::string, int> first;
            for (int i = hp->graph_first_net[g]; i < hp->graph_first_net[g + 1]; ++i) {
                // only networks the plan holds whole (every slice, its 1/2 counted) share values
                const size_t li = (size_t)(i - hp->graph_first_net[g]);
                const bool part = (li < graphs[g].sel_slices.size() && !graphs[g].sel_slices[li].empty()) ||
                                  (li < graphs[g].sel_owner.size() && !graphs[g].sel_owner[li]);
                if (key[i].empty() || part) continue;
                auto it = first.emplace(key[i], i);
                if (!it.second) rep[i] = it.first->second;
            }
        }
    }
    std::vector<Adjacency> adjs(graphs.size());
    for (size_t g = 0; g < graphs.size(); ++g) adjs[g] = graph_adjacency(graphs[g]);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (;;) {
            int i = next.fetch_add(1);
            if (i >= n_nets) break;
            int g = (int)(std::upper_bound(hp->graph_first_net.begin(), hp->graph_first_net.end(), i) -
                          hp->graph_first_net.begin()) - 1;
            Network& net = hp->nets[i];
            net.graph = g;
            net.edge = graphs[g].edge_of((size_t)(i - hp->graph_first_net[g]));
            build_network(graphs[g], adjs[g], cfg.p, net.edge, &net);
            net.rep = rep[i];
            if (net.rep >= 0) continue;  // takes its representative's value: nothing to plan
            if (cfg.slice_width > 0) slice_network(&net, cfg.slice_width, cfg.max_slice_bits);
            {
                const size_t li = (size_t)(i - hp->graph_first_net[g]);
                if (li < graphs[g].sel_slices.size()) {
                    net.slices = graphs[g].sel_slices[li];
                    for (uint32_t s : net.slices)
                        if (s >= (1u << net.slice_bits)) {
                            status[i] = QT_EINVAL;  // a slice the network does not have
                            break;
                        }
                    if (status[i] != QT_OK) continue;
                }
                if (li < graphs[g].sel_owner.size()) net.owner = graphs[g].sel_owner[li] != 0;
            }
            std::vector<int> best_order, ord;
            double best_cost = 0, c = 0;
            int best_w = 0, w = 0;
            order_min_fill(net, false, 0, &best_order, &best_cost, &best_w);
            // a restart's order is kept if cheaper and, with slicing, no wider than the target
            // (or the greedy width, if the slice-bit budget left that wider)
            const int w_cap = cfg.slice_width > 0 ? std::max(cfg.slice_width, best_w) : cfg.max_width;
            for (int r = 0; r < (best_w >= cfg.restart_min_width ? cfg.restarts : 0); ++r) {
                // seeded by the network's identity (graph, edge), so that subset, shard and pass
                // plans of a graph order each network as the whole graph's plan does
                const uint64_t id = ((uint64_t)g << 32) | (uint64_t)(uint32_t)net.edge;
                order_min_fill(net, true, mix64(cfg.seed ^ mix64(id * 1315423911ull + r)), &ord, &c, &w);
                if (c < best_cost && w <= w_cap) {
                    best_cost = c;
                    best_order = ord;
                    best_w = w;
                }
            }
            if (best_w > cfg.max_width) {
                status[i] = QT_EWIDTH;
                continue;
            }
            NetPlan& np = hp->nplans[i];
            np.order = best_order;
            status[i] = make_buckets(net, best_order, cfg.max_width, &np);
            if (status[i] == QT_OK && cfg.merge) merge_chains(&np);
        }
    };
    unsigned nthreads = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
    nthreads = std::min<unsigned>(nthreads, (unsigned)n_nets);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t + 1 < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int s : status)
        if (s != QT_OK) return s;
    const int rc = layout_plan(hp);
    hp->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

// Everything after the networks, their orders and buckets: tile choice,
// device layout, fused units, claim order, reverse-sweep tasks. Rerun by the
// autotuner for each candidate configuration (hp->cfg).
int layout_plan(HostPlan* hp) {
    const PlanConfig& cfg = hp->cfg;
    const std::vector<GraphIn>& graphs = hp->graphs;
    const int n_nets = hp->graph_first_net.back();
    hp->op_src.clear();
    hp->op_leaf_kind.clear();
    hp->op_leaf_layer.clear();
    hp->op_rank.clear();
    hp->bucket_level.clear();
    hp->bucket_var.clear();
    hp->bucket_var2.clear();
    hp->bucket_var3.clear();
    hp->root_bucket.clear();
    hp->sim_seconds = 0;

    // ---- flatten ---------------------------------------------------------
    const uint64_t esize = cfg.dtype == 1 ? 16 : 8;
    const uint64_t align = 128 / esize;
    const int L = leaf_slots_per_graph(cfg.p);
    const uint64_t leaf_vals = (uint64_t)graphs.size() * L * kLeafSlots;
    hp->dleaf_off = cfg.with_grad ? leaf_vals : 0;
    hp->leaf_elems = align_up(cfg.with_grad ? 2 * leaf_vals : leaf_vals, align);
    hp->op_param.clear();
    hp->net_graph.clear();
    uint64_t off = hp->leaf_elems;
    hp->net_first_bucket.assign(1, 0);
    hp->net_first_root.assign(1, 0);
    hp->buckets.clear();
    hp->operands.clear();
    hp->max_width = 0;
    hp->n_levels = 0;
    hp->sum_2w = hp->alg_bytes = hp->flops = 0;
    std::fill(hp->width_hist, hp->width_hist + 64, 0);
    hp->bucket_slice.clear();
    {
        // sizes of the flat arrays, so that they grow once
        size_t nb = 0, no = 0;
        for (int i = 0; i < n_nets; ++i) {
            if (hp->nets[i].rep >= 0) continue;
            size_t ops = 0;
            for (const HBucket& B : hp->nplans[i].buckets) ops += B.ops.size();
            nb += hp->nplans[i].buckets.size() * hp->nets[i].n_emitted();
            no += ops * hp->nets[i].n_emitted();
        }
        hp->buckets.reserve(nb);
        hp->bucket_level.reserve(nb);
        hp->bucket_var.reserve(nb);
        hp->bucket_var2.reserve(nb);
        hp->bucket_var3.reserve(nb);
        hp->bucket_slice.reserve(nb);
        hp->operands.reserve(no);
        hp->op_src.reserve(no);
        hp->op_leaf_kind.reserve(no);
        hp->op_leaf_layer.reserve(no);
        hp->op_rank.reserve(no);
        hp->op_leaf_sub.reserve(no);
        hp->op_param.reserve(no);
    }
    hp->op_leaf_sub.clear();
    hp->net_first_factor.assign(1, 0);
    hp->factor.clear();
    hp->factor_param.clear();
    hp->graph_owned.assign(graphs.size(), 0);
    hp->n_unique = 0;
    hp->net_weight.clear();
    hp->n_slices = 0;
    for (int i = 0; i < n_nets; ++i) {
        const NetPlan& np = hp->nplans[i];
        const Network& net = hp->nets[i];
        if (net.rep >= 0) {
            // the representative's value: its factor list (it comes earlier)
            for (uint32_t f = hp->net_first_factor[net.rep]; f < hp->net_first_factor[net.rep + 1]; ++f) {
                const uint64_t w = hp->factor[f];
                const int8_t fp = hp->factor_param[f];
                hp->factor.push_back(w);
                hp->factor_param.push_back(fp);
            }
        }
        // every slice of the network: the same buckets, its own gate entries
        for (uint32_t k = 0; k < (net.rep >= 0 ? 0u : net.n_emitted()); ++k) {
            const uint32_t sl = net.slice_at(k);
            const uint32_t base = (uint32_t)hp->buckets.size();
            const size_t root0 = hp->root_bucket.size();
            for (size_t lb = 0; lb < np.buckets.size(); ++lb) {
                const HBucket& B = np.buckets[lb];
                HBucket merged_view;  // only merged buckets need a device view of their own
                if (B.n_sum > 1) merged_view = device_view(B);
                const HBucket& V = B.n_sum > 1 ? merged_view : B;
                DBucket d{};
                d.op_begin = (uint32_t)hp->operands.size();
                d.n_ops = (uint8_t)B.ops.size();
                d.n_out = (uint8_t)(B.width - 1);
                int cb = 0;
                bool fold = false;
                const int tcap = cfg.tile_cap[width_class(d.n_out)];
                pick_tile(V, net, tcap > 0 ? tcap : cfg.chunk_log2 > 0 ? cfg.chunk_log2 : kDefaultTileBits,
                          cfg.dtype == 1 ? kStageElemsC128 : kStageElemsC64, B.n_sum - 1, &cb, &fold);
                d.chunk_bits = (uint8_t)cb;
                d.flags = (uint8_t)((fold ? kBucketFoldLeaves : 0) | ((B.n_sum - 1) << 3));
                {
                    const uint32_t low = (1u << cb) - 1u;
                    uint32_t foot = 0, ns = 0, nl = 0, lu = 0, lh = 0;
                    for (const HOperand& op : V.ops) {
                        if (fold && foldable(op)) {
                            nl++;
                            lu |= op.mask & low;
                            lh |= op.mask & ~low;
                        } else {
                            foot += (1u << __builtin_popcount(op.smask)) << __builtin_popcount(op.mask & low);
                            ns++;
                        }
                    }
                    d.total_foot = foot;
                    d.n_staged = (uint8_t)ns;
                    d.n_leaves = (uint8_t)nl;
                    d.leaf_u = lu;
                    d.leaf_hi = lh;
                }
                d.parent = B.parent >= 0 ? base + (uint32_t)B.parent : kNone;
                d.n_deps = (uint32_t)B.n_deps;
                d.n_tasks = 1u << (d.n_out - cb);
                d.net = (uint32_t)i;
                d.out_off = off;
                off += align_up(1ull << (B.width - B.n_sum), align);
                double opbytes = 0;
                uint32_t next_soff = 0, next_staged = 0, next_leaf = 0;
                for (size_t t = 0; t < B.ops.size(); ++t) {
                    const HOperand& op = V.ops[t];
                    DOperand o{};
                    o.mask = op.mask;
                    o.src = kNone;
                    o.folded = (d.flags & kBucketFoldLeaves) && foldable(op);
                    o.smask = (uint8_t)B.ops[t].smask;
                    if (o.folded) {
                        o.slot = (uint8_t)next_leaf++;
                    } else {
                        o.slot = (uint8_t)next_staged++;
                        o.soff = (uint16_t)next_soff;
                        next_soff += (1u << __builtin_popcount(op.smask)) << __builtin_popcount(op.mask & ((1u << d.chunk_bits) - 1u));
                    }
                    if (op.src >= 0) {
                        o.off = 0;  // set below, once every result has its offset
                        o.flags = 0;
                    } else {
                        const Leaf& lf = net.leaves[op.leaf];
                        o.off = ((uint64_t)net.graph * L + leaf_index(lf.kind, lf.layer)) * kLeafSlots +
                                (lf.fix >= 0 ? 2u * ((sl >> lf.fix) & 1u) : 0u);
                        o.flags = kOpLeaf;
                    }
                    hp->operands.push_back(o);
                    hp->op_src.push_back(op.src >= 0 ? (int32_t)(base + op.src) : -1);
                    hp->op_leaf_kind.push_back(op.src >= 0 ? -1 : net.leaves[op.leaf].kind);
                    hp->op_leaf_layer.push_back(op.src >= 0 ? -1 : net.leaves[op.leaf].layer);
                    hp->op_rank.push_back(op.rank);
                    hp->op_leaf_sub.push_back(op.src >= 0 || net.leaves[op.leaf].fix < 0
                                                  ? 0
                                                  : (int32_t)(2u * ((sl >> net.leaves[op.leaf].fix) & 1u)));
                    {
                        int8_t prm = -1;
                        if (op.src < 0) {
                            const Leaf& lf = net.leaves[op.leaf];
                            if (lf.kind == QT_LEAF_ZZ || lf.kind == QT_LEAF_ZZ_CONJ) prm = (int8_t)lf.layer;
                            if (lf.kind == QT_LEAF_RX || lf.kind == QT_LEAF_RX_CONJ) prm = (int8_t)(cfg.p + lf.layer);
                        }
                        hp->op_param.push_back(prm);
                    }
                    opbytes += std::ldexp(1.0, op.rank);
                }
                hp->buckets.push_back(d);
                hp->bucket_level.push_back(B.level);
                hp->bucket_var.push_back(B.var);
                hp->bucket_var2.push_back(B.var2);
                hp->bucket_var3.push_back(B.var3);
                hp->bucket_slice.push_back((int32_t)sl);
                if (B.parent < 0) hp->root_bucket.push_back(base + (uint32_t)lb);
                hp->max_width = std::max(hp->max_width, B.width);
                hp->n_levels = std::max(hp->n_levels, B.level + 1);
                hp->width_hist[B.width]++;
                hp->sum_2w += std::ldexp(1.0, B.width);
                hp->alg_bytes += (double)esize * (opbytes + std::ldexp(1.0, B.width - B.n_sum));
                {
                    // a merged bucket counts the flops of its unmerged buckets: the
                    // bucket of s0 (products of its operands, sums over s0), then each
                    // consumer's gate products and its sum; operand t belongs to the
                    // bucket of its earliest summed variable
                    double n_k[4] = {0, 0, 0, 0};
                    for (const HOperand& op : B.ops) n_k[__builtin_ctz(op.smask)] += 1;
                    for (int v = 0; v < B.n_sum; ++v)
                        hp->flops += std::ldexp(1.0, B.width - v) * 6.0 * (n_k[v] - (v == 0 ? 1 : 0)) +
                                     std::ldexp(1.0, B.width - v - 1) * 2.0;
                }
            }
            // the slice's factors of the network's value: its root results,
            // then the entries of its fully fixed gates
            bool first = true;
            auto push_factor = [&](uint64_t e, int8_t prm) {
                hp->factor.push_back(e | (first ? kFirstFactor : 0));
                hp->factor_param.push_back(prm);
                first = false;
            };
            for (size_t r = root0; r < hp->root_bucket.size(); ++r)
                push_factor(hp->buckets[hp->root_bucket[r]].out_off, kFactorRoot);
            for (const FixedLeaf& fl : net.fixed) {
                uint32_t e = (sl >> fl.f[0]) & 1u;
                if (fl.rank == 2) e += 2u * ((sl >> fl.f[1]) & 1u);
                int8_t prm = -1;
                if (fl.kind == QT_LEAF_ZZ || fl.kind == QT_LEAF_ZZ_CONJ) prm = (int8_t)fl.layer;
                if (fl.kind == QT_LEAF_RX || fl.kind == QT_LEAF_RX_CONJ) prm = (int8_t)(cfg.p + fl.layer);
                push_factor(((uint64_t)net.graph * L + leaf_index(fl.kind, fl.layer)) * kLeafSlots + e, prm);
            }
            hp->n_slices++;
        }
        hp->n_unique += net.rep < 0 ? 1 : 0;
        if (net.rep >= 0) {  // the reverse sweep seeds a representative once for its whole class
            if (hp->net_weight.empty()) hp->net_weight.assign(n_nets, 1);
            hp->net_weight[net.rep]++;
            hp->net_weight[i] = 0;
        }
        hp->net_first_factor.push_back((uint32_t)hp->factor.size());
        if ((int)hp->graph_owned.size() <= net.graph) hp->graph_owned.resize(net.graph + 1, 0);
        hp->graph_owned[net.graph] += net.owner ? 1 : 0;
        hp->net_first_bucket.push_back((uint32_t)hp->buckets.size());
        hp->net_first_root.push_back((uint32_t)hp->root_bucket.size());
        hp->net_graph.push_back((uint32_t)net.graph);
    }
    // intermediate operands point at their producer's result and name it
    for (size_t o = 0; o < hp->operands.size(); ++o)
        if (hp->op_src[o] >= 0) {
            const DBucket& src = hp->buckets[hp->op_src[o]];
            hp->operands[o].off = src.out_off;
            hp->operands[o].src = (uint32_t)hp->op_src[o];
            hp->operands[o].src_tiles = src.n_tasks;
        }
    hp->arena_elems = off;
    hp->cot_off = 0;
    hp->total_elems = off;
    if (cfg.with_grad) {
        hp->cot_off = off;  // cotangent of each result mirrors the result region
        hp->total_elems = off + (off - hp->leaf_elems);
    }

    // ---- tasks in level order, grouped into work items ---------------------
    const uint32_t nb = (uint32_t)hp->buckets.size();
    hp->by_level.resize(nb);
    for (uint32_t b = 0; b < nb; ++b) hp->by_level[b] = b;
    // level order (a topological order); within a level the largest buckets
    // first, so that a level ends on small tasks
    std::stable_sort(hp->by_level.begin(), hp->by_level.end(), [&](uint32_t a, uint32_t b) {
        if (hp->bucket_level[a] != hp->bucket_level[b]) return hp->bucket_level[a] < hp->bucket_level[b];
        return hp->buckets[a].n_out > hp->buckets[b].n_out;
    });
    hp->level_first_bucket.assign(hp->n_levels + 1, 0);
    for (uint32_t b : hp->by_level) hp->level_first_bucket[hp->bucket_level[b] + 1]++;
    for (int l = 0; l < hp->n_levels; ++l) hp->level_first_bucket[l + 1] += hp->level_first_bucket[l];
    // Work groups: a bucket's tiles are handed out in groups of group_tiles
    // consecutive tiles, so a warp reads the bucket's descriptors once per group.
    hp->runs.clear();
    hp->n_tiles = 0;
    hp->n_groups = 0;
    for (uint32_t b : hp->by_level) {
        DBucket& d = hp->buckets[b];
        const uint32_t rt = cfg.run_tiles > 0 ? (uint32_t)cfg.run_tiles : (uint32_t)kRunTiles;
        d.group_tiles = std::min(rt, d.n_tasks);
        d.n_groups = (d.n_tasks + d.group_tiles - 1) / d.group_tiles;
        hp->n_tiles += d.n_tasks;
        hp->n_groups += d.n_groups;
    }
    form_units(hp, cfg.dtype == 1 ? kStageElemsC128 : kStageElemsC64);
    if (cfg.order == 1) {
        // ready queue: groups of buckets without producers open it (fused units
        // among them), in level order with the largest buckets first; every
        // other bucket appends its groups when its last producer finishes
        for (uint32_t b : hp->by_level) {
            const DBucket& d = hp->buckets[b];
            if (d.flags & kBucketInUnit) continue;
            if (d.flags & kBucketUnitRoot) {
                hp->runs.push_back(unit_run(*hp, b));
            } else if (d.n_deps == 0) {
                for (uint32_t c = 0; c < d.n_tasks; c += d.group_tiles)
                    hp->runs.push_back(DRun{b, c, std::min(d.group_tiles, d.n_tasks - c), d.op_begin, 0, 0, 0, d.n_ops});
            }
        }
    } else {
        simulate_order(hp);
    }
    // reverse sweep: tiles of every bucket, level by level (a bucket's result
    // cotangent is complete once its consumer, at a higher level, is done)
    hp->bwd_bucket.clear();
    hp->bwd_tile.clear();
    hp->bwd_level_begin.assign(1, 0);
    hp->op_bwd.assign(hp->operands.size(), kBwdNone);
    hp->op_roff.assign(hp->operands.size(), 0);
    hp->bwd_zero.clear();
    if (cfg.with_grad) {
        // Each result has one consumer, so its cotangent comes from one bucket:
        // entries are stored once where the operand carries every output bit,
        // or summed in shared memory over the tile's bits it lacks; only
        // operands lacking bits above the tile take atomic adds (and a zeroed
        // cotangent).
        const uint64_t cot_delta = hp->cot_off - hp->leaf_elems;
        for (uint32_t b = 0; b < nb; ++b) {
            const DBucket& d = hp->buckets[b];
            const uint32_t outm = d.n_out ? ((1u << d.n_out) - 1u) : 0u;
            const int tb = std::min<int>(d.n_out, kBwdTileBits);
            const uint32_t low = (1u << tb) - 1u;
            uint32_t used = 0;
            for (uint32_t i = d.op_begin; i < d.op_begin + d.n_ops; ++i) {
                const DOperand& o = hp->operands[i];
                int8_t mode;
                if (o.flags & kOpLeaf) {
                    mode = hp->op_param[i] >= 0 ? kBwdGate : kBwdNone;
                } else if (o.mask == outm) {
                    mode = kBwdDirect;
                } else {
                    const uint32_t fp = 2u << __builtin_popcount(o.mask & low);
                    const bool hi_free = (outm & ~low & ~o.mask) != 0u;
                    if (used + fp <= (uint32_t)kBwdRedElems) {
                        mode = hi_free ? kBwdRedAtomic : kBwdRedStore;
                        hp->op_roff[i] = (uint16_t)used;
                        used += fp;
                    } else {
                        mode = kBwdAtomic;
                    }
                    if (mode != kBwdRedStore) {
                        const DBucket& src = hp->buckets[o.src];
                        const uint64_t n = 1ull << result_bits(src);
                        for (uint64_t c = 0; c < n; c += kZeroChunk) {
                            hp->bwd_zero.push_back(src.out_off + cot_delta + c);
                            hp->bwd_zero.push_back(std::min<uint64_t>(kZeroChunk, n - c));
                        }
                    }
                }
                hp->op_bwd[i] = mode;
            }
        }
        // tasks by level, and within a level by operand-count class (one
        // launch each): bwd_level_begin[kBwdClasses * lv + c] starts class c
        for (int lv = 0; lv < hp->n_levels; ++lv) {
            for (int cls = 0; cls < kBwdClasses; ++cls) {
                if (cls > 0) hp->bwd_level_begin.push_back((uint32_t)hp->bwd_bucket.size());
                for (uint32_t i = hp->level_first_bucket[lv]; i < hp->level_first_bucket[lv + 1]; ++i) {
                    const uint32_t b = hp->by_level[i];
                    if (bwd_op_class(hp->buckets[b].n_ops) != cls) continue;
                    const int tb = std::min<int>(hp->buckets[b].n_out, kBwdTileBits);
                    for (uint32_t t = 0; t < (1u << (hp->buckets[b].n_out - tb)); ++t) {
                        hp->bwd_bucket.push_back(b);
                        hp->bwd_tile.push_back(t);
                    }
                }
            }
            hp->bwd_level_begin.push_back((uint32_t)hp->bwd_bucket.size());
        }
    }
    return QT_OK;
}

// ---------------------------------------------------------------------------
// Contraction of caller-supplied tensors over binary indices (the paper's
// "tncontract" benchmark, §II-E), planned with the same bucket elimination
// (§II-B), merged eliminations (§II-C) and device layout as the energy plans.
// ---------------------------------------------------------------------------
int build_contract_plan(const std::vector<std::vector<int>>& labels, const std::vector<int>& out_labels, int dtype,
                        int sim_workers, ContractPlan* cp) {
    *cp = ContractPlan();
    cp->dtype = dtype;
    const int n_in = (int)labels.size();
    if (n_in < 1 || n_in > kMaxOps || (dtype != 0 && dtype != 1)) return QT_EINVAL;
    // variables: the distinct labels in order of first appearance
    std::vector<int> count;  // operands holding each variable
    std::unordered_map<int, int> var_of;
    for (const auto& L : labels) {
        if (L.empty() || L.size() > (size_t)kMaxOutBits) return QT_EINVAL;
        std::set<int> seen;
        for (int l : L) {
            if (l < 0 || !seen.insert(l).second) return QT_EINVAL;
            auto it = var_of.emplace(l, (int)count.size());
            if (it.second) count.push_back(0);
            count[it.first->second]++;
        }
    }
    const int V = (int)count.size();
    if (V > kMaxOutBits) return QT_EINVAL;
    std::vector<uint8_t> free_var(V, 0);
    {
        std::set<int> seen;
        for (int l : out_labels) {
            auto it = var_of.find(l);
            if (it == var_of.end() || !seen.insert(l).second) return QT_EINVAL;
            free_var[it->second] = 1;
        }
    }
    // elimination order: the summed variables (those in more operands first),
    // then the output's bits from the lowest (its last label) up
    std::vector<int> order;
    for (int v = 0; v < V; ++v)
        if (!free_var[v]) order.push_back(v);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return count[a] > count[b]; });
    const int S = (int)order.size();
    if (S == 0) return QT_EINVAL;  // nothing summed: not a contraction
    for (int k = (int)out_labels.size() - 1; k >= 0; --k) order.push_back(var_of[out_labels[k]]);
    std::vector<int> pos(V);
    for (int i = 0; i < V; ++i) pos[order[i]] = i;
    // bucket elimination of the summed variables (as make_buckets); an operand
    // whose labels are all free would need an outer product: refused
    struct Tens {
        std::vector<int> vars;  // by rank
        int src;
    };
    std::vector<Tens> pool;
    std::vector<std::vector<int>> bucket_of(V);
    for (int t = 0; t < n_in; ++t) {
        Tens T;
        for (int l : labels[t]) T.vars.push_back(var_of[l]);
        std::sort(T.vars.begin(), T.vars.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        if (free_var[T.vars[0]]) return QT_EINVAL;
        T.src = -1 - t;  // caller's operand t
        bucket_of[T.vars[0]].push_back((int)pool.size());
        pool.push_back(std::move(T));
    }
    NetPlan np;
    for (int step = 0; step < S; ++step) {
        const int v = order[step];
        auto& list = bucket_of[v];
        std::vector<int> uni;
        for (int t : list)
            for (int x : pool[t].vars) uni.push_back(x);
        std::sort(uni.begin(), uni.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
        const int w = (int)uni.size();
        if (list.empty() || (int)list.size() > kMaxOps) return QT_EWIDTH;
        HBucket B;
        B.var = v;
        B.width = w;
        B.parent = -1;
        B.n_deps = 0;
        B.level = 0;
        const int bid = (int)np.buckets.size();
        for (int t : list) {
            const Tens& T = pool[t];
            HOperand op;
            op.src = T.src >= 0 ? T.src : -1;
            op.leaf = T.src >= 0 ? -1 : -1 - T.src;
            op.rank = (int)T.vars.size();
            op.mask = 0;
            for (size_t i = 1; i < T.vars.size(); ++i)
                op.mask |= 1u << ((int)(std::find(uni.begin() + 1, uni.end(), T.vars[i]) - uni.begin()) - 1);
            if (T.src >= 0) {
                B.n_deps++;
                np.buckets[T.src].parent = bid;
                B.level = std::max(B.level, np.buckets[T.src].level + 1);
            }
            B.ops.push_back(op);
        }
        list.clear();
        if (w > 1) {
            Tens R;
            R.vars.assign(uni.begin() + 1, uni.end());
            R.src = bid;
            bucket_of[R.vars[0]].push_back((int)pool.size());
            pool.push_back(std::move(R));
        }
        np.buckets.push_back(std::move(B));
    }
    // one result must remain, over exactly the output's variables
    int left = 0, last = -1;
    for (int k = S; k < V; ++k)
        for (int t : bucket_of[order[k]]) {
            left++;
            last = t;
        }
    int roots = 0;
    for (const HBucket& B : np.buckets) roots += B.parent < 0;
    if (roots != 1 || np.buckets.back().parent >= 0) return QT_EINVAL;  // pieces that would need an outer product
    if (out_labels.empty() ? left != 0 : (left != 1 || pool[last].vars.size() != out_labels.size()))
        return QT_EINVAL;
    merge_chains(&np);
    // ---- device layout: the caller's operands (permuted) first, then the results
    const uint64_t esize = dtype == 1 ? 16 : 8;
    const uint64_t align = 128 / esize;
    uint64_t off = 0;
    for (int t = 0; t < n_in; ++t) {
        const int r = (int)labels[t].size();
        std::vector<int> vars;
        for (int l : labels[t]) vars.push_back(var_of[l]);
        std::vector<int> byrank = vars;
        std::sort(byrank.begin(), byrank.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        std::vector<uint8_t> src_bit(r);
        for (int k = 0; k < r; ++k) {
            const int a = (int)(std::find(vars.begin(), vars.end(), byrank[k]) - vars.begin());  // C-order axis
            src_bit[k] = (uint8_t)(r - 1 - a);
        }
        cp->in_rank.push_back(r);
        cp->in_off.push_back(off);
        cp->in_src_bit.push_back(std::move(src_bit));
        off += align_up(std::max<uint64_t>(1ull << r, kLeafSlots), align);
    }
    Network none;
    for (const HBucket& B : np.buckets) {
        HBucket merged_view;
        if (B.n_sum > 1) merged_view = device_view(B);
        const HBucket& Vw = B.n_sum > 1 ? merged_view : B;
        DBucket d{};
        d.op_begin = (uint32_t)cp->operands.size();
        d.n_ops = (uint8_t)B.ops.size();
        d.n_out = (uint8_t)(B.width - 1);
        int cb = 0;
        bool fold = false;
        const int stage = dtype == 1 ? kStageElemsC128 : kStageElemsC64;
        pick_tile(Vw, none, kDefaultTileBits, stage, B.n_sum - 1, &cb, &fold);
        d.chunk_bits = (uint8_t)cb;
        d.flags = (uint8_t)((fold ? kBucketFoldLeaves : 0) | ((B.n_sum - 1) << 3));
        const uint32_t low = (1u << cb) - 1u;
        uint32_t foot = 0, ns = 0, nl = 0, lu = 0, lh = 0;
        for (const HOperand& op : Vw.ops) {
            if (fold && foldable(op)) {
                nl++;
                lu |= op.mask & low;
                lh |= op.mask & ~low;
            } else {
                foot += (1u << __builtin_popcount(op.smask)) << __builtin_popcount(op.mask & low);
                ns++;
            }
        }
        if (foot > (uint32_t)stage) return QT_EWIDTH;  // no tile's footprints fit the stage
        d.total_foot = foot;
        d.n_staged = (uint8_t)ns;
        d.n_leaves = (uint8_t)nl;
        d.leaf_u = lu;
        d.leaf_hi = lh;
        d.parent = B.parent >= 0 ? (uint32_t)B.parent : kNone;
        d.n_deps = (uint32_t)B.n_deps;
        d.n_tasks = 1u << (d.n_out - cb);
        d.out_off = off;
        off += align_up(std::max<uint64_t>(1ull << (B.width - B.n_sum), kLeafSlots), align);
        double opbytes = 0;
        uint32_t next_soff = 0, next_staged = 0, next_leaf = 0;
        for (size_t t = 0; t < B.ops.size(); ++t) {
            const HOperand& op = Vw.ops[t];
            DOperand o{};
            o.mask = op.mask;
            o.src = kNone;
            o.folded = fold && foldable(op);
            o.smask = (uint8_t)B.ops[t].smask;
            if (o.folded) {
                o.slot = (uint8_t)next_leaf++;
            } else {
                o.slot = (uint8_t)next_staged++;
                o.soff = (uint16_t)next_soff;
                next_soff += (1u << __builtin_popcount(op.smask)) << __builtin_popcount(op.mask & low);
            }
            if (op.src >= 0) {
                o.src = (uint32_t)op.src;
                o.off = cp->buckets[op.src].out_off;
                o.src_tiles = cp->buckets[op.src].n_tasks;
            } else {
                o.off = cp->in_off[op.leaf];
                o.flags = kOpLeaf;  // written before the bucket kernel starts
            }
            cp->operands.push_back(o);
            opbytes += std::ldexp(1.0, op.rank);
        }
        cp->buckets.push_back(d);
        cp->widths.push_back(B.width);
        cp->max_width = std::max(cp->max_width, B.width);
        cp->alg_bytes += (double)esize * (opbytes + std::ldexp(1.0, B.width - B.n_sum));
        double n_k[4] = {0, 0, 0, 0};
        for (const HOperand& op : B.ops) n_k[__builtin_ctz(op.smask)] += 1;
        for (int v = 0; v < B.n_sum; ++v)  // complex multiply-adds: 8 flops each (4 real mul, 4 real add)
            cp->flops += 8.0 * (std::ldexp(1.0, B.width - v) * (n_k[v] - (v == 0 ? 1 : 0) + 0.5));
    }
    cp->operands.resize(cp->operands.size() + kMaxOps, DOperand{});  // kernels read a bucket's operands in 16s
    cp->out_off = cp->buckets.back().out_off;
    cp->out_rank = (int)out_labels.size();
    cp->n_summed = S;
    cp->arena_elems = off;
    // work groups: spread each bucket over the grid (it runs alone once its producer is done)
    const uint32_t W = (uint32_t)std::max(1, sim_workers);
    for (uint32_t b = 0; b < (uint32_t)cp->buckets.size(); ++b) {
        DBucket& d = cp->buckets[b];
        d.group_tiles = lone_group_tiles(d.n_tasks, W, kRunTiles);
        d.n_groups = (d.n_tasks + d.group_tiles - 1) / d.group_tiles;
        for (uint32_t c = 0; c < d.n_tasks; c += d.group_tiles)
            cp->runs.push_back(DRun{b, c, std::min(d.group_tiles, d.n_tasks - c), d.op_begin, d.n_deps, 0, 0, d.n_ops});
    }
    return QT_OK;
}

}  // namespace qt
