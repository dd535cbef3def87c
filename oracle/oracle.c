/*
 * CPU oracle for the QAOA MaxCut edge expectations e_jk = <g,b| Z_j Z_k |g,b>.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header
 * or table with the CUDA path and never calls it.
 *
 * Everything is complex128 (C99 `double complex`), written as plain loops.
 *
 * Problem (§II-A and §II-B of the paper):
 *   MaxCut cost C = 1/2 sum_{(ij) in E} (1 - Z_i Z_j)                    (Eq. 1)
 *   |g,b>_p = prod_k e^{-i b_k B} e^{-i g_k C} |+>,  B = sum_i X_i        (Eq. 2)
 *   <C> = |E|/2 - 1/2 sum_{jk in E} e_jk   (edge decomposition, §II-B)
 *
 * Gate convention (the paper's Eq. 2 up to a rescaling of gamma, see the
 * design notes): layer k applies, in this order,
 *   ZZ phase on every edge (a,b):  exp(-i gamma_k s_a s_b),  s(x) = 1 - 2x,
 *   mixer on every qubit:          exp(-i beta_k X) = [[c, -i s], [-i s, c]],
 * starting from |+>^N.  Z|0> = +|0>.
 *
 * Three routes:
 *   1. state vector over all 2^N amplitudes           (oracle_sv_*)
 *   2. bucket elimination of each edge's lightcone      (oracle_bucket_*)
 *      tensor network, with this file's own network
 *      builder and its own min-degree order (or, for
 *      the large N=1000 p=5 networks, its own greedy
 *      min-fill order; both break ties at random)
 *   3. brute-force sum over every variable assignment   (oracle_edge_brute)
 *      of one lightcone network
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_ETOOBIG -3

/* ------------------------------------------------------------------------ */
/* threads                                                                    */
/* ------------------------------------------------------------------------ */

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check_graph(int n, int m, const int32_t *edges) {
    if (n < 2 || m < 1 || !edges) return OR_EINVAL;
    for (int e = 0; e < m; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return OR_EINVAL;
    }
    return OR_OK;
}

static inline double spin(uint64_t z, int q) { return ((z >> q) & 1u) ? -1.0 : 1.0; }

/* ------------------------------------------------------------------------ */
/* Route 1: state vector                                                      */
/* ------------------------------------------------------------------------ */

/*
 * Evolve |+>^n through p layers, each gate with its own angle, then return
 * e[e] = <psi| Z_a Z_b |psi> for every edge.
 *   zz_angles[k*m + e]  angle of the ZZ phase gate of edge e in layer k
 *   x_angles[k*n + q]   angle of the mixer of qubit q in layer k
 * Per-gate angles let the parameter-shift gradient shift one gate at a time.
 * Eq. 2 of the paper with the gate convention of the header.
 */
int oracle_sv_zz_gates(int n, int m, const int32_t *edges, int p,
                       const double *zz_angles, const double *x_angles, double *zz_out) {
    if (check_graph(n, m, edges) != OR_OK || p < 1 || n > 34) return OR_EINVAL;
    const uint64_t dim = (uint64_t)1 << n;
    cplx *psi = (cplx *)malloc(dim * sizeof(cplx));
    if (!psi) return OR_ENOMEM;
    const double amp = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
    for (uint64_t z = 0; z < dim; ++z) psi[z] = amp;

    for (int k = 0; k < p; ++k) {
        /* diagonal cost layer: psi[z] *= exp(-i sum_e theta_e s_a(z) s_b(z)) */
#pragma omp parallel for schedule(static)
        for (uint64_t z = 0; z < dim; ++z) {
            double phase = 0.0;
            for (int e = 0; e < m; ++e)
                phase += zz_angles[(size_t)k * m + e] * spin(z, edges[2 * e]) * spin(z, edges[2 * e + 1]);
            psi[z] *= cexp(-I * phase);
        }
        /* mixer layer: exp(-i theta X) on each qubit, as in-place pair updates */
        for (int q = 0; q < n; ++q) {
            const double c = cos(x_angles[(size_t)k * n + q]);
            const double s = sin(x_angles[(size_t)k * n + q]);
            const uint64_t low = ((uint64_t)1 << q) - 1;
#pragma omp parallel for schedule(static)
            for (uint64_t i = 0; i < dim / 2; ++i) {
                uint64_t z0 = ((i & ~low) << 1) | (i & low); /* bit q is 0 */
                uint64_t z1 = z0 | ((uint64_t)1 << q);
                cplx a = psi[z0], b = psi[z1];
                psi[z0] = c * a - I * s * b;
                psi[z1] = -I * s * a + c * b;
            }
        }
    }

    /* <Z_a Z_b> = sum_z |psi_z|^2 s_a(z) s_b(z) */
    for (int e = 0; e < m; ++e) zz_out[e] = 0.0;
#pragma omp parallel
    {
        double *acc = (double *)calloc((size_t)m, sizeof(double));
#pragma omp for schedule(static)
        for (uint64_t z = 0; z < dim; ++z) {
            double pr = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
            for (int e = 0; e < m; ++e) acc[e] += pr * spin(z, edges[2 * e]) * spin(z, edges[2 * e + 1]);
        }
#pragma omp critical
        for (int e = 0; e < m; ++e) zz_out[e] += acc[e];
        free(acc);
    }
    free(psi);
    return OR_OK;
}

/* Same, with one gamma and one beta per layer (Eq. 2 as written). */
int oracle_sv_zz(int n, int m, const int32_t *edges, int p,
                 const double *gammas, const double *betas, double *zz_out) {
    if (p < 1) return OR_EINVAL;
    double *ga = (double *)malloc(sizeof(double) * (size_t)p * m);
    double *xa = (double *)malloc(sizeof(double) * (size_t)p * n);
    if (!ga || !xa) { free(ga); free(xa); return OR_ENOMEM; }
    for (int k = 0; k < p; ++k) {
        for (int e = 0; e < m; ++e) ga[(size_t)k * m + e] = gammas[k];
        for (int q = 0; q < n; ++q) xa[(size_t)k * n + q] = betas[k];
    }
    int rc = oracle_sv_zz_gates(n, m, edges, p, ga, xa, zz_out);
    free(ga);
    free(xa);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Lightcone tensor network of one edge (§II-B)                              */
/* ------------------------------------------------------------------------ */

/* One tensor of rank 1 or 2 over binary variables.
 * Entry index: bit i of the index is the value of vars[i]. */
typedef struct {
    int rank;
    int vars[2];
    cplx data[4];
} leaf_t;

typedef struct {
    int nvars;
    int ntens;
    int cap;
    leaf_t *t;
    int *qubit_vars; /* per qubit: number of variables on its wire (0 = outside) */
} network_t;

static void net_free(network_t *net) {
    free(net->t);
    free(net->qubit_vars);
    memset(net, 0, sizeof(*net));
}

static int net_push(network_t *net, leaf_t t) {
    if (net->ntens == net->cap) {
        int cap = net->cap ? 2 * net->cap : 64;
        leaf_t *nt = (leaf_t *)realloc(net->t, sizeof(leaf_t) * (size_t)cap);
        if (!nt) return OR_ENOMEM;
        net->t = nt;
        net->cap = cap;
    }
    net->t[net->ntens++] = t;
    return OR_OK;
}

static leaf_t vec1(int v, cplx a0, cplx a1) {
    leaf_t t;
    memset(&t, 0, sizeof(t));
    t.rank = 1;
    t.vars[0] = v;
    t.vars[1] = -1;
    t.data[0] = a0;
    t.data[1] = a1;
    return t;
}

/* exp(-i g s_a s_b) on (a, b); the conjugate for the bra side. */
static leaf_t zz_phase(int a, int b, double g, int conj_) {
    leaf_t t;
    memset(&t, 0, sizeof(t));
    t.rank = 2;
    t.vars[0] = a;
    t.vars[1] = b;
    for (int xa = 0; xa < 2; ++xa)
        for (int xb = 0; xb < 2; ++xb) {
            double ss = (1 - 2 * xa) * (1 - 2 * xb);
            cplx v = cexp(-I * g * ss);
            t.data[xa | (xb << 1)] = conj_ ? conj(v) : v;
        }
    return t;
}

/* <new| exp(-i b X) |old> on (old, new); the conjugate for the bra side. */
static leaf_t mixer(int old_v, int new_v, double b, int conj_) {
    leaf_t t;
    memset(&t, 0, sizeof(t));
    t.rank = 2;
    t.vars[0] = old_v;
    t.vars[1] = new_v;
    for (int xo = 0; xo < 2; ++xo)
        for (int xn = 0; xn < 2; ++xn) {
            cplx v = (xo == xn) ? cos(b) : -I * sin(b);
            t.data[xo | (xn << 1)] = conj_ ? conj(v) : v;
        }
    return t;
}

/*
 * Distance from the edge {j,k} to every vertex, by breadth-first search over
 * the whole graph. -1 marks a vertex farther than p (or unreachable).
 */
static void edge_distances(int n, int m, const int32_t *edges, int j, int k, int p, int *dist) {
    for (int q = 0; q < n; ++q) dist[q] = -1;
    dist[j] = 0;
    dist[k] = 0;
    for (int d = 0; d < p; ++d) {
        for (int e = 0; e < m; ++e) {
            int a = edges[2 * e], b = edges[2 * e + 1];
            if (dist[a] == d && dist[b] < 0) dist[b] = d + 1;
            if (dist[b] == d && dist[a] < 0) dist[a] = d + 1;
        }
    }
}

/*
 * Build the lightcone network of edge `eidx` (§II-B).
 * Gates outside the causal cone of Z_j Z_k cancel against their conjugates:
 *   the mixer of layer k (1-based) acts on qubit q when dist(q) <= p - k,
 *   the ZZ gate of layer k on edge (a,b) when min(dist(a), dist(b)) <= p - k.
 * Ket side: |+> on each qubit of the cone, then per layer the ZZ phases on the
 * current variables and a fresh variable behind every mixer. Z on the current
 * variables of j and k. Bra side: the mirror image with conjugated tensors,
 * layers in reverse, ending in <+|. Diagonal gates create no variables.
 */
static int build_network(int n, int m, const int32_t *edges, int p,
                         const double *gammas, const double *betas, int eidx, network_t *net) {
    memset(net, 0, sizeof(*net));
    int *dist = (int *)malloc(sizeof(int) * (size_t)n);
    int *cur = (int *)malloc(sizeof(int) * (size_t)n);
    net->qubit_vars = (int *)calloc((size_t)n, sizeof(int));
    if (!dist || !cur || !net->qubit_vars) { free(dist); free(cur); net_free(net); return OR_ENOMEM; }
    int j = edges[2 * eidx], k = edges[2 * eidx + 1];
    edge_distances(n, m, edges, j, k, p, dist);
    const double r = 1.0 / sqrt(2.0);
    int rc = OR_OK;

    for (int q = 0; q < n && rc == OR_OK; ++q) {
        if (dist[q] < 0) continue;
        cur[q] = net->nvars++;
        net->qubit_vars[q] = 1;
        rc = net_push(net, vec1(cur[q], r, r));
    }
    for (int layer = 1; layer <= p && rc == OR_OK; ++layer) {
        for (int e = 0; e < m && rc == OR_OK; ++e) {
            int a = edges[2 * e], b = edges[2 * e + 1];
            int da = dist[a] < 0 ? 1 << 30 : dist[a], db = dist[b] < 0 ? 1 << 30 : dist[b];
            if ((da < db ? da : db) <= p - layer) rc = net_push(net, zz_phase(cur[a], cur[b], gammas[layer - 1], 0));
        }
        for (int q = 0; q < n && rc == OR_OK; ++q) {
            if (dist[q] < 0 || dist[q] > p - layer) continue;
            int nv = net->nvars++;
            net->qubit_vars[q] += 1;
            rc = net_push(net, mixer(cur[q], nv, betas[layer - 1], 0));
            cur[q] = nv;
        }
    }
    if (rc == OR_OK) rc = net_push(net, vec1(cur[j], 1.0, -1.0));
    if (rc == OR_OK) rc = net_push(net, vec1(cur[k], 1.0, -1.0));
    for (int layer = p; layer >= 1 && rc == OR_OK; --layer) {
        for (int q = 0; q < n && rc == OR_OK; ++q) {
            if (dist[q] < 0 || dist[q] > p - layer) continue;
            int nv = net->nvars++;
            net->qubit_vars[q] += 1;
            rc = net_push(net, mixer(cur[q], nv, betas[layer - 1], 1));
            cur[q] = nv;
        }
        for (int e = 0; e < m && rc == OR_OK; ++e) {
            int a = edges[2 * e], b = edges[2 * e + 1];
            int da = dist[a] < 0 ? 1 << 30 : dist[a], db = dist[b] < 0 ? 1 << 30 : dist[b];
            if ((da < db ? da : db) <= p - layer) rc = net_push(net, zz_phase(cur[a], cur[b], gammas[layer - 1], 1));
        }
    }
    for (int q = 0; q < n && rc == OR_OK; ++q)
        if (dist[q] >= 0) rc = net_push(net, vec1(cur[q], r, r));
    free(dist);
    free(cur);
    if (rc != OR_OK) net_free(net);
    return rc;
}

/* Structure of edge `eidx`'s network: variable count, tensor count and the
 * number of variables on each qubit's wire (0 outside the lightcone). */
int oracle_edge_network_shape(int n, int m, const int32_t *edges, int p, int eidx,
                              int *nvars, int *ntens, int *qubit_vars) {
    if (check_graph(n, m, edges) != OR_OK || p < 1 || eidx < 0 || eidx >= m) return OR_EINVAL;
    double *zero = (double *)calloc((size_t)p, sizeof(double));
    network_t net;
    int rc = build_network(n, m, edges, p, zero, zero, eidx, &net);
    free(zero);
    if (rc != OR_OK) return rc;
    *nvars = net.nvars;
    *ntens = net.ntens;
    if (qubit_vars) memcpy(qubit_vars, net.qubit_vars, sizeof(int) * (size_t)n);
    net_free(&net);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Route 3: brute force over all variable assignments                        */
/* ------------------------------------------------------------------------ */

/* value = sum over all 2^V assignments of the product of every tensor entry:
 * the definition of contracting the whole network. */
static cplx contract_brute(const network_t *net) {
    const uint64_t total = (uint64_t)1 << net->nvars;
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (uint64_t a = 0; a < total; ++a) {
        cplx prod = 1.0;
        for (int t = 0; t < net->ntens; ++t) {
            const leaf_t *x = &net->t[t];
            int idx = (int)((a >> x->vars[0]) & 1u);
            if (x->rank == 2) idx |= (int)((a >> x->vars[1]) & 1u) << 1;
            prod *= x->data[idx];
        }
        re += creal(prod);
        im += cimag(prod);
    }
    return re + I * im;
}

int oracle_edge_brute(int n, int m, const int32_t *edges, int p,
                      const double *gammas, const double *betas, int eidx, double *out_re_im) {
    if (check_graph(n, m, edges) != OR_OK || p < 1 || eidx < 0 || eidx >= m) return OR_EINVAL;
    network_t net;
    int rc = build_network(n, m, edges, p, gammas, betas, eidx, &net);
    if (rc != OR_OK) return rc;
    if (net.nvars > 30) { net_free(&net); return OR_ETOOBIG; }
    cplx v = contract_brute(&net);
    out_re_im[0] = creal(v);
    out_re_im[1] = cimag(v);
    net_free(&net);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Route 2: bucket elimination (§II-B)                                       */
/* ------------------------------------------------------------------------ */

static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * Elimination order: repeatedly take a variable of minimum degree in the
 * interaction graph (variables adjacent when they share a tensor), breaking
 * ties at random, join its remaining neighbours into a clique and drop it.
 * The paper leaves its ordering algorithm unspecified (§II-D); every order
 * gives the same value, which is what makes this route a check on the other.
 */
static int min_degree_order(const network_t *net, uint64_t seed, int *order) {
    const int V = net->nvars;
    unsigned char *adj = (unsigned char *)calloc((size_t)V * V, 1);
    int *deg = (int *)calloc((size_t)V, sizeof(int));
    unsigned char *done = (unsigned char *)calloc((size_t)V, 1);
    int *cand = (int *)malloc(sizeof(int) * (size_t)V);
    int *nb = (int *)malloc(sizeof(int) * (size_t)V);
    if (!adj || !deg || !done || !cand || !nb) {
        free(adj); free(deg); free(done); free(cand); free(nb);
        return OR_ENOMEM;
    }
#define ADJ(a, b) adj[(size_t)(a) * V + (b)]
    for (int t = 0; t < net->ntens; ++t) {
        if (net->t[t].rank != 2) continue;
        int a = net->t[t].vars[0], b = net->t[t].vars[1];
        if (a != b && !ADJ(a, b)) {
            ADJ(a, b) = ADJ(b, a) = 1;
            deg[a]++;
            deg[b]++;
        }
    }
    uint64_t rng = seed;
    for (int step = 0; step < V; ++step) {
        int best = 1 << 30, nc = 0;
        for (int v = 0; v < V; ++v) {
            if (done[v]) continue;
            if (deg[v] < best) { best = deg[v]; nc = 0; }
            if (deg[v] == best) cand[nc++] = v;
        }
        int v = cand[splitmix64(&rng) % (uint64_t)nc];
        order[step] = v;
        done[v] = 1;
        int nn = 0;
        for (int a = 0; a < V; ++a)
            if (ADJ(v, a)) nb[nn++] = a;
        for (int i = 0; i < nn; ++i) {
            ADJ(v, nb[i]) = ADJ(nb[i], v) = 0;
            deg[nb[i]]--;
        }
        for (int i = 0; i < nn; ++i)
            for (int j2 = i + 1; j2 < nn; ++j2) {
                int a = nb[i], b = nb[j2];
                if (!ADJ(a, b)) {
                    ADJ(a, b) = ADJ(b, a) = 1;
                    deg[a]++;
                    deg[b]++;
                }
            }
    }
#undef ADJ
    free(adj); free(deg); free(done); free(cand); free(nb);
    return OR_OK;
}

/*
 * Greedy min-fill order (§II-D leaves the ordering heuristic open): at each
 * step eliminate a variable whose neighbours in the interaction graph need
 * the fewest new edges to become a clique; ties are broken at random
 * (splitmix64 seeded by `seed`). Eliminating v joins its neighbours.
 */
static int min_fill_order(const network_t *net, uint64_t seed, int *order) {
    const int V = net->nvars;
    unsigned char *adj = (unsigned char *)calloc((size_t)V * V, 1);
    unsigned char *done = (unsigned char *)calloc((size_t)V, 1);
    int *cand = (int *)malloc(sizeof(int) * (size_t)V);
    int *nb = (int *)malloc(sizeof(int) * (size_t)V);
    if (!adj || !done || !cand || !nb) {
        free(adj); free(done); free(cand); free(nb);
        return OR_ENOMEM;
    }
#define ADJ(a, b) adj[(size_t)(a) * V + (b)]
    for (int t = 0; t < net->ntens; ++t) {
        if (net->t[t].rank != 2) continue;
        int a = net->t[t].vars[0], b = net->t[t].vars[1];
        if (a != b) ADJ(a, b) = ADJ(b, a) = 1;
    }
    uint64_t rng = seed;
    for (int step = 0; step < V; ++step) {
        long best = -1;
        int nc = 0;
        for (int v = 0; v < V; ++v) {
            if (done[v]) continue;
            int nn = 0;
            for (int a = 0; a < V; ++a)
                if (ADJ(v, a)) nb[nn++] = a;
            long fill = 0;
            for (int i = 0; i < nn; ++i)
                for (int j2 = i + 1; j2 < nn; ++j2)
                    if (!ADJ(nb[i], nb[j2])) fill++;
            if (best < 0 || fill < best) { best = fill; nc = 0; }
            if (fill == best) cand[nc++] = v;
        }
        int v = cand[splitmix64(&rng) % (uint64_t)nc];
        order[step] = v;
        done[v] = 1;
        int nn = 0;
        for (int a = 0; a < V; ++a)
            if (ADJ(v, a)) nb[nn++] = a;
        for (int i = 0; i < nn; ++i) ADJ(v, nb[i]) = ADJ(nb[i], v) = 0;
        for (int i = 0; i < nn; ++i)
            for (int j2 = i + 1; j2 < nn; ++j2) ADJ(nb[i], nb[j2]) = ADJ(nb[j2], nb[i]) = 1;
    }
#undef ADJ
    free(adj); free(done); free(cand); free(nb);
    return OR_OK;
}

/* A dense tensor over binary variables: bit i of an entry's index is the
 * value of vars[i]. rank 0 is a scalar. */
typedef struct {
    int rank;
    int *vars;
    cplx *data;
} dense_t;

static void dense_free(dense_t *d) {
    free(d->vars);
    free(d->data);
    d->vars = NULL;
    d->data = NULL;
}

/*
 * Contract one bucket (§II-B): multiply every tensor of the bucket and sum
 * over the bucket variable v. The result's variables are all the others
 * that appear in the bucket; its width is their count plus one.
 * Entries are decoded one by one from the output index, the plain way.
 */
static int contract_bucket(dense_t *ops, int nops, int v, int max_out_rank, dense_t *out) {
    int *ov = (int *)malloc(sizeof(int) * 64);
    if (!ov) return OR_ENOMEM;
    int r = 0;
    for (int t = 0; t < nops; ++t)
        for (int i = 0; i < ops[t].rank; ++i) {
            int x = ops[t].vars[i], seen = (x == v);
            for (int j = 0; j < r && !seen; ++j) seen = (ov[j] == x);
            if (!seen) {
                if (r >= 63 || r >= max_out_rank) { free(ov); return OR_ETOOBIG; }
                ov[r++] = x;
            }
        }
    /* where each operand's index bits come from: -1 for v, else output bit */
    int **src = (int **)malloc(sizeof(int *) * (size_t)nops);
    if (!src) { free(ov); return OR_ENOMEM; }
    for (int t = 0; t < nops; ++t) {
        src[t] = (int *)malloc(sizeof(int) * (size_t)(ops[t].rank + 1));
        for (int i = 0; i < ops[t].rank; ++i) {
            int x = ops[t].vars[i];
            src[t][i] = -1;
            for (int j = 0; j < r; ++j)
                if (ov[j] == x) src[t][i] = j;
        }
    }
    const uint64_t size = (uint64_t)1 << r;
    cplx *res = (cplx *)malloc(sizeof(cplx) * size);
    if (!res) {
        for (int t = 0; t < nops; ++t) free(src[t]);
        free(src); free(ov);
        return OR_ENOMEM;
    }
#pragma omp parallel for schedule(static) if (size >= 4096)
    for (uint64_t o = 0; o < size; ++o) {
        cplx acc = 0.0;
        for (int x = 0; x < 2; ++x) {
            cplx prod = 1.0;
            for (int t = 0; t < nops; ++t) {
                uint64_t idx = 0;
                for (int i = 0; i < ops[t].rank; ++i) {
                    uint64_t bit = src[t][i] < 0 ? (uint64_t)x : (o >> src[t][i]) & 1u;
                    idx |= bit << i;
                }
                prod *= ops[t].data[idx];
            }
            acc += prod;
        }
        res[o] = acc;
    }
    for (int t = 0; t < nops; ++t) free(src[t]);
    free(src);
    out->rank = r;
    out->vars = ov;
    out->data = res;
    return OR_OK;
}

/*
 * Bucket elimination of one network (§II-B): every tensor goes to the bucket
 * of its earliest variable in the order; buckets are contracted in order and
 * each result joins the bucket of its own earliest variable. Scalars multiply
 * into the value. *max_width receives the largest bucket width (the count of
 * distinct variables in a bucket, the summed one included).
 */
static int eliminate(const network_t *net, const int *order, int max_width, cplx *value, int *max_w) {
    const int V = net->nvars;
    int *pos = (int *)malloc(sizeof(int) * (size_t)V);
    /* bucket lists as linked lists over a growing tensor pool */
    int cap = net->ntens + V + 8;
    dense_t *pool = (dense_t *)calloc((size_t)cap, sizeof(dense_t));
    int *next = (int *)malloc(sizeof(int) * (size_t)cap);
    int *head = (int *)malloc(sizeof(int) * (size_t)V);
    if (!pos || !pool || !next || !head) { free(pos); free(pool); free(next); free(head); return OR_ENOMEM; }
    for (int i = 0; i < V; ++i) { pos[order[i]] = i; head[i] = -1; }
    int np = 0, rc = OR_OK;
    cplx result = 1.0;
    *max_w = 0;

    for (int t = 0; t < net->ntens; ++t) {
        const leaf_t *x = &net->t[t];
        dense_t d;
        d.rank = x->rank;
        d.vars = (int *)malloc(sizeof(int) * 2);
        d.data = (cplx *)malloc(sizeof(cplx) * 4);
        d.vars[0] = x->vars[0];
        d.vars[1] = x->vars[1];
        for (int i = 0; i < 4; ++i) d.data[i] = x->data[i];
        int first = d.vars[0];
        if (d.rank == 2 && pos[d.vars[1]] < pos[first]) first = d.vars[1];
        pool[np] = d;
        next[np] = head[first];
        head[first] = np;
        np++;
    }
    for (int step = 0; step < V && rc == OR_OK; ++step) {
        int v = order[step];
        int nops = 0;
        for (int i = head[v]; i >= 0; i = next[i]) nops++;
        if (nops == 0) continue;
        dense_t *ops = (dense_t *)malloc(sizeof(dense_t) * (size_t)nops);
        int k = 0;
        for (int i = head[v]; i >= 0; i = next[i]) ops[k++] = pool[i];
        dense_t res;
        rc = contract_bucket(ops, nops, v, max_width - 1, &res);
        for (int i = 0; i < nops; ++i) dense_free(&ops[i]);
        free(ops);
        head[v] = -1;
        if (rc != OR_OK) break;
        if (res.rank + 1 > *max_w) *max_w = res.rank + 1;
        if (res.rank == 0) {
            result *= res.data[0];
            dense_free(&res);
            continue;
        }
        int first = res.vars[0];
        for (int i = 1; i < res.rank; ++i)
            if (pos[res.vars[i]] < pos[first]) first = res.vars[i];
        if (np == cap) {
            cap *= 2;
            pool = (dense_t *)realloc(pool, sizeof(dense_t) * (size_t)cap);
            next = (int *)realloc(next, sizeof(int) * (size_t)cap);
        }
        pool[np] = res;
        next[np] = head[first];
        head[first] = np;
        np++;
    }
    for (int i = 0; i < V; ++i)
        for (int j = head[i]; j >= 0; j = next[j]) dense_free(&pool[j]);
    free(pos); free(pool); free(next); free(head);
    *value = result;
    return rc;
}

/* The value of edge `eidx`'s network by bucket elimination under the
 * min-degree order drawn with `seed`; width limit `max_width` (inclusive). */
int oracle_edge_bucket(int n, int m, const int32_t *edges, int p, const double *gammas,
                       const double *betas, int eidx, uint64_t seed, int max_width,
                       double *out_re_im, int *max_w) {
    if (check_graph(n, m, edges) != OR_OK || p < 1 || eidx < 0 || eidx >= m) return OR_EINVAL;
    network_t net;
    int rc = build_network(n, m, edges, p, gammas, betas, eidx, &net);
    if (rc != OR_OK) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)net.nvars);
    rc = order ? min_degree_order(&net, seed, order) : OR_ENOMEM;
    cplx v = 0.0;
    int w = 0;
    if (rc == OR_OK) rc = eliminate(&net, order, max_width, &v, &w);
    free(order);
    net_free(&net);
    if (rc != OR_OK) return rc;
    out_re_im[0] = creal(v);
    out_re_im[1] = cimag(v);
    if (max_w) *max_w = w;
    return OR_OK;
}

/* As oracle_edge_bucket, with the order chosen by `order_kind`: 0 min-degree,
 * 1 greedy min-fill (both with random ties drawn from `seed`). */
int oracle_edge_bucket_order(int n, int m, const int32_t *edges, int p, const double *gammas,
                             const double *betas, int eidx, int order_kind, uint64_t seed, int max_width,
                             double *out_re_im, int *max_w) {
    if (check_graph(n, m, edges) != OR_OK || p < 1 || eidx < 0 || eidx >= m) return OR_EINVAL;
    if (order_kind != 0 && order_kind != 1) return OR_EINVAL;
    network_t net;
    int rc = build_network(n, m, edges, p, gammas, betas, eidx, &net);
    if (rc != OR_OK) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)net.nvars);
    if (!order) rc = OR_ENOMEM;
    else rc = order_kind == 1 ? min_fill_order(&net, seed, order) : min_degree_order(&net, seed, order);
    cplx v = 0.0;
    int w = 0;
    if (rc == OR_OK) rc = eliminate(&net, order, max_width, &v, &w);
    free(order);
    net_free(&net);
    if (rc != OR_OK) return rc;
    out_re_im[0] = creal(v);
    out_re_im[1] = cimag(v);
    if (max_w) *max_w = w;
    return OR_OK;
}

/* Every edge's value by bucket elimination; zz_re_im holds (re, im) pairs. */
int oracle_bucket_zz(int n, int m, const int32_t *edges, int p, const double *gammas,
                     const double *betas, uint64_t seed, int max_width, double *zz_re_im,
                     int *max_w) {
    int wmax = 0;
    for (int e = 0; e < m; ++e) {
        int w = 0;
        int rc = oracle_edge_bucket(n, m, edges, p, gammas, betas, e, seed + (uint64_t)e, max_width,
                                    zz_re_im + 2 * e, &w);
        if (rc != OR_OK) return rc;
        if (w > wmax) wmax = w;
    }
    if (max_w) *max_w = wmax;
    return OR_OK;
}
