/*
 * qt.h -- C ABI of libqtgb: QAOA MaxCut energy by lightcone bucket elimination
 * on one GB300 (sm_103a).
 *
 * What is computed (paper §II-A and §II-B):
 *   C = 1/2 sum_{(ij) in E} (1 - Z_i Z_j)                              (Eq. 1)
 *   |g,b>_p = prod_{k=1..p} e^{-i b_k B} e^{-i g_k C} |+>^N,  B = sum X   (Eq. 2)
 *   <C>_p = |E|/2 - 1/2 sum_{jk in E} e_jk,  e_jk = <g,b| Z_j Z_k |g,b>
 * Each e_jk is the value of the tensor network of edge jk's lightcone,
 * contracted by bucket elimination (§II-B): buckets are taken in elimination
 * order; a bucket's tensors are multiplied and summed over the bucket index,
 * and the result joins a later bucket.
 *
 * Angle convention: layer k applies exp(-i gamma_k s_a s_b) on each edge (a,b)
 * with s(x) = 1 - 2x, then exp(-i beta_k X) on each qubit. The paper's Eq. 2
 * corresponds to gamma_paper = -2 * gamma (a global phase aside).
 *
 * Conventions for every call:
 *  - Return 0 (QT_OK) or a negative QT_E* code; qt_error_string() names it.
 *    No output is written on error, and no C++ exception crosses the ABI.
 *  - Graphs are simple and undirected, vertices 0..n-1, edges given as
 *    int32 pairs. Edge outputs follow the input edge order.
 *  - The caller owns every array it passes. Pointers marked "host or device"
 *    are classified with cudaPointerGetAttributes; device pointers must be on
 *    the plan's device.
 *  - Calls with `stream == NULL` are synchronous. With a stream, device
 *    outputs are valid once the stream has synchronised; host outputs are
 *    always valid on return (the call waits for its own copies).
 *  - A plan is used by one call at a time (per plan, not per process).
 */
#ifndef QT_H
#define QT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define QT_OK 0
#define QT_EINVAL -1   /* bad argument: null pointer, self-loop, duplicate edge, vertex out of range, p < 1
                          (a graph without edges is valid: no networks, energy 0) */
#define QT_EWIDTH -2   /* a bucket is wider than qt_plan_opts.max_width, or has more than 16 operands */
#define QT_ENOMEM -3   /* host or device allocation failed, or over qt_plan_opts.arena_bytes */
#define QT_ECUDA -4    /* a CUDA runtime call failed (no device, launch failure, ...) */
#define QT_ETIMEOUT -5 /* a kernel's bounded wait on a bucket dependency ran out */
#define QT_EBOUNDS -6  /* a kernel found an operand index outside its tensor */
#define QT_ESTATE -7   /* call not valid for this plan (wrong dtype/mode, gradient not planned, ...) */

typedef struct qt_plan_s *qt_plan_t; /* opaque; owns the host plan and its device memory */

typedef enum { QT_C64 = 0, QT_C128 = 1 } qt_dtype;

/* How qt_energy runs the bucket schedule. */
typedef enum {
    QT_SCHED_PERSISTENT = 0, /* one persistent kernel drains a device-side dependency
                                queue of bucket tiles; captured in a CUDA graph */
    QT_SCHED_PER_BUCKET = 1  /* the plain form: one kernel launch per bucket, in order */
} qt_sched;

/* Plan options. A zero-initialised struct selects every default. */
typedef struct {
    qt_dtype dtype;        /* element type of every tensor: complex64 (FP32 arithmetic) or complex128 */
    qt_sched sched;        /* schedule used by qt_energy (default persistent) */
    int32_t order_restarts;/* extra randomised greedy min-fill orders per network; the order
                              with the smallest sum of 2^width is kept. 0 (default): 64 restarts for
                              the networks whose plain greedy order reaches width 18, none for the
                              others; > 0: that many for every network; negative: none (the plain
                              greedy order) */
    uint64_t order_seed;   /* seed of the randomised restarts */
    int32_t max_width;     /* largest bucket width allowed, the summed index included
                              (default 31, at most 31) */
    size_t arena_bytes;    /* cap on device memory for tensors (default: no cap beyond the device) */
    int32_t with_grad;     /* nonzero: also allocate what qt_energy_grad needs */
    uint64_t spin_limit;   /* polls of a dependency counter before a kernel gives up with
                              QT_ETIMEOUT (default 2^23, each poll sleeps ~0.1-1 us) */
    int32_t chunk_log2;    /* most outputs per tile, log2 (default 0: 9, i.e. 512 outputs); smaller
                              when a bucket's operand footprints do not fit the 8 KB stage */
    int32_t host_only;     /* nonzero: plan on the host only (statistics, export); no device
                              memory is touched and every evaluation call returns QT_ESTATE */
    int32_t run_tiles;     /* most tiles of one bucket handed out per claim (default 0: 12) */
    int32_t trace;         /* nonzero: run the instrumented persistent kernel, which counts
                              per-warp cycles by phase (read with qt_trace_counters) */
    int32_t order;         /* claim order of the persistent kernel: 0 (default) the order of a
                              critical-path list-scheduling simulation made at plan time, each
                              group starting once its producers are done; 1 a device-side ready
                              queue, first come first served */
    int32_t no_fuse;       /* nonzero: no fused units (by default, subtrees of small buckets, at most
                              256 outputs each, run as one work group contracted in a warp's shared
                              memory; never for gradient plans or the per-bucket schedule) */
    int32_t autotune;      /* > 0: autotune the tile shapes at plan time (persistent schedule, device
                              plans): per bucket-width class (output bits <= 6, 7..10, 11..14, 15..19,
                              >= 20) the most tile bits, then the group size, each candidate timed on
                              the device over `autotune` evaluations; the choice is in qt_plan_stats */
    int8_t tile_cap[8];    /* most tile bits (log2 outputs per tile, 1..11) per width class, 0: default
                              (chunk_log2, else 9); the first 5 entries are used */
    int32_t no_merge;      /* merged eliminations: a bucket of 2^10 outputs or more and the consumer
                              that only extends it become one bucket summing both variables, the
                              intermediate never written. 0 (default): energy plans of the persistent
                              schedule merge, gradient plans do not (their reverse sweep ran slower);
                              negative: gradient plans merge too; positive: no plan merges. The
                              per-bucket schedule never merges */
    size_t adjoint_budget_bytes; /* gradient plans (single graph): device bytes for results and their
                              cotangents; a plan that needs more runs in passes that fit, over its
                              networks' slices (each pass saves its own results and seeds each slice
                              from its own factors; energies and gradients are summed over passes); a
                              slice that alone exceeds it gives QT_ENOMEM. 0: no budget */
    int32_t slice_width;   /* index slicing: a network whose greedy order is wider than this target
                              gets variables fixed, one at a time, until it is not (or max_slice_bits
                              are fixed); its value is the sum over the 2^s assignments of the fixed
                              variables of networks without them, all contracted in the same launch.
                              2..31: the target; 0: the default target (22 complex64, 20 complex128);
                              -1: no slicing. Gradient plans too: each slice's root cotangents are the
                              products of its other factors, and a gate entry fixed by slicing adds its
                              own derivative term */
    int32_t max_slice_bits;/* most variables fixed per network (1..16); 0: 8 */
    int32_t dedup;         /* nonzero: lightcone deduplication. Within each graph, networks whose
                              lightcones are isomorphic (the qubits within distance p of the edge,
                              labelled by distance) are contracted once: the others take that
                              network's value; in gradient plans the reverse sweep seeds it once for
                              its whole class. A budget (energy_budget_bytes, or
                              adjoint_budget_bytes with gradients) that the deduplicated plan fits
                              keeps it; one it exceeds runs every network in passes, without
                              deduplication. A shard deduplicates the networks it holds whole.
                              0: every network is contracted */
    size_t energy_budget_bytes; /* energy plans (single graph): device bytes for the gate tables and
                              results; a plan that needs more runs in passes that fit, over the
                              networks' slices (opts.slice_width), on one shared arena; per-edge values
                              and the energy are summed over passes; a slice that alone exceeds it
                              gives QT_ENOMEM. 0: no budget */
} qt_plan_opts;

/* Plan statistics. Widths count the summed index (inclusive); a bucket of
 * width w writes 2^(w-1) entries. */
typedef struct {
    int32_t n_graphs;
    int32_t n_networks;     /* one per edge of every graph */
    int64_t n_buckets;
    int64_t n_operands;
    int32_t max_width;
    int32_t p;
    double sum_2w;          /* sum over buckets of 2^width */
    double alg_bytes;       /* algorithmic bytes of one energy evaluation: every operand read
                               once plus every output written once, at the plan's dtype */
    double flops;           /* complex multiply-adds of one evaluation x 8 real flops */
    int64_t arena_bytes;    /* device bytes of the tensor arena */
    int64_t n_tasks;        /* output tiles over all buckets */
    int64_t n_items;        /* persistent-kernel work groups (ready-queue entries, one claim each) */
    int32_t n_levels;       /* longest dependency chain, in buckets */
    int32_t dtype;
    int64_t width_hist[64]; /* buckets per width */
    double plan_seconds;    /* host time spent building the plan */
    double sim_seconds;     /* makespan predicted by the plan-time schedule simulation (0: none) */
    int64_t n_units;        /* fused units (small subtrees run as one work group) */
    int64_t n_fused;        /* buckets inside fused units, their roots included */
    int32_t tile_cap[8];    /* most tile bits per width class in effect (5 used) */
    int32_t run_tiles;      /* most tiles per work group in effect */
    double tune_seconds;    /* host time spent autotuning (0 without opts.autotune) */
    int32_t tune_candidates;/* configurations the autotuner laid out and timed */
    int32_t n_passes;       /* plans over opts.adjoint_budget_bytes (gradients, passes over networks) or
                               opts.energy_budget_bytes (energies, passes over slices); 1 otherwise */
    int32_t slice_bits;     /* most variables fixed in any one network (opts.slice_width) */
    int64_t n_slices;       /* slices over all networks (1 per network without slicing) */
    int64_t n_unique;       /* networks contracted (opts.dedup: the others share their values) */
    int64_t pass_arena_bytes; /* plans in passes: device bytes of the arena the passes share (the
                               largest pass); 0 otherwise */
} qt_plan_stats;

/* One bucket of the schedule as seen by host-side inspection (tests). */
typedef struct {
    int32_t network;   /* network (edge) it belongs to, numbered over all graphs */
    int32_t width;     /* inclusive width w */
    int32_t n_ops;     /* operands (leaf gate tensors and earlier results) */
    int32_t op_begin;  /* first operand in the qt_operand_info array */
    int32_t parent;    /* bucket that consumes this bucket's result; -1 for a root (scalar) */
    int32_t n_deps;    /* operands that are results of earlier buckets */
    int32_t level;     /* 0 for buckets whose operands are all leaves */
    int32_t var;       /* the summed variable, numbered within the network */
    int32_t tile_log2; /* log2 of the outputs per tile of the persistent kernel (a merged bucket's
                          tiles run over (o, s1), s1 lowest: 2^(tile_log2 - n_sum + 1) results) */
    uint32_t tile_bits;/* the output bits that vary within a tile (popcount = tile_log2): the
                          lowest ones, so tile c holds outputs c * 2^tile_log2 + j */
    uint32_t folded;   /* operands (bit i: the bucket's i-th) folded into the per-tile gate table */
    uint32_t unit_role;/* 0: scheduled on its own; 1: inside a fused unit; 2: the root of a fused unit */
    int32_t n_sum;     /* summed variables (more than 1: merged eliminations); outputs 2^(width - n_sum) */
    int32_t var2;      /* a merged bucket's second summed variable (its consumer's), else -1 */
    int32_t var3;      /* a third summed variable (the consumer's consumer's), else -1; merges take
                          two variables per bucket, so -1 */
    int32_t slice;     /* the slice of its network the bucket belongs to (0 without slicing); in a
                          sliced network, variables are numbered after removing the fixed ones */
} qt_bucket_info;

/* One operand of a bucket. With one summed variable (smask = 1) the operand's
 * entry for output index o and summed value x is at element 2*pext(o, mask) + x. */
typedef struct {
    int32_t src;       /* producing bucket, or -1 for a leaf gate tensor */
    int32_t leaf_kind; /* for leaves: QT_LEAF_* below, else -1 */
    int32_t leaf_layer;/* for ZZ and mixer leaves: layer 0..p-1, else -1 */
    uint32_t mask;     /* output bits this operand carries */
    int32_t rank;      /* index bits of the operand (summed bits included) */
    uint32_t smask;    /* summed variables it carries; its entry for output o and summed values s is
                          2^popc(smask) * pext(o, mask) + pext(s, smask) */
    int32_t leaf_sub;  /* leaves: element offset into the gate tensor's entries: 2 * (fixed value)
                          for a gate with one variable fixed by slicing (entries for the free
                          variable x at leaf_sub + x), else 0 */
    int32_t pad;
} qt_operand_info;

/* A gate tensor of a sliced network whose variables are all fixed: in slice
 * `slice` of `network` the network's value is multiplied by entry `entry` of
 * the gate (QT_LEAF_* kind, layer as in qt_operand_info). */
typedef struct {
    int32_t network;
    int32_t slice;
    int32_t leaf_kind;
    int32_t leaf_layer;
    int32_t entry;
    int32_t pad;
} qt_fixed_info;

/* The arrays the device kernels read (host-side inspection and tests): per
 * bucket its result's arena offset, operands, tile outputs (n_out; a merged
 * bucket's outputs are (o, s1) with s1 as bit 0) and summed variables; per
 * operand its arena offset (a gate's slot plus any slice offset, or the
 * producer's result), its mask over the bucket's tile outputs, whether its
 * entries pair over the bucket's first summed variable (then entry
 * 2 * pext(o, mask) + x, else pext(o, mask)), and whether it is a gate; the
 * epilogue's factor lists (arena offsets, bit 63 on each slice's first factor;
 * per network factors [net_first_factor[i], net_first_factor[i + 1])) and per
 * graph the networks whose 1/2 the energy counts. Arena layout: per graph
 * 2 + 4p gate tensors of 4 entries from element 0 (|+>, Z, then per layer ZZ,
 * ZZ*, mixer, mixer*), entry x + 2y. Any pointer may be NULL; *n_factors
 * receives the factor count (call once with factor NULL to size it). */
typedef struct {
    uint64_t out_off;
    int32_t op_begin;
    int32_t n_ops;
    int32_t n_out;
    int32_t n_sum;
} qt_dev_bucket;

typedef struct {
    uint64_t off;
    uint32_t mask;
    int32_t pairs_x;
    int32_t leaf;
    int32_t pad;
} qt_dev_operand;

int qt_plan_export_device(qt_plan_t plan, qt_dev_bucket *buckets, qt_dev_operand *operands,
                          uint32_t *net_first_factor, uint64_t *factor, int32_t *graph_owned,
                          int64_t *n_factors);

/* Pass k (0 <= k < qt_plan_stats.n_passes) of a plan that runs in passes,
 * for host-side inspection: *pass is a handle owned by `plan` (valid while
 * it lives; do not free it), pass_edges (may be NULL, else n_edges int32 of
 * room) receives the graph edges of the pass's networks in its order, and
 * *n_edges their count. QT_ESTATE for a plan without passes. */
int qt_plan_pass(qt_plan_t plan, int32_t k, qt_plan_t *pass, int32_t *pass_edges, int32_t *n_edges);

/* Lightcone deduplication (host-side inspection): rep[i] = the network whose
 * value network i takes (i itself when it is contracted); n_networks int32. */
int qt_plan_export_reps(qt_plan_t plan, int32_t *rep);

/* The fixed gate entries of every slice (host-side inspection). `out` holds
 * at least *n_out entries on entry, or is NULL to ask for the count; *n_out
 * receives the count. */
int qt_plan_export_fixed(qt_plan_t plan, qt_fixed_info *out, int64_t *n_out);

#define QT_LEAF_PLUS 0   /* [1, 1]/sqrt 2: |+> and <+| */
#define QT_LEAF_ZOBS 1   /* [1, -1]: the observable Z on an edge endpoint */
#define QT_LEAF_ZZ 2     /* exp(-i gamma_k s_a s_b) */
#define QT_LEAF_ZZ_CONJ 3
#define QT_LEAF_RX 4     /* <new| exp(-i beta_k X) |old> */
#define QT_LEAF_RX_CONJ 5

/*
 * Build the plan for one graph (§II-B): each edge's lightcone network with the
 * ZZ-phase gates as rank-2 diagonal tensors, a greedy min-fill elimination
 * order, the bucket schedule with every tensor's index bits sorted by
 * elimination rank, and the device memory for it. Host-side work, then one
 * upload. `edges`: host, 2*n_edges int32. `opts` may be NULL. On success
 * *out owns device memory until qt_plan_free.
 */
int qt_plan(int32_t n_vertices, int32_t n_edges, const int32_t *edges, int32_t p,
            const qt_plan_opts *opts, qt_plan_t *out);

/*
 * A plan for the networks of selected edges only: `sel` (host, n_sel indices
 * into `edges`, any order, no repeats needed) picks the lightcones to plan.
 * qt_energy then reports edge_zz in selection order and, as energy, the
 * selected edges' share of <C>: n_sel/2 - 1/2 sum_sel e_jk. The lightcones
 * still see the whole graph.
 */
int qt_plan_subset(int32_t n_vertices, int32_t n_edges, const int32_t *edges, int32_t p, int32_t n_sel,
                   const int32_t *sel, const qt_plan_opts *opts, qt_plan_t *out);

/*
 * One plan over several graphs, evaluated together by qt_energy_batch.
 * n_vertices[g], n_edges[g] per graph; `edges` holds every graph's pairs back
 * to back (host). All graphs share p; each gets its own angles.
 */
int qt_plan_batch(int32_t n_graphs, const int32_t *n_vertices, const int32_t *n_edges,
                  const int32_t *edges, int32_t p, const qt_plan_opts *opts, qt_plan_t *out);

/* Statistics of a plan (host only). */
/*
 * One rank's share of a graph's lightcone networks, for splitting one energy
 * over `world` processes (one GPU each). Every network is planned on the host
 * for its cost (sum over its buckets of 2^width); the units are the networks'
 * slices (opts.slice_width; one per unsliced network), each costing its
 * slice's sum, and go to ranks by longest-processing-time-first (the
 * costliest unit to the least loaded rank). The plan holds the units of rank
 * `rank`: its qt_energy gives, per edge of the shard, the sum of e_jk over the
 * rank's slices of that edge's network (the whole e_jk when the rank holds
 * them all), and the partial energy: the rank holding a network's slice 0
 * counts the edge's 1/2, every rank subtracts 1/2 of its partial e_jk. The
 * full e_jk, E and gradient are sums over ranks (one reduction of 2p + 1
 * doubles for E and the gradient; gradient plans are never sliced).
 * shard_edges (may be NULL, else n_edges int32 of room) receives the rank's
 * edges in increasing order, *n_shard their count. A rank with no unit gets
 * a plan of no networks (energy 0). Options as for qt_plan.
 */
int qt_plan_shard(int32_t n_vertices, int32_t n_edges, const int32_t *edges, int32_t p, int32_t world,
                  int32_t rank, const qt_plan_opts *opts, qt_plan_t *out, int32_t *shard_edges,
                  int32_t *n_shard);

int qt_plan_stats_get(qt_plan_t plan, qt_plan_stats *out);

/* Copy the schedule out for inspection (host only). `buckets` holds
 * stats.n_buckets entries, `operands` stats.n_operands; either may be NULL. */
int qt_plan_export(qt_plan_t plan, qt_bucket_info *buckets, qt_operand_info *operands);

/* Number of variables on each qubit wire of network `network` (host,
 * n_vertices of its graph entries; 0 for qubits outside the lightcone). */
int qt_plan_network_wires(qt_plan_t plan, int32_t network, int32_t *vars_per_qubit);

/* One work group of the persistent kernel's queue, as seen by host-side
 * inspection (tests): tiles [first_tile, first_tile + n_tiles) of `bucket`,
 * or, when unit_buckets > 0, a fused unit of that many buckets rooted at
 * `bucket` (n_tiles 1). */
typedef struct {
    int32_t bucket;
    int32_t first_tile;
    int32_t n_tiles;
    int32_t unit_buckets;
} qt_group_info;

/* The static part of the queue in claim order (qt_plan_stats.n_items groups
 * with the default order; with the ready-queue order, only the groups of
 * buckets without producers, the rest being published at run time). `groups`
 * holds at least n_items entries; *n_out receives the count. */
int qt_plan_export_groups(qt_plan_t plan, qt_group_info *groups, int64_t *n_out);

/* A fused unit (host-side inspection, tests): the subtree of n_buckets buckets
 * rooted at `root`, whose program starts at record first_rec of the plan's
 * unit program. */
typedef struct {
    int32_t root;
    int32_t n_buckets;
    int64_t first_rec;
} qt_unit_info;

/* One record of the unit program, as the kernel reads it. A program is a
 * sequence of steps; a step is either one bucket over the whole warp -- a
 * header (a = n_out | n_ops << 8 | 1 << 16 for the unit's root; b = the
 * result's element offset in the warp's shared-memory scratch, unused for the
 * root, whose result goes to its arena offset) followed by its operand records
 * -- or several independent buckets run at once, one output per lane: a step
 * record (a = records of the step | 1 << 18 | items << 20 | lanes used << 24;
 * b = offsets of items 1..3 from the step record, 8 bits each; off = each
 * lane's item, 2 bits per lane), then each item's header (off = its first lane)
 * and operand records. Operand record: a = the operand's mask over the
 * bucket's outputs (its entry for output o and summed value x is 2 pext(o, a)
 * + x); b bit 0 = 1 for a result held in scratch (off = its scratch offset), 0
 * for a gate tensor (off = its arena offset); b bit 1 = 1 when the mask is one
 * run of bits, starting at bit b >> 8. */
typedef struct {
    uint32_t a;
    uint32_t b;
    uint64_t off;
} qt_unit_rec;

/* The fused units of a plan and their programs (0 of each without units).
 * With units/recs NULL only the counts are written; otherwise the arrays hold
 * at least *n_units and *n_recs entries (as returned by a first call). */
int qt_plan_export_units(qt_plan_t plan, qt_unit_info *units, qt_unit_rec *recs, int64_t *n_units,
                         int64_t *n_recs);

/*
 * Energy of a single-graph plan: edge_zz[e] = e_jk of edge e (n_edges doubles,
 * host or device, may be NULL), *energy = |E|/2 - 1/2 sum e_jk (host or
 * device, may be NULL). gammas/betas: p doubles each, host or device.
 * Per-edge values are the real part of each network's value, accumulated to
 * double at the end; the arithmetic inside runs in the plan's dtype.
 */
int qt_energy(qt_plan_t plan, const double *gammas, const double *betas, double *edge_zz,
              double *energy, void *cuda_stream);

/*
 * Energies of every graph of a batch plan in one pass: gammas/betas hold
 * n_graphs*p doubles (graph-major), energies n_graphs doubles, edge_zz the
 * per-edge values of all graphs back to back (may be NULL).
 */
int qt_energy_batch(qt_plan_t plan, const double *gammas, const double *betas, double *energies,
                    double *edge_zz, void *cuda_stream);

/*
 * Energy and its gradient dE/dgamma_k, dE/dbeta_k (k = 1..p) by the adjoint
 * of the bucket elimination: a reverse sweep over the saved results. The plan
 * must have been built with opts.with_grad. For batch plans the outputs are
 * per graph (n_graphs, n_graphs*p, n_graphs*p). Host or device pointers.
 */
int qt_energy_grad(qt_plan_t plan, const double *gammas, const double *betas, double *energy,
                   double *dE_dgamma, double *dE_dbeta, void *cuda_stream);

/* Imaginary parts of the per-edge network values from the last evaluation
 * (host, n_edges doubles): a consistency check, zero up to rounding. */
int qt_last_imag(qt_plan_t plan, double *edge_imag);

/* Wait for the plan's work on `cuda_stream` and report a kernel-side error
 * (QT_ETIMEOUT, QT_EBOUNDS) raised since the previous check. */
int qt_sync(qt_plan_t plan, void *cuda_stream);

/* Average device time per launch of the plan's main kernel over the calls made
 * since the last reset, measured with CUDA events on the launch stream.
 * *launches receives the count. reset != 0 clears the counters. */
int qt_kernel_time(qt_plan_t plan, double *avg_ms, int64_t *launches, int32_t reset);

/*
 * Time the persistent kernel on the tiles of one bucket alone (no other bucket
 * runs, no consumer is notified). The tiles form work groups of at most the
 * plan's group size, spread evenly over every warp of the grid in whole
 * rounds (as a bucket that has the GPU to itself is scheduled). `reps` launches back to back after one
 * warm-up launch, on the plan's own stream, each preceded by a reset of the
 * kernel's 256-byte control word; CUDA events around the whole sequence, so
 * the host's launch latency overlaps the previous launch. *avg_ms receives the
 * mean per launch (the resets included), *bytes (may be NULL) the bucket's
 * algorithmic bytes (every operand read once, the result written once). The operands hold whatever the last
 * evaluation left (run qt_energy first for meaningful data; the timing does
 * not depend on the values). Persistent plans only; host call, synchronous.
 */
int qt_bucket_time(qt_plan_t plan, int64_t bucket, int32_t reps, double *avg_ms, double *bytes);

/* Phase counters of the last persistent run of a plan built with opts.trace,
 * summed over warps: totals[0..6] = cycles spent claiming work (and the
 * kernel's tail), reading run descriptors, checking and waiting for producers,
 * starting bulk copies, waiting for copies to land, contracting tiles, and
 * publishing finished runs; totals[7] = tiles, totals[8] = runs, totals[9] =
 * cycles spent building the folded gate tables. *n_warps receives the number of warps launched. Host call; waits
 * for the plan's work to finish. QT_ESTATE if the plan was built without trace. */
int qt_trace_counters(qt_plan_t plan, uint64_t *totals, int64_t *n_warps);

/* Per-bucket timeline of the last persistent run of a traced plan:
 * start_end_ns[2b] = %globaltimer (ns) when the first group of bucket b was
 * taken up, start_end_ns[2b+1] = when its last group finished. Host, 2 *
 * n_buckets entries; waits for the plan's work. QT_ESTATE without opts.trace. */
int qt_trace_bucket_times(qt_plan_t plan, uint64_t *start_end_ns);

/* Fault injection for tests: on the device, raise the number of output tiles
 * bucket `bucket` must complete by one, so the bucket consuming its result can
 * never start. The next persistent run must end with QT_ETIMEOUT (its bounded
 * wait runs out) rather than wait forever. Use a plan that is then freed. */
int qt_debug_stall_bucket(qt_plan_t plan, int64_t bucket);

/*
 * Energy without any device allocation. The paper has no counterpart: this
 * entry point serves callers that must not allocate device memory during the
 * call, e.g. code running inside a custom allocator or memory pool, or a host
 * that fixes its device-memory footprint at start-up and forbids cudaMalloc
 * afterwards. qt_energy's plans own device memory made by qt_plan; this call
 * instead runs the same persistent kernel with all of its device memory (plan
 * arrays, counters, queue, gate tables and intermediate results) inside one
 * static device array of QT_NOALLOC_SCRATCH_BYTES, built into the library.
 *
 *  - plan: any plan, typically one made with opts.host_only = 1 (no device
 *    memory at all). Single-graph or batch plans; the plan's dtype is used, its
 *    schedule option is not (the persistent kernel always runs).
 *  - gammas/betas: n_graphs*p doubles each (graph-major), host or device.
 *  - energies: n_graphs doubles, edge_zz: the per-edge values of every graph
 *    back to back; host or device, either may be NULL. Written only on success.
 *  - cuda_stream: the work is queued there (NULL: the default stream); the call
 *    waits for it to finish before returning, so it is synchronous.
 * Returns QT_ENOMEM (with qt_last_error_detail() naming both sizes) if the plan
 * needs more than QT_NOALLOC_SCRATCH_BYTES, checked before any CUDA call, and
 * QT_ETIMEOUT / QT_EBOUNDS as qt_energy does. It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 * Set-up: the first call on each device (with that device current) looks up
 * the array's device address with cudaGetSymbolAddress and sets the kernel's
 * shared-memory attribute; make that first call before any stream capture.
 * From then on the array stays resident on every device that made a call,
 * until the process exits.
 * Every call, from every thread and plan, shares the one array and leaves its
 * contents behind; each call resets what must start at zero. Calls whose GPU
 * work overlaps (concurrent host threads, or different streams) race on the
 * array and give wrong results: serialise them.
 */
#define QT_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20) /* 64 MiB of device memory */
int qt_energy_noalloc(qt_plan_t plan, const double *gammas, const double *betas, double *energies,
                      double *edge_zz, void *cuda_stream);

/*
 * Measured FMA throughput of the current device's CUDA cores, in TFLOP/s
 * (an FMA counts 2 flops): FP32 for QT_C64, FP64 for QT_C128. Independent
 * FMA chains on every SM, timed with CUDA events after a warm-up launch; a
 * few milliseconds of GPU time. This is the arithmetic roofline of the
 * contraction kernels (the paper has no counterpart: it reports flops
 * against its V100's datasheet peak, §III-C). Allocates and frees a small
 * buffer; synchronous.
 */
int qt_fma_peak(int32_t dtype, double *tflops);

void qt_plan_free(qt_plan_t plan);

/* ---- contraction of caller tensors over binary indices ---------------------
 * The paper's "tncontract" benchmark expression (§II-E, synthetic datasets;
 * Table III "Tensor Network Random Contraction"): tensors whose every index
 * has size 2, contracted as
 *     out[K] = sum over the labels not in K of  prod_t  T_t[L_t]
 * (the labels not in the output are summed). It runs on the bucket
 * elimination of the energy plans (§II-B; merged eliminations, §II-C): the
 * summed labels are eliminated first, each bucket's label bit 0 of its
 * operands, and the output's labels take the next elimination ranks in the
 * output's bit order, so the last bucket writes the output. */
typedef struct qt_contract_s *qt_contract_t;  /* opaque; owns its device memory */

typedef struct {
    int32_t n_buckets;   /* buckets of the elimination (merged ones counted once) */
    int32_t max_width;   /* widest bucket, its summed labels included */
    int32_t n_summed;    /* labels summed */
    int32_t n_merged;    /* buckets that sum two labels */
    double alg_bytes;    /* bytes of the buckets: every operand read once, every result written once */
    double copy_bytes;   /* bytes of the copies: each input read and written in the arena's layout, the
                            result read and the output written */
    int64_t arena_bytes; /* device memory the plan holds for tensors */
    int32_t widths[32];  /* the first 32 buckets' widths */
} qt_contract_stats;

/* Plan a contraction. n_ops operands (1..16); operand t has ranks[t] labels
 * (1..30), listed consecutively in `labels` (host) in C order: its first label
 * is its slowest axis, its last label bit 0 of its flat index. Labels are
 * non-negative ints, distinct within an operand; equal labels in two operands
 * are the same index. `out_labels` (host, out_rank of them, may be 0 for a
 * scalar) lists the output's labels in C order; each must occur in an operand.
 * Every operand must hold at least one summed label (an operand of output
 * labels only would need an outer product), and the buckets must end in one
 * result: QT_EINVAL otherwise. At most 30 distinct labels; QT_EWIDTH if a
 * bucket has more than 16 operands or no tile of it fits the kernel's
 * shared-memory stage. host_only != 0: no device memory (stats only). Device
 * memory: the arena (every operand permuted, every result) plus small tables;
 * the plan is bound to the current device. */
int qt_contract_plan(int32_t n_ops, const int32_t *ranks, const int32_t *labels, int32_t out_rank,
                     const int32_t *out_labels, qt_dtype dtype, int32_t host_only, qt_contract_t *out);

/* Run a planned contraction. ops[t]: device pointer to operand t, 2^ranks[t]
 * elements of the plan's dtype as interleaved (re, im) pairs -- the layout of
 * a contiguous complex64 / complex128 array -- in C order over its labels;
 * out: device pointer to 2^out_rank elements, written the same way. Pointers
 * 16-byte aligned; the caller owns them. With cuda_stream == NULL the call
 * waits and returns any kernel-side error; with a stream it only enqueues
 * (copies in, the bucket kernel, the copy out) and qt_contract_sync reports
 * the kernel-side status. One call at a time per plan. */
int qt_contract_run(qt_contract_t c, const void *const *ops, void *out, void *cuda_stream);

/* Wait for `cuda_stream` and return the kernel-side status of the plan's
 * last run (QT_OK, QT_ETIMEOUT or QT_EBOUNDS). */
int qt_contract_sync(qt_contract_t c, void *cuda_stream);

int qt_contract_stats_get(qt_contract_t c, qt_contract_stats *out);

void qt_contract_free(qt_contract_t c);

const char *qt_error_string(int code);

/* Library version string. */
const char *qt_version(void);

/* Text describing the last QT_ECUDA / QT_ENOMEM failure on the calling thread
 * (the failing CUDA call and its error name); empty if none. Owned by the
 * library; valid until the next call on this thread. */
const char *qt_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* QT_H */
