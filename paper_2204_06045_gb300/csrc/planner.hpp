// Host-side planner: graph -> lightcone networks -> elimination orders ->
// bucket schedule -> flat device layout.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>

#include "qt_internal.hpp"

namespace qt {

// A gate tensor of the network (rank 1 or 2). Kinds follow QT_LEAF_* in qt.h.
struct Leaf {
    int kind;
    int layer;  // 0-based layer for ZZ / mixer tensors, -1 otherwise
    int rank;
    int v[2];
    int fix = -1;  // sliced networks: a rank-2 gate with one variable fixed, the fixed variable's
                   // slice bit (its entries for the other variable x are at x + 2 * value)
};

// A gate tensor of a sliced network whose variables are all fixed: a scalar
// per slice, entry val(f[0]) (rank 1) or val(f[0]) + 2 val(f[1]) (rank 2).
struct FixedLeaf {
    int kind;
    int layer;
    int rank;
    int f[2];  // slice bits of its variables
};

struct Network {
    int graph = 0;
    int edge = 0;  // edge index within its graph
    int nvars = 0;
    std::vector<Leaf> leaves;
    std::vector<int> wire_vars;  // variables on each qubit's wire
    // index slicing: 2^slice_bits slices, slice s fixing variable k of
    // fixed_vars (numbered in the unsliced network) to bit k of s
    int slice_bits = 0;
    std::vector<int> fixed_vars;
    std::vector<FixedLeaf> fixed;
    std::vector<uint32_t> slices;  // the slices this plan contracts, increasing (empty: all)
    bool owner = true;             // the plan counts the network's 1/2 in the energy (sharded slices: one plan does)
    int rep = -1;                  // lightcone deduplication: the earlier network of the same graph whose
                                   // value this one takes (it is not contracted); -1: contracted itself
    uint32_t n_emitted() const { return slices.empty() ? (1u << slice_bits) : (uint32_t)slices.size(); }
    uint32_t slice_at(uint32_t k) const { return slices.empty() ? k : slices[k]; }
};

struct HOperand {
    int src;        // local bucket producing it, or -1 for a leaf
    int leaf;       // leaf index in the network, or -1
    uint32_t mask;  // output bits it carries
    int rank;       // its index bits, the summed ones included
    uint32_t smask = 1;  // summed variables it carries (bit k: the bucket's k-th summed variable)
};

struct HBucket {
    int var;
    int width;  // inclusive: the summed variables count
    int parent; // local id of the consuming bucket, -1 for a scalar result
    int n_deps;
    int level;
    int n_sum = 1;  // summed variables (more than 1: merged eliminations)
    int var2 = -1;  // merged: the second summed variable (the absorbed consumer's)
    int var3 = -1;  // merged: the third (the consumer's consumer's)
    std::vector<HOperand> ops;
};

struct NetPlan {
    std::vector<int> order;
    std::vector<HBucket> buckets;  // in elimination order
    double cost = 0;               // sum of 2^width
    int max_width = 0;
};

struct GraphIn {
    int n = 0;
    std::vector<std::pair<int, int>> edges;
    std::vector<int> sel;  // edges whose networks are planned; empty: every edge
    // per planned network (parallel to sel): the slices to contract (empty:
    // all) and whether this plan counts the network's 1/2 in the energy
    std::vector<std::vector<uint32_t>> sel_slices;
    std::vector<uint8_t> sel_owner;
    size_t n_nets() const { return sel.empty() ? edges.size() : sel.size(); }
    int edge_of(size_t i) const { return sel.empty() ? (int)i : sel[i]; }
};

struct PlanConfig {
    int p = 1;
    int dtype = 0;  // 0 complex64, 1 complex128
    int restarts = 0;
    int restart_min_width = 0;  // restarts only for networks whose plain greedy order reaches this width
    uint64_t seed = 0;
    int max_width = 31;
    int chunk_log2 = 0;
    int run_tiles = 0;
    int order = 0;        // 0: claim order from a critical-path list-scheduling simulation; 1: ready queue
    int sim_workers = 1824;  // warps assumed by the simulation
    bool with_grad = false;
    bool fuse = false;       // form fused units of small subtrees (persistent energy plans)
    int tile_cap[kWidthClasses] = {0, 0, 0, 0, 0};  // most tile bits per bucket-width class (0: chunk_log2 / default)
    bool merge = false;      // merge chains of eliminations (a bucket and the parent that only extends it)
    bool dedup = false;      // contract one network per isomorphism class of lightcones (per graph)
    int slice_width = 0;     // > 0: slice networks whose greedy width exceeds it (forward plans)
    int max_slice_bits = 0;  // most variables fixed per network
};

// The flat plan: what gets uploaded plus host-side bookkeeping.
struct HostPlan {
    PlanConfig cfg;
    std::vector<GraphIn> graphs;
    std::vector<Network> nets;
    std::vector<NetPlan> nplans;

    std::vector<int> graph_first_net;   // n_graphs + 1
    std::vector<uint32_t> net_first_bucket;  // n_nets + 1
    std::vector<DBucket> buckets;       // network-contiguous, elimination order within a network
    std::vector<DOperand> operands;
    std::vector<int32_t> op_src;        // global producing bucket, -1 for leaves
    std::vector<int32_t> op_leaf_kind;
    std::vector<int32_t> op_leaf_layer;
    std::vector<int32_t> op_rank;
    std::vector<int32_t> bucket_level;
    std::vector<int32_t> bucket_var;
    std::vector<int32_t> bucket_var2;
    std::vector<int32_t> bucket_var3;
    std::vector<int32_t> bucket_slice;  // the slice of its network a bucket belongs to
    std::vector<int32_t> op_leaf_sub;   // leaf operands: element offset within the gate tensor (sliced gates)
    // epilogue: per network, factors of its value (arena element offsets, bit
    // 63 set on the first factor of each slice): value = sum over slices of
    // the product of the slice's factors (root results and fixed gate entries)
    std::vector<uint32_t> net_first_factor;  // n_nets + 1
    std::vector<uint64_t> factor;
    std::vector<int8_t> factor_param;        // per factor: kFactorRoot for a root result, else the fixed gate's
                                             // angle (k: gamma_k, p+k: beta_k) or -1 (|+>, Z)
    std::vector<int32_t> graph_owned;        // per graph: networks whose 1/2 the energy counts
    std::vector<int32_t> net_weight;         // deduplicated plans: per network, the networks sharing its
                                             // value (0 for a duplicate); empty without duplicates
    uint64_t n_slices = 0;               // slices over all networks (1 per unsliced network)
    uint64_t n_unique = 0;               // networks contracted (the others take a representative's value)
    std::vector<DRun> runs;             // static claim order (all groups, or the groups of buckets without producers)
    std::vector<URec> unit_prog;        // fused units' programs, unit by unit (padded by kURecWindow records)
    uint64_t n_units = 0;
    uint64_t n_fused = 0;               // buckets inside fused units (roots included)
    uint64_t n_tiles = 0;
    uint64_t n_groups = 0;              // queue length: groups over all buckets
    double sim_seconds = 0;             // makespan of the host simulation (0 if not simulated)
    std::vector<uint32_t> root_bucket;  // every root bucket (scalar result)
    std::vector<uint32_t> net_first_root;  // n_nets + 1 into root_bucket
    std::vector<uint32_t> level_first_bucket;  // buckets sorted by level (for the adjoint)
    std::vector<uint32_t> by_level;

    uint64_t leaf_elems = 0;   // leaf table size in elements (gate values, then their derivatives with_grad)
    uint64_t dleaf_off = 0;    // element offset of the derivative table (gradient plans)
    std::vector<int8_t> op_param;        // per operand: parameter of a gate tensor (k: gamma_k, p+k: beta_k), -1 none
    std::vector<int8_t> op_bwd;          // per operand: kBwd* treatment in the reverse sweep
    std::vector<uint16_t> op_roff;       // per operand: offset of its in-tile sum in the warp's shared memory
    std::vector<uint64_t> bwd_zero;      // cotangent pieces to zero before the sweep: (element offset, count) pairs
    std::vector<uint32_t> net_graph;     // graph of each network
    std::vector<uint32_t> bwd_bucket;    // reverse sweep: (bucket, tile) tasks, deepest level last
    std::vector<uint32_t> bwd_tile;
    std::vector<uint32_t> bwd_level_begin;  // kBwdClasses * n_levels + 1 offsets into the task arrays:
                                            // level lv, operand-count class c starts at kBwdClasses * lv + c
    uint64_t arena_elems = 0;  // leaf table + results
    uint64_t cot_off = 0;      // start of the cotangent region (gradient plans)
    uint64_t total_elems = 0;
    int max_width = 0;
    int n_levels = 0;
    double sum_2w = 0, alg_bytes = 0, flops = 0;
    int64_t width_hist[64] = {0};
    double plan_seconds = 0;
};

// A contraction of tensors over binary indices in one expression (the paper's
// "tncontract" benchmark, §II-E): out[K] = sum over the labels not in K of the
// product of the operands, each operand given by its labels in C order (its
// last label is bit 0 of its flat index). It runs as a chain of buckets: the
// summed labels are eliminated first (each bucket's variable is bit 0 of its
// operands, as in the energy plans), and the free labels take the next ranks
// in the output's bit order, so the last result is the output, bit for bit.
struct ContractPlan {
    int dtype = 0;
    std::vector<int> in_rank;                 // per input
    std::vector<uint64_t> in_off;             // per input: element offset of its permuted copy in the arena
    std::vector<std::vector<uint8_t>> in_src_bit;  // per input, per internal bit k: the bit of the caller's flat
                                                   // index (C order) it comes from
    std::vector<DBucket> buckets;             // in elimination order (a chain or a tree ending in one result)
    std::vector<DOperand> operands;           // padded by kMaxOps
    std::vector<DRun> runs;                   // static claim order: every group, producers first
    uint64_t out_off = 0;
    int out_rank = 0;
    uint64_t arena_elems = 0;
    int n_summed = 0;
    int max_width = 0;
    double alg_bytes = 0;  // every bucket's operands read once and result written once
    double flops = 0;      // 8 per complex multiply-add of the buckets (the paper's complex FLOP count)
    std::vector<int> widths;  // per bucket, the summed labels included
};

// labels: per operand, its labels in C order (any non-negative ints, distinct
// within an operand); out_labels: the output's, in C order. Every output label
// must appear in an operand and every operand must carry at least one summed
// label; at most 30 distinct labels, 16 operands. Returns QT_OK, QT_EINVAL or
// QT_EWIDTH.
int build_contract_plan(const std::vector<std::vector<int>>& labels, const std::vector<int>& out_labels, int dtype,
                        int sim_workers, ContractPlan* cp);

// Returns QT_OK or a QT_E* code.
int build_host_plan(const std::vector<GraphIn>& graphs, const PlanConfig& cfg, HostPlan* out);
// Recompute the layout stages (tiles, device arrays, units, claim order) of a
// plan whose networks are built, for the configuration in hp->cfg.
int layout_plan(HostPlan* hp);

// Tiles per work group for a bucket that has the grid's `warps` to itself:
// the fewest whole rounds of `warps` groups of at most `cap` tiles, with the
// tiles shared evenly, so that no warp is left a round that the others skip.
inline uint32_t lone_group_tiles(uint32_t n_tasks, uint32_t warps, uint32_t cap) {
    if (n_tasks == 0 || warps == 0 || cap == 0) return 1;
    const uint64_t per_round = (uint64_t)warps * cap;
    const uint64_t rounds = (n_tasks + per_round - 1) / per_round;
    return (uint32_t)((n_tasks + rounds * warps - 1) / (rounds * warps));
}

int leaf_slots_per_graph(int p);
int leaf_index(int kind, int layer);

}  // namespace qt
