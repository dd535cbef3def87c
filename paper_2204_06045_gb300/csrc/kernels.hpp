// Launch wrappers for the CUDA kernels (called only by the C ABI layer).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "qt_internal.hpp"

namespace qt {

// Device view of a plan, passed to kernels by value.
struct DevPlan {
    const DBucket* buckets;
    const DOperand* ops;
    const DRun* runs;       // the queue's first n_static positions: groups of buckets without producers
    uint32_t n_static;
    uint32_t n_groups;      // queue length
    uint32_t n_buckets;
    DSlot* slots;           // queue positions n_static.. n_groups-1, published at run time
    uint32_t* tiles_done;   // n_buckets: tiles written so far
    uint32_t* prod_done;    // n_buckets: producers finished so far (ready-queue order)
    DControl* ctl;
    void* arena;            // complex64 or complex128 elements
    uint64_t spin_limit;
    uint64_t* trace;        // per-warp phase counters (kTraceSlots each), or null: untraced kernel
    uint32_t isolated;      // nonzero: run only the groups in `runs` and notify no consumer
    unsigned long long* bucket_times;  // traced runs: per bucket, first group start and last group end (ns)
    const URec* unit_prog;      // fused units' programs (DRun.unit_begin - 1 indexes them)
    uint32_t has_units;         // nonzero: the plan has fused units (the kernel variant that runs them)
};

// Phase counters of the traced persistent kernel, per warp (cycles unless noted).
constexpr int kTraceSlots = 10;
enum : int {
    kTrClaim = 0,   // claiming work items, and the kernel's tail
    kTrPrep = 1,    // reading run descriptors and gate tensors
    kTrDeps = 2,    // checking and waiting for producers
    kTrIssue = 3,   // starting bulk copies
    kTrWait = 4,    // waiting for bulk copies to land
    kTrCompute = 5, // contracting tiles and storing results
    kTrFinish = 6,  // publishing finished runs
    kTrTiles = 7,   // count of tiles
    kTrRuns = 8,    // count of runs
    kTrGate = 9     // building the folded gate table of a tile
};

// Everything the epilogue reads and writes.
struct DevEpilogue {
    const DBucket* buckets;
    const uint32_t* net_first_root;  // n_nets + 1
    const uint32_t* root_bucket;
    const int32_t* graph_first_net;  // n_graphs + 1
    const uint32_t* net_first_factor;  // n_nets + 1
    const uint64_t* factor;  // arena element offsets; kFirstFactor marks the first factor of each slice
    const int8_t* factor_param;  // per factor: kFactorRoot, a fixed gate's angle, or -1
    const int32_t* graph_owned;  // n_graphs: networks whose 1/2 the energy counts (all, unless sharded by slice)
    const int32_t* net_weight;   // gradient plans with deduplicated networks: per network, the networks
                                 // sharing its value (its class; 0 for a duplicate); null: 1 each
    int32_t n_graphs;
    const void* arena;
    double* zz;        // n_nets
    double* zz_imag;   // n_nets
    double* energies;  // n_graphs
};

// Everything the reverse sweep reads and writes.
struct DevBwd {
    const DBucket* buckets;
    const DOperand* ops;
    const int8_t* op_param;     // per operand: gate parameter (k: gamma_k, p+k: beta_k), -1 none
    const int8_t* op_bwd;       // per operand: kBwd* treatment
    const uint16_t* op_roff;    // per operand: offset of its in-tile sum in the warp's shared memory
    const uint32_t* net_graph;  // graph of each network
    const uint32_t* task_bucket;// tasks of one level: (bucket, tile)
    const uint32_t* task_tile;
    uint32_t n_tasks;
    int32_t p;
    void* arena;
    uint64_t cot_delta;         // cotangent of the result at offset X lives at X + cot_delta
    uint64_t dleaf_delta;       // derivative of the gate tensor at offset X lives at X + dleaf_delta
    double* grad;               // n_graphs x 2p accumulators: sum Re <cotangent, dT/dtheta>
};

cudaError_t launch_leaf_fill(int dtype, const double* angles, int n_graphs, int p, void* arena, uint64_t dleaf_off,
                             cudaStream_t s);
// Reverse-sweep seeds: every root result's cotangent, and the derivative terms of the gate
// entries that slicing fixed (added to grad, n_graphs x 2p, before the -1/2 of k_grad_final).
cudaError_t launch_seed_roots(int dtype, const DevEpilogue& de, int n_nets, uint64_t cot_delta, uint64_t dleaf_delta,
                              double* grad, int p, const uint32_t* net_graph, cudaStream_t s);
// op_class: the level's tasks of buckets with exactly 1..5 operands (0..4), at most 8 (5) or 16 (6)
cudaError_t launch_backward(int dtype, int op_class, const DevBwd& db, cudaStream_t s);
// Function attributes of the reverse-sweep kernels (the shared-memory size
// above the default); once per process and element type, before any capture.
cudaError_t prepare_backward(int dtype);

cudaError_t launch_zero_ranges(int dtype, void* arena, const uint64_t* ranges, uint32_t n_ranges, cudaStream_t s);
cudaError_t launch_grad_final(const double* grad, int n_graphs, int p, double* dgamma, double* dbeta, cudaStream_t s);
cudaError_t launch_persistent(int dtype, int grid, const DevPlan& dp, cudaStream_t s);
cudaError_t launch_per_bucket(int dtype, uint32_t bucket, uint32_t n_tasks, const DevPlan& dp, cudaStream_t s);
cudaError_t launch_epilogue(int dtype, const DevEpilogue& de, cudaStream_t s);
int persistent_blocks_per_sm(int dtype);
cudaError_t launch_clear_ends(unsigned long long* t, size_t n, cudaStream_t s);
constexpr int kPersistentThreads = 128;  // 4 warps; each warp owns its shared-memory stages
size_t persistent_smem_bytes(int dtype);

// Records a failed CUDA call for qt_last_error_detail; returns QT_ENOMEM or QT_ECUDA.
int report_cuda_error(cudaError_t e, const char* file, const char* what, int line);

}  // namespace qt
