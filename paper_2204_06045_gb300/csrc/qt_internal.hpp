// Internal plan layout shared by the host planner and the CUDA kernels.
//
// A plan is a list of buckets (§II-B). Bucket b sums its variable v out of the
// product of its operands. All of b's operands contain v, and every tensor's
// index bits are ordered by elimination rank with the earliest variable as
// bit 0, so v is bit 0 of every operand. The output's bits are the other
// variables of the bucket, also in rank order. An operand t therefore carries
// a subset of the output bits, given by `mask`, and its entry for output index
// o and summed value x sits at element 2 * pext(o, mask) + x.
#pragma once
#include <cstdint>

namespace qt {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kMaxOutBits = 30;  // outputs of at most 2^30 entries (width 31)
constexpr int kMaxOps = 16;      // operands per bucket
constexpr int kLeafSlots = 4;    // every leaf tensor occupies 4 elements
// Persistent kernel staging: every operand's footprint in one output tile is a
// contiguous block, copied into a per-warp shared-memory stage of this many
// elements (8 KB for both element types). Gate tensors whose tile bits number
// at most kLeafBits are folded into one product table instead.
constexpr int kStageElemsC64 = 1024;
constexpr int kStageElemsC128 = 512;
constexpr int kLeafBits = 5;
constexpr int kMaxFoldLeaves = 8;
constexpr uint8_t kBucketFoldLeaves = 1;
constexpr int kRunTiles = 16;  // tiles of one bucket handed out per claim

// One bucket on the device. 32 bytes.
struct DBucket {
    uint64_t out_off;   // element offset of the result in the arena
    uint32_t op_begin;  // first operand in the operand array
    uint8_t n_ops;      // operand count
    uint8_t flags;      // kBucketFoldLeaves: gate tensors go through the per-tile product table
    uint8_t n_out;      // output bits (width - 1)
    uint8_t chunk_bits; // log2 of the outputs per task
    uint32_t parent;    // consuming bucket, kNone for a root (scalar result)
    uint32_t n_deps;    // operands produced by earlier buckets
    uint32_t n_tasks;   // tasks (output chunks) = 2^(n_out - chunk_bits)
    uint32_t net;       // network index
};
static_assert(sizeof(DBucket) == 32, "DBucket layout");

// One operand on the device. 16 bytes.
struct DOperand {
    uint64_t off;  // element offset of the operand's tensor in the arena
    uint32_t mask; // output bits the operand carries
    uint32_t flags;// bit 0 (kOpLeaf): a gate tensor; otherwise bits 1..31 hold the producing bucket
};
static_assert(sizeof(DOperand) == 16, "DOperand layout");
constexpr uint32_t kOpLeaf = 1u;

// A run of consecutive tiles of one bucket, the unit a persistent warp
// prepares once (descriptors, gate values, dependency check). 16 bytes.
struct DRun {
    uint32_t bucket;
    uint32_t chunk_begin;
    uint32_t n_chunks;
    uint32_t pad;
};
static_assert(sizeof(DRun) == 16, "DRun layout");

// Counters the persistent kernel uses; zeroed before every run.
struct DControl {
    uint32_t next_item;  // next work item to claim
    int32_t error;       // first kernel-side error (QT_E* code), 0 if none
    uint32_t err_bucket; // bucket at which the error was raised
    uint32_t pad;
};

}  // namespace qt
