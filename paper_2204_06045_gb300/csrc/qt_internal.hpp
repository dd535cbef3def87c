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
constexpr int kMaxOps = 32;      // operands per bucket
constexpr int kLeafSlots = 4;    // every leaf tensor occupies 4 elements
constexpr int kAlignElems128 = 8;// 128-byte alignment in complex128 elements (16 for complex64)

// One bucket on the device. 32 bytes.
struct DBucket {
    uint64_t out_off;   // element offset of the result in the arena
    uint32_t op_begin;  // first operand in the operand array
    uint16_t n_ops;     // operand count
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
    uint32_t flags;// kOpLeaf: a gate tensor written before the contraction starts
};
static_assert(sizeof(DOperand) == 16, "DOperand layout");
constexpr uint32_t kOpLeaf = 1u;

// Counters the persistent kernel uses; zeroed before every run.
struct DControl {
    uint32_t next_item;  // next work item to claim
    int32_t error;       // first kernel-side error (QT_E* code), 0 if none
    uint32_t err_bucket; // bucket at which the error was raised
    uint32_t pad;
};

}  // namespace qt
