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
// elements (QT_STAGE_BYTES, 8 KB by default, for both element types). Gate tensors whose tile bits number
// at most kLeafBits are folded into one product table instead.
#ifndef QT_STAGE_BYTES
#define QT_STAGE_BYTES 8192
#endif
constexpr int kStageElemsC64 = QT_STAGE_BYTES / 8;
constexpr int kStageElemsC128 = QT_STAGE_BYTES / 16;
constexpr int kLeafBits = 5;
constexpr int kMaxFoldLeaves = 8;
constexpr uint8_t kBucketFoldLeaves = 1;
constexpr uint8_t kBucketInUnit = 2;    // inside a fused unit, not its root: never claimed on its own
constexpr uint8_t kBucketUnitRoot = 4;  // the root (last bucket) of a fused unit
// Merged eliminations: flags bits 3..4 hold n_sum - 1, the bucket's summed
// variables beyond the first. In the planner (and the exported plan) an
// operand's entry for output o and summed values s is at
// 2^popc(smask) * pext(o, mask) + pext(s, smask). On the device a bucket
// summing s0 and then s1 is laid out as the bucket of s0 alone, whose outputs
// are (o, s1) with s1 as bit 0: its tiles contract s0 as usual, and the
// epilogue adds the two outputs of each lane (s1 = 0, 1) into result o. The
// consumer's gate tensors (no s0) are folded into the gate table with equal
// entries for both values of s0. The planner's chains and device view take
// more summed variables (s2 as device bit 1); the kernel's epilogues take two.
constexpr int kMaxSum = 2;          // summed variables per bucket, at most
constexpr int bucket_n_sum(uint8_t flags) { return 1 + ((flags >> 3) & 3); }
// Epilogue factor lists (element offsets into the arena): this bit marks the
// first factor of a slice's product.
constexpr uint64_t kFirstFactor = 1ull << 63;
constexpr int8_t kFactorRoot = -2;  // a factor that is a root result (the others are fixed gate entries)
// Fused units: a subtree of small buckets (every output count at most
// 2^kFuseOutBits, every non-gate operand produced inside the subtree) is one
// work group; one warp contracts its buckets in elimination order with the
// intermediates in its shared-memory stage and writes only the root's result.
#ifndef QT_FUSE_OUT_BITS
#define QT_FUSE_OUT_BITS 8
#endif
constexpr int kFuseOutBits = QT_FUSE_OUT_BITS;
constexpr int kRunTiles = 12;        // tiles of one bucket handed out per claim (default)
constexpr int kBwdTileBits = 9;      // outputs per reverse-sweep tile, log2 (512: 3% faster than 256 on N=50 p=4 c64; 1024 slower)
constexpr int kBwdRedElems = 1024;   // per-warp shared-memory elements for in-tile cotangent sums
constexpr uint32_t kZeroChunk = 1u << 16;  // elements per block of the cotangent zeroing kernel
// Reverse-sweep launches per level: buckets of exactly 1, 2, 3, 4 or 5 operands
// (compile-time counts), then at most 8, then at most 16.
constexpr int kBwdClasses = 7;
constexpr int bwd_op_class(int n_ops) { return n_ops <= 5 ? n_ops - 1 : n_ops <= 8 ? 5 : 6; }
// How the reverse sweep treats an operand (per operand, fixed at plan time).
enum : int8_t {
    kBwdNone = 0,       // a gate tensor without an angle (|+>, Z)
    kBwdGate = 1,       // a gate tensor of an angle: Re <cotangent, dT/dangle> summed per angle
    kBwdDirect = 2,     // a result carrying every output bit: each cotangent entry stored once
    kBwdRedStore = 3,   // summed over the tile's missing bits in shared memory, then stored
    kBwdRedAtomic = 4,  // as 3, but other tiles add to the same entries: atomic adds
    kBwdAtomic = 5      // no room in shared memory: atomic adds per output (zeroed first)
};
constexpr int kDefaultTileBits = 9;  // at most 512 outputs per tile (default); measured best on GB300
// Bucket-width classes of the tile autotuner, by output bits: <= 6, 7..10,
// 11..14, 15..19, >= 20.
constexpr int kWidthClasses = 5;
constexpr int width_class(int n_out) { return n_out <= 6 ? 0 : n_out <= 10 ? 1 : n_out <= 14 ? 2 : n_out <= 19 ? 3 : 4; }

// One bucket on the device. 64 bytes.
struct DBucket {
    uint64_t out_off;   // element offset of the result in the arena
    uint32_t op_begin;  // first operand in the operand array
    uint8_t n_ops;      // operand count
    uint8_t flags;      // kBucketFoldLeaves: gate tensors go through the per-tile product table
    uint8_t n_out;      // output bits of the tiles (width - 1); the result has n_out + 1 - n_sum
    uint8_t chunk_bits; // log2 of the outputs per tile
    uint32_t parent;    // consuming bucket, kNone for a root (scalar result)
    uint32_t n_deps;    // operands produced by earlier buckets
    uint32_t n_tasks;   // tiles = 2^(n_out - chunk_bits)
    uint32_t net;       // network index
    // staging of one tile (persistent kernel), fixed by the planner
    uint32_t total_foot;// staged elements per tile
    uint8_t n_staged;   // operands copied into the stage buffer
    uint8_t n_leaves;   // gate tensors folded into the product table
    uint16_t scr_off;   // kBucketInUnit: element offset of its result in the warp's stage
    uint32_t leaf_u;    // folded gate masks within the tile
    uint32_t leaf_hi;   // folded gate masks above the tile (nonzero: the table changes per tile)
    uint32_t group_tiles; // tiles per work group (the unit a warp claims)
    uint32_t n_groups;    // ceil(n_tasks / group_tiles); 1 for a unit root, 0 inside a unit
    uint32_t unit_begin;  // kBucketUnitRoot: 1 + the unit's first record in the unit programs
    uint32_t unit_count;  // kBucketUnitRoot: the unit's buckets (the root last)
};
static_assert(sizeof(DBucket) == 64, "DBucket layout");
// index bits of a bucket's result
constexpr int result_bits(const DBucket& d) { return d.n_out + 1 - bucket_n_sum(d.flags); }

// One operand on the device. 32 bytes.
struct DOperand {
    uint64_t off;      // element offset of the operand's tensor in the arena
    uint32_t mask;     // output bits the operand carries (tile outputs: s1 is bit 0 when merged)
    uint32_t flags;    // kOpLeaf: a gate tensor (written before the contraction starts)
    uint32_t src;      // producing bucket, kNone for a gate tensor
    uint32_t src_tiles;// the producer's tile count
    uint16_t soff;     // staged: element offset of its tile footprint in the stage buffer
    uint8_t slot;      // position among the staged operands, or among the folded gate tensors
    uint8_t folded;    // 1: folded into the per-tile gate table
    uint8_t smask;     // summed variables it carries: bit 0 s0 (the entry pair's x), bit 1 s1
    uint8_t pad[3];
};
static_assert(sizeof(DOperand) == 32, "DOperand layout");
constexpr uint32_t kOpLeaf = 1u;

// A group of consecutive tiles of one bucket: what one claim hands a warp,
// which reads the bucket's descriptors once for all of them. 32 bytes.
struct DRun {
    uint32_t bucket;
    uint32_t chunk_begin;
    uint32_t n_chunks;
    uint32_t op_begin;  // the bucket's first operand (saves a dependent load)
    uint32_t n_deps;    // producers that must finish before the group may start (static order: each
                        // operand's producer has counted all its tiles; ready queue: 0)
    uint32_t unit_begin;// fused unit: 1 + its first record in the unit programs (0: an ordinary group)
    uint32_t unit_count;// fused unit: its buckets (the root last)
    uint32_t n_ops;     // the bucket's operand count (the dependency check reads its producers from them)
};
static_assert(sizeof(DRun) == 32, "DRun layout");

// A published slot of the ready queue: a group whose bucket's producers have
// all finished. 16 bytes.
struct DSlot {
    uint32_t bucket;
    uint32_t chunk_begin;
    uint32_t op_begin;
    uint32_t n_chunks;  // written last (release); nonzero marks the slot as published
};
static_assert(sizeof(DSlot) == 16, "DSlot layout");

// A fused unit's program: for each bucket, in elimination order, a header
// record then one record per operand. 16 bytes.
//   header:  a = n_out | n_ops << 8 | (1 << 16 if the unit's root), b = stage
//            offset of the result (not the root), off = its first lane in a step
//   operand: a = mask, b bit 0 = 1 for an intermediate of the unit (off: its
//            stage offset), 0 for a gate tensor (off: arena offset); b bit 1 =
//            1 if the mask is one run of bits, starting at bit b >> 8 (the
//            entry index is then (o & mask) >> (b >> 8))
//   step:    several independent buckets run together, one output per lane:
//            a = records of the step (this one included) | kUnitStep | items
//            << 20 | lanes used << 24, b = offsets of items 1..3 from this
//            record (8 bits each), off = the item of each lane (2 bits each);
//            item i's header and operand records follow in order
struct URec {
    uint32_t a;
    uint32_t b;
    uint64_t off;
};
static_assert(sizeof(URec) == 16, "URec layout");
constexpr int kURecWindow = 32;  // records a warp holds at once (one per lane)
constexpr uint32_t kUnitStep = 1u << 18;  // marks a step record

// Counters the persistent kernel uses; zeroed before every run.
struct DControl {
    uint32_t next_item;  // next queue position to claim
    int32_t error;       // first kernel-side error (QT_E* code), 0 if none
    uint32_t err_bucket; // bucket at which the error was raised
    uint32_t next_free;  // next free slot of the dynamic part of the queue
};

}  // namespace qt
