// CUDA kernels for bucket elimination on sm_103a.
//
//  k_leaf_fill    gate tensors of every graph from its angles (FP64 -> dtype)
//  k_persistent   one launch drains every bucket of the plan: warps claim work
//                 items in a level-sorted task list, wait (bounded) until the
//                 bucket's producers are done, contract one tile of the bucket
//                 and signal its consumer
//  k_per_bucket   the plain form: one launch per bucket, stream-ordered
//  k_epilogue     per-network scalar -> <Z_jZ_k> and the FP64 energy sum
//
// Bucket contraction (§II-B): out[o] = sum_{x in {0,1}} prod_t T_t[2 pext(o, M_t) + x].
// The summed variable is bit 0 of every operand, so the x = 0 / x = 1 pair of
// an operand is contiguous: one 16-byte load for complex64, two for
// complex128. A lane owns two consecutive outputs; when an operand carries
// output bit 0, its two pairs are contiguous too (32 bytes).
#include <cuda_runtime.h>

#include "../../include/qt.h"
#include "device_common.cuh"
#include "kernels.hpp"

namespace qt {
namespace {

constexpr int kWarps = kPersistentThreads / 32;
static_assert(kMaxSum == 2, "the tile epilogues add the two outputs of a lane: two summed variables at most");
constexpr int kUnroll = 4;  // iterations of 64 outputs in flight per warp

// The (x = 0, x = 1) entries at element e (even) of a tensor. Gate tensors are
// written by an earlier kernel and read through the read-only path;
// results of earlier buckets are read at L2 (`.cg`), since the same kernel
// may have written them from another SM.
__device__ __forceinline__ Pair<float2> ld_pair(const float2* T, uint64_t e, bool leaf) {
    const float4* p = reinterpret_cast<const float4*>(T + e);
    return unpack_pair(leaf ? __ldg(p) : __ldcg(p));
}
__device__ __forceinline__ Pair<double2> ld_pair(const double2* T, uint64_t e, bool leaf) {
    const double2* p = T + e;
    return unpack_pair(leaf ? __ldg(p) : __ldcg(p), leaf ? __ldg(p + 1) : __ldcg(p + 1));
}

// A pair through a generic pointer (shared memory, or a tensor written before this kernel).
__device__ __forceinline__ Pair<float2> ld_pair_smem(const float2* p) {
    return unpack_pair(*reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ Pair<double2> ld_pair_smem(const double2* p) { return unpack_pair(p[0], p[1]); }

// Outputs o and o + 1 (o even): one pair.
__device__ __forceinline__ void st_two(float2* out, uint64_t o, float2 a, float2 b) {
    *reinterpret_cast<float4*>(out + o) = pack_pair(a, b);
}
__device__ __forceinline__ void st_two(double2* out, uint64_t o, double2 a, double2 b) {
    out[o] = make_double2(a.x, b.x);
    out[o + 1] = make_double2(a.y, b.y);
}

struct OpStage {
    uint64_t off;
    uint32_t mask;
    uint32_t chunk_base;  // pext(first output of the tile, mask)
    uint32_t flags;
    uint32_t pad;
};

// One tile (2^chunk_bits outputs starting at chunk << chunk_bits) of bucket B,
// computed by one warp. Output index bits: bit 0 picks one of the lane's two
// outputs, bits 1..5 the lane, bits 6..chunk_bits-1 the iteration.
template <typename R>
__device__ __forceinline__ void contract_tile(const DBucket& B, uint32_t chunk, const OpStage* so,
                                              typename CT<R>::c* arena, int lane) {
    using C = typename CT<R>::c;
    const int cb = B.chunk_bits;
    const int n_ops = B.n_ops;
    const int lane_bits = cb >= 6 ? 5 : (cb >= 1 ? cb - 1 : 0);
    const bool active = (lane >> lane_bits) == 0;
    const uint32_t niter = cb >= 6 ? 1u << (cb - 6) : 1u;
    const uint32_t lane_mask = (1u << (lane_bits + 1)) - 1u;
    const uint32_t obase = chunk << cb;
    C* out = arena + B.out_off;
    for (uint32_t i0 = 0; i0 < niter; i0 += kUnroll) {
        C acc[kUnroll][2][2];
        for (int t = 0; t < n_ops; ++t) {
            const OpStage op = so[t];
            const uint32_t M = op.mask;
            const uint32_t lbase = pext_u32((uint32_t)lane << 1, M & lane_mask);
            const uint32_t mi = cb >= 6 ? (M >> 6) & (niter - 1u) : 0u;
            const int si = __popc(M & 63u);
            const bool contig = (mi & (mi + 1u)) == 0u;
            const bool b0 = (M & 1u) != 0u;
            const bool leaf = (op.flags & kOpLeaf) != 0u;
            const C* T = arena + op.off;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const uint32_t i = i0 + u;
                if (i < niter && active) {
                    const uint32_t ip = contig ? (i & mi) : pext_u32(i, mi);
                    const uint64_t e = 2ull * (uint64_t)(op.chunk_base + lbase + (ip << si));
                    Pair<C> a = ld_pair(T, e, leaf);
                    Pair<C> b = b0 ? ld_pair(T, e + 2, leaf) : a;
                    if (t == 0) {
                        acc[u][0][0] = a.v0;
                        acc[u][0][1] = a.v1;
                        acc[u][1][0] = b.v0;
                        acc[u][1][1] = b.v1;
                    } else {
                        acc[u][0][0] = cmul(acc[u][0][0], a.v0);
                        acc[u][0][1] = cmul(acc[u][0][1], a.v1);
                        acc[u][1][0] = cmul(acc[u][1][0], b.v0);
                        acc[u][1][1] = cmul(acc[u][1][1], b.v1);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t i = i0 + u;
            if (i < niter && active) {
                C r0 = cadd(acc[u][0][0], acc[u][0][1]);
                C r1 = cadd(acc[u][1][0], acc[u][1][1]);
                if (B.n_out == 0) {
                    elem_st(out, 0, r0);  // scalar result: one output
                } else {
                    st_two(out, (uint64_t)obase + ((uint64_t)i << 6) + ((uint64_t)lane << 1), r0, r1);
                }
            }
        }
    }
}

__device__ __forceinline__ void stage_ops(const DBucket& B, uint32_t chunk, const DOperand* ops, OpStage* so, int lane) {
    if (lane < B.n_ops) {
        const DOperand o = ops[B.op_begin + lane];
        OpStage s;
        s.off = o.off;
        s.mask = o.mask;
        s.chunk_base = pext_u32(chunk << B.chunk_bits, o.mask);
        s.flags = o.flags;
        s.pad = 0;
        so[lane] = s;
    }
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *reinterpret_cast<const volatile int32_t*>(p); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Persistent kernel with shared-memory staging (Blackwell bulk copies).
//
// Within an aligned tile of 2^cb outputs starting at o0, operand t (mask M)
// touches exactly the 2^(popc(M & (2^cb-1)) + 1) contiguous elements starting
// at 2 * pext(o0, M). One cp.async.bulk per operand moves that block into the
// warp's stage buffer and an mbarrier counts the bytes in. Each warp keeps
// two stages, so the copy for its next tile is in flight while it contracts
// the current one from shared memory; results go straight to global memory.
//
// Work is claimed in items of runs (consecutive tiles of one bucket). A run's
// descriptors and gate tensors are read once into a run slot; the gate tensors
// of a bucket are multiplied into one small per-tile table. When a run's last
// tile is written the warp adds the run's tile count to the bucket's counter
// (release); a consumer run polls its producers' counters (acquire) until they
// reach the producers' tile counts, at most spin_limit polls.
// ---------------------------------------------------------------------------

constexpr int kPW = kPersistentThreads / 32;  // warps per block
constexpr int kLeafTab = 2 << kLeafBits;       // entries of the folded gate table
constexpr int kUnrollS = 2;                    // 64-output iterations in flight when reading shared memory
constexpr int kFast = 4;                       // most operands of the unrolled tile loop
constexpr int kPmBits = 7;                     // premultiplied operands: most tile bits of the footprint
constexpr int kPmK = (1 << kPmBits) / 32;      // their footprint pairs per lane
// Premultiplied operands in complex128 only, where the tile loop is bound by
// FP64 throughput and a product saved per output is time saved (C2 7.0 ->
// 5.7 ms); the complex64 loop is latency-bound, and the extra dependent
// shared-memory round trip per tile cost more than it saved (+5%).
template <typename R>
struct UsePm {
    static constexpr bool value = sizeof(R) == 8;
};

template <typename R>
struct StageCfg;
template <>
struct StageCfg<float> {
    static constexpr int elems = kStageElemsC64;
};
template <>
struct StageCfg<double> {
    static constexpr int elems = kStageElemsC128;
};

// Everything about one run that does not change from tile to tile.
template <typename R>
struct RunSlot {
    uint64_t out_off;
    uint64_t goff[kMaxOps];    // staged operands: element offset in the arena
    uint32_t gmask[kMaxOps];   // staged operands: full masks
    uint16_t soff[kMaxOps];    // staged operands: element offset in the stage buffer
    uint32_t lmask[kMaxFoldLeaves];
    uint8_t lx[kMaxFoldLeaves];  // 1: the folded tensor's entries pair over x; 0: it lacks x (merged buckets)
    typename CT<R>::c lval[kMaxFoldLeaves][kLeafSlots];  // the folded gate tensors
    uint32_t bucket, chunk_begin, n_chunks;
    uint32_t parent, n_tasks;
    uint32_t leaf_u;      // folded gate masks within the tile
    uint32_t leaf_hi;     // nonzero if a folded gate mask has bits above the tile
    uint32_t total_foot;  // staged elements per tile
    uint8_t n_out, cb, n_staged, n_leaves;
    uint8_t n_ops;
    uint8_t merged;       // 1: merged eliminations (s0, s1): each lane's two outputs add into one result
    uint32_t bad;         // the plan's footprint exceeds the stage: not computed
    // per-group constants of the unrolled tile loop, for the staged operands
    // and the gate table (at most kFast of them)
    uint8_t n_fast;                  // operands of the tile loop; 0: the generic loop
    uint8_t loff[kFast][32];         // each lane's pair index within the footprint
    uint16_t dstep[kFast][5];        // pair-index step of tile bits 6..10
    uint8_t n_hi;                    // folded tensors whose output bit lies above the tile
    uint8_t hi_idx[kMaxFoldLeaves];  // their slots
    uint8_t hi_shift[kMaxFoldLeaves];// position of that bit within the chunk index
    uint8_t hi_ebit[kMaxFoldLeaves]; // bit of a gate-table entry's index holding the tensor's bit in the tile
    uint8_t lsh[kMaxFoldLeaves][2];  // folded tensors within the tile: the bits of a table entry's index
                                     // that give bits 0 and 1 of the tensor's entry (31: none); 255: above
    // A staged operand whose tile bits include the gate table's and number
    // fewer than the tile's: each tile multiplies its footprint by the table
    // (pm_f pairs, written past every footprint, at pm_dst) and the tile loop
    // reads that product instead of the operand and the table.
    uint8_t pm;                      // the operand (255: none)
    uint16_t pm_f;                   // its footprint pairs
    uint16_t pm_dst;                 // element offset of the product in the stage
    uint8_t pm_e[kPmK][32];          // gate-table pair of footprint pair lane + 32 k
    uint32_t unit_begin;             // a fused unit: 1 + its first entry in the unit list (0: none)
    uint32_t unit_count;
};

template <typename R>
struct alignas(128) WarpSmem {
    typename CT<R>::c stage[2][StageCfg<R>::elems];
    typename CT<R>::c leaf_tab[kLeafTab];
    RunSlot<R> slot[2];
    unsigned long long bar[2];
};

// Three blocks of the complex64 kernel per SM (228 KB of shared memory per
// SM, 1 KB of it reserved per block), two of the complex128 one.
static_assert(sizeof(WarpSmem<float>) * kPW + 1024 <= 233472 / 3, "complex64 persistent kernel: 3 blocks per SM");
static_assert(sizeof(WarpSmem<double>) * kPW + 1024 <= 233472 / 2, "complex128 persistent kernel: 2 blocks per SM");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Queue positions are claimed with one atomic each; lane 0 claims the next
// position as soon as it takes the current one, so the claim's round trip
// overlaps the work.
struct Cursor {
    uint32_t reserved = 0;
    __device__ uint32_t claim(const DevPlan& dp, int lane) {
        uint32_t q = 0;
        if (lane == 0) q = ld_volatile(&dp.ctl->error) != 0 ? dp.n_groups : atomicAdd(&dp.ctl->next_item, 1u);
        return q;
    }
    __device__ uint32_t start(const DevPlan& dp, int lane) {
        const uint32_t q = claim(dp, lane);
        reserved = claim(dp, lane);
        return __shfl_sync(kFull, q, 0);
    }
    __device__ uint32_t next(const DevPlan& dp, int lane) {
        const uint32_t q = reserved;
        reserved = claim(dp, lane);
        return __shfl_sync(kFull, q, 0);
    }
};

// A static-order group's dependency check: lane t holds operand t's producer
// and the tile count it must reach (kNone: nothing to wait for).
struct DepCheck {
    uint32_t src = kNone, need = 0;
    __device__ bool ready(const DevPlan& dp) const {
        const bool ok = src == kNone || ld_acquire(&dp.tiles_done[src]) >= need;
        return __all_sync(kFull, ok);
    }
};

// The group at queue position q, if it may start (non-blocking): a position of
// the static order once its bucket's producers have all finished -- lane t
// reads, with acquire, the tile counter of operand t's producer (kept in *dc
// for later polls) -- a position of the ready queue once it has been published.
__device__ __forceinline__ bool group_at(const DevPlan& dp, uint32_t q, DRun* out, int lane, DepCheck* dc) {
    uint32_t ok = 1;
    DRun r{};
    *dc = DepCheck{};
    if (q < dp.n_static) {
        r = dp.runs[q];
        if (r.n_deps) {
            if (lane < (int)r.n_ops) {
                const DOperand& o = dp.ops[r.op_begin + lane];
                dc->src = o.src;
                dc->need = o.src_tiles;
            }
            ok = dc->ready(dp);
        }
    } else {
        if (lane == 0) {
            const DSlot* sl = dp.slots + (q - dp.n_static);
            const uint32_t n = ld_acquire(&sl->n_chunks);
            ok = n != 0;
            if (ok) r = DRun{sl->bucket, sl->chunk_begin, n, sl->op_begin, 0u, 0u, 0u, 0u};
        }
        ok = __shfl_sync(kFull, ok, 0);
        r.bucket = __shfl_sync(kFull, r.bucket, 0);
        r.chunk_begin = __shfl_sync(kFull, r.chunk_begin, 0);
        r.n_chunks = __shfl_sync(kFull, r.n_chunks, 0);
        r.op_begin = __shfl_sync(kFull, r.op_begin, 0);
    }
    *out = r;
    return ok != 0;
}

// Bounded wait until position q may start; records QT_ETIMEOUT on expiry.
// `checked`: group_at has already read position q into *out and dc, so a
// static-order position polls only its producers' counters.
__device__ bool wait_group(const DevPlan& dp, uint32_t q, DRun* out, int lane, DepCheck& dc, bool checked) {
    uint64_t polls = 0;
    const bool counters_only = checked && q < dp.n_static;
    while (counters_only ? !dc.ready(dp) : !group_at(dp, q, out, lane, &dc)) {
        const bool err = ld_volatile(&dp.ctl->error) != 0;
        if (__any_sync(kFull, err)) return false;
        if (++polls > dp.spin_limit) {
            if (lane == 0 && atomicCAS(&dp.ctl->error, 0, QT_ETIMEOUT) == 0) dp.ctl->err_bucket = q;
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Read group `run` into slot `sl`: bucket header, staged operands, folded gate
// values (all laid out by the planner). Lane t < n_staged also gets the
// compressed index of the group's first tile in its operand's bits above the
// tile (pext(o0, M) is that index shifted left by the operand's tile bits).
template <typename R, bool Units>
__device__ void prep_run(const DevPlan& dp, WarpSmem<R>& ws, int sl, const DRun& run, int lane, uint32_t* cbase,
                         bool results_ready = true) {
    using C = typename CT<R>::c;
    if (Units && run.unit_begin) {  // a fused unit: nothing to stage, no gate table
        RunSlot<R>& us = ws.slot[sl];
        if (lane == 0) {
            const DBucket B = dp.buckets[run.bucket];
            us.out_off = B.out_off;
            us.bucket = run.bucket;
            us.chunk_begin = 0;
            us.n_chunks = B.n_tasks;  // the whole unit is one "tile" of its root, which counts as all of them
            us.parent = B.parent;
            us.n_tasks = B.n_tasks;
            us.leaf_u = 0;
            us.leaf_hi = 0;
            us.total_foot = 0;
            us.n_out = B.n_out;
            us.cb = B.n_out;
            us.n_staged = 0;
            us.n_leaves = 0;
            us.bad = 0;
            us.n_fast = 0;
            us.pm = 255;
            us.n_hi = 0;
            us.merged = 0;
            us.unit_begin = run.unit_begin;
            us.unit_count = run.unit_count;
        }
        __syncwarp();
        *cbase = 0;
        return;
    }
    DOperand op{};
    if (lane < kMaxOps) op = dp.ops[run.op_begin + lane];  // the operand array is padded by kMaxOps
    const DBucket B = dp.buckets[run.bucket];
    RunSlot<R>& rs = ws.slot[sl];
    const bool has = lane < B.n_ops;
    // an operand without x (a merged bucket's consumer gates) is always folded
    const bool fits = B.total_foot <= (uint32_t)StageCfg<R>::elems && B.n_leaves <= kMaxFoldLeaves &&
                      __all_sync(kFull, !has || op.folded || (op.smask & 1u));
    if (has && fits) {
        if (op.folded) {
            // a gate tensor (4 slots) or an earlier result of rank <= 2, which
            // this launch wrote from another SM: read that one at L2; its
            // allocation is 128-byte aligned, so 4 entries stay inside it
            rs.lmask[op.slot] = op.mask;
            rs.lx[op.slot] = op.smask & 1u;
            const C* T = static_cast<const C*>(dp.arena) + op.off;
            if ((op.flags & kOpLeaf) || results_ready) {
#pragma unroll
                for (int i = 0; i < kLeafSlots; ++i)
                    rs.lval[op.slot][i] = (op.flags & kOpLeaf) ? elem_ld(T, i) : elem_ldcg(T, i);
            }
        } else {
            rs.goff[op.slot] = op.off;
            rs.gmask[op.slot] = op.mask;
            rs.soff[op.slot] = op.soff;
        }
    }
    if (lane == 0) {
        rs.out_off = B.out_off;
        rs.bucket = run.bucket;
        rs.chunk_begin = run.chunk_begin;
        rs.n_chunks = run.n_chunks;
        rs.parent = B.parent;
        rs.n_tasks = B.n_tasks;
        rs.leaf_u = B.leaf_u;
        rs.leaf_hi = B.leaf_hi;
        rs.total_foot = B.total_foot;
        rs.n_out = B.n_out;
        rs.cb = B.chunk_bits;
        rs.n_staged = B.n_staged;
        rs.n_leaves = B.n_leaves;
        rs.n_ops = B.n_ops;
        rs.merged = (uint8_t)(bucket_n_sum(B.flags) - 1);
        rs.unit_begin = 0;
        rs.unit_count = 0;
        rs.bad = !fits;
        if (!fits && atomicCAS(&dp.ctl->error, 0, QT_EBOUNDS) == 0) dp.ctl->err_bucket = run.bucket;
    }
    __syncwarp();
    *cbase = 0;
    if (lane < rs.n_staged) *cbase = pext_u32(run.chunk_begin, rs.gmask[lane] >> rs.cb);
    // constants of the unrolled tile loop: lane offsets, iteration steps, and
    // the folded tensors whose single output bit lies above the tile
    const uint32_t low = (1u << rs.cb) - 1u;
    const int nf = rs.n_staged + (rs.n_leaves ? 1 : 0);
    const bool fast = !rs.bad && rs.cb >= 6 && rs.cb <= 11 && nf <= kFast;
    for (int t = 0; t < nf && fast; ++t) {
        const uint32_t m = t < rs.n_staged ? (rs.gmask[t] & low) : rs.leaf_u;
        rs.loff[t][lane] = (uint8_t)pext_u32((uint32_t)lane << 1, m & 63u);
        if (lane < 5) {
            const int bit = 6 + lane;
            rs.dstep[t][lane] = ((m >> bit) & 1u) ? (uint16_t)(1u << __popc(m & ((1u << bit) - 1u))) : (uint16_t)0;
        }
    }
    if (lane < rs.n_leaves) {
        // table entry e = 2 j + x, j the tile outputs of leaf_u compressed: the
        // tensor's entry index takes x (if it pairs over x) and then its output
        // bits, the k-th of which is bit 1 + (its rank within leaf_u) of e
        const uint32_t lm = rs.lmask[lane];
        const uint32_t b0 = lm & (0u - lm), b1 = (lm & (lm - 1u)) & (0u - (lm & (lm - 1u)));  // its lowest two bits
        const uint32_t p0 = 1u + __popc(rs.leaf_u & (b0 - 1u)), p1 = 1u + __popc(rs.leaf_u & (b1 - 1u));
        uint32_t s0 = 31u, s1 = 31u;
        if (lm & ~low)
            s0 = 255u;
        else if (rs.lx[lane]) {
            s0 = 0u;
            if (b0) s1 = p0;
        } else {
            if (b0) s0 = p0;
            if (b1) s1 = p1;
        }
        rs.lsh[lane][0] = (uint8_t)s0;
        rs.lsh[lane][1] = (uint8_t)s1;
    }
    // the premultiplied operand: the smallest footprint that carries every
    // tile bit of the gate table, if smaller than the tile and the stage has
    // room for the product past the footprints
    uint32_t pm = 255u, pmb = 32u;
    if (UsePm<R>::value && fast && rs.n_leaves) {
        for (int t = 0; t < rs.n_staged; ++t) {
            const uint32_t m = rs.gmask[t] & low;
            const uint32_t nb = __popc(m);
            if ((rs.leaf_u & ~m) == 0u && nb < pmb) {
                pm = (uint32_t)t;
                pmb = nb;
            }
        }
        if (pm != 255u &&
            (pmb >= rs.cb || pmb > (uint32_t)kPmBits || rs.total_foot + (2u << pmb) > (uint32_t)StageCfg<R>::elems))
            pm = 255u;
    }
    if (UsePm<R>::value && pm != 255u) {
        const uint32_t cl = pext_u32(rs.leaf_u, rs.gmask[pm] & low);  // the table's bits in the footprint index
#pragma unroll
        for (int k = 0; k < kPmK; ++k) rs.pm_e[k][lane] = (uint8_t)pext_u32((uint32_t)lane + 32u * k, cl);
    }
    if (lane == 0) {
        rs.n_fast = fast ? (uint8_t)(nf - (pm != 255u ? 1 : 0)) : (uint8_t)0;
        rs.pm = (uint8_t)pm;
        rs.pm_f = (uint16_t)(pm != 255u ? 1u << pmb : 0u);
        rs.pm_dst = (uint16_t)rs.total_foot;
        uint8_t nh = 0;
        for (int l = 0; l < rs.n_leaves; ++l)
            if (rs.lmask[l] & ~low) {
                rs.hi_idx[nh] = (uint8_t)l;
                rs.hi_shift[nh] = (uint8_t)(31 - __clz(rs.lmask[l]) - rs.cb);
                // with x the tensor's bit in the tile is x (entry bit 0); without
                // x it is one of the output bits in leaf_u (rank <= 2)
                const uint32_t lb = rs.lmask[l] & low;
                rs.hi_ebit[nh] = rs.lx[l] ? (uint8_t)0 : (uint8_t)(1 + __popc(rs.leaf_u & (lb - 1u)));
                ++nh;
            }
        rs.n_hi = nh;
    }
    __syncwarp();
}

// A group prepared before its producers finished: read the earlier results
// folded into its gate table (rank <= 2, read at L2) now that they are done.
template <typename R>
__device__ void load_folded_results(const DevPlan& dp, WarpSmem<R>& ws, int sl, const DRun& run, int lane) {
    RunSlot<R>& rs = ws.slot[sl];
    if (!rs.bad && lane < rs.n_ops) {
        const DOperand op = dp.ops[run.op_begin + lane];
        if (op.folded && !(op.flags & kOpLeaf)) {
            const typename CT<R>::c* T = static_cast<const typename CT<R>::c*>(dp.arena) + op.off;
#pragma unroll
            for (int i = 0; i < kLeafSlots; ++i) rs.lval[op.slot][i] = elem_ldcg(T, i);
        }
    }
    __syncwarp();
}

// Append every group of bucket p to the queue (its last producer just finished).
__device__ void publish_bucket(const DevPlan& dp, uint32_t p, int lane) {
    const DBucket& B = dp.buckets[p];
    const uint32_t ng = B.n_groups, gt = B.group_tiles, nt = B.n_tasks, ob = B.op_begin;
    uint32_t base = 0;
    if (lane == 0) {
        base = atomicAdd(&dp.ctl->next_free, ng);
        if (base + ng > dp.n_groups - dp.n_static) {  // cannot happen with a consistent plan
            if (atomicCAS(&dp.ctl->error, 0, QT_EBOUNDS) == 0) dp.ctl->err_bucket = p;
            base = 0xffffffffu;
        }
    }
    base = __shfl_sync(kFull, base, 0);
    if (base == 0xffffffffu) return;
    for (uint32_t k = lane; k < ng; k += 32) {
        DSlot* sl = dp.slots + base + k;
        sl->bucket = p;
        sl->chunk_begin = k * gt;
        sl->op_begin = ob;
        const uint32_t n = min(gt, nt - k * gt);
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&sl->n_chunks), "r"(n) : "memory");
    }
}

// Start the bulk copies of tile `chunk` of the group in slot `sl` into stage
// `st`. Lane t < n_staged keeps in `cbase` the compressed index of the
// current tile in its operand's bits above the tile; for the next tile of the
// group it is advanced in place: going from chunk c-1 to c clears the trailing
// ones of c-1 (their r operand bits below bit t = ctz(c) give back 2^r - 1)
// and sets bit t (worth 2^r if the operand carries it).
// Returns true if copies were issued (the stage's barrier will complete).
// The group's copy parameters are read from its slot once, at its first
// tile, into `is` (registers): the tiles of a group are issued in order, and
// no other group's are issued between them.
template <typename R>
struct IssueState {
    const typename CT<R>::c* src;  // this lane's staged operand
    uint32_t dst;                  // its footprint's element offset in a stage
    uint32_t mh;                   // its mask's bits above the tile
    uint32_t plow;                 // its tile bits: the footprint is 2 << plow elements
    uint32_t tx;                   // bytes of one tile's copies, every operand
    uint32_t n_issued;             // tiles of the group issued so far
    bool on;                       // copies to issue (the plan's footprints fit, something is staged)
    bool lane_on;                  // this lane copies an operand
};

template <typename R>
__device__ __forceinline__ bool issue_tile(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, uint32_t chunk,
                                           bool first, int lane, uint32_t& cbase, IssueState<R>& is,
                                           uint32_t& pm_dirty) {
    using C = typename CT<R>::c;
    if (first) {
        const RunSlot<R>& rs = ws.slot[sl];
        is.on = !(rs.bad || rs.total_foot == 0);
        is.tx = rs.total_foot * (uint32_t)sizeof(C);
        is.lane_on = lane < rs.n_staged;
        is.n_issued = 0;
        if (is.lane_on) {
            const uint32_t m = rs.gmask[lane];
            is.mh = m >> rs.cb;
            is.plow = __popc(m & ((1u << rs.cb) - 1u));
            is.src = static_cast<const C*>(dp.arena) + rs.goff[lane];
            is.dst = rs.soff[lane];
        }
    }
    if (!is.on) return false;
    // The stage's previous contents were read into registers and consumed
    // before the caller's __syncwarp, so the copies may overwrite it now.
    if (lane == 0) mbar_expect_tx(&ws.bar[st], is.tx);
    if (UsePm<R>::value && is.n_issued < 2u && ((pm_dirty >> st) & 1u)) {
        // the stage's last tile was another group's, which wrote a
        // premultiplied footprint past its own footprints (generic stores),
        // where this group's copies may land: order those stores first. A
        // group's own products never overlap its copies.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        pm_dirty &= ~(1u << st);
    }
    ++is.n_issued;
    __syncwarp();
    if (is.lane_on) {
        if (!first) {
            const uint32_t t = __ffs(chunk) - 1u;
            const uint32_t r = __popc(is.mh & ((1u << t) - 1u));
            cbase = cbase - ((1u << r) - 1u) + (((is.mh >> t) & 1u) << r);
        }
        bulk_g2s(&ws.stage[st][is.dst], is.src + 2ull * ((uint64_t)cbase << is.plow), (2u << is.plow) * (uint32_t)sizeof(C),
                 &ws.bar[st]);
    }
    return true;
}

// Any number of operands (descriptors re-read from shared memory per use).
template <typename R>
__device__ void tile_from_smem_generic(const WarpSmem<R>& ws, int sl, int st, typename CT<R>::c* out, uint32_t chunk,
                                       int lane) {
    using C = typename CT<R>::c;
    const RunSlot<R>& rs = ws.slot[sl];
    const int cb = rs.cb;
    const int n = rs.n_staged + (rs.n_leaves ? 1 : 0);
    const int lane_bits = cb >= 6 ? 5 : (cb >= 1 ? cb - 1 : 0);
    const bool active = (lane >> lane_bits) == 0;
    const uint32_t niter = cb >= 6 ? 1u << (cb - 6) : 1u;
    const uint32_t lane_mask = (1u << (lane_bits + 1)) - 1u;
    const uint32_t low = (1u << cb) - 1u;
    const uint32_t o0 = chunk << cb;
    if (!active) return;
    for (uint32_t i0 = 0; i0 < niter; i0 += kUnrollS) {
        C acc[kUnrollS][2][2];
        for (int t = 0; t < n; ++t) {
            const bool is_tab = t == rs.n_staged;
            const uint32_t m = is_tab ? rs.leaf_u : (rs.gmask[t] & low);
            const C* base = is_tab ? ws.leaf_tab : ws.stage[st] + rs.soff[t];
            const uint32_t lb = pext_u32((uint32_t)lane << 1, m & lane_mask);
            const uint32_t mi = cb >= 6 ? (m >> 6) & (niter - 1u) : 0u;
            const int si = __popc(m & 63u);
            const bool b0 = (m & 1u) != 0u;
#pragma unroll
            for (int u = 0; u < kUnrollS; ++u) {
                const uint32_t i = i0 + u;
                if (i < niter) {
                    const uint32_t e = 2u * (lb + (pext_u32(i, mi) << si));
                    const Pair<C> a = ld_pair_smem(base + e);
                    const Pair<C> b = b0 ? ld_pair_smem(base + e + 2) : a;
                    if (t == 0) {
                        acc[u][0][0] = a.v0;
                        acc[u][0][1] = a.v1;
                        acc[u][1][0] = b.v0;
                        acc[u][1][1] = b.v1;
                    } else {
                        acc[u][0][0] = cmul(acc[u][0][0], a.v0);
                        acc[u][0][1] = cmul(acc[u][0][1], a.v1);
                        acc[u][1][0] = cmul(acc[u][1][0], b.v0);
                        acc[u][1][1] = cmul(acc[u][1][1], b.v1);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnrollS; ++u) {
            const uint32_t i = i0 + u;
            if (i < niter) {
                const C r0 = cadd(acc[u][0][0], acc[u][0][1]);
                const C r1 = cadd(acc[u][1][0], acc[u][1][1]);
                if (rs.n_out == 0) {
                    elem_st(out, 0, r0);
                } else if (rs.merged == 0) {
                    st_two(out, (uint64_t)o0 + ((uint64_t)i << 6) + ((uint64_t)lane << 1), r0, r1);
                } else {  // merged: outputs (o, s1 = 0, 1) add into result o
                    elem_st(out, ((uint64_t)o0 >> 1) + ((uint64_t)i << 5) + (uint64_t)lane, cadd(r0, r1));
                }
            }
        }
    }
}

// Shared-memory reads of the tile loop use 32-bit shared addresses. The loads
// are ordinary (non-volatile) asm so the compiler may schedule them freely;
// each address carries `tok`, an opaque zero produced after the last wait or
// barrier, so no load can be hoisted above the point its data became valid.
__device__ __forceinline__ uint32_t opaque_zero() {
    uint32_t z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
}

// Arithmetic of the tile loop on one output's entry pair (x = 0, 1): load from
// shared memory, multiply by another operand's pair, sum over x, and add two
// outputs' pairs (a merged bucket's s1 = 0 and 1). complex64 keeps the pair as
// packed real and imaginary parts, so a complex product of both x is four
// f32x2 instructions (and one integer sign flip) instead of eight; complex128
// multiplies each entry in FP64.
template <typename R>
struct TileMath;
template <>
struct TileMath<float> {
    struct P {
        f32x2 re, im;
    };
    static __device__ __forceinline__ P load(uint32_t a) {
        P r;
        asm("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(r.re), "=l"(r.im) : "r"(a));
        return r;
    }
    static __device__ __forceinline__ P mul(P p, P a) {
        P r;
        r.re = x2_fma(p.re, a.re, x2_neg(x2_mul(p.im, a.im)));
        r.im = x2_fma(p.re, a.im, x2_mul(p.im, a.re));
        return r;
    }
    static __device__ __forceinline__ float2 xsum(P p) {
        return make_float2(x2_lo(p.re) + x2_hi(p.re), x2_lo(p.im) + x2_hi(p.im));
    }
    static __device__ __forceinline__ P add(P a, P b) { return {x2_add(a.re, b.re), x2_add(a.im, b.im)}; }
    static __device__ __forceinline__ void store(uint32_t a, P v) {
        asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(a), "l"(v.re), "l"(v.im) : "memory");
    }
};
template <>
struct TileMath<double> {
    using P = Pair<double2>;
    static __device__ __forceinline__ P load(uint32_t a) {
        double2 re, im;
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(re.x), "=d"(re.y) : "r"(a));
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(im.x), "=d"(im.y) : "r"(a + 16u));
        return unpack_pair(re, im);
    }
    static __device__ __forceinline__ P mul(P p, P a) { return {cmul(p.v0, a.v0), cmul(p.v1, a.v1)}; }
    static __device__ __forceinline__ double2 xsum(P p) { return cadd(p.v0, p.v1); }
    static __device__ __forceinline__ P add(P a, P b) { return {cadd(a.v0, b.v0), cadd(a.v1, b.v1)}; }
    static __device__ __forceinline__ void store(uint32_t a, P v) {
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.v0.x), "d"(v.v1.x) : "memory");
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a + 16u), "d"(v.v0.y), "d"(v.v1.y) : "memory");
    }
};

// Outputs o, o + 1 (o even) of a result: one planar pair, one store.
__device__ __forceinline__ void stg_two(float2* p, float2 a, float2 b) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a.x), "f"(b.x), "f"(a.y), "f"(b.y));
}
__device__ __forceinline__ void stg_two(double2* p, double2 a, double2 b) {
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(a.x), "d"(b.x));
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p + 1), "d"(a.y), "d"(b.y));
}
// One output per lane, lane l writing output l of `p` (32 consecutive
// outputs, p even): lanes 2k and 2k + 1 hold one pair, which lane 2k stores.
template <typename C>
__device__ __forceinline__ void stg_lanes(C* p, C v, int lane) {
    C w;
    w.x = __shfl_xor_sync(kFull, v.x, 1);
    w.y = __shfl_xor_sync(kFull, v.y, 1);
    if ((lane & 1) == 0) stg_two(p + lane, v, w);
}

// The tile loop for tiles of at least 64 outputs (cb >= 6): N operands in
// shared memory, the last of which may be the folded gate table. A lane owns
// outputs 2*lane + {0,1} + 64*i, i < 2^(cb-6); an operand's pair for such an
// output sits at the lane's offset (loff) plus the steps (dstep) of the set
// bits of i, all fixed per group. U = 2^UB iterations are unrolled per trip
// (cb >= 6 + UB), the trips running over i's bits above bit UB - 1, which
// keeps the code small: every bucket shape runs one of a few loop bodies per
// operand count. A merged bucket (s0, s1) adds a lane's two outputs (s1 = 0,
// 1) into one result, lane + 32*i.
template <typename R, int N, int U, bool Exact>
__device__ __forceinline__ void tile_loop(const uint32_t (&sbase)[N], const uint32_t (&smask)[N],
                                          const RunSlot<R>& rs, typename CT<R>::c* out, int lane, int n_rt) {
    using C = typename CT<R>::c;
    using M = TileMath<R>;
    constexpr uint32_t PB = 2 * sizeof(C);  // bytes of one (x = 0, x = 1) pair
    constexpr int UB = U == 1 ? 0 : U == 2 ? 1 : U == 4 ? 2 : 3;
    constexpr int HB = 5 - UB;  // iteration bits above the unrolled ones (tiles of at most 2^11 outputs)
    uint32_t a0[N], second[N], du[N][UB > 0 ? UB : 1], dh[N][HB];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        a0[t] = sbase[t] + PB * rs.loff[t][lane];
        second[t] = (smask[t] & 1u) ? PB : 0u;  // the lane's second output uses the next pair
#pragma unroll
        for (int k = 0; k < UB; ++k) du[t][k] = PB * rs.dstep[t][k];
#pragma unroll
        for (int k = 0; k < HB; ++k) dh[t][k] = PB * rs.dstep[t][UB + k];
    }
    const uint32_t trips = 1u << (rs.cb - 6 - UB);
    const bool merged = rs.merged != 0;
    for (uint32_t j = 0; j < trips; ++j) {
        uint32_t qb[N];
#pragma unroll
        for (int t = 0; t < N; ++t) {
            qb[t] = a0[t];
#pragma unroll
            for (int k = 0; k < HB; ++k) qb[t] += ((j >> k) & 1u) ? dh[t][k] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            typename M::P p0, p1;  // the lane's two outputs, each an (x = 0, 1) pair of products
#pragma unroll
            for (int t = 0; t < N; ++t) {
                if (!Exact && t >= n_rt) break;  // a uniform branch: the operand count of the group
                uint32_t q = qb[t];
#pragma unroll
                for (int k = 0; k < UB; ++k)
                    if ((u >> k) & 1) q += du[t][k];
                const typename M::P a = M::load(q);
                typename M::P b = a;
                if (second[t]) b = M::load(q + second[t]);
                if (t == 0) {
                    p0 = a;
                    p1 = b;
                } else {
                    p0 = M::mul(p0, a);
                    p1 = M::mul(p1, b);
                }
            }
            const uint32_t i = j * U + (uint32_t)u;
            if (merged)
                stg_lanes(out + i * 32, M::xsum(M::add(p0, p1)), lane);
            else
                stg_two(out + (i * 64 + 2 * lane), M::xsum(p0), M::xsum(p1));
        }
    }
}

// N operands (Exact), or at most N with n of them used.
template <typename R, int N, bool Exact>
__device__ __forceinline__ void run_tile_n(const WarpSmem<R>& ws, int sl, int st, typename CT<R>::c* out,
                                           uint32_t chunk, int lane, int n) {
    using C = typename CT<R>::c;
    const RunSlot<R>& rs = ws.slot[sl];
    const uint32_t low = (1u << rs.cb) - 1u;
    const uint32_t tok = opaque_zero();  // after the stage wait and the gate table's barrier
    uint32_t sbase[N], smask[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        const bool is_tab = t == rs.n_staged;  // never with a premultiplied operand: N = n_staged then
        const uint32_t off = (UsePm<R>::value && t == rs.pm) ? rs.pm_dst : rs.soff[t];
        sbase[t] = tok + (is_tab ? smem_u32(ws.leaf_tab) : smem_u32(ws.stage[st] + off));
        smask[t] = is_tab ? rs.leaf_u : (rs.gmask[t] & low);
    }
    C* tile_out = out + ((uint64_t)chunk << (rs.cb - rs.merged));
    // complex128, bound by FP64 throughput, gains nothing from two iterations
    // in flight and loses to their registers (5.66 vs 5.79 ms on C2)
    if (rs.cb == 6 || sizeof(R) == 8)
        tile_loop<R, N, 1, Exact>(sbase, smask, rs, tile_out, lane, n);
    else
        tile_loop<R, N, 2, Exact>(sbase, smask, rs, tile_out, lane, n);
}

// Wait (bounded) until the copies into stage st have landed. Returns false
// if the wait ran out or the run cannot be computed.
template <typename R>
__device__ bool wait_stage(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, uint32_t& phase, int lane) {
    const RunSlot<R>& rs = ws.slot[sl];
    if (rs.bad) return false;
    if (rs.total_foot > 0) {
        const uint32_t par = (phase >> st) & 1u;
        uint64_t polls = 0;
        while (!mbar_try_wait(&ws.bar[st], par)) {
            if (++polls > dp.spin_limit) {
                if (lane == 0 && atomicCAS(&dp.ctl->error, 0, QT_ETIMEOUT) == 0) dp.ctl->err_bucket = rs.bucket;
                return false;
            }
        }
        phase ^= 1u << st;
    }
    return true;
}

// The folded gate table of a tile: entry 2j + x is the product of the folded
// tensors at tile output pdep(j, leaf_u) and summed value x; a tensor without
// x (a merged bucket's consumer gates) gives both x the same factor. Tensors
// whose bits lie inside the tile give a table over the tile bits that is the
// same for every tile of a group: each lane keeps its two entries in `tlow`.
// A tensor with a bit above the tile (one at most: rank <= 2) takes one of two
// values per tile. Within the tile it depends on one bit of the entry index
// (hi_ebit): x, or for a tensor without x its output bit in leaf_u (s1 or s2,
// the lowest output bits, so the entry bit is at most 2). The table of a tile
// is tlow times those tensors' entries; each lane computes its own factor,
// the same for both of its entries (e and e + 32).
template <typename R>
__device__ __forceinline__ void gate_table(WarpSmem<R>& ws, const RunSlot<R>& rs, uint32_t chunk, bool first,
                                           typename CT<R>::c (&tlow)[2], uint32_t& hi_key, int lane) {
    using C = typename CT<R>::c;
    const uint32_t nent = 2u << __popc(rs.leaf_u);
    if (first) {
        C v0, v1;  // entries lane and lane + 32
        v0.x = v1.x = (R)1;
        v0.y = v1.y = (R)0;
        const uint32_t e0 = (uint32_t)lane, e1 = e0 + 32u;
        for (int l = 0; l < rs.n_leaves; ++l) {
            const uint32_t s0 = rs.lsh[l][0], s1 = rs.lsh[l][1];
            if (s0 == 255u) continue;  // a bit above the tile: per tile, below
            v0 = cmul(v0, rs.lval[l][((e0 >> s0) & 1u) | (((e0 >> s1) & 1u) << 1)]);
            v1 = cmul(v1, rs.lval[l][((e1 >> s0) & 1u) | (((e1 >> s1) & 1u) << 1)]);
        }
        tlow[0] = v0;
        tlow[1] = v1;
    }
    // the table changes only when one of the high output bits changes
    uint32_t key = 0;
    for (int h = 0; h < rs.n_hi; ++h) key |= ((chunk >> rs.hi_shift[h]) & 1u) << h;
    if (!first && key == hi_key) return;
    hi_key = key;
    C f;
    f.x = (R)1;
    f.y = (R)0;
    for (int h = 0; h < rs.n_hi; ++h) {
        const int l = rs.hi_idx[h];
        const uint32_t y = (key >> h) & 1u;  // the tensor's bit above the tile
        f = cmul(f, rs.lval[l][2u * y + (((uint32_t)lane >> rs.hi_ebit[h]) & 1u)]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t e = (uint32_t)lane + 32u * h;
        if (e < nent) elem_st(ws.leaf_tab, e, cmul(tlow[h], f));
    }
    __syncwarp();
}

// A fused unit: its buckets run in steps, intermediates in stage st (free: a
// unit stages nothing), the root's result to the arena. A step is one bucket
// over the whole warp (one output per lane at a time), or several independent
// buckets of at most 16 outputs that the planner packed together, one output
// per lane (a step record gives each lane its bucket). The unit's program is
// read through two windows of kURecWindow records (one per lane each,
// coalesced loads): once the next step starts in the second window, the
// windows move on by one and the next one is requested. A step's records go
// to the warp's gate-table area (unused by units) for its output loop.
__device__ __forceinline__ URec shfl_rec(const URec& r, int src) {
    URec o;
    o.a = __shfl_sync(kFull, r.a, src);
    o.b = __shfl_sync(kFull, r.b, src);
    o.off = __shfl_sync(kFull, r.off, src);
    return o;
}
// Record i (< 2 kURecWindow) of the two windows.
__device__ __forceinline__ URec window_rec(const URec& cur, const URec& nxt, uint32_t i) {
    const URec rc = shfl_rec(cur, (int)(i & (kURecWindow - 1)));
    const URec rn = shfl_rec(nxt, (int)(i & (kURecWindow - 1)));
    return i < (uint32_t)kURecWindow ? rc : rn;
}

// One output o of a bucket whose operand records are ops[0..n_ops).
template <typename R>
__device__ __forceinline__ typename CT<R>::c unit_output(const URec* ops, uint32_t n_ops, uint32_t o,
                                                         typename CT<R>::c* scr, typename CT<R>::c* arena) {
    using C = typename CT<R>::c;
    C a0, a1;
    a0.x = a1.x = (R)1;
    a0.y = a1.y = (R)0;
    for (uint32_t t = 0; t < n_ops; ++t) {
        const URec d = ops[t];
        const uint32_t e = 2u * ((d.b & 2u) ? (o & d.a) >> (d.b >> 8) : pext_u32(o, d.a));
        const C* src = (d.b & 1u) ? scr + d.off : arena + d.off;
        const Pair<C> v = ld_pair_smem(src + e);  // shared memory, or a gate tensor
        a0 = cmul(a0, v.v0);
        a1 = cmul(a1, v.v1);
    }
    return cadd(a0, a1);
}

template <typename R>
__device__ void run_unit(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, int lane) {
    using C = typename CT<R>::c;
    static_assert(sizeof(URec) * kURecWindow <= sizeof(ws.leaf_tab), "a step's records");
    static_assert(kURecWindow == 32 && kMaxOps + 1 <= kURecWindow, "a step's records fit a window");
    URec* recs = reinterpret_cast<URec*>(ws.leaf_tab);
    const RunSlot<R>& rs = ws.slot[sl];
    C* scr = ws.stage[st];
    C* arena = static_cast<C*>(dp.arena);
    // the program is padded by two windows past the last unit
    const URec* prog = dp.unit_prog + (rs.unit_begin - 1u);
    uint32_t pos = 0, base = 0;  // next record; the windows hold records [base, base + 2 kURecWindow)
    URec cur = prog[lane], nxt = prog[kURecWindow + lane];
    for (uint32_t k = 0; k < rs.unit_count;) {
        // a step spans at most 32 records, so pos - base < 64 here and one move suffices
        if (pos >= base + kURecWindow) {
            base += kURecWindow;
            cur = nxt;
            nxt = prog[base + kURecWindow + lane];
        }
        const URec h = shfl_rec(cur, (int)(pos - base));
        if (h.a & kUnitStep) {
            // several buckets: stage the step's records, then each lane
            // computes one output of its bucket
            const uint32_t n_recs = h.a & 0x3fu, n_items = (h.a >> 20) & 7u, used = (h.a >> 24) & 0x3fu;
            const URec r = window_rec(cur, nxt, pos + (uint32_t)lane - base);
            if ((uint32_t)lane < n_recs) recs[lane] = r;
            pos += n_recs;
            k += n_items;
            __syncwarp();
            if ((uint32_t)lane < used) {
                const uint32_t q = (uint32_t)(h.off >> (2 * lane)) & 3u;
                const uint32_t at = q == 0 ? 1u : (h.b >> (8 * (q - 1))) & 0xffu;
                const URec hq = recs[at];
                const uint32_t n_ops = (hq.a >> 8) & 0xffu;
                const uint32_t o = (uint32_t)lane - (uint32_t)hq.off;
                elem_st(scr + hq.b, o, unit_output<R>(recs + at + 1, n_ops, o, scr, arena));
            }
        } else {
            // one bucket over the whole warp
            const uint32_t n_out = h.a & 0xffu, n_ops = (h.a >> 8) & 0xffu;
            const bool root = (h.a >> 16) & 1u;
            const URec r = window_rec(cur, nxt, pos + 1u + (uint32_t)lane - base);  // lane t: operand t
            if ((uint32_t)lane < n_ops) recs[lane] = r;
            pos += 1u + n_ops;
            ++k;
            __syncwarp();
            C* dst = root ? arena + rs.out_off : scr + h.b;
            for (uint32_t o = lane; o < (1u << n_out); o += 32) elem_st(dst, o, unit_output<R>(recs, n_ops, o, scr, arena));
        }
        __syncwarp();
    }
    // the stage will be a bulk-copy target again: order these generic writes
    // before later async-proxy writes to it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
}

// Contract tile `chunk` of the group in slot sl from stage st.
// The premultiplied operand's footprint in stage st times the gate table
// (entry pairs over x on both sides), stored past the stage's footprints.
template <typename R>
__device__ __forceinline__ void premultiply(WarpSmem<R>& ws, const RunSlot<R>& rs, int st, int lane) {
    using M = TileMath<R>;
    constexpr uint32_t PB = 2 * sizeof(typename CT<R>::c);
    const uint32_t tok = opaque_zero();  // after the stage wait and the gate table's barrier
    const uint32_t src = tok + smem_u32(ws.stage[st] + rs.soff[rs.pm]);
    const uint32_t tab = tok + smem_u32(ws.leaf_tab);
    const uint32_t dst = smem_u32(ws.stage[st] + rs.pm_dst);
    const uint32_t f = rs.pm_f;
#pragma unroll
    for (int k = 0; k < kPmK; ++k) {
        const uint32_t j = (uint32_t)lane + 32u * (uint32_t)k;
        if (j < f) M::store(dst + PB * j, M::mul(M::load(src + PB * j), M::load(tab + PB * rs.pm_e[k][lane])));
    }
    __syncwarp();
}

template <typename R, bool Units, typename Clock>
__device__ void contract_tile(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, uint32_t chunk, bool first_of_run,
                              typename CT<R>::c (&tlow)[2], uint32_t& hi_key, uint32_t& pm_dirty, int lane,
                              Clock& clk) {
    using C = typename CT<R>::c;
    const RunSlot<R>& rs = ws.slot[sl];
    if (Units && rs.unit_begin) {
        run_unit<R>(dp, ws, sl, st, lane);
        return;
    }
    // the table changes within a group only if a folded tensor has a bit above the tile
    if (rs.n_leaves && (first_of_run || rs.n_hi)) gate_table<R>(ws, rs, chunk, first_of_run, tlow, hi_key, lane);
    if (UsePm<R>::value && rs.pm != 255u) {
        premultiply<R>(ws, rs, st, lane);
        pm_dirty |= 1u << st;
    }
    clk.lap(kTrGate);
    C* out = static_cast<C*>(dp.arena) + rs.out_off;
    switch (rs.n_fast) {
        case 1: run_tile_n<R, 1, true>(ws, sl, st, out, chunk, lane, 1); break;
        case 2: run_tile_n<R, 2, true>(ws, sl, st, out, chunk, lane, 2); break;
        case 3: run_tile_n<R, 3, true>(ws, sl, st, out, chunk, lane, 3); break;
        case 4: run_tile_n<R, 4, true>(ws, sl, st, out, chunk, lane, 4); break;
        default: tile_from_smem_generic<R>(ws, sl, st, out, chunk, lane); break;
    }
    __syncwarp();
}

// A group's tiles are all written. Count them. In the static order that is
// all: a consumer reads its producers' tile counters itself. In the ready-queue
// order the warp that completes the bucket counts one producer of the parent
// done, and the warp that completes the parent's last producer publishes the
// parent's groups.
template <typename R>
__device__ __forceinline__ void finish_group(const DevPlan& dp, const RunSlot<R>& rs, int lane) {
    fence_proxy_async_global();  // results become visible to later bulk copies
    __syncwarp();
    uint32_t push = 0;
    const uint32_t parent = rs.parent;
    if (dp.isolated) return;
    if (dp.n_static == dp.n_groups) {
        // static order: consumers read this counter themselves, so one release
        // reduction, without waiting for its result, completes the group
        if (lane == 0)
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&dp.tiles_done[rs.bucket]), "r"(rs.n_chunks)
                         : "memory");
        __syncwarp();
        return;
    }
    if (lane == 0) {
        // acquire-release adds: the group that completes the bucket has
        // acquired the other groups' results before it releases them (with its
        // own) to the consumer, whose dependency check is an acquire load
        const uint32_t done = atom_add_acq_rel(&dp.tiles_done[rs.bucket], rs.n_chunks) + rs.n_chunks;
        if (done == rs.n_tasks && parent != kNone) {
            const uint32_t pd = atom_add_acq_rel(&dp.prod_done[parent], 1u) + 1u;
            push = pd == dp.buckets[parent].n_deps;
        }
    }
    push = __shfl_sync(kFull, push, 0);
    if (push && dp.n_static < dp.n_groups) publish_bucket(dp, parent, lane);  // ready-queue order only
    __syncwarp();
}

// Per-warp cycle counters of the kernel's phases (the traced instantiation
// only; the plain one compiles every call away).
template <bool On>
struct PhaseClock {
    uint64_t acc[kTraceSlots];
    long long t0;
    __device__ void begin() {
        if (On) {
#pragma unroll
            for (int i = 0; i < kTraceSlots; ++i) acc[i] = 0;
            t0 = clock64();
        }
    }
    __device__ void lap(int phase) {
        if (On) {
            const long long t = clock64();
            acc[phase] += (uint64_t)(t - t0);
            t0 = t;
        }
    }
    __device__ void count(int slot, uint32_t n) {
        if (On) acc[slot] += n;
    }
    __device__ void store(const DevPlan& dp, int lane) {
        if (On && lane == 0 && dp.trace) {
            const uint32_t w = blockIdx.x * kPW + (threadIdx.x >> 5);
#pragma unroll
            for (int i = 0; i < kTraceSlots; ++i) dp.trace[(size_t)w * kTraceSlots + i] = acc[i];
        }
    }
};

#ifndef QT_PERSISTENT_MIN_BLOCKS
#define QT_PERSISTENT_MIN_BLOCKS 3
#endif

// Traced runs: each bucket's earliest group start and latest group end.
template <bool On>
__device__ __forceinline__ void mark_bucket(const DevPlan& dp, uint32_t b, bool end, int lane) {
    if (On && lane == 0 && dp.bucket_times) {
        const unsigned long long t = globaltimer_ns();
        if (end)
            atomicMax(&dp.bucket_times[2 * b + 1], t);
        else
            atomicMin(&dp.bucket_times[2 * b], t);
    }
}

// Units: the plan has fused units (a separate instantiation, so that plans
// without them run the tile loop alone).
template <typename R, bool Trace, bool Units>
__global__ void __launch_bounds__(kPersistentThreads, QT_PERSISTENT_MIN_BLOCKS) k_persistent(DevPlan dp) {
    using C = typename CT<R>::c;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<R>& ws = reinterpret_cast<WarpSmem<R>*>(smem_raw)[warp];
    PhaseClock<Trace> clk;
    clk.begin();
    if (lane == 0) {
        mbar_init(&ws.bar[0], 1);
        mbar_init(&ws.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    bool pending[2] = {false, false};
    Cursor cur;
    const uint32_t qa = cur.start(dp, lane);
    clk.lap(kTrClaim);
    if (qa < dp.n_groups) {
        // tile A is contracted from stage st (group in slot sa) while the
        // copies for tile B, the next one, are in flight
        int sa = 0, st = 0;
        uint32_t cbase = 0, hi_key = 0;
        C tlow[2];
        IssueState<R> iss{};
        uint32_t pm_dirty = 0;  // stages holding a premultiplied footprint (bit per stage)
        DRun ra;
        DepCheck dca;
        bool ok = wait_group(dp, qa, &ra, lane, dca, false);
        clk.lap(kTrDeps);
        if (ok) {
            prep_run<R, Units>(dp, ws, sa, ra, lane, &cbase);
            mark_bucket<Trace>(dp, ra.bucket, false, lane);
            clk.lap(kTrPrep);
            clk.count(kTrRuns, 1);
            if (lane == 0) fence_proxy_async_global();  // producers' results before this warp's copies
            __syncwarp();
            pending[st] = issue_tile<R>(dp, ws, sa, st, ra.chunk_begin, true, lane, cbase, iss, pm_dirty);
            clk.lap(kTrIssue);
        }
        uint32_t a_chunk = ra.chunk_begin, a_left = ra.n_chunks;
        bool a_first = true;
        while (ok) {
            int sb = sa;
            uint32_t b_chunk = a_chunk + 1, b_left = a_left - 1, qb = 0;
            bool b_valid = true, b_first = false, b_issued = false, b_prepped = false;
            DRun rb;
            DepCheck dcb;
            bool b_checked = false;  // group_at read position qb into rb and dcb
            if (a_left > 1) {
                pending[st ^ 1] = issue_tile<R>(dp, ws, sb, st ^ 1, b_chunk, false, lane, cbase, iss, pm_dirty);
                b_issued = true;
                clk.lap(kTrIssue);
            } else {
                qb = cur.next(dp, lane);
                b_valid = qb < dp.n_groups;
                clk.lap(kTrClaim);
                b_checked = b_valid;
                if (b_valid && group_at(dp, qb, &rb, lane, &dcb)) {
                    sb = sa ^ 1;
                    prep_run<R, Units>(dp, ws, sb, rb, lane, &cbase);
                    mark_bucket<Trace>(dp, rb.bucket, false, lane);
                    clk.lap(kTrPrep);
                    clk.count(kTrRuns, 1);
                    if (lane == 0) fence_proxy_async_global();
                    __syncwarp();
                    pending[st ^ 1] = issue_tile<R>(dp, ws, sb, st ^ 1, rb.chunk_begin, true, lane, cbase, iss, pm_dirty);
                    b_issued = true;
                    b_chunk = rb.chunk_begin;
                    b_left = rb.n_chunks;
                    b_first = true;
                    clk.lap(kTrIssue);
                } else if (b_valid && qb < dp.n_static) {
                    // not ready yet: prepare everything that does not depend
                    // on its producers while tile A is contracted
                    sb = sa ^ 1;
                    prep_run<R, Units>(dp, ws, sb, rb, lane, &cbase, false);
                    b_prepped = true;
                    clk.lap(kTrPrep);
                }
            }
            if (!wait_stage<R>(dp, ws, sa, st, phase, lane)) break;
            clk.lap(kTrWait);
            contract_tile<R, Units>(dp, ws, sa, st, a_chunk, a_first, tlow, hi_key, pm_dirty, lane, clk);
            clk.lap(kTrCompute);
            clk.count(kTrTiles, 1);
            pending[st] = false;
            if (a_left == 1) {
                mark_bucket<Trace>(dp, ws.slot[sa].bucket, true, lane);
                finish_group<R>(dp, ws.slot[sa], lane);
                clk.lap(kTrFinish);
            }
            if (!b_valid) break;
            if (!b_issued) {
                // the next group was not yet published when looked at: wait for it now
                if (!wait_group(dp, qb, &rb, lane, dcb, b_checked)) break;
                clk.lap(kTrDeps);
                sb = sa ^ 1;
                if (!b_prepped) prep_run<R, Units>(dp, ws, sb, rb, lane, &cbase);
                mark_bucket<Trace>(dp, rb.bucket, false, lane);
                clk.lap(kTrPrep);
                clk.count(kTrRuns, 1);
                if (lane == 0) fence_proxy_async_global();
                __syncwarp();
                pending[st ^ 1] = issue_tile<R>(dp, ws, sb, st ^ 1, rb.chunk_begin, true, lane, cbase, iss, pm_dirty);
                // a group prepared before its producers finished reads the
                // results folded into its gate table now, while its copies fly
                if (b_prepped) load_folded_results<R>(dp, ws, sb, rb, lane);
                b_chunk = rb.chunk_begin;
                b_left = rb.n_chunks;
                b_first = true;
                clk.lap(kTrIssue);
            }
            sa = sb;
            a_chunk = b_chunk;
            a_left = b_left;
            a_first = b_first;
            st ^= 1;
        }
    }
    // On an error exit, let copies still in flight land before the block's
    // shared memory is released (bounded).
    for (int s2 = 0; s2 < 2; ++s2) {
        if (!pending[s2]) continue;
        const uint32_t par = (phase >> s2) & 1u;
        for (uint64_t polls = 0; polls < dp.spin_limit && !mbar_try_wait(&ws.bar[s2], par); ++polls) {
        }
    }
    clk.lap(kTrClaim);
    clk.store(dp, lane);
}

template <typename R>
__global__ void __launch_bounds__(kPersistentThreads) k_per_bucket(DevPlan dp, uint32_t b) {
    using C = typename CT<R>::c;
    __shared__ OpStage s_ops[kWarps][kMaxOps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const DBucket B = dp.buckets[b];
    const uint32_t chunk = blockIdx.x * kWarps + warp;
    if (chunk >= B.n_tasks) return;
    stage_ops(B, chunk, dp.ops, s_ops[warp], lane);
    __syncwarp();
    contract_tile<R>(B, chunk, s_ops[warp], static_cast<C*>(dp.arena), lane);
}

// Gate tensors of every graph. Slot layout per graph: 0 |+> (and <+|),
// 1 the observable Z, then for each layer l: ZZ(gamma_l), its conjugate,
// the mixer exp(-i beta_l X), its conjugate. Entry x + 2y: x is the bit of the
// tensor's earlier variable. Both rank-2 kinds are symmetric in (x, y).
template <typename R>
__global__ void k_leaf_fill(const double* angles, int n_graphs, int p, typename CT<R>::c* arena, uint64_t dleaf_off) {
    using C = typename CT<R>::c;
    const int L = 2 + 4 * p;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_graphs * L) return;
    const int g = idx / L, s = idx % L;
    const double* gam = angles + (size_t)g * p;                      // all gammas first,
    const double* bet = angles + (size_t)n_graphs * p + (size_t)g * p;  // then all betas
    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    double dre[4] = {0, 0, 0, 0}, dim[4] = {0, 0, 0, 0};  // d/dgamma_l or d/dbeta_l of the same entries
    if (s == 0) {
        re[0] = re[1] = 0.70710678118654752440;
    } else if (s == 1) {
        re[0] = 1.0;
        re[1] = -1.0;
    } else {
        const int l = (s - 2) / 4, k = (s - 2) % 4;
        const double sign = (k == 1 || k == 3) ? -1.0 : 1.0;  // conjugate flips the imaginary part
        for (int y = 0; y < 2; ++y)
            for (int x = 0; x < 2; ++x) {
                if (k < 2) {
                    // exp(-/+ i g a), a = s_x s_y; its derivative is -/+ i a times itself
                    const double ss = (1 - 2 * x) * (1 - 2 * y);
                    double sn, cs;
                    sincos(gam[l] * ss, &sn, &cs);
                    re[x + 2 * y] = cs;
                    im[x + 2 * y] = -sign * sn;
                    dre[x + 2 * y] = -ss * sn;
                    dim[x + 2 * y] = -sign * ss * cs;
                } else {
                    // [[c, -/+ i s], [-/+ i s, c]]; derivative [[-s, -/+ i c], [-/+ i c, -s]]
                    double sn, cs;
                    sincos(bet[l], &sn, &cs);
                    re[x + 2 * y] = x == y ? cs : 0.0;
                    im[x + 2 * y] = x == y ? 0.0 : -sign * sn;
                    dre[x + 2 * y] = x == y ? -sn : 0.0;
                    dim[x + 2 * y] = x == y ? 0.0 : -sign * cs;
                }
            }
    }
    C* T = arena + (size_t)idx * kLeafSlots;
    for (int i = 0; i < 4; ++i) {
        C v;
        v.x = (R)re[i];
        v.y = (R)im[i];
        elem_st(T, i, v);
    }
    if (dleaf_off) {
        C* D = T + dleaf_off;
        for (int i = 0; i < 4; ++i) {
            C v;
            v.x = (R)dre[i];
            v.y = (R)dim[i];
            elem_st(D, i, v);
        }
    }
}

// One block per graph: each network's value is the product of its scalar
// results (one per connected piece; normally one), taken in FP64; its real
// part is <Z_jZ_k>. Then E = |E|/2 - 1/2 sum_jk <Z_jZ_k>, summed in edge order.
template <typename R>
__global__ void k_epilogue(DevEpilogue de) {
    using C = typename CT<R>::c;
    const C* arena = static_cast<const C*>(de.arena);
    const int g = blockIdx.x;
    const int first = de.graph_first_net[g], last = de.graph_first_net[g + 1];
    for (int net = first + threadIdx.x; net < last; net += blockDim.x) {
        // the network's value: over its slices (one without slicing), the
        // product of the slice's root results and fixed gate entries, summed
        double sr = 0.0, si = 0.0, vr = 1.0, vi = 0.0;
        const uint32_t f0 = de.net_first_factor[net], f1 = de.net_first_factor[net + 1];
        for (uint32_t f = f0; f < f1; ++f) {
            const uint64_t w = de.factor[f];
            if ((w & kFirstFactor) && f != f0) {
                sr += vr;
                si += vi;
                vr = 1.0;
                vi = 0.0;
            }
            const C v = elem_ld(arena, w & ~kFirstFactor);
            const double xr = (double)v.x, xi = (double)v.y;
            const double nr = vr * xr - vi * xi, ni = vr * xi + vi * xr;
            vr = nr;
            vi = ni;
        }
        de.zz[net] = sr + vr;
        de.zz_imag[net] = si + vi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int net = first; net < last; ++net) s += de.zz[net];
        de.energies[g] = 0.5 * (double)de.graph_owned[g] - 0.5 * s;
    }
}

}  // namespace

cudaError_t launch_leaf_fill(int dtype, const double* angles, int n_graphs, int p, void* arena, uint64_t dleaf_off,
                             cudaStream_t s) {
    const int total = n_graphs * (2 + 4 * p);
    const int threads = 128, blocks = (total + threads - 1) / threads;
    if (dtype == QT_C128)
        k_leaf_fill<double><<<blocks, threads, 0, s>>>(angles, n_graphs, p, static_cast<double2*>(arena), dleaf_off);
    else
        k_leaf_fill<float><<<blocks, threads, 0, s>>>(angles, n_graphs, p, static_cast<float2*>(arena), dleaf_off);
    return cudaGetLastError();
}

__global__ void k_clear_ends(unsigned long long* t, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) t[2 * i + 1] = 0ull;
}

cudaError_t launch_clear_ends(unsigned long long* t, size_t n, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_clear_ends<<<blocks, 256, 0, s>>>(t, n);
    return cudaGetLastError();
}

size_t persistent_smem_bytes(int dtype) {
    return dtype == QT_C128 ? sizeof(WarpSmem<double>) * kPW : sizeof(WarpSmem<float>) * kPW;
}

template <typename R, bool Trace, bool Units>
static void launch_k(int grid, size_t smem, const DevPlan& dp, cudaStream_t s) {
    k_persistent<R, Trace, Units><<<grid, kPersistentThreads, smem, s>>>(dp);
}

template <typename R>
static void launch_k(int grid, size_t smem, const DevPlan& dp, cudaStream_t s) {
    const bool tr = dp.trace != nullptr, un = dp.has_units != 0;
    if (tr)
        un ? launch_k<R, true, true>(grid, smem, dp, s) : launch_k<R, true, false>(grid, smem, dp, s);
    else
        un ? launch_k<R, false, true>(grid, smem, dp, s) : launch_k<R, false, false>(grid, smem, dp, s);
}

cudaError_t launch_persistent(int dtype, int grid, const DevPlan& dp, cudaStream_t s) {
    const size_t smem = persistent_smem_bytes(dtype);
    if (dtype == QT_C128)
        launch_k<double>(grid, smem, dp, s);
    else
        launch_k<float>(grid, smem, dp, s);
    return cudaGetLastError();
}

cudaError_t launch_per_bucket(int dtype, uint32_t bucket, uint32_t n_tasks, const DevPlan& dp, cudaStream_t s) {
    const uint32_t blocks = (n_tasks + kWarps - 1) / kWarps;
    if (dtype == QT_C128)
        k_per_bucket<double><<<blocks, kPersistentThreads, 0, s>>>(dp, bucket);
    else
        k_per_bucket<float><<<blocks, kPersistentThreads, 0, s>>>(dp, bucket);
    return cudaGetLastError();
}

cudaError_t launch_epilogue(int dtype, const DevEpilogue& de, cudaStream_t s) {
    if (dtype == QT_C128)
        k_epilogue<double><<<de.n_graphs, 256, 0, s>>>(de);
    else
        k_epilogue<float><<<de.n_graphs, 256, 0, s>>>(de);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t set_smem_attributes(int smem) {
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_persistent<R, false, false>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_persistent<R, false, true>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_persistent<R, true, false>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_persistent<R, true, true>, a, smem);
    return e;
}

int persistent_blocks_per_sm(int dtype) {
    const size_t smem = persistent_smem_bytes(dtype);
    int n = 0, n2 = 0;
    cudaError_t e;
    if (dtype == QT_C128) {
        e = set_smem_attributes<double>((int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<double, false, false>, kPersistentThreads, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_persistent<double, false, true>, kPersistentThreads, smem);
    } else {
        e = set_smem_attributes<float>((int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<float, false, false>, kPersistentThreads, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_persistent<float, false, true>, kPersistentThreads, smem);
    }
    n = n < n2 ? n : n2;  // one grid size serves every instantiation
    return e == cudaSuccess && n > 0 ? n : 0;
}

}  // namespace qt
