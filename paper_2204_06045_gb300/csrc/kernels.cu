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
#include "kernels.hpp"

namespace qt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kPersistentThreads / 32;
constexpr int kUnroll = 4;  // iterations of 64 outputs in flight per warp

template <typename R>
struct CT;
template <>
struct CT<float> {
    using c = float2;
};
template <>
struct CT<double> {
    using c = double2;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename C>
struct Pair {
    C v0, v1;
};

// The (x = 0, x = 1) entries at element e (even) of a tensor. Gate tensors are
// written by an earlier kernel and read through the read-only path;
// results of earlier buckets are read at L2 (`.cg`), since the same kernel
// may have written them from another SM.
__device__ __forceinline__ Pair<float2> ld_pair(const float2* T, uint64_t e, bool leaf) {
    const float4* p = reinterpret_cast<const float4*>(T + e);
    float4 v = leaf ? __ldg(p) : __ldcg(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double2> ld_pair(const double2* T, uint64_t e, bool leaf) {
    const double2* p = T + e;
    double2 a = leaf ? __ldg(p) : __ldcg(p);
    double2 b = leaf ? __ldg(p + 1) : __ldcg(p + 1);
    return {a, b};
}

__device__ __forceinline__ Pair<float2> ld_pair_smem(const float2* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double2> ld_pair_smem(const double2* p) { return {p[0], p[1]}; }

__device__ __forceinline__ void st_two(float2* out, uint64_t o, float2 a, float2 b) {
    *reinterpret_cast<float4*>(out + o) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_two(double2* out, uint64_t o, double2 a, double2 b) {
    out[o] = a;
    out[o + 1] = b;
}

// Bits of x selected by m, packed to the low end (parallel bit extract).
__device__ __forceinline__ uint32_t pext_u32(uint32_t x, uint32_t m) {
    uint32_t r = 0, t = x & m;
    while (t) {
        uint32_t low = t & (0u - t);
        r |= 1u << __popc(m & (low - 1u));
        t ^= low;
    }
    return r;
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
                    out[0] = r0;  // scalar result: one output
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

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *reinterpret_cast<const volatile int32_t*>(p); }

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
    typename CT<R>::c lval[kMaxFoldLeaves][kLeafSlots];  // the folded gate tensors
    uint32_t bucket, chunk_begin, n_chunks;
    uint32_t leaf_u;      // folded gate masks within the tile
    uint32_t leaf_hi;     // nonzero if a folded gate mask has bits above the tile
    uint32_t total_foot;  // staged elements per tile
    uint8_t n_out, cb, n_staged, n_leaves;
    uint32_t bad;         // the plan's footprint exceeds the stage: not computed
};

template <typename R>
struct alignas(128) WarpSmem {
    typename CT<R>::c stage[2][StageCfg<R>::elems];
    typename CT<R>::c leaf_tab[kLeafTab];
    RunSlot<R> slot[2];
    unsigned long long bar[2];
};

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
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bits of j deposited at the set bits of m (parallel bit deposit).
__device__ __forceinline__ uint32_t pdep_u32(uint32_t j, uint32_t m) {
    uint32_t r = 0;
    for (uint32_t k = 0; m; ++k) {
        const uint32_t low = m & (0u - m);
        if ((j >> k) & 1u) r |= low;
        m ^= low;
    }
    return r;
}

// Exclusive prefix sum over the warp.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane, uint32_t* total) {
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    *total = __shfl_sync(kFull, x, 31);
    return x - v;
}

// The claimed work of one warp, walked tile by tile. The next item is
// claimed as soon as the current one is taken, so the claim's round trip
// overlaps the work.
struct Cursor {
    uint32_t r = 0, r_end = 0;  // runs of the current item
    uint32_t c = 0;             // tiles handed out from run r
    uint32_t reserved = 0;      // next item (lane 0), claimed ahead
    bool have_reserved = false;

    __device__ uint32_t claim(const DevPlan& dp, int lane) {
        uint32_t item = 0;
        if (lane == 0) item = ld_volatile(&dp.ctl->error) != 0 ? dp.n_items : atomicAdd(&dp.ctl->next_item, 1u);
        return item;
    }
    // Advance to the next run; false when the warp's work is done.
    __device__ bool next_run(const DevPlan& dp, int lane) {
        ++r;
        c = 0;
        if (r < r_end) return true;
        uint32_t item = have_reserved ? reserved : claim(dp, lane);
        item = __shfl_sync(kFull, item, 0);
        if (item >= dp.n_items) return false;
        reserved = claim(dp, lane);
        have_reserved = true;
        r = dp.item_begin[item];
        r_end = dp.item_begin[item + 1];
        return true;
    }
    __device__ bool start(const DevPlan& dp, int lane) {
        r = 0xffffffffu;  // next_run() wraps it to 0 >= r_end and claims an item
        r_end = 0;
        return next_run(dp, lane);
    }
};

// Read run `ri` into slot `sl`: bucket, operands, folded gate values. Each
// lane returns the producer it must wait for (kNone if none) and that
// producer's tile count.
template <typename R>
__device__ void prep_run(const DevPlan& dp, WarpSmem<R>& ws, int sl, uint32_t ri, int lane, uint32_t* dep_b,
                         uint32_t* dep_need) {
    using C = typename CT<R>::c;
    const DRun run = dp.runs[ri];
    const DBucket B = dp.buckets[run.bucket];
    RunSlot<R>& rs = ws.slot[sl];
    const int cb = B.chunk_bits;
    const uint32_t low = (1u << cb) - 1u;
    const bool fold = (B.flags & kBucketFoldLeaves) != 0;
    DOperand op{};
    const bool has = lane < B.n_ops;
    if (has) op = dp.ops[B.op_begin + lane];
    const bool leaf = has && (op.flags & kOpLeaf);
    const bool folded = fold && leaf;
    const bool staged = has && !folded;
    const uint32_t foot = staged ? (2u << __popc(op.mask & low)) : 0u;
    uint32_t total_foot, n_staged, n_leaves;
    const uint32_t soff = warp_excl_scan(foot, lane, &total_foot);
    const uint32_t spos = warp_excl_scan(staged ? 1u : 0u, lane, &n_staged);
    const uint32_t lpos = warp_excl_scan(folded ? 1u : 0u, lane, &n_leaves);
    const uint32_t leaf_u = __reduce_or_sync(kFull, folded ? (op.mask & low) : 0u);
    const uint32_t leaf_hi = __reduce_or_sync(kFull, folded ? (op.mask & ~low) : 0u);
    const bool fits = total_foot <= (uint32_t)StageCfg<R>::elems && n_leaves <= (uint32_t)kMaxFoldLeaves;
    if (staged && fits) {
        rs.goff[spos] = op.off;
        rs.gmask[spos] = op.mask;
        rs.soff[spos] = (uint16_t)soff;
    }
    if (folded && fits) {
        rs.lmask[lpos] = op.mask;
        const C* T = static_cast<const C*>(dp.arena) + op.off;
#pragma unroll
        for (int i = 0; i < kLeafSlots; ++i) rs.lval[lpos][i] = T[i];
    }
    if (lane == 0) {
        rs.out_off = B.out_off;
        rs.bucket = run.bucket;
        rs.chunk_begin = run.chunk_begin;
        rs.n_chunks = run.n_chunks;
        rs.leaf_u = leaf_u;
        rs.leaf_hi = leaf_hi;
        rs.total_foot = total_foot;
        rs.n_out = B.n_out;
        rs.cb = (uint8_t)cb;
        rs.n_staged = (uint8_t)n_staged;
        rs.n_leaves = (uint8_t)n_leaves;
        rs.bad = !fits;
        if (!fits && atomicCAS(&dp.ctl->error, 0, QT_EBOUNDS) == 0) dp.ctl->err_bucket = run.bucket;
    }
    *dep_b = (has && !leaf) ? (op.flags >> 1) : kNone;
    *dep_need = *dep_b != kNone ? dp.buckets[*dep_b].n_tasks : 0u;
    __syncwarp();
}

// True once every producer has written all its tiles (one poll per lane).
__device__ __forceinline__ bool deps_met(const DevPlan& dp, uint32_t dep_b, uint32_t need) {
    const bool ok = dep_b == kNone || ld_acquire(&dp.chunks_done[dep_b]) >= need;
    return __all_sync(kFull, ok);
}

// Bounded wait for the producers; on expiry records QT_ETIMEOUT.
__device__ bool wait_deps_run(const DevPlan& dp, uint32_t dep_b, uint32_t need, uint32_t b, int lane) {
    uint64_t polls = 0;
    while (!deps_met(dp, dep_b, need)) {
        const bool err = ld_volatile(&dp.ctl->error) != 0;
        if (__any_sync(kFull, err)) return false;
        if (++polls > dp.spin_limit) {
            if (lane == 0 && atomicCAS(&dp.ctl->error, 0, QT_ETIMEOUT) == 0) dp.ctl->err_bucket = b;
            return false;
        }
        __nanosleep(100);
    }
    return true;
}

// Start the bulk copies of tile `chunk` of the run in slot `sl` into stage `st`.
// Returns true if copies were issued (the stage's barrier will complete).
template <typename R>
__device__ __forceinline__ bool issue_tile(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, uint32_t chunk, int lane) {
    using C = typename CT<R>::c;
    const RunSlot<R>& rs = ws.slot[sl];
    if (rs.bad || rs.total_foot == 0) return false;
    fence_proxy_async_smem();  // earlier reads of this stage come before the new copies
    __syncwarp();
    if (lane == 0) mbar_expect_tx(&ws.bar[st], rs.total_foot * (uint32_t)sizeof(C));
    __syncwarp();
    if (lane < rs.n_staged) {
        const uint32_t m = rs.gmask[lane];
        const C* src = static_cast<const C*>(dp.arena) + rs.goff[lane] + 2ull * pext_u32(chunk << rs.cb, m);
        const uint32_t foot = 2u << __popc(m & ((1u << rs.cb) - 1u));
        bulk_g2s(&ws.stage[st][rs.soff[lane]], src, foot * (uint32_t)sizeof(C), &ws.bar[st]);
    }
    return true;
}

// N operands from shared memory (the last may be the folded gate table), a
// tile of 2^cb outputs written straight to global memory.
template <typename R, int N>
__device__ __forceinline__ void tile_from_smem(const typename CT<R>::c* const (&base)[N], const uint32_t (&mask)[N],
                                               typename CT<R>::c* out, int cb, int n_out, uint32_t o0, int lane) {
    using C = typename CT<R>::c;
    const int lane_bits = cb >= 6 ? 5 : (cb >= 1 ? cb - 1 : 0);
    const bool active = (lane >> lane_bits) == 0;
    const uint32_t niter = cb >= 6 ? 1u << (cb - 6) : 1u;
    const uint32_t lane_mask = (1u << (lane_bits + 1)) - 1u;
    uint32_t lb[N], mi[N];
    int si[N];
    bool b0[N], contig[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        lb[t] = pext_u32((uint32_t)lane << 1, mask[t] & lane_mask);
        mi[t] = cb >= 6 ? (mask[t] >> 6) & (niter - 1u) : 0u;
        si[t] = __popc(mask[t] & 63u);
        b0[t] = (mask[t] & 1u) != 0u;
        contig[t] = (mi[t] & (mi[t] + 1u)) == 0u;
    }
    if (!active) return;
    for (uint32_t i0 = 0; i0 < niter; i0 += kUnrollS) {
        C acc[kUnrollS][2][2];
#pragma unroll
        for (int t = 0; t < N; ++t) {
#pragma unroll
            for (int u = 0; u < kUnrollS; ++u) {
                const uint32_t i = i0 + u;
                if (i < niter) {
                    const uint32_t ip = contig[t] ? (i & mi[t]) : pext_u32(i, mi[t]);
                    const uint32_t e = 2u * (lb[t] + (ip << si[t]));
                    const Pair<C> a = ld_pair_smem(base[t] + e);
                    const Pair<C> b = b0[t] ? ld_pair_smem(base[t] + e + 2) : a;
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
                if (n_out == 0)
                    out[0] = r0;
                else
                    st_two(out, (uint64_t)o0 + ((uint64_t)i << 6) + ((uint64_t)lane << 1), r0, r1);
            }
        }
    }
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
                if (rs.n_out == 0)
                    out[0] = r0;
                else
                    st_two(out, (uint64_t)o0 + ((uint64_t)i << 6) + ((uint64_t)lane << 1), r0, r1);
            }
        }
    }
}

template <typename R, int N>
__device__ __forceinline__ void run_tile_n(const WarpSmem<R>& ws, int sl, int st, typename CT<R>::c* out,
                                           uint32_t chunk, int lane) {
    using C = typename CT<R>::c;
    const RunSlot<R>& rs = ws.slot[sl];
    const uint32_t low = (1u << rs.cb) - 1u;
    const C* base[N];
    uint32_t mask[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        const bool is_tab = t == rs.n_staged;
        base[t] = is_tab ? ws.leaf_tab : ws.stage[st] + rs.soff[t];
        mask[t] = is_tab ? rs.leaf_u : (rs.gmask[t] & low);
    }
    tile_from_smem<R, N>(base, mask, out, rs.cb, rs.n_out, chunk << rs.cb, lane);
}

// Wait for stage st, (re)build the gate table, contract tile `chunk` of the
// run in slot sl. Returns false if the bounded wait ran out.
template <typename R>
__device__ bool compute_tile(const DevPlan& dp, WarpSmem<R>& ws, int sl, int st, uint32_t chunk, bool first_of_run,
                             uint32_t& phase, int lane) {
    using C = typename CT<R>::c;
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
    const uint32_t o0 = chunk << rs.cb;
    if (rs.n_leaves && (first_of_run || rs.leaf_hi)) {
        const uint32_t nent = 2u << __popc(rs.leaf_u);
        for (uint32_t e = lane; e < nent; e += 32) {
            const uint32_t x = e & 1u;
            const uint32_t o = o0 | pdep_u32(e >> 1, rs.leaf_u);
            C v = rs.lval[0][2u * pext_u32(o, rs.lmask[0]) + x];
            for (int l = 1; l < rs.n_leaves; ++l) v = cmul(v, rs.lval[l][2u * pext_u32(o, rs.lmask[l]) + x]);
            ws.leaf_tab[e] = v;
        }
        __syncwarp();
    }
    C* out = static_cast<C*>(dp.arena) + rs.out_off;
    const int n = rs.n_staged + (rs.n_leaves ? 1 : 0);
    switch (n) {
        case 1: run_tile_n<R, 1>(ws, sl, st, out, chunk, lane); break;
        case 2: run_tile_n<R, 2>(ws, sl, st, out, chunk, lane); break;
        case 3: run_tile_n<R, 3>(ws, sl, st, out, chunk, lane); break;
        default: tile_from_smem_generic<R>(ws, sl, st, out, chunk, lane); break;
    }
    __syncwarp();
    return true;
}

// A run's tiles are all written: publish them to consumers.
__device__ __forceinline__ void finish_run(const DevPlan& dp, uint32_t bucket, uint32_t n_chunks, int lane) {
    fence_proxy_async_global();  // results become visible to later bulk copies
    __syncwarp();
    if (lane == 0) red_release_add(&dp.chunks_done[bucket], n_chunks);
    __syncwarp();
}

template <typename R>
__global__ void __launch_bounds__(kPersistentThreads, 3) k_persistent(DevPlan dp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<R>& ws = reinterpret_cast<WarpSmem<R>*>(smem_raw)[warp];
    if (lane == 0) {
        mbar_init(&ws.bar[0], 1);
        mbar_init(&ws.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    bool pending[2] = {false, false};
    Cursor cur;
    if (cur.start(dp, lane)) {
        // tile A: being computed (slot sa, stage st); tile B: the next one
        int sa = 0, st = 0;
        uint32_t dep_b, dep_need;
        prep_run<R>(dp, ws, sa, cur.r, lane, &dep_b, &dep_need);
        uint32_t a_chunk = ws.slot[sa].chunk_begin, a_left = ws.slot[sa].n_chunks;
        bool a_first = true;
        bool ok = wait_deps_run(dp, dep_b, dep_need, ws.slot[sa].bucket, lane);
        if (ok) {
            if (lane == 0) fence_proxy_async_global();
            __syncwarp();
            pending[st] = issue_tile<R>(dp, ws, sa, st, a_chunk, lane);
        }
        while (ok) {
            // the next tile: same run, or the first tile of the next run
            int sb = sa;
            uint32_t b_chunk = a_chunk + 1, b_left = a_left - 1;
            bool b_valid = true, b_first = false, b_issued = false;
            uint32_t bdep = kNone, bneed = 0;
            if (a_left == 1) {
                b_valid = cur.next_run(dp, lane);
                if (b_valid) {
                    sb = sa ^ 1;
                    prep_run<R>(dp, ws, sb, cur.r, lane, &bdep, &bneed);
                    b_chunk = ws.slot[sb].chunk_begin;
                    b_left = ws.slot[sb].n_chunks;
                    b_first = true;
                }
            }
            if (b_valid && deps_met(dp, bdep, bneed)) {
                if (b_first && lane == 0) fence_proxy_async_global();
                __syncwarp();
                pending[st ^ 1] = issue_tile<R>(dp, ws, sb, st ^ 1, b_chunk, lane);
                b_issued = true;
            }
            if (!compute_tile<R>(dp, ws, sa, st, a_chunk, a_first, phase, lane)) break;
            pending[st] = false;
            if (a_left == 1) finish_run(dp, ws.slot[sa].bucket, ws.slot[sa].n_chunks, lane);
            if (!b_valid) break;
            if (!b_issued) {
                if (!wait_deps_run(dp, bdep, bneed, ws.slot[sb].bucket, lane)) break;
                if (lane == 0) fence_proxy_async_global();
                __syncwarp();
                pending[st ^ 1] = issue_tile<R>(dp, ws, sb, st ^ 1, b_chunk, lane);
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
__global__ void k_leaf_fill(const double* angles, int n_graphs, int p, typename CT<R>::c* arena) {
    using C = typename CT<R>::c;
    const int L = 2 + 4 * p;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_graphs * L) return;
    const int g = idx / L, s = idx % L;
    const double* gam = angles + (size_t)g * p;                      // all gammas first,
    const double* bet = angles + (size_t)n_graphs * p + (size_t)g * p;  // then all betas
    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
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
                    const double ss = (1 - 2 * x) * (1 - 2 * y);
                    double sn, cs;
                    sincos(gam[l] * ss, &sn, &cs);
                    re[x + 2 * y] = cs;
                    im[x + 2 * y] = -sign * sn;
                } else {
                    double sn, cs;
                    sincos(bet[l], &sn, &cs);
                    re[x + 2 * y] = x == y ? cs : 0.0;
                    im[x + 2 * y] = x == y ? 0.0 : -sign * sn;
                }
            }
    }
    C* T = arena + (size_t)idx * kLeafSlots;
    for (int i = 0; i < 4; ++i) {
        C v;
        v.x = (R)re[i];
        v.y = (R)im[i];
        T[i] = v;
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
        double vr = 1.0, vi = 0.0;
        for (uint32_t r = de.net_first_root[net]; r < de.net_first_root[net + 1]; ++r) {
            const C v = arena[de.buckets[de.root_bucket[r]].out_off];
            const double xr = (double)v.x, xi = (double)v.y;
            const double nr = vr * xr - vi * xi, ni = vr * xi + vi * xr;
            vr = nr;
            vi = ni;
        }
        de.zz[net] = vr;
        de.zz_imag[net] = vi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int net = first; net < last; ++net) s += de.zz[net];
        de.energies[g] = 0.5 * (double)(last - first) - 0.5 * s;
    }
}

}  // namespace

cudaError_t launch_leaf_fill(int dtype, const double* angles, int n_graphs, int p, void* arena, cudaStream_t s) {
    const int total = n_graphs * (2 + 4 * p);
    const int threads = 128, blocks = (total + threads - 1) / threads;
    if (dtype == QT_C128)
        k_leaf_fill<double><<<blocks, threads, 0, s>>>(angles, n_graphs, p, static_cast<double2*>(arena));
    else
        k_leaf_fill<float><<<blocks, threads, 0, s>>>(angles, n_graphs, p, static_cast<float2*>(arena));
    return cudaGetLastError();
}

size_t persistent_smem_bytes(int dtype) {
    return dtype == QT_C128 ? sizeof(WarpSmem<double>) * kPW : sizeof(WarpSmem<float>) * kPW;
}

cudaError_t launch_persistent(int dtype, int grid, const DevPlan& dp, cudaStream_t s) {
    const size_t smem = persistent_smem_bytes(dtype);
    if (dtype == QT_C128)
        k_persistent<double><<<grid, kPersistentThreads, smem, s>>>(dp);
    else
        k_persistent<float><<<grid, kPersistentThreads, smem, s>>>(dp);
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

int persistent_blocks_per_sm(int dtype) {
    const size_t smem = persistent_smem_bytes(dtype);
    int n = 0;
    cudaError_t e;
    if (dtype == QT_C128) {
        e = cudaFuncSetAttribute(k_persistent<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<double>, kPersistentThreads, smem);
    } else {
        e = cudaFuncSetAttribute(k_persistent<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<float>, kPersistentThreads, smem);
    }
    return e == cudaSuccess && n > 0 ? n : 0;
}

}  // namespace qt
