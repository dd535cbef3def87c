// CUDA kernels of the reverse sweep (the adjoint of bucket elimination) on
// sm_103a: root seeding, one launch per level and operand-count class of
// k_backward, zeroing of atomically updated cotangents, and the final scaling.
#include <cuda_runtime.h>

#include "../../include/qt.h"
#include "device_common.cuh"
#include "kernels.hpp"

namespace qt {
namespace {

// ---------------------------------------------------------------------------
// Reverse sweep (the adjoint of bucket elimination).
//
// A network's value V is a polynomial in the gate entries, so dV/dtheta =
// sum over gate tensors g and entries i of (dV/dT_g[i]) (dT_g[i]/dtheta). The
// cotangent of bucket b's result, Rbar, is complete once b's consumer has
// been swept; the cotangent contribution to operand s from output o and
// summed value x is Rbar[o] * prod_{t != s} T_t[2 pext(o, M_t) + x]. Results
// of earlier buckets receive these contributions in their cotangent buffers
// (atomically, since several outputs may share an entry); gate tensors turn
// them at once into Re(contribution * dT_g/dtheta), summed per parameter.
// E = |E|/2 - 1/2 sum Re V, so dE/dtheta = -1/2 times those sums.
// ---------------------------------------------------------------------------

// The seeds of one network (one thread): its value is the sum over its
// slices of the product of the slice's factors -- root results and the gate
// entries slicing fixed (one slice, with root results only, when unsliced).
// A root's cotangent is the product of its slice's other factors; a fixed
// entry of an angle's gate adds Re(product of the other factors x the entry's
// derivative) to that angle's sum. Both carry the network's weight: the
// networks sharing its value (deduplicated plans; 1 otherwise), 0 for a
// duplicate, which has no buckets of its own.
template <typename R>
__global__ void k_seed_roots(DevEpilogue de, int n_nets, uint64_t cot_delta, uint64_t dleaf_delta, double* grad,
                             int p, const uint32_t* net_graph) {
    using C = typename CT<R>::c;
    C* arena = static_cast<C*>(const_cast<void*>(de.arena));
    const int net = blockIdx.x * blockDim.x + threadIdx.x;
    if (net >= n_nets) return;
    const double w = de.net_weight ? (double)de.net_weight[net] : 1.0;
    if (w == 0.0) return;
    const uint32_t f0 = de.net_first_factor[net], f1 = de.net_first_factor[net + 1];
    double* g = grad + (size_t)net_graph[net] * 2 * p;
    for (uint32_t a = f0; a < f1;) {
        uint32_t b = a + 1;  // the slice's factors are [a, b)
        while (b < f1 && !(de.factor[b] & kFirstFactor)) ++b;
        for (uint32_t j = a; j < b; ++j) {
            const int8_t kind = de.factor_param[j];
            if (kind == -1) continue;  // a fixed entry of |+> or Z: no angle
            double vr = w, vi = 0.0;  // the product of the other factors
            for (uint32_t k = a; k < b; ++k) {
                if (k == j) continue;
                const C v = elem_ld(arena, de.factor[k] & ~kFirstFactor);
                const double nr = vr * (double)v.x - vi * (double)v.y, ni = vr * (double)v.y + vi * (double)v.x;
                vr = nr;
                vi = ni;
            }
            const uint64_t off = de.factor[j] & ~kFirstFactor;
            if (kind == kFactorRoot) {
                C c;
                c.x = (R)vr;
                c.y = (R)vi;
                elem_st(arena, off + cot_delta, c);
            } else {
                const C d = elem_ld(arena, off + dleaf_delta);
                atomicAdd(g + kind, vr * (double)d.x - vi * (double)d.y);
            }
        }
        a = b;
    }
}

constexpr int kBwdWarps = 4;  // warps per block of the reverse sweep, one (bucket, tile) task each

// One tile (2^tb outputs, tb = min(n_out, kBwdTileBits)) of one bucket's
// reverse sweep, by one warp. Lane l takes outputs o = obase + l + 32 k. For
// each output it forms, for both x at once, c_s = Rbar[o] prod_{t != s}
// T_t[2 pext(o, M_t) + x] and hands it to operand s by its mode. An operand's
// pair index pext(o, M) is split, as in the forward tile loop, into the
// tile's part (once per task), the lane's part and the steps of the iteration
// bits, so no output pays for a bit-by-bit extract.
//
// An operand's entry pair (x = 0, 1) is one value of BwdMath<R>::P: complex64
// holds it as packed real and packed imaginary parts (f32x2), as it is stored
// (planar pairs), so one packed complex product serves both x; complex128
// holds the two entries and multiplies each in FP64. A value that does not
// depend on x (the result's cotangent, the merged consumer's gate entries) is
// repeated for both x. The products of the other operands take 3n - 4 pair
// products per output (prefix times suffix; none by the identity). In-tile
// sums go to the warp's shared buffer with plain read-add-writes: after the
// shuffles, the lanes left own distinct entries (they differ in a bit the
// operand carries), in every iteration. Gate sums are compensated per x and
// lane in complex64 (FP32), plain in complex128, then reduced in FP64.
struct PC {
    f32x2 re, im;
};
template <typename R>
struct BwdMath;
template <>
struct BwdMath<float> {
    using P = PC;
    using RP = f32x2;  // a real value per x
    static __device__ __forceinline__ P mul(P a, P b) {
        return {x2_fma(a.re, b.re, x2_neg(x2_mul(a.im, b.im))), x2_fma(a.re, b.im, x2_mul(a.im, b.re))};
    }
    static __device__ __forceinline__ P splat(float2 v) { return {x2_pack(v.x, v.x), x2_pack(v.y, v.y)}; }
    static __device__ __forceinline__ P ldg(const float2* p) {  // read-only path
        P r;
        asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(r.re), "=l"(r.im) : "l"(p));
        return r;
    }
    static __device__ __forceinline__ void stg(float2* p, P v) {
        asm volatile("st.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(v.re), "l"(v.im) : "memory");
    }
    static __device__ __forceinline__ void sadd(float2* p, P v) {  // shared memory
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
        f32x2 re, im;
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(re), "=l"(im) : "r"(a) : "memory");
        re = x2_add(re, v.re);
        im = x2_add(im, v.im);
        asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(a), "l"(re), "l"(im) : "memory");
    }
    static __device__ __forceinline__ P shfl_add(P v, int m) {
        return {x2_add(v.re, __shfl_xor_sync(kFull, v.re, m)), x2_add(v.im, __shfl_xor_sync(kFull, v.im, m))};
    }
    static __device__ __forceinline__ RP re_prod(P c, P d) { return x2_fma(c.re, d.re, x2_neg(x2_mul(c.im, d.im))); }
    static __device__ __forceinline__ RP add(RP a, RP b) { return x2_add(a, b); }
    static __device__ __forceinline__ RP sub(RP a, RP b) { return x2_add(a, x2_neg(b)); }
    static __device__ __forceinline__ double sum(RP a) { return (double)x2_lo(a) + (double)x2_hi(a); }
    static __device__ __forceinline__ float2 at(P v, int x) {
        return x ? make_float2(x2_hi(v.re), x2_hi(v.im)) : make_float2(x2_lo(v.re), x2_lo(v.im));
    }
    static __device__ __forceinline__ P zero() { return {0ull, 0ull}; }
    static __device__ __forceinline__ RP rzero() { return 0ull; }
};
template <>
struct BwdMath<double> {
    using P = Pair<double2>;
    using RP = double2;
    static __device__ __forceinline__ P mul(P a, P b) { return {cmul(a.v0, b.v0), cmul(a.v1, b.v1)}; }
    static __device__ __forceinline__ P splat(double2 v) { return {v, v}; }
    static __device__ __forceinline__ P ldg(const double2* p) { return unpack_pair(__ldg(p), __ldg(p + 1)); }
    static __device__ __forceinline__ void stg(double2* p, P v) {
        p[0] = make_double2(v.v0.x, v.v1.x);
        p[1] = make_double2(v.v0.y, v.v1.y);
    }
    static __device__ __forceinline__ void sadd(double2* p, P v) {  // shared memory
        double2 re = p[0], im = p[1];
        re.x += v.v0.x;
        re.y += v.v1.x;
        im.x += v.v0.y;
        im.y += v.v1.y;
        p[0] = re;
        p[1] = im;
    }
    static __device__ __forceinline__ double2 shfl2(double2 v, int m) {
        return make_double2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
    }
    static __device__ __forceinline__ P shfl_add(P v, int m) { return {cadd(v.v0, shfl2(v.v0, m)), cadd(v.v1, shfl2(v.v1, m))}; }
    static __device__ __forceinline__ RP re_prod(P c, P d) {
        return make_double2(c.v0.x * d.v0.x - c.v0.y * d.v0.y, c.v1.x * d.v1.x - c.v1.y * d.v1.y);
    }
    static __device__ __forceinline__ RP add(RP a, RP b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ RP sub(RP a, RP b) { return make_double2(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ double sum(RP a) { return a.x + a.y; }
    static __device__ __forceinline__ double2 at(P v, int x) { return x ? v.v1 : v.v0; }
    static __device__ __forceinline__ P zero() { return {double2{0.0, 0.0}, double2{0.0, 0.0}}; }
    static __device__ __forceinline__ RP rzero() { return double2{0.0, 0.0}; }
};

// 16-byte asynchronous copies global -> shared (no registers), and the wait
// for all of this thread's.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename R, int NMAX, bool Exact>
__device__ void bwd_tile(const DevBwd& db, uint32_t b, uint32_t tile, int lane, typename CT<R>::c* red) {
    using C = typename CT<R>::c;
    using M = BwdMath<R>;
    using P = typename M::P;
    using RP = typename M::RP;
    constexpr int KB = kBwdTileBits - 5;  // iteration bits at most
    C* arena = static_cast<C*>(db.arena);
    const DBucket B = db.buckets[b];
    const int n = Exact ? NMAX : (int)B.n_ops;
    const int tb = min((int)B.n_out, kBwdTileBits);
    const int kb = tb > 5 ? tb - 5 : 0;
    const uint32_t low = (1u << tb) - 1u;
    const uint32_t lmask = low & 31u;
    const bool active = ((uint32_t)lane & ~lmask) == 0u;
    const uint32_t obase = tile << tb;
    const C* rbar = arena + B.out_off + db.cot_delta;
    const uint32_t rshift = bucket_n_sum(B.flags) - 1;  // a merged bucket's outputs (o, s1) share result o
    // operand t: with x, opp = its pair base[t] (the tile's block, pair-aligned);
    // without x (gates), opp = the tensor's first entry and nb = base[t]
    C* opp[NMAX];
    uint32_t nb[NMAX], mask[NMAX], lo[NMAX], step[NMAX][KB], roff[NMAX];
    bool px[NMAX];
    int mode[NMAX], prm[NMAX];
    uint32_t red_elems = 0;
#pragma unroll
    for (int t = 0; t < NMAX; ++t) {
        opp[t] = arena;
        nb[t] = mask[t] = lo[t] = roff[t] = 0;
        px[t] = true;
        mode[t] = kBwdNone;
        prm[t] = -1;
#pragma unroll
        for (int k = 0; k < KB; ++k) step[t][k] = 0;
        if (t < n) {
            const uint32_t i = B.op_begin + t;
            const DOperand o = db.ops[i];
            mask[t] = o.mask;
            px[t] = (o.smask & 1u) != 0u;
            mode[t] = db.op_bwd[i];
            prm[t] = db.op_param[i];
            roff[t] = db.op_roff[i];
            const uint32_t base = pext_u32(obase, o.mask);
            opp[t] = arena + o.off + (px[t] ? 2ull * base : 0ull);
            nb[t] = px[t] ? 0u : base;
            lo[t] = pext_u32((uint32_t)lane & lmask, o.mask & lmask);
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                const int bit = 5 + k;
                step[t][k] = (k < kb && ((o.mask >> bit) & 1u)) ? (1u << __popc(o.mask & ((1u << bit) - 1u))) : 0u;
            }
            if (mode[t] == kBwdRedStore || mode[t] == kBwdRedAtomic)
                red_elems = max(red_elems, roff[t] + (2u << __popc(o.mask & low)));
        }
    }
    for (uint32_t e = lane; e < red_elems; e += 32) red[e] = C{};
    // The tile's entries of the result's cotangent (at least one pair; the
    // block starts on a pair: obase >> rshift is even or 0), copied once into
    // the buffer's unused end when it fits, instead of a global load in every
    // iteration below.
    const uint32_t rcount = max(2u, (1u << tb) >> rshift);
    const bool rstaged = red_elems + rcount <= (uint32_t)kBwdRedElems;
    C* const rsm = red + red_elems;  // red_elems is even: pair-aligned
    if (rstaged) {
        const char* src = reinterpret_cast<const char*>(rbar + (obase >> rshift));
        char* dst = reinterpret_cast<char*>(rsm);
        const uint32_t chunks = rcount * (uint32_t)sizeof(C) / 16u;
        for (uint32_t i = (uint32_t)lane; i < chunks; i += 32u) cp_async16(dst + 16u * i, src + 16u * i);
        cp_async_wait_all();
    }
    __syncwarp();
    RP acc[NMAX], comp[NMAX];  // compensated sums of Re(c dT), per x
#pragma unroll
    for (int t = 0; t < NMAX; ++t) acc[t] = comp[t] = M::rzero();
    const uint64_t dld = db.dleaf_delta, cot = db.cot_delta;
    for (uint32_t k = 0; k < (1u << kb); ++k) {
        const uint32_t o = obase + (k << 5) + ((uint32_t)lane & lmask);
        P r = M::zero();
        if (active) r = M::splat(rstaged ? elem_ld(rsm, (o - obase) >> rshift) : elem_ldg(rbar, o >> rshift));
        P v[NMAX];
        uint32_t li[NMAX];
#pragma unroll
        for (int t = 0; t < NMAX; ++t) {
            uint32_t q = lo[t];
#pragma unroll
            for (int kk = 0; kk < KB; ++kk)
                if ((k >> kk) & 1u) q += step[t][kk];
            li[t] = q;
            if (t < n) v[t] = px[t] ? M::ldg(opp[t] + 2u * q) : M::splat(elem_ldg(opp[t], nb[t] + q));
        }
        // suffix products suf[t] = prod_{u > t} v[u] (none for the last operand)
        P suf[NMAX];
#pragma unroll
        for (int t = NMAX - 2; t >= 0; --t) {
            if (t < n - 1) suf[t] = (t == n - 2) ? v[t + 1] : M::mul(v[t + 1], suf[t + 1]);
        }
        P pre = r;
#pragma unroll
        for (int t = 0; t < NMAX; ++t) {
            if (t < n) {
                const int md = mode[t];
                if (md != kBwdNone) {
                    const P c = (t == n - 1) ? pre : M::mul(pre, suf[t]);  // Rbar[o] prod_{u != t} v[u]
                    if (md == kBwdGate) {
                        const P d = px[t] ? M::ldg(opp[t] + dld + 2u * li[t]) : M::splat(elem_ldg(opp[t] + dld, nb[t] + li[t]));
                        if (sizeof(R) == 8) {
                            // FP64: a lane's few hundred terms need no compensation
                            acc[t] = M::add(acc[t], M::re_prod(c, d));
                        } else {
                            const RP y = M::sub(M::re_prod(c, d), comp[t]);
                            const RP s2 = M::add(acc[t], y);
                            comp[t] = M::sub(M::sub(s2, acc[t]), y);
                            acc[t] = s2;
                        }
                    } else if (md == kBwdDirect) {
                        if (active) M::stg(opp[t] + cot + 2u * li[t], c);
                    } else if (md == kBwdRedStore || md == kBwdRedAtomic) {
                        // lanes that differ only in bits the operand lacks
                        // add to the same entry: sum them by shuffles first
                        P w = c;
                        const uint32_t miss = lmask & ~mask[t];
#pragma unroll
                        for (int i = 0; i < 5; ++i)
                            if ((miss >> i) & 1u) w = M::shfl_add(w, 1 << i);
                        if (active && ((uint32_t)lane & miss) == 0u) M::sadd(red + roff[t] + 2u * li[t], w);
                    } else if (md == kBwdAtomic) {
                        if (active) {
                            elem_atomic_add(opp[t] + cot, 2ull * li[t], M::at(c, 0));
                            elem_atomic_add(opp[t] + cot, 2ull * li[t] + 1, M::at(c, 1));
                        }
                    }
                }
                if (t < n - 1) pre = M::mul(pre, v[t]);
            }
        }
    }
    __syncwarp();
    // in-tile sums (planar pairs, as stored): the operand's entries for this
    // tile are one contiguous block
#pragma unroll
    for (int t = 0; t < NMAX; ++t) {
        if (t < n && (mode[t] == kBwdRedStore || mode[t] == kBwdRedAtomic)) {
            const uint32_t fp = 2u << __popc(mask[t] & low);
            C* dst = opp[t] + cot;
            const C* src = red + roff[t];
            for (uint32_t e = lane; e < fp; e += 32) {
                if (mode[t] == kBwdRedStore)
                    elem_st(dst, e, elem_ld(src, e));
                else
                    elem_atomic_add(dst, e, elem_ld(src, e));
            }
        }
    }
    const uint32_t g = db.net_graph[B.net];
#pragma unroll
    for (int t = 0; t < NMAX; ++t) {
        if (t < n && mode[t] == kBwdGate) {
            double s2 = M::sum(acc[t]) - M::sum(comp[t]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s2 += __shfl_xor_sync(kFull, s2, d);
            if (lane == 0) atomicAdd(&db.grad[(size_t)g * 2 * db.p + prm[t]], s2);
        }
    }
}

// One launch per level and operand-count class (buckets of at most NMAX
// operands), so that each instantiation keeps its own register budget.
// Blocks per SM at least: complex64 4 (3 for more than four operands: 2),
// complex128 3 (its 64 KB of shared memory per block allow no more), 2.
template <typename R, int NMAX, bool Exact>
__global__ void __launch_bounds__(kBwdWarps * 32, NMAX <= 4 ? (sizeof(R) == 4 ? 4 : 3) : 2) k_backward(DevBwd db) {
    using C = typename CT<R>::c;
    extern __shared__ __align__(16) unsigned char bwd_smem[];
    C* red = reinterpret_cast<C*>(bwd_smem) + (threadIdx.x >> 5) * kBwdRedElems;
    const uint32_t w = blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= db.n_tasks) return;
    bwd_tile<R, NMAX, Exact>(db, db.task_bucket[w], db.task_tile[w], lane, red);
}

// Zero the cotangent pieces that receive atomic adds: (offset, count) pairs,
// one block per piece (pieces are at most kZeroChunk elements).
template <typename R>
__global__ void k_zero_ranges(typename CT<R>::c* arena, const uint64_t* ranges, uint32_t n) {
    using C = typename CT<R>::c;
    for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
        C* p = arena + ranges[2 * r];
        const uint32_t cnt = (uint32_t)ranges[2 * r + 1];
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) elem_st(p, i, C{});
    }
}

__global__ void k_grad_final(const double* grad, int n_graphs, int p, double* dgamma, double* dbeta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_graphs * p) return;
    const int g = i / p, k = i % p;
    dgamma[i] = -0.5 * grad[(size_t)g * 2 * p + k];
    dbeta[i] = -0.5 * grad[(size_t)g * 2 * p + p + k];
}

}  // namespace

cudaError_t launch_seed_roots(int dtype, const DevEpilogue& de, int n_nets, uint64_t cot_delta, uint64_t dleaf_delta,
                              double* grad, int p, const uint32_t* net_graph, cudaStream_t s) {
    if (n_nets == 0) return cudaSuccess;  // a plan of graphs without edges
    const int blocks = (n_nets + 127) / 128;
    if (dtype == QT_C128)
        k_seed_roots<double><<<blocks, 128, 0, s>>>(de, n_nets, cot_delta, dleaf_delta, grad, p, net_graph);
    else
        k_seed_roots<float><<<blocks, 128, 0, s>>>(de, n_nets, cot_delta, dleaf_delta, grad, p, net_graph);
    return cudaGetLastError();
}

template <typename R>
constexpr size_t bwd_smem() {
    return (size_t)kBwdWarps * kBwdRedElems * sizeof(typename CT<R>::c);
}

template <typename R, int NMAX, bool Exact>
static cudaError_t bwd_attr() {
    if (bwd_smem<R>() <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_backward<R, NMAX, Exact>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bwd_smem<R>());
}

template <typename R>
static cudaError_t prepare_bwd() {
    const cudaError_t es[] = {bwd_attr<R, 1, true>(), bwd_attr<R, 2, true>(), bwd_attr<R, 3, true>(),
                              bwd_attr<R, 4, true>(), bwd_attr<R, 5, true>(),  bwd_attr<R, 8, false>(),
                              bwd_attr<R, kMaxOps, false>()};
    for (cudaError_t e : es)
        if (e != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename R, int NMAX, bool Exact>
static cudaError_t launch_bwd(const DevBwd& db, cudaStream_t s) {
    const uint32_t blocks = (db.n_tasks + kBwdWarps - 1) / kBwdWarps;
    k_backward<R, NMAX, Exact><<<blocks, kBwdWarps * 32, bwd_smem<R>(), s>>>(db);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_bwd_class(int op_class, const DevBwd& db, cudaStream_t s) {
    switch (op_class) {
        case 0: return launch_bwd<R, 1, true>(db, s);
        case 1: return launch_bwd<R, 2, true>(db, s);
        case 2: return launch_bwd<R, 3, true>(db, s);
        case 3: return launch_bwd<R, 4, true>(db, s);
        case 4: return launch_bwd<R, 5, true>(db, s);
        case 5: return launch_bwd<R, 8, false>(db, s);
        default: return launch_bwd<R, kMaxOps, false>(db, s);
    }
}

cudaError_t launch_backward(int dtype, int op_class, const DevBwd& db, cudaStream_t s) {
    if (db.n_tasks == 0) return cudaSuccess;
    return dtype == QT_C128 ? launch_bwd_class<double>(op_class, db, s) : launch_bwd_class<float>(op_class, db, s);
}

cudaError_t prepare_backward(int dtype) { return dtype == QT_C128 ? prepare_bwd<double>() : prepare_bwd<float>(); }

cudaError_t launch_zero_ranges(int dtype, void* arena, const uint64_t* ranges, uint32_t n_ranges, cudaStream_t s) {
    if (n_ranges == 0) return cudaSuccess;
    const uint32_t blocks = n_ranges < 65535u ? n_ranges : 65535u;
    if (dtype == QT_C128)
        k_zero_ranges<double><<<blocks, 256, 0, s>>>(static_cast<double2*>(arena), ranges, n_ranges);
    else
        k_zero_ranges<float><<<blocks, 256, 0, s>>>(static_cast<float2*>(arena), ranges, n_ranges);
    return cudaGetLastError();
}

cudaError_t launch_grad_final(const double* grad, int n_graphs, int p, double* dgamma, double* dbeta, cudaStream_t s) {
    const int n = n_graphs * p;
    k_grad_final<<<(n + 127) / 128, 128, 0, s>>>(grad, n_graphs, p, dgamma, dbeta);
    return cudaGetLastError();
}

}  // namespace qt
