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

// Bounded wait until `need` producers of a bucket have finished. Gives up
// after `limit` polls (each followed by a short sleep) or as soon as another
// warp has reported an error; returns 0 then.
__device__ int wait_deps(const uint32_t* ctr, uint32_t need, uint64_t limit, DControl* ctl, uint32_t b) {
    uint64_t polls = 0;
    while (ld_acquire(ctr) < need) {
        if (ld_volatile(&ctl->error) != 0) return 0;
        if (++polls > limit) {
            if (atomicCAS(&ctl->error, 0, QT_ETIMEOUT) == 0) ctl->err_bucket = b;
            return 0;
        }
        __nanosleep(100);
    }
    return 1;
}

template <typename R>
__global__ void __launch_bounds__(kPersistentThreads) k_persistent(DevPlan dp) {
    using C = typename CT<R>::c;
    __shared__ OpStage s_ops[kWarps][kMaxOps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* arena = static_cast<C*>(dp.arena);
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = ld_volatile(&dp.ctl->error) != 0 ? dp.n_items : atomicAdd(&dp.ctl->next_item, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= dp.n_items) return;
        const uint32_t t_end = dp.item_begin[item + 1];
        for (uint32_t t = dp.item_begin[item]; t < t_end; ++t) {
            const uint32_t b = dp.task_bucket[t];
            const uint32_t chunk = dp.task_chunk[t];
            const DBucket B = dp.buckets[b];
            if (B.n_deps) {
                int ok = 1;
                if (lane == 0) ok = wait_deps(&dp.deps_done[b], B.n_deps, dp.spin_limit, dp.ctl, b);
                ok = __shfl_sync(kFull, ok, 0);
                if (!ok) return;
            }
            stage_ops(B, chunk, dp.ops, s_ops[warp], lane);
            __syncwarp();
            contract_tile<R>(B, chunk, s_ops[warp], arena, lane);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                const uint32_t prev = atomicAdd(&dp.chunks_done[b], 1u);
                if (prev + 1u == B.n_tasks && B.parent != kNone) {
                    __threadfence();
                    atomicAdd(&dp.deps_done[B.parent], 1u);
                }
            }
            __syncwarp();
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

cudaError_t launch_persistent(int dtype, int grid, const DevPlan& dp, cudaStream_t s) {
    if (dtype == QT_C128)
        k_persistent<double><<<grid, kPersistentThreads, 0, s>>>(dp);
    else
        k_persistent<float><<<grid, kPersistentThreads, 0, s>>>(dp);
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
    int n = 0;
    cudaError_t e = dtype == QT_C128
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<double>, kPersistentThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<float>, kPersistentThreads, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

}  // namespace qt
