// Contraction of caller-supplied tensors over binary indices: the paper's
// "tncontract" benchmark expression (§II-E), out[K] = sum over the labels not
// in K of the product of the operands, run by the bucket-elimination kernel of
// the energy plans (§II-B, merged eliminations §II-C).
//
//  k_permute_in      a caller's tensor (interleaved complex, C order over its
//                    labels) into the arena's layout: index bits in elimination
//                    rank (the summed labels lowest), entries in planar pairs
//  k_persistent      the plan's chain of buckets (kernels.cu)
//  k_out_interleave  the last result (the output's labels in the output's bit
//                    order) to the caller's interleaved complex array
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/qt.h"
#include "device_common.cuh"
#include "kernels.hpp"
#include "planner.hpp"

namespace qt {
namespace {

constexpr int kPermTileBits = 5;  // the low bits on either side that one permuting tile covers
constexpr int kPermThreads = 256;

// One caller tensor's permuting copy. A tile holds the 2^tbits elements that
// differ only in the tensor's internal bits 0..4 and in the internal bits that
// come from the caller's bits 0..4; one block per value of the other bits (hbits
// of them). Tile elements are numbered two ways: in the caller's bit order
// (e_usr, for coalesced reads) and in the internal bit order (e_int, for
// coalesced writes).
struct PermDesc {
    const void* src;        // the caller's tensor
    uint64_t dst_off;       // element offset of its copy in the arena
    const uint32_t* uoff;   // per e_usr: the element's offset within the tile, caller's index
    const uint16_t* sidx;   // per e_usr: its e_int
    const uint32_t* joff;   // per e_int: its offset within the tile, internal index
    uint32_t tbits, hbits;
    uint8_t hint[32];       // the block's bits: internal positions,
    uint8_t huser[32];      // and the caller's
};

template <typename R>
__global__ void __launch_bounds__(kPermThreads) k_permute_in(PermDesc pd, typename CT<R>::c* arena) {
    using C = typename CT<R>::c;
    extern __shared__ __align__(16) unsigned char perm_smem[];
    C* tile = reinterpret_cast<C*>(perm_smem);
    const uint32_t ntile = 1u << pd.tbits;
    uint64_t bi = 0, bu = 0;
    for (uint32_t h = 0; h < pd.hbits; ++h)
        if ((blockIdx.x >> h) & 1u) {
            bi |= 1ull << pd.hint[h];
            bu |= 1ull << pd.huser[h];
        }
    const C* src = static_cast<const C*>(pd.src) + bu;
    for (uint32_t e = threadIdx.x; e < ntile; e += blockDim.x) tile[__ldg(pd.sidx + e)] = __ldg(src + __ldg(pd.uoff + e));
    __syncthreads();
    // internal bit 0 is a tile bit (e_int bit 0), so e_int and e_int + 1 form a pair
    C* dst = arena + pd.dst_off + bi;
    for (uint32_t e = 2u * threadIdx.x; e < ntile; e += 2u * blockDim.x) {
        const uint32_t j = __ldg(pd.joff + e);
        C* p = dst + j;
        if constexpr (sizeof(R) == 4) {
            *reinterpret_cast<float4*>(p) = pack_pair(tile[e], tile[e + 1]);
        } else {
            p[0] = make_double2(tile[e].x, tile[e + 1].x);
            p[1] = make_double2(tile[e].y, tile[e + 1].y);
        }
    }
}

// The result (n elements, planar pairs) to the caller's interleaved array.
template <typename R>
__global__ void k_out_interleave(const typename CT<R>::c* res, uint64_t n, typename CT<R>::c* out) {
    using C = typename CT<R>::c;
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (n == 1) {
        if (i == 0) out[0] = elem_ld(res, 0);
        return;
    }
    if (2 * i >= n) return;
    const C* p = res + 2 * i;
    if constexpr (sizeof(R) == 4) {
        const Pair<float2> v = unpack_pair(__ldg(reinterpret_cast<const float4*>(p)));
        *reinterpret_cast<float4*>(out + 2 * i) = make_float4(v.v0.x, v.v0.y, v.v1.x, v.v1.y);
    } else {
        const Pair<double2> v = unpack_pair(__ldg(p), __ldg(p + 1));
        out[2 * i] = v.v0;
        out[2 * i + 1] = v.v1;
    }
}

// Host side of one tensor's permuting copy: its tile tables.
struct PermHost {
    uint32_t tbits = 0, hbits = 0;
    std::vector<uint32_t> uoff, joff;
    std::vector<uint16_t> sidx;
    uint8_t hint[32] = {}, huser[32] = {};
};

PermHost perm_tables(const std::vector<uint8_t>& src_bit) {
    PermHost ph;
    const int r = (int)src_bit.size();
    std::vector<int> T, H;  // internal bit positions
    for (int k = 0; k < r; ++k)
        (k < kPermTileBits || src_bit[k] < kPermTileBits ? T : H).push_back(k);
    ph.tbits = (uint32_t)T.size();
    ph.hbits = (uint32_t)H.size();
    for (size_t h = 0; h < H.size(); ++h) {
        ph.hint[h] = (uint8_t)H[h];
        ph.huser[h] = src_bit[H[h]];
    }
    std::vector<int> Tu(T.size());  // tile bits in the caller's bit order (indices into T)
    for (size_t q = 0; q < T.size(); ++q) Tu[q] = (int)q;
    std::sort(Tu.begin(), Tu.end(), [&](int a, int b) { return src_bit[T[a]] < src_bit[T[b]]; });
    const uint32_t n = 1u << ph.tbits;
    ph.uoff.resize(n);
    ph.sidx.resize(n);
    ph.joff.resize(n);
    for (uint32_t e = 0; e < n; ++e) {
        uint32_t ei = 0, uo = 0, jo = 0;
        for (size_t q = 0; q < T.size(); ++q) {
            if ((e >> q) & 1u) {
                ei |= 1u << Tu[q];
                uo |= 1u << src_bit[T[Tu[q]]];
                jo |= 1u << T[q];
            }
        }
        ph.sidx[e] = (uint16_t)ei;
        ph.uoff[e] = uo;
        ph.joff[e] = jo;
    }
    return ph;
}

#define QTC_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return qt::report_cuda_error(e_, "contract.cu", #call, __LINE__); \
    } while (0)

}  // namespace
}  // namespace qt

struct qt_contract_s {
    qt::ContractPlan cp;
    int device = 0;
    int grid = 0;
    size_t esize = 8;
    void* d_arena = nullptr;
    void* d_static = nullptr;
    void* d_counters = nullptr;
    size_t counters_bytes = 0;
    int32_t* h_err = nullptr;
    qt::DevPlan dp{};
    std::vector<qt::PermHost> perm;
    std::vector<qt::PermDesc> pd;  // device table pointers filled in; src set per run
    ~qt_contract_s() {
        if (d_arena || d_static || d_counters || h_err) cudaSetDevice(device);
        if (d_arena) cudaFree(d_arena);
        if (d_static) cudaFree(d_static);
        if (d_counters) cudaFree(d_counters);
        if (h_err) cudaFreeHost(h_err);
    }
};

namespace {

template <typename T>
size_t bytes_of(const std::vector<T>& v) {
    return v.size() * sizeof(T);
}

int contract_upload(qt_contract_t C) {
    using namespace qt;
    const ContractPlan& cp = C->cp;
    QTC_CUDA(cudaGetDevice(&C->device));
    const size_t arena_bytes = (size_t)cp.arena_elems * C->esize;
    size_t free_b = 0, total_b = 0;
    QTC_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (arena_bytes + (256u << 20) > free_b) return QT_ENOMEM;
    QTC_CUDA(cudaMalloc(&C->d_arena, std::max<size_t>(arena_bytes, 256)));
    // static arrays: buckets, operands, groups, then each input's tile tables
    struct Piece {
        const void* src;
        size_t bytes;
        size_t off;
    };
    std::vector<Piece> pieces = {{cp.buckets.data(), bytes_of(cp.buckets), 0},
                                 {cp.operands.data(), bytes_of(cp.operands), 0},
                                 {cp.runs.data(), bytes_of(cp.runs), 0}};
    for (const PermHost& ph : C->perm) {
        pieces.push_back({ph.uoff.data(), bytes_of(ph.uoff), 0});
        pieces.push_back({ph.sidx.data(), bytes_of(ph.sidx), 0});
        pieces.push_back({ph.joff.data(), bytes_of(ph.joff), 0});
    }
    size_t total = 0;
    for (auto& pc : pieces) {
        pc.off = total;
        total += (pc.bytes + 255) / 256 * 256;
    }
    QTC_CUDA(cudaMalloc(&C->d_static, std::max<size_t>(total, 256)));
    std::vector<char> staging(total);
    for (auto& pc : pieces)
        if (pc.bytes) std::memcpy(staging.data() + pc.off, pc.src, pc.bytes);
    QTC_CUDA(cudaMemcpy(C->d_static, staging.data(), total, cudaMemcpyHostToDevice));
    char* base = static_cast<char*>(C->d_static);
    const uint32_t nb = (uint32_t)cp.buckets.size();
    const size_t ctl_bytes = 256;
    C->counters_bytes = ctl_bytes + ((size_t)2 * nb * sizeof(uint32_t) + 255) / 256 * 256;
    QTC_CUDA(cudaMalloc(&C->d_counters, C->counters_bytes));
    QTC_CUDA(cudaMemset(C->d_counters, 0, C->counters_bytes));
    QTC_CUDA(cudaHostAlloc((void**)&C->h_err, 2 * sizeof(int32_t), cudaHostAllocDefault));
    C->h_err[0] = C->h_err[1] = 0;
    DevPlan& dp = C->dp;
    dp.buckets = reinterpret_cast<const DBucket*>(base + pieces[0].off);
    dp.ops = reinterpret_cast<const DOperand*>(base + pieces[1].off);
    dp.runs = reinterpret_cast<const DRun*>(base + pieces[2].off);
    dp.n_static = dp.n_groups = (uint32_t)cp.runs.size();
    dp.n_buckets = nb;
    dp.slots = nullptr;  // static order only: nothing is published at run time
    char* cbase = static_cast<char*>(C->d_counters);
    dp.ctl = reinterpret_cast<DControl*>(cbase);
    dp.tiles_done = reinterpret_cast<uint32_t*>(cbase + ctl_bytes);
    dp.prod_done = dp.tiles_done + nb;
    dp.arena = C->d_arena;
    dp.spin_limit = 1ull << 23;
    dp.trace = nullptr;
    dp.isolated = 0;
    dp.bucket_times = nullptr;
    dp.unit_prog = nullptr;
    dp.has_units = 0;
    for (size_t t = 0; t < C->perm.size(); ++t) {
        const PermHost& ph = C->perm[t];
        PermDesc d{};
        d.dst_off = cp.in_off[t];
        d.uoff = reinterpret_cast<const uint32_t*>(base + pieces[3 + 3 * t].off);
        d.sidx = reinterpret_cast<const uint16_t*>(base + pieces[4 + 3 * t].off);
        d.joff = reinterpret_cast<const uint32_t*>(base + pieces[5 + 3 * t].off);
        d.tbits = ph.tbits;
        d.hbits = ph.hbits;
        std::memcpy(d.hint, ph.hint, sizeof(d.hint));
        std::memcpy(d.huser, ph.huser, sizeof(d.huser));
        C->pd.push_back(d);
    }
    int sms = 0;
    QTC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C->device));
    const int per_sm = persistent_blocks_per_sm(cp.dtype);
    if (per_sm <= 0) return QT_ECUDA;
    C->grid = sms * per_sm;
    return QT_OK;
}

template <typename R>
int contract_launch(qt_contract_t C, const void* const* ops, void* out, cudaStream_t s) {
    using namespace qt;
    using Cx = typename CT<R>::c;
    const ContractPlan& cp = C->cp;
    for (size_t t = 0; t < C->pd.size(); ++t) {
        PermDesc d = C->pd[t];
        d.src = ops[t];
        const size_t smem = ((size_t)1 << d.tbits) * sizeof(Cx);
        k_permute_in<R><<<1u << d.hbits, kPermThreads, smem, s>>>(d, static_cast<Cx*>(C->d_arena));
        QTC_CUDA(cudaGetLastError());
    }
    QTC_CUDA(cudaMemsetAsync(C->d_counters, 0, C->counters_bytes, s));
    QTC_CUDA(launch_persistent(cp.dtype, C->grid, C->dp, s));
    const uint64_t n = 1ull << cp.out_rank;
    const uint64_t threads = n == 1 ? 1 : n / 2;
    k_out_interleave<R><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        static_cast<const Cx*>(C->d_arena) + cp.out_off, n, static_cast<Cx*>(out));
    QTC_CUDA(cudaGetLastError());
    QTC_CUDA(cudaMemcpyAsync(C->h_err, &C->dp.ctl->error, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return QT_OK;
}

}  // namespace

extern "C" {

int qt_contract_plan(int32_t n_ops, const int32_t* ranks, const int32_t* labels, int32_t out_rank,
                     const int32_t* out_labels, qt_dtype dtype, int32_t host_only, qt_contract_t* out) {
    if (!out || n_ops < 1 || n_ops > 16 || !ranks || !labels || out_rank < 0 || (out_rank > 0 && !out_labels))
        return QT_EINVAL;
    if (dtype != QT_C64 && dtype != QT_C128) return QT_EINVAL;
    *out = nullptr;
    std::vector<std::vector<int>> ls(n_ops);
    size_t k = 0;
    for (int t = 0; t < n_ops; ++t) {
        if (ranks[t] < 1 || ranks[t] > 30) return QT_EINVAL;
        ls[t].assign(labels + k, labels + k + ranks[t]);
        k += (size_t)ranks[t];
    }
    std::vector<int> ol(out_labels, out_labels + out_rank);
    std::unique_ptr<qt_contract_s> C(new (std::nothrow) qt_contract_s());
    if (!C) return QT_ENOMEM;
    C->esize = dtype == QT_C128 ? 16 : 8;
    int sms = 152, dev = 0;
    if (!host_only && cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    int rc;
    try {
        rc = qt::build_contract_plan(ls, ol, dtype, sms * 4 * (dtype == QT_C128 ? 2 : 3), &C->cp);
        if (rc == QT_OK)
            for (const auto& sb : C->cp.in_src_bit) C->perm.push_back(qt::perm_tables(sb));
    } catch (const std::bad_alloc&) {
        return QT_ENOMEM;
    }
    if (rc != QT_OK) return rc;
    if (!host_only) {
        rc = contract_upload(C.get());
        if (rc != QT_OK) return rc;
    }
    *out = C.release();
    return QT_OK;
}

int qt_contract_run(qt_contract_t C, const void* const* ops, void* out, void* cuda_stream) {
    if (!C || !ops || !out) return QT_EINVAL;
    if (!C->d_arena) return QT_ESTATE;  // a host-only plan
    for (size_t t = 0; t < C->cp.in_rank.size(); ++t)
        if (!ops[t]) return QT_EINVAL;
    QTC_CUDA(cudaSetDevice(C->device));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int rc = C->cp.dtype == QT_C128 ? contract_launch<double>(C, ops, out, s) : contract_launch<float>(C, ops, out, s);
    if (rc != QT_OK || cuda_stream) return rc;
    return qt_contract_sync(C, nullptr);
}

int qt_contract_sync(qt_contract_t C, void* cuda_stream) {
    if (!C) return QT_EINVAL;
    if (!C->d_arena) return QT_ESTATE;
    QTC_CUDA(cudaSetDevice(C->device));
    QTC_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    const int32_t err = C->h_err[0];
    C->h_err[0] = 0;
    return err;
}

int qt_contract_stats_get(qt_contract_t C, qt_contract_stats* out) {
    if (!C || !out) return QT_EINVAL;
    const qt::ContractPlan& cp = C->cp;
    std::memset(out, 0, sizeof(*out));
    out->n_buckets = (int32_t)cp.buckets.size();
    out->max_width = cp.max_width;
    out->n_summed = cp.n_summed;
    for (const qt::DBucket& d : cp.buckets) out->n_merged += qt::bucket_n_sum(d.flags) > 1;
    out->alg_bytes = cp.alg_bytes;
    double io = 0;
    for (int r : cp.in_rank) io += 2.0 * std::ldexp(1.0, r);  // each input read, and written permuted
    io += 2.0 * std::ldexp(1.0, cp.out_rank);                  // the result read, the output written
    out->copy_bytes = io * (double)C->esize;
    out->arena_bytes = (int64_t)(cp.arena_elems * C->esize);
    for (size_t b = 0; b < cp.widths.size() && b < 32; ++b) out->widths[b] = cp.widths[b];
    return QT_OK;
}

void qt_contract_free(qt_contract_t C) {
    if (!C) return;
    if (C->d_arena) {
        cudaSetDevice(C->device);
        cudaDeviceSynchronize();
    }
    delete C;
}

}  // extern "C"
