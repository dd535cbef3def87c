// C ABI of libqtgb (declared in include/qt.h): plan ownership, device
// memory, the CUDA graph of one energy evaluation, and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/qt.h"
#include "kernels.hpp"
#include "planner.hpp"

namespace {

constexpr int kRing = 512;  // event pairs for per-launch kernel timing
constexpr int kAutoRestarts = 64;      // default randomised min-fill restarts of a wide network
constexpr int kAutoRestartWidth = 18;  // "wide": its plain greedy order reaches this bucket width

}  // namespace

struct qt_plan_s {
    qt::HostPlan hp;
    int device = 0;
    int dtype = QT_C64;
    int sched = QT_SCHED_PERSISTENT;
    uint64_t spin_limit = 1ull << 23;
    size_t esize = 8;

    // device memory
    void* d_arena = nullptr;
    size_t arena_bytes = 0;
    void* d_static = nullptr;  // plan arrays
    void* d_counters = nullptr;  // chunks_done | deps_done | control
    size_t counters_bytes = 0;
    qt::DevPlan dp{};
    qt::DevEpilogue de{};
    double* d_angles = nullptr;  // gammas (n_graphs*p) then betas (n_graphs*p)
    double* d_out = nullptr;     // zz | zz_imag | energies
    int32_t* h_err = nullptr;    // pinned copy of the kernel error word
    int grid = 0;

    // execution
    cudaStream_t stream = nullptr;  // internal stream (NULL-stream calls and graph capture)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_nodes[2] = {nullptr, nullptr};
    cudaEvent_t cap_ev[2] = {nullptr, nullptr};
    cudaEvent_t ring[kRing][2] = {};
    bool ring_pending[kRing] = {};
    uint64_t calls = 0;
    double time_ms = 0;
    int64_t timed = 0;
    bool err_pending = false;
    bool host_only = false;
    bool trace = false;
    uint64_t* d_trace = nullptr;
    unsigned long long* d_btimes = nullptr;
    // gradient plans
    void* d_bwd = nullptr;       // op_param | net_graph | backward task arrays
    double* d_grad = nullptr;    // n_graphs x 2p accumulators, then dgamma | dbeta
    const uint64_t* d_zero = nullptr;  // cotangent pieces zeroed before each reverse sweep (inside d_bwd)
    uint32_t n_zero = 0;
    qt::DevBwd db{};
    // the reverse sweep as one CUDA graph: within a level, the operand-count
    // classes (independent launches) run on parallel branches
    cudaGraphExec_t bwd_exec = nullptr;
    cudaStream_t side[qt::kBwdClasses - 1] = {};
    cudaEvent_t bwd_ev[qt::kBwdClasses] = {};

    // autotuning record
    double tune_seconds = 0;
    int32_t tune_candidates = 0;
    // gradient plans over a memory budget: the networks run in passes, each a
    // plan of its own on one shared arena (owned here, d_arena of the parts)
    std::vector<std::unique_ptr<qt_plan_s>> parts;
    std::vector<std::vector<int32_t>> part_edges;
    void* d_shared = nullptr;
    bool arena_external = false;  // d_arena belongs to the plan that holds this one

    // Free every device-side resource and forget it (the host plan stays).
    void release_device() {
        if (stream) cudaStreamSynchronize(stream);
        if (bwd_exec) cudaGraphExecDestroy(bwd_exec);
        bwd_exec = nullptr;
        for (auto& st : side) {
            if (st) cudaStreamDestroy(st);
            st = nullptr;
        }
        for (auto& e : bwd_ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        ev_nodes[0] = ev_nodes[1] = nullptr;
        for (auto& e : cap_ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
        for (int i = 0; i < kRing; ++i) {
            for (auto& e : ring[i]) {
                if (e) cudaEventDestroy(e);
                e = nullptr;
            }
            ring_pending[i] = false;
        }
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
        void* dev[] = {arena_external ? nullptr : d_arena, d_static, d_counters, d_angles, d_out, d_trace, d_btimes,
                       d_bwd, d_grad};
        for (void* q : dev)
            if (q) cudaFree(q);
        d_arena = d_static = d_counters = d_bwd = nullptr;
        d_angles = d_out = d_grad = nullptr;
        d_trace = nullptr;
        d_btimes = nullptr;
        d_zero = nullptr;
        if (h_err) cudaFreeHost(h_err);
        h_err = nullptr;
        calls = 0;
        time_ms = 0;
        timed = 0;
        err_pending = false;
    }

    ~qt_plan_s() {
        parts.clear();  // before the arena they share
        if (d_shared) cudaFree(d_shared);
        release_device();
    }
};

namespace {

thread_local char g_detail[512] = "";

int cuda_fail(cudaError_t e, const char* what, int line) {
    std::snprintf(g_detail, sizeof(g_detail), "%s failed at capi.cu:%d: %s (%s)", what, line, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QT_ENOMEM : QT_ECUDA;
}

}  // namespace

namespace qt {
// The same report for the other C-ABI sources (the text qt_last_error_detail returns).
int report_cuda_error(cudaError_t e, const char* file, const char* what, int line) {
    std::snprintf(g_detail, sizeof(g_detail), "%s failed at %s:%d: %s (%s)", what, file, line, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QT_ENOMEM : QT_ECUDA;
}
}  // namespace qt

namespace {

#define QT_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call, __LINE__); \
    } while (0)

bool is_host_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
}

template <typename T>
size_t bytes_of(const std::vector<T>& v) {
    return v.size() * sizeof(T);
}

int upload(qt_plan_t P) {
    qt::HostPlan& hp = P->hp;
    QT_CUDA(cudaGetDevice(&P->device));
    // tensors
    P->arena_bytes = (size_t)hp.total_elems * P->esize;
    if (!P->arena_external) {
        size_t free_b = 0, total_b = 0;
        QT_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if (P->arena_bytes + (256u << 20) > free_b) return QT_ENOMEM;
        QT_CUDA(cudaMalloc(&P->d_arena, std::max<size_t>(P->arena_bytes, 256)));
    }

    // static plan arrays, one allocation, 256-byte aligned pieces
    std::vector<uint32_t> u_graph_first_net(hp.graph_first_net.begin(), hp.graph_first_net.end());
    // operand array padded so a warp may read kMaxOps entries from any bucket's first operand
    std::vector<qt::DOperand> ops_padded(hp.operands);
    ops_padded.resize(hp.operands.size() + qt::kMaxOps, qt::DOperand{});
    struct Piece {
        const void* src;
        size_t bytes;
        size_t off;
    };
    std::vector<Piece> pieces = {
        {hp.buckets.data(), bytes_of(hp.buckets), 0},         {ops_padded.data(), bytes_of(ops_padded), 0},
        {nullptr, 0, 0},                                       {hp.runs.data(), bytes_of(hp.runs), 0},
        {nullptr, 0, 0},                                       {hp.net_first_root.data(), bytes_of(hp.net_first_root), 0},
        {hp.root_bucket.data(), bytes_of(hp.root_bucket), 0}, {u_graph_first_net.data(), bytes_of(u_graph_first_net), 0},
        {hp.unit_prog.data(), bytes_of(hp.unit_prog), 0},     {hp.net_first_factor.data(), bytes_of(hp.net_first_factor), 0},
        {hp.factor.data(), bytes_of(hp.factor), 0},            {hp.graph_owned.data(), bytes_of(hp.graph_owned), 0},
        {hp.net_weight.data(), bytes_of(hp.net_weight), 0},   {hp.factor_param.data(), bytes_of(hp.factor_param), 0},
    };
    size_t total = 0;
    for (auto& pc : pieces) {
        pc.off = total;
        total += (pc.bytes + 255) / 256 * 256;
    }
    QT_CUDA(cudaMalloc(&P->d_static, std::max<size_t>(total, 256)));
    std::vector<char> staging(total);
    for (auto& pc : pieces)
        if (pc.bytes) std::memcpy(staging.data() + pc.off, pc.src, pc.bytes);
    QT_CUDA(cudaMemcpy(P->d_static, staging.data(), total, cudaMemcpyHostToDevice));
    char* base = static_cast<char*>(P->d_static);

    // zeroed before every persistent run: control word, per-bucket tile and
    // producer counters, and the published part of the ready queue
    const uint32_t nb = (uint32_t)hp.buckets.size();
    const uint64_t n_dyn = hp.n_groups - hp.runs.size();
    const size_t ctl_bytes = 256;
    const size_t cnt_bytes = ((size_t)2 * nb * sizeof(uint32_t) + 255) / 256 * 256;
    P->counters_bytes = ctl_bytes + cnt_bytes + (size_t)n_dyn * sizeof(qt::DSlot);
    QT_CUDA(cudaMalloc(&P->d_counters, P->counters_bytes));
    QT_CUDA(cudaMemset(P->d_counters, 0, P->counters_bytes));

    const int n_graphs = (int)hp.graphs.size();
    const int n_nets = (int)hp.nets.size();
    QT_CUDA(cudaMalloc((void**)&P->d_angles, sizeof(double) * 2 * n_graphs * hp.cfg.p));
    QT_CUDA(cudaMalloc((void**)&P->d_out, sizeof(double) * (2 * n_nets + n_graphs)));
    QT_CUDA(cudaHostAlloc((void**)&P->h_err, 2 * sizeof(int32_t), cudaHostAllocDefault));
    P->h_err[0] = P->h_err[1] = 0;

    qt::DevPlan& dp = P->dp;
    dp.buckets = reinterpret_cast<const qt::DBucket*>(base + pieces[0].off);
    dp.ops = reinterpret_cast<const qt::DOperand*>(base + pieces[1].off);
    dp.runs = reinterpret_cast<const qt::DRun*>(base + pieces[3].off);
    dp.unit_prog = reinterpret_cast<const qt::URec*>(base + pieces[8].off);
    dp.has_units = hp.n_units > 0 ? 1u : 0u;
    dp.n_static = (uint32_t)hp.runs.size();
    dp.n_groups = (uint32_t)hp.n_groups;
    dp.n_buckets = nb;
    char* cbase = static_cast<char*>(P->d_counters);
    dp.ctl = reinterpret_cast<qt::DControl*>(cbase);
    dp.tiles_done = reinterpret_cast<uint32_t*>(cbase + ctl_bytes);
    dp.prod_done = dp.tiles_done + nb;
    dp.slots = reinterpret_cast<qt::DSlot*>(cbase + ctl_bytes + cnt_bytes);
    dp.arena = P->d_arena;
    dp.spin_limit = P->spin_limit;

    qt::DevEpilogue& de = P->de;
    de.buckets = dp.buckets;
    de.net_first_root = reinterpret_cast<const uint32_t*>(base + pieces[5].off);
    de.root_bucket = reinterpret_cast<const uint32_t*>(base + pieces[6].off);
    de.graph_first_net = reinterpret_cast<const int32_t*>(base + pieces[7].off);
    de.net_first_factor = reinterpret_cast<const uint32_t*>(base + pieces[9].off);
    de.factor = reinterpret_cast<const uint64_t*>(base + pieces[10].off);
    de.factor_param = reinterpret_cast<const int8_t*>(base + pieces[13].off);
    de.graph_owned = reinterpret_cast<const int32_t*>(base + pieces[11].off);
    de.net_weight = hp.net_weight.empty() ? nullptr : reinterpret_cast<const int32_t*>(base + pieces[12].off);
    de.n_graphs = n_graphs;
    de.arena = P->d_arena;
    de.zz = P->d_out;
    de.zz_imag = P->d_out + n_nets;
    de.energies = P->d_out + 2 * n_nets;

    int sms = 0;
    QT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
    const int per_sm = qt::persistent_blocks_per_sm(P->dtype);
    if (per_sm <= 0) {
        std::snprintf(g_detail, sizeof(g_detail), "persistent kernel does not fit an SM (%zu bytes of shared memory)",
                      qt::persistent_smem_bytes(P->dtype));
        return QT_ECUDA;
    }
    P->grid = sms * per_sm;
    if (P->trace) {
        const size_t tb = (size_t)P->grid * (qt::kPersistentThreads / 32) * qt::kTraceSlots * sizeof(uint64_t);
        QT_CUDA(cudaMalloc((void**)&P->d_trace, tb));
        QT_CUDA(cudaMemset(P->d_trace, 0, tb));
        P->dp.trace = P->d_trace;
        QT_CUDA(cudaMalloc((void**)&P->d_btimes, hp.buckets.size() * 2 * sizeof(unsigned long long)));
        P->dp.bucket_times = P->d_btimes;
    } else {
        P->dp.trace = nullptr;
        P->dp.bucket_times = nullptr;
    }
    QT_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    QT_CUDA(cudaEventCreate(&P->cap_ev[0]));
    QT_CUDA(cudaEventCreate(&P->cap_ev[1]));
    for (auto& r : P->ring) {
        QT_CUDA(cudaEventCreate(&r[0]));
        QT_CUDA(cudaEventCreate(&r[1]));
    }
    if (hp.cfg.with_grad) {
        // op_param | net_graph | task buckets | task tiles | op_bwd | op_roff | zero ranges
        Piece pc[7] = {{hp.op_param.data(), bytes_of(hp.op_param), 0},   {hp.net_graph.data(), bytes_of(hp.net_graph), 0},
                       {hp.bwd_bucket.data(), bytes_of(hp.bwd_bucket), 0}, {hp.bwd_tile.data(), bytes_of(hp.bwd_tile), 0},
                       {hp.op_bwd.data(), bytes_of(hp.op_bwd), 0},         {hp.op_roff.data(), bytes_of(hp.op_roff), 0},
                       {hp.bwd_zero.data(), bytes_of(hp.bwd_zero), 0}};
        size_t tot = 0;
        for (auto& x : pc) {
            x.off = tot;
            tot += (x.bytes + 255) / 256 * 256;
        }
        QT_CUDA(cudaMalloc(&P->d_bwd, std::max<size_t>(tot, 256)));
        char* q = static_cast<char*>(P->d_bwd);
        for (auto& x : pc)
            if (x.bytes) QT_CUDA(cudaMemcpy(q + x.off, x.src, x.bytes, cudaMemcpyHostToDevice));
        const size_t b0 = pc[1].off, b1 = pc[2].off - pc[1].off, b2 = pc[3].off - pc[2].off;
        QT_CUDA(cudaMalloc((void**)&P->d_grad, sizeof(double) * 4 * n_graphs * hp.cfg.p));
        qt::DevBwd& db = P->db;
        db.buckets = dp.buckets;
        db.ops = dp.ops;
        db.op_param = reinterpret_cast<const int8_t*>(q);
        db.net_graph = reinterpret_cast<const uint32_t*>(q + b0);
        db.task_bucket = reinterpret_cast<const uint32_t*>(q + b0 + b1);
        db.task_tile = reinterpret_cast<const uint32_t*>(q + b0 + b1 + b2);
        db.op_bwd = reinterpret_cast<const int8_t*>(q + pc[4].off);
        db.op_roff = reinterpret_cast<const uint16_t*>(q + pc[5].off);
        P->d_zero = reinterpret_cast<const uint64_t*>(q + pc[6].off);
        P->n_zero = (uint32_t)(hp.bwd_zero.size() / 2);
        db.p = hp.cfg.p;
        db.arena = P->d_arena;
        db.cot_delta = hp.cot_off - hp.leaf_elems;
        db.dleaf_delta = hp.dleaf_off;
        db.grad = P->d_grad;
    }
    return QT_OK;
}

// Everything one evaluation runs after the angles are in place, on stream s.
int enqueue_eval(qt_plan_t P, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    qt::HostPlan& hp = P->hp;
    QT_CUDA(qt::launch_leaf_fill(P->dtype, P->d_angles, (int)hp.graphs.size(), hp.cfg.p, P->d_arena, hp.dleaf_off, s));
    if (P->sched == QT_SCHED_PERSISTENT) {
        QT_CUDA(cudaMemsetAsync(P->d_counters, 0, P->counters_bytes, s));
        if (P->d_btimes) {  // starts to all ones (min), ends to zero (max)
            QT_CUDA(cudaMemsetAsync(P->d_btimes, 0xff, hp.buckets.size() * 2 * sizeof(unsigned long long), s));
            QT_CUDA(qt::launch_clear_ends(P->d_btimes, hp.buckets.size(), s));
        }
        QT_CUDA(cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal));
        QT_CUDA(qt::launch_persistent(P->dtype, P->grid, P->dp, s));
        QT_CUDA(cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal));
    } else {
        QT_CUDA(cudaEventRecord(e0, s));
        for (size_t b = 0; b < hp.buckets.size(); ++b)
            QT_CUDA(qt::launch_per_bucket(P->dtype, (uint32_t)b, hp.buckets[b].n_tasks, P->dp, s));
        QT_CUDA(cudaEventRecord(e1, s));
    }
    QT_CUDA(qt::launch_epilogue(P->dtype, P->de, s));
    QT_CUDA(cudaMemcpyAsync(P->h_err, &P->dp.ctl->error, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return QT_OK;
}

int ensure_graph(qt_plan_t P) {
    if (P->exec) return QT_OK;
    QT_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_eval(P, P->stream, P->cap_ev[0], P->cap_ev[1]);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (rc != QT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture", __LINE__);
    P->graph = g;
    size_t n = 0;
    QT_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    QT_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        QT_CUDA(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        QT_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        if (ev == P->cap_ev[0]) P->ev_nodes[0] = nd;
        if (ev == P->cap_ev[1]) P->ev_nodes[1] = nd;
    }
    if (!P->ev_nodes[0] || !P->ev_nodes[1]) {
        std::snprintf(g_detail, sizeof(g_detail), "timing event nodes not found in the captured graph");
        return QT_ECUDA;
    }
    QT_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
    return QT_OK;
}

void harvest_slot(qt_plan_t P, int slot) {
    if (!P->ring_pending[slot]) return;
    if (cudaEventSynchronize(P->ring[slot][1]) == cudaSuccess) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, P->ring[slot][0], P->ring[slot][1]) == cudaSuccess) {
            P->time_ms += ms;
            P->timed++;
        }
    }
    cudaGetLastError();
    P->ring_pending[slot] = false;
}

int check_error_word(qt_plan_t P) {
    int32_t e = P->h_err[0];
    if (e != 0) {
        P->h_err[0] = 0;
        return e;
    }
    return QT_OK;
}

// One evaluation: angles in, run, results out.
int run_eval(qt_plan_t P, const double* gammas, const double* betas, void* stream_v,
             double* zz_out, double* energies_out, bool all_nets_out) {
    const int G = (int)P->hp.graphs.size();
    const int p = P->hp.cfg.p;
    const int n_nets = (int)P->hp.nets.size();
    if (!gammas || !betas) return QT_EINVAL;
    if (P->host_only) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    cudaStream_t s = stream_v ? static_cast<cudaStream_t>(stream_v) : P->stream;
    QT_CUDA(cudaMemcpyAsync(P->d_angles, gammas, sizeof(double) * G * p, cudaMemcpyDefault, s));
    QT_CUDA(cudaMemcpyAsync(P->d_angles + (size_t)G * p, betas, sizeof(double) * G * p, cudaMemcpyDefault, s));

    const int slot = (int)(P->calls % kRing);
    harvest_slot(P, slot);
    if (P->sched == QT_SCHED_PERSISTENT) {
        int rc = ensure_graph(P);
        if (rc != QT_OK) return rc;
        QT_CUDA(cudaGraphExecEventRecordNodeSetEvent(P->exec, P->ev_nodes[0], P->ring[slot][0]));
        QT_CUDA(cudaGraphExecEventRecordNodeSetEvent(P->exec, P->ev_nodes[1], P->ring[slot][1]));
        QT_CUDA(cudaGraphLaunch(P->exec, s));
    } else {
        int rc = enqueue_eval(P, s, P->ring[slot][0], P->ring[slot][1]);
        if (rc != QT_OK) return rc;
    }
    P->ring_pending[slot] = true;
    P->calls++;
    P->err_pending = true;

    bool host_out = false;
    if (zz_out) {
        size_t nz = all_nets_out ? (size_t)n_nets : (size_t)n_nets;
        QT_CUDA(cudaMemcpyAsync(zz_out, P->de.zz, sizeof(double) * nz, cudaMemcpyDefault, s));
        host_out |= is_host_ptr(zz_out);
    }
    if (energies_out) {
        QT_CUDA(cudaMemcpyAsync(energies_out, P->de.energies, sizeof(double) * G, cudaMemcpyDefault, s));
        host_out |= is_host_ptr(energies_out);
    }
    if (host_out || !stream_v) {
        QT_CUDA(cudaStreamSynchronize(s));
        P->err_pending = false;
        return check_error_word(P);
    }
    return QT_OK;
}

// Mean device time of the persistent kernel over `reps` evaluations (after
// one warm-up) at fixed probe angles, on the plan as uploaded.
int time_probe(qt_plan_t P, int reps, double* ms) {
    const int G = (int)P->hp.graphs.size(), p = P->hp.cfg.p;
    std::vector<double> g((size_t)G * p, 0.4), b((size_t)G * p, 0.3);
    int rc = run_eval(P, g.data(), b.data(), nullptr, nullptr, nullptr, true);  // warm-up
    if (rc != QT_OK) return rc;
    for (int i = 0; i < kRing; ++i) harvest_slot(P, i);
    P->time_ms = 0;
    P->timed = 0;
    for (int r = 0; r < reps; ++r) {
        rc = run_eval(P, g.data(), b.data(), nullptr, nullptr, nullptr, true);
        if (rc != QT_OK) return rc;
    }
    for (int i = 0; i < kRing; ++i) harvest_slot(P, i);
    if (P->timed == 0) return QT_ECUDA;
    *ms = P->time_ms / (double)P->timed;
    return QT_OK;
}

// Autotuner of the tile shapes (§III-C: per-bucket kernel choices). For each
// bucket-width class present, in turn, try every cap on the tile's outputs
// (2^6 .. 2^11, within the class's widths) with the best settings so far,
// then groups of 8 and 32 tiles; keep a change only if the probe time drops
// by 1% or more. Each candidate is laid out, uploaded and timed on the
// device; the plan ends uploaded with the best settings.
int autotune(qt_plan_t P, int reps) {
    auto t0 = std::chrono::steady_clock::now();
    qt::HostPlan& hp = P->hp;
    int max_out[qt::kWidthClasses] = {-1, -1, -1, -1, -1};
    for (const auto& d : hp.buckets) {
        const int c = qt::width_class(d.n_out);
        max_out[c] = std::max(max_out[c], (int)d.n_out);
    }
    auto trial = [&](const qt::PlanConfig& cfg, double* ms) {
        P->release_device();
        hp.cfg = cfg;
        int rc = qt::layout_plan(&hp);
        if (rc == QT_OK) rc = upload(P);
        if (rc == QT_OK) rc = time_probe(P, reps, ms);
        P->tune_candidates++;
        return rc;
    };
    qt::PlanConfig best = hp.cfg;
    double best_ms = 0;
    int rc = trial(best, &best_ms);
    if (rc != QT_OK) return rc;
    const int def_cap = best.chunk_log2 > 0 ? best.chunk_log2 : qt::kDefaultTileBits;
    for (int c = 0; c < qt::kWidthClasses; ++c) {
        if (max_out[c] <= 6) continue;  // tiles of 64 outputs or fewer: nothing to choose
        const int cur = best.tile_cap[c] > 0 ? best.tile_cap[c] : def_cap;
        for (int cap = 6; cap <= std::min(11, max_out[c]); ++cap) {
            if (cap == cur) continue;
            qt::PlanConfig cfg = best;
            cfg.tile_cap[c] = cap;
            double ms = 0;
            rc = trial(cfg, &ms);
            if (rc != QT_OK) return rc;
            if (ms < 0.99 * best_ms) {
                best_ms = ms;
                best = cfg;
            }
        }
    }
    for (int rt : {8, 16, 32}) {
        qt::PlanConfig cfg = best;
        cfg.run_tiles = rt;
        double ms = 0;
        rc = trial(cfg, &ms);
        if (rc != QT_OK) return rc;
        if (ms < 0.99 * best_ms) {
            best_ms = ms;
            best = cfg;
        }
    }
    // the chosen settings, stated explicitly
    for (int c = 0; c < qt::kWidthClasses; ++c)
        if (best.tile_cap[c] == 0) best.tile_cap[c] = def_cap;
    P->release_device();
    hp.cfg = best;
    rc = qt::layout_plan(&hp);
    if (rc == QT_OK) rc = upload(P);
    P->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

qt_plan_opts default_opts() {
    qt_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    return o;
}

int make_plan(const std::vector<qt::GraphIn>& graphs, int32_t p, const qt_plan_opts* opts_in, qt_plan_t* out);

// A gradient plan over opts.adjoint_budget_bytes: its networks are packed, in
// edge order, into passes whose saved results and cotangents fit the budget
// (with the leaf tables); each pass is a plan of its own, all on one arena of
// the largest pass's size. A network that alone exceeds the budget is refused
// (QT_ENOMEM): networks are not split. Single-graph plans only.
// A plan over a memory budget runs in passes, each a sub-plan of one graph on
// one shared arena. Gradient plans pass over whole networks (results and
// their cotangents); energy plans over networks' slices (results only), a
// pass counting an edge's 1/2 only if it holds the network's slice 0.
int make_passes(qt_plan_t P, const std::vector<qt::GraphIn>& graphs, int32_t p, const qt_plan_opts& o) {
    const qt::HostPlan& hp = P->hp;
    if (graphs.size() != 1) return QT_ESTATE;
    const bool grad = hp.cfg.with_grad;
    const size_t budget = grad ? o.adjoint_budget_bytes : o.energy_budget_bytes;
    const size_t leaf_bytes = (size_t)hp.leaf_elems * P->esize;
    if (leaf_bytes >= budget) return QT_ENOMEM;
    const size_t room = budget - leaf_bytes;
    const qt::GraphIn& g0 = graphs[0];
    struct Pass {
        std::vector<int32_t> edges;
        std::vector<std::vector<uint32_t>> slices;
        std::vector<uint8_t> owner;
    };
    std::vector<Pass> passes(1);
    size_t cur_bytes = 0;
    for (size_t i = 0; i < hp.nets.size(); ++i) {
        const qt::Network& net = hp.nets[i];
        const uint32_t n_sl = 1u << net.slice_bits;
        std::vector<size_t> nb(n_sl, 0);  // per slice: results (and cotangents), 128-byte aligned
        for (uint32_t b = hp.net_first_bucket[i]; b < hp.net_first_bucket[i + 1]; ++b)
            nb[hp.bucket_slice[b]] += (grad ? 2 : 1) * (((size_t)1 << qt::result_bits(hp.buckets[b])) * P->esize + 128);
        for (uint32_t s = 0; s < n_sl; ++s) {
            if (nb[s] > room) return QT_ENOMEM;
            if (cur_bytes + nb[s] > room && !passes.back().edges.empty()) {
                passes.emplace_back();
                cur_bytes = 0;
            }
            Pass& ps = passes.back();
            const int32_t e = (int32_t)g0.edge_of(i);
            if (ps.edges.empty() || ps.edges.back() != e) {
                ps.edges.push_back(e);
                ps.slices.emplace_back();
                ps.owner.push_back(0);
            }
            ps.slices.back().push_back(s);
            if (s == 0) ps.owner.back() = 1;
            cur_bytes += nb[s];
        }
    }
    if (passes.back().edges.empty()) passes.pop_back();
    qt_plan_opts so = o;
    so.adjoint_budget_bytes = 0;
    so.energy_budget_bytes = 0;
    so.host_only = 1;
    so.autotune = 0;
    so.dedup = 0;
    size_t arena = 0;
    for (Pass& ps : passes) {
        std::vector<qt::GraphIn> gs(1);
        gs[0].n = g0.n;
        gs[0].edges = g0.edges;
        gs[0].sel = ps.edges;
        gs[0].sel_slices = ps.slices;  // a network's slices may sit in several passes (gradients too:
        gs[0].sel_owner = ps.owner;    // each slice's roots are seeded from its own factors)
        P->part_edges.push_back(ps.edges);
        qt_plan_t part = nullptr;
        const int rc = make_plan(gs, p, &so, &part);
        if (rc != QT_OK) return rc;
        P->parts.emplace_back(part);
        arena = std::max(arena, (size_t)part->hp.total_elems * P->esize);
    }
    if (o.host_only) return QT_OK;
    size_t free_b = 0, total_b = 0;
    QT_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (arena + (256u << 20) > free_b) return QT_ENOMEM;
    QT_CUDA(cudaMalloc(&P->d_shared, std::max<size_t>(arena, 256)));
    for (auto& part : P->parts) {
        part->host_only = false;
        part->arena_external = true;
        part->d_arena = P->d_shared;
        const int rc = upload(part.get());
        if (rc != QT_OK) return rc;
    }
    return QT_OK;
}

// Energy (and gradient) of a plan that runs in passes: each pass in turn on
// the shared arena; per-edge values scattered to the graph's edge order,
// partial energies and gradients summed in FP64 on the host.
int run_passes(qt_plan_t P, const double* gammas, const double* betas, double* edge_zz, double* energy,
               double* dg, double* db, void* stream, bool grad) {
    const int p = P->hp.cfg.p;
    const qt::GraphIn& g0 = P->hp.graphs[0];
    const size_t m = P->hp.nets.size();  // outputs: one per planned network, in the plan's order
    std::vector<int64_t> pos(g0.edges.size(), -1);
    for (size_t i = 0; i < m; ++i) pos[g0.edge_of(i)] = (int64_t)i;
    std::vector<double> g(p), b(p), zz(m, 0.0), gs(p, 0.0), bs(p, 0.0);
    QT_CUDA(cudaMemcpy(g.data(), gammas, sizeof(double) * p, cudaMemcpyDefault));
    QT_CUDA(cudaMemcpy(b.data(), betas, sizeof(double) * p, cudaMemcpyDefault));
    double E = 0.0;
    for (size_t k = 0; k < P->parts.size(); ++k) {
        qt_plan_t part = P->parts[k].get();
        const auto& pe = P->part_edges[k];
        std::vector<double> pz(pe.size()), pg(p), pb(p);
        double pE = 0.0;
        int rc = grad ? qt_energy_grad(part, g.data(), b.data(), &pE, pg.data(), pb.data(), stream)
                      : qt_energy(part, g.data(), b.data(), pz.data(), &pE, stream);
        if (rc != QT_OK) return rc;
        if (grad) {
            for (int i = 0; i < p; ++i) {
                gs[i] += pg[i];
                bs[i] += pb[i];
            }
        }
        for (size_t i = 0; i < pe.size(); ++i) zz[pos[pe[i]]] += pz[i];  // energy passes may split a network's slices
        E += pE;
    }
    if (edge_zz) QT_CUDA(cudaMemcpy(edge_zz, zz.data(), sizeof(double) * m, cudaMemcpyDefault));
    if (energy) QT_CUDA(cudaMemcpy(energy, &E, sizeof(double), cudaMemcpyDefault));
    if (grad && dg) QT_CUDA(cudaMemcpy(dg, gs.data(), sizeof(double) * p, cudaMemcpyDefault));
    if (grad && db) QT_CUDA(cudaMemcpy(db, bs.data(), sizeof(double) * p, cudaMemcpyDefault));
    return QT_OK;
}

int make_plan(const std::vector<qt::GraphIn>& graphs, int32_t p, const qt_plan_opts* opts_in, qt_plan_t* out) {
    if (!out) return QT_EINVAL;
    *out = nullptr;
    qt_plan_opts o = opts_in ? *opts_in : default_opts();
    if (o.dtype != QT_C64 && o.dtype != QT_C128) return QT_EINVAL;
    if (o.sched != QT_SCHED_PERSISTENT && o.sched != QT_SCHED_PER_BUCKET) return QT_EINVAL;
    qt::PlanConfig cfg;
    cfg.p = p;
    cfg.dtype = o.dtype;
    // order restarts: by default 64 for the networks whose plain greedy order is
    // wide (their buckets carry the bytes); measured on the N=30 p=4 workload:
    // 3.42 -> 2.31 GB per evaluation, kernel 1.21 -> 1.06 ms (complex64)
    cfg.restarts = o.order_restarts > 0 ? o.order_restarts : o.order_restarts == 0 ? kAutoRestarts : 0;
    cfg.restart_min_width = o.order_restarts == 0 ? kAutoRestartWidth : 0;
    cfg.seed = o.order_seed;
    cfg.max_width = o.max_width > 0 ? o.max_width : 31;
    cfg.chunk_log2 = o.chunk_log2;
    cfg.run_tiles = o.run_tiles;
    cfg.order = o.order;
    if (o.order < 0 || o.order > 1) return QT_EINVAL;
    {
        // warps of the persistent grid (the schedule simulation and the group
        // sizes of wide buckets assume them): 4 per block, 3 blocks per SM for
        // complex64 and 2 for complex128; 152 SMs when planning without a GPU
        int sms = 152, dev = 0;
        if (!o.host_only && cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        cfg.sim_workers = sms * 4 * (o.dtype == QT_C128 ? 2 : 3);
    }
    if (o.run_tiles < 0 || o.run_tiles > 4096) return QT_EINVAL;
    cfg.with_grad = o.with_grad != 0;
    cfg.fuse = o.sched == QT_SCHED_PERSISTENT && !cfg.with_grad && o.no_fuse == 0;
    // the per-bucket kernel sums one variable per bucket: merging is a
    // persistent-schedule option (fused units take only unmerged subtrees).
    // Gradient plans merge only when asked (no_merge < 0): their reverse sweep
    // ran slower on merged buckets (N=50 p=4: complex64 21.8 vs 20.0 ms)
    cfg.merge = o.sched == QT_SCHED_PERSISTENT && (o.no_merge < 0 || (o.no_merge == 0 && !cfg.with_grad));
    if (o.slice_width < -1 || o.slice_width == 1 || o.slice_width > 31) return QT_EINVAL;
    if (o.max_slice_bits < 0 || o.max_slice_bits > 16) return QT_EINVAL;
    // default target widths: measured best on the N=30 p=4 and N=1000 p=5 networks
    const int sw = o.slice_width == 0 ? (o.dtype == QT_C128 ? 20 : 22) : std::max(0, o.slice_width);
    cfg.slice_width = sw;
    cfg.max_slice_bits = o.max_slice_bits ? o.max_slice_bits : 8;
    // a duplicate network takes its representative's value within one plan, so passes do
    // not deduplicate; the choice waits until the deduplicated plan's size is known
    cfg.dedup = o.dedup != 0;
    for (int c = 0; c < qt::kWidthClasses; ++c) {
        if (o.tile_cap[c] != 0 && (o.tile_cap[c] < 1 || o.tile_cap[c] > 11)) return QT_EINVAL;
        cfg.tile_cap[c] = o.tile_cap[c];
    }
    if (o.autotune < 0 || o.autotune > 1000 || (o.autotune > 0 && o.sched != QT_SCHED_PERSISTENT)) return QT_EINVAL;
    if (cfg.chunk_log2 < 0 || cfg.chunk_log2 > 24) return QT_EINVAL;
    std::unique_ptr<qt_plan_s> P(new (std::nothrow) qt_plan_s());
    if (!P) return QT_ENOMEM;
    P->dtype = o.dtype;
    P->sched = o.sched;
    P->esize = o.dtype == QT_C128 ? 16 : 8;
    P->spin_limit = o.spin_limit ? o.spin_limit : (1ull << 23);
    int rc;
    try {
        rc = qt::build_host_plan(graphs, cfg, &P->hp);
    } catch (const std::bad_alloc&) {
        return QT_ENOMEM;
    } catch (...) {
        return QT_EINVAL;
    }
    if (rc != QT_OK) return rc;
    P->arena_bytes = (size_t)P->hp.total_elems * P->esize;
    const size_t budget = cfg.with_grad ? o.adjoint_budget_bytes : o.energy_budget_bytes;
    const bool passes = budget > 0 && P->arena_bytes > budget;
    if (passes && cfg.dedup) {
        // over budget even deduplicated: plan every network, then split it into passes
        cfg.dedup = false;
        P->hp = qt::HostPlan();
        try {
            rc = qt::build_host_plan(graphs, cfg, &P->hp);
        } catch (const std::bad_alloc&) {
            return QT_ENOMEM;
        } catch (...) {
            return QT_EINVAL;
        }
        if (rc != QT_OK) return rc;
        P->arena_bytes = (size_t)P->hp.total_elems * P->esize;
    }
    if (o.arena_bytes && P->arena_bytes > o.arena_bytes) return QT_ENOMEM;
    P->host_only = o.host_only != 0;
    P->trace = o.trace != 0;
    if (passes) {
        rc = make_passes(P.get(), graphs, p, o);
        if (rc != QT_OK) return rc;
        *out = P.release();
        return QT_OK;
    }
    if (!P->host_only) {
        rc = o.autotune > 0 ? autotune(P.get(), o.autotune) : upload(P.get());
        if (rc != QT_OK) return rc;
    }
    *out = P.release();
    return QT_OK;
}

}  // namespace

extern "C" {

int qt_plan(int32_t n_vertices, int32_t n_edges, const int32_t* edges, int32_t p, const qt_plan_opts* opts,
            qt_plan_t* out) {
    if (n_edges < 0 || (n_edges > 0 && !edges) || n_vertices < 1) return QT_EINVAL;
    std::vector<qt::GraphIn> gs(1);
    gs[0].n = n_vertices;
    for (int e = 0; e < n_edges; ++e) gs[0].edges.emplace_back(edges[2 * e], edges[2 * e + 1]);
    return make_plan(gs, p, opts, out);
}

int qt_plan_subset(int32_t n_vertices, int32_t n_edges, const int32_t* edges, int32_t p, int32_t n_sel,
                   const int32_t* sel, const qt_plan_opts* opts, qt_plan_t* out) {
    if (!edges || n_edges < 1 || n_vertices < 2 || n_sel < 1 || !sel) return QT_EINVAL;
    std::vector<qt::GraphIn> gs(1);
    gs[0].n = n_vertices;
    for (int e = 0; e < n_edges; ++e) gs[0].edges.emplace_back(edges[2 * e], edges[2 * e + 1]);
    gs[0].sel.assign(sel, sel + n_sel);
    return make_plan(gs, p, opts, out);
}

int qt_plan_shard(int32_t n_vertices, int32_t n_edges, const int32_t* edges, int32_t p, int32_t world, int32_t rank,
                  const qt_plan_opts* opts, qt_plan_t* out, int32_t* shard_edges, int32_t* n_shard) {
    if (!out || !n_shard || world < 1 || rank < 0 || rank >= world) return QT_EINVAL;
    if (n_edges < 0 || (n_edges > 0 && !edges) || n_vertices < 1) return QT_EINVAL;
    // every network planned on the host, for its cost (sum of 2^width)
    qt_plan_opts ho = opts ? *opts : default_opts();
    ho.host_only = 1;
    ho.autotune = 0;
    ho.dedup = 0;  // every network's own cost (a shard deduplicates within itself)
    qt_plan_t full = nullptr;
    int rc = qt_plan(n_vertices, n_edges, edges, p, &ho, &full);
    if (rc != QT_OK) return rc;
    // units: every slice of every network (one per unsliced network), each
    // costing its slice's sum of 2^width
    struct Unit {
        double cost;
        int edge;
        uint32_t slice;
    };
    std::vector<Unit> units;
    std::vector<uint32_t> n_sl(n_edges);
    for (int e = 0; e < n_edges; ++e) {
        n_sl[e] = 1u << full->hp.nets[e].slice_bits;
        for (uint32_t s = 0; s < n_sl[e]; ++s) units.push_back(Unit{full->hp.nplans[e].cost, e, s});
    }
    qt_plan_free(full);
    // LPT: the costliest unit first (ties: lower edge, then slice), to the least loaded rank (ties: lower rank)
    std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.cost > b.cost; });
    std::vector<double> load(world, 0.0);
    std::vector<std::vector<uint32_t>> my_slices(n_edges);
    std::vector<uint8_t> my_owner(n_edges, 0);
    for (const Unit& u : units) {
        const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[r] += u.cost;
        if (r != rank) continue;
        my_slices[u.edge].push_back(u.slice);
        if (u.slice == 0) my_owner[u.edge] = 1;  // the rank holding slice 0 counts the edge's 1/2
    }
    std::vector<int32_t> mine;
    for (int e = 0; e < n_edges; ++e)
        if (!my_slices[e].empty()) mine.push_back(e);
    *n_shard = (int32_t)mine.size();
    if (shard_edges && !mine.empty()) std::memcpy(shard_edges, mine.data(), mine.size() * sizeof(int32_t));
    std::vector<qt::GraphIn> gs(1);
    gs[0].n = n_vertices;
    if (!mine.empty()) {  // an empty shard is a graph without edges: no networks, energy 0
        for (int e = 0; e < n_edges; ++e) gs[0].edges.emplace_back(edges[2 * e], edges[2 * e + 1]);
        gs[0].sel = mine;
        for (int e : mine) {
            std::sort(my_slices[e].begin(), my_slices[e].end());
            // all of a network's slices: leave the selection empty (the plain plan)
            gs[0].sel_slices.push_back(my_slices[e].size() == n_sl[e] ? std::vector<uint32_t>() : my_slices[e]);
            gs[0].sel_owner.push_back(my_owner[e]);
        }
    }
    return make_plan(gs, p, opts, out);
}

int qt_plan_batch(int32_t n_graphs, const int32_t* n_vertices, const int32_t* n_edges, const int32_t* edges,
                  int32_t p, const qt_plan_opts* opts, qt_plan_t* out) {
    if (n_graphs < 1 || !n_vertices || !n_edges) return QT_EINVAL;
    int64_t total_edges = 0;
    for (int g = 0; g < n_graphs; ++g) total_edges += n_edges[g] > 0 ? n_edges[g] : 0;
    if (total_edges > 0 && !edges) return QT_EINVAL;
    std::vector<qt::GraphIn> gs(n_graphs);
    size_t at = 0;
    for (int g = 0; g < n_graphs; ++g) {
        if (n_edges[g] < 0 || n_vertices[g] < 1) return QT_EINVAL;
        gs[g].n = n_vertices[g];
        for (int e = 0; e < n_edges[g]; ++e, ++at) gs[g].edges.emplace_back(edges[2 * at], edges[2 * at + 1]);
    }
    return make_plan(gs, p, opts, out);
}

int qt_plan_stats_get(qt_plan_t P, qt_plan_stats* out) {
    if (!P || !out) return QT_EINVAL;
    std::memset(out, 0, sizeof(*out));
    const qt::HostPlan& hp = P->hp;
    out->n_graphs = (int32_t)hp.graphs.size();
    out->n_networks = (int32_t)hp.nets.size();
    out->n_buckets = (int64_t)hp.buckets.size();
    out->n_operands = (int64_t)hp.operands.size();
    out->max_width = hp.max_width;
    out->p = hp.cfg.p;
    out->sum_2w = hp.sum_2w;
    out->alg_bytes = hp.alg_bytes;
    out->flops = hp.flops;
    out->arena_bytes = (int64_t)P->arena_bytes;  // what the device arena takes (or would take)
    out->n_tasks = (int64_t)hp.n_tiles;
    out->n_items = (int64_t)hp.n_groups;
    out->n_levels = hp.n_levels;
    out->dtype = P->dtype;
    std::memcpy(out->width_hist, hp.width_hist, sizeof(out->width_hist));
    out->plan_seconds = hp.plan_seconds;
    out->sim_seconds = hp.sim_seconds;
    out->n_units = (int64_t)hp.n_units;
    out->n_fused = (int64_t)hp.n_fused;
    const int def_cap = hp.cfg.chunk_log2 > 0 ? hp.cfg.chunk_log2 : qt::kDefaultTileBits;
    for (int c = 0; c < 8; ++c)
        out->tile_cap[c] = c < qt::kWidthClasses ? (hp.cfg.tile_cap[c] > 0 ? hp.cfg.tile_cap[c] : def_cap) : 0;
    out->run_tiles = hp.cfg.run_tiles > 0 ? hp.cfg.run_tiles : qt::kRunTiles;
    out->tune_seconds = P->tune_seconds;
    out->tune_candidates = P->tune_candidates;
    out->n_passes = P->parts.empty() ? 1 : (int32_t)P->parts.size();
    out->slice_bits = 0;
    for (const qt::Network& net : hp.nets) out->slice_bits = std::max(out->slice_bits, (int32_t)net.slice_bits);
    out->n_slices = (int64_t)hp.n_slices;
    out->n_unique = (int64_t)hp.n_unique;
    out->pass_arena_bytes = 0;
    for (const auto& part : P->parts)
        out->pass_arena_bytes = std::max<int64_t>(out->pass_arena_bytes, (int64_t)part->hp.total_elems * part->esize);
    return QT_OK;
}

int qt_plan_export(qt_plan_t P, qt_bucket_info* buckets, qt_operand_info* operands) {
    if (!P) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    if (buckets) {
        for (size_t b = 0; b < hp.buckets.size(); ++b) {
            const qt::DBucket& d = hp.buckets[b];
            qt_bucket_info& o = buckets[b];
            o.network = (int32_t)d.net;
            o.width = d.n_out + 1;
            o.n_ops = d.n_ops;
            o.op_begin = (int32_t)d.op_begin;
            o.parent = d.parent == qt::kNone ? -1 : (int32_t)d.parent;
            o.n_deps = (int32_t)d.n_deps;
            o.level = hp.bucket_level[b];
            o.var = hp.bucket_var[b];
            o.tile_log2 = d.chunk_bits;
            o.tile_bits = (1u << d.chunk_bits) - 1u;
            o.folded = 0;
            for (uint32_t i = 0; i < d.n_ops; ++i)
                if (hp.operands[d.op_begin + i].folded) o.folded |= 1u << i;
            o.unit_role = (d.flags & qt::kBucketInUnit) ? 1u : (d.flags & qt::kBucketUnitRoot) ? 2u : 0u;
            o.n_sum = qt::bucket_n_sum(d.flags);
            o.var2 = hp.bucket_var2[b];
            o.var3 = hp.bucket_var3[b];
            o.slice = hp.bucket_slice[b];
        }
    }
    if (operands) {
        for (size_t i = 0; i < hp.operands.size(); ++i) {
            qt_operand_info& o = operands[i];
            o.src = hp.op_src[i];
            o.leaf_kind = hp.op_leaf_kind[i];
            o.leaf_layer = hp.op_leaf_layer[i];
            o.rank = hp.op_rank[i];
            o.smask = hp.operands[i].smask;
            o.mask = hp.operands[i].mask;
            o.leaf_sub = hp.op_leaf_sub[i];
            o.pad = 0;
        }
        // a merged bucket's operands carry s1 (and s2) in the low bits of their device masks
        for (const qt::DBucket& d : hp.buckets) {
            const int m = qt::bucket_n_sum(d.flags) - 1;
            if (m == 0) continue;
            for (uint32_t i = d.op_begin; i < d.op_begin + d.n_ops; ++i) operands[i].mask >>= m;
        }
    }
    return QT_OK;
}

int qt_plan_export_device(qt_plan_t P, qt_dev_bucket* buckets, qt_dev_operand* operands, uint32_t* net_first_factor,
                          uint64_t* factor, int32_t* graph_owned, int64_t* n_factors) {
    if (!P) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    if (buckets)
        for (size_t b = 0; b < hp.buckets.size(); ++b) {
            const qt::DBucket& d = hp.buckets[b];
            buckets[b] = qt_dev_bucket{d.out_off, (int32_t)d.op_begin, (int32_t)d.n_ops, (int32_t)d.n_out,
                                       (int32_t)qt::bucket_n_sum(d.flags)};
        }
    if (operands)
        for (size_t i = 0; i < hp.operands.size(); ++i) {
            const qt::DOperand& o = hp.operands[i];
            operands[i] = qt_dev_operand{o.off, o.mask, (int32_t)(o.smask & 1u), (o.flags & qt::kOpLeaf) ? 1 : 0, 0};
        }
    if (net_first_factor)
        std::memcpy(net_first_factor, hp.net_first_factor.data(), hp.net_first_factor.size() * sizeof(uint32_t));
    if (factor && !hp.factor.empty()) std::memcpy(factor, hp.factor.data(), hp.factor.size() * sizeof(uint64_t));
    if (graph_owned && !hp.graph_owned.empty())
        std::memcpy(graph_owned, hp.graph_owned.data(), hp.graph_owned.size() * sizeof(int32_t));
    if (n_factors) *n_factors = (int64_t)hp.factor.size();
    return QT_OK;
}

int qt_plan_pass(qt_plan_t P, int32_t k, qt_plan_t* pass, int32_t* pass_edges, int32_t* n_edges) {
    if (!P || !pass || !n_edges) return QT_EINVAL;
    if (P->parts.empty()) return QT_ESTATE;
    if (k < 0 || k >= (int32_t)P->parts.size()) return QT_EINVAL;
    *pass = P->parts[k].get();
    const auto& pe = P->part_edges[k];
    *n_edges = (int32_t)pe.size();
    if (pass_edges && !pe.empty()) std::memcpy(pass_edges, pe.data(), pe.size() * sizeof(int32_t));
    return QT_OK;
}

int qt_plan_export_reps(qt_plan_t P, int32_t* rep) {
    if (!P || !rep) return QT_EINVAL;
    for (size_t i = 0; i < P->hp.nets.size(); ++i) rep[i] = P->hp.nets[i].rep >= 0 ? P->hp.nets[i].rep : (int32_t)i;
    return QT_OK;
}

int qt_plan_export_fixed(qt_plan_t P, qt_fixed_info* out, int64_t* n_out) {
    if (!P || !n_out) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    int64_t k = 0;
    for (size_t i = 0; i < hp.nets.size(); ++i) {
        const qt::Network& net = hp.nets[i];
        for (uint32_t j = 0; j < net.n_emitted(); ++j)
            for (const qt::FixedLeaf& fl : net.fixed) {
                const uint32_t sl = net.slice_at(j);
                if (out) {
                    qt_fixed_info& f = out[k];
                    f.network = (int32_t)i;
                    f.slice = (int32_t)sl;
                    f.leaf_kind = fl.kind;
                    f.leaf_layer = fl.layer;
                    f.entry = (int32_t)(((sl >> fl.f[0]) & 1u) + (fl.rank == 2 ? 2u * ((sl >> fl.f[1]) & 1u) : 0u));
                    f.pad = 0;
                }
                ++k;
            }
    }
    *n_out = k;
    return QT_OK;
}

int qt_plan_export_groups(qt_plan_t P, qt_group_info* groups, int64_t* n_out) {
    if (!P || !groups || !n_out) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    for (size_t i = 0; i < hp.runs.size(); ++i) {
        const qt::DRun& r = hp.runs[i];
        groups[i] = qt_group_info{(int32_t)r.bucket, (int32_t)r.chunk_begin, (int32_t)r.n_chunks,
                                  r.unit_begin ? (int32_t)r.unit_count : 0};
    }
    *n_out = (int64_t)hp.runs.size();
    return QT_OK;
}

int qt_plan_export_units(qt_plan_t P, qt_unit_info* units, qt_unit_rec* recs, int64_t* n_units, int64_t* n_recs) {
    if (!P || !n_units || !n_recs) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    static_assert(sizeof(qt_unit_rec) == sizeof(qt::URec), "unit record layout");
    int64_t nu = 0;
    for (size_t b = 0; b < hp.buckets.size(); ++b) {
        const qt::DBucket& d = hp.buckets[b];
        if (!(d.flags & qt::kBucketUnitRoot)) continue;
        if (units) units[nu] = qt_unit_info{(int32_t)b, (int32_t)d.unit_count, (int64_t)d.unit_begin - 1};
        ++nu;
    }
    if (recs)
        for (size_t i = 0; i < hp.unit_prog.size(); ++i) {
            const qt::URec& r = hp.unit_prog[i];
            recs[i] = qt_unit_rec{r.a, r.b, r.off};
        }
    *n_units = nu;
    *n_recs = (int64_t)hp.unit_prog.size();
    return QT_OK;
}

int qt_plan_network_wires(qt_plan_t P, int32_t network, int32_t* vars_per_qubit) {
    if (!P || !vars_per_qubit || network < 0 || network >= (int32_t)P->hp.nets.size()) return QT_EINVAL;
    const qt::Network& net = P->hp.nets[network];
    for (size_t q = 0; q < net.wire_vars.size(); ++q) vars_per_qubit[q] = net.wire_vars[q];
    return QT_OK;
}

int qt_energy(qt_plan_t P, const double* gammas, const double* betas, double* edge_zz, double* energy,
              void* cuda_stream) {
    if (!P) return QT_EINVAL;
    if (!P->parts.empty()) return run_passes(P, gammas, betas, edge_zz, energy, nullptr, nullptr, cuda_stream, false);
    if (P->hp.graphs.size() != 1) return QT_ESTATE;
    return run_eval(P, gammas, betas, cuda_stream, edge_zz, energy, false);
}

int qt_energy_batch(qt_plan_t P, const double* gammas, const double* betas, double* energies, double* edge_zz,
                    void* cuda_stream) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P) return QT_EINVAL;
    return run_eval(P, gammas, betas, cuda_stream, edge_zz, energies, true);
}

// The reverse sweep's launches, in order: zero the atomically updated
// cotangents and the angle sums, seed the roots, then every level from the
// roots down (its operand-count classes forked onto the side streams and
// joined again), then the final scaling.
cudaError_t enqueue_sweep(qt_plan_t P, cudaStream_t s) {
    const qt::HostPlan& hp = P->hp;
    const int G = (int)hp.graphs.size(), p = hp.cfg.p;
    cudaError_t e = qt::launch_zero_ranges(P->dtype, P->d_arena, P->d_zero, P->n_zero, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_grad, 0, sizeof(double) * 2 * G * p, s);
    if (e == cudaSuccess)
        e = qt::launch_seed_roots(P->dtype, P->de, (int)hp.nets.size(), P->db.cot_delta, P->db.dleaf_delta, P->d_grad,
                                  p, P->db.net_graph, s);
    for (int lv = hp.n_levels - 1; lv >= 0 && e == cudaSuccess; --lv) {
        int used = 0;
        e = cudaEventRecord(P->bwd_ev[0], s);  // the level's fork point
        for (int cls = 0; cls < qt::kBwdClasses && e == cudaSuccess; ++cls) {
            const uint32_t i0 = hp.bwd_level_begin[qt::kBwdClasses * lv + cls];
            const uint32_t i1 = hp.bwd_level_begin[qt::kBwdClasses * lv + cls + 1];
            if (i1 == i0) continue;
            qt::DevBwd db = P->db;
            db.task_bucket += i0;
            db.task_tile += i0;
            db.n_tasks = i1 - i0;
            cudaStream_t t = used == 0 ? s : P->side[used - 1];
            if (used > 0) e = cudaStreamWaitEvent(t, P->bwd_ev[0], 0);
            if (e == cudaSuccess) e = qt::launch_backward(P->dtype, cls, db, t);
            ++used;
        }
        for (int j = 1; j < used && e == cudaSuccess; ++j) {  // join
            e = cudaEventRecord(P->bwd_ev[j], P->side[j - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P->bwd_ev[j], 0);
        }
    }
    double* d_dg = P->d_grad + 2 * G * p;
    if (e == cudaSuccess) e = qt::launch_grad_final(P->d_grad, G, p, d_dg, d_dg + G * p, s);
    return e;
}

int ensure_bwd_graph(qt_plan_t P) {
    if (P->bwd_exec) return QT_OK;
    QT_CUDA(qt::prepare_backward(P->dtype));
    for (auto& st : P->side)
        if (!st) QT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto& ev : P->bwd_ev)
        if (!ev) QT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    QT_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_sweep(P, P->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (e == cudaSuccess) e = ce;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->bwd_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        P->bwd_exec = nullptr;
        return cuda_fail(e, "reverse sweep graph", __LINE__);
    }
    return QT_OK;
}

int qt_energy_grad(qt_plan_t P, const double* gammas, const double* betas, double* energy, double* dE_dgamma,
                   double* dE_dbeta, void* cuda_stream) {
    if (!P) return QT_EINVAL;
    if (!P->parts.empty()) {
        if (!gammas || !betas) return QT_EINVAL;
        return run_passes(P, gammas, betas, nullptr, energy, dE_dgamma, dE_dbeta, cuda_stream, true);
    }
    if (P->host_only || !P->hp.cfg.with_grad) return QT_ESTATE;
    const qt::HostPlan& hp = P->hp;
    const int G = (int)hp.graphs.size(), p = hp.cfg.p;
    // forward pass: every result stays in the arena
    int rc = run_eval(P, gammas, betas, cuda_stream, nullptr, nullptr, true);
    if (rc != QT_OK) return rc;
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : P->stream;
    // reverse sweep
    rc = ensure_bwd_graph(P);
    if (rc != QT_OK) return rc;
    QT_CUDA(cudaGraphLaunch(P->bwd_exec, s));
    double* d_dg = P->d_grad + 2 * G * p;
    double* d_db = d_dg + G * p;
    QT_CUDA(cudaMemcpyAsync(P->h_err, &P->dp.ctl->error, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    bool host_out = false;
    if (energy) {
        QT_CUDA(cudaMemcpyAsync(energy, P->de.energies, sizeof(double) * G, cudaMemcpyDefault, s));
        host_out |= is_host_ptr(energy);
    }
    if (dE_dgamma) {
        QT_CUDA(cudaMemcpyAsync(dE_dgamma, d_dg, sizeof(double) * G * p, cudaMemcpyDefault, s));
        host_out |= is_host_ptr(dE_dgamma);
    }
    if (dE_dbeta) {
        QT_CUDA(cudaMemcpyAsync(dE_dbeta, d_db, sizeof(double) * G * p, cudaMemcpyDefault, s));
        host_out |= is_host_ptr(dE_dbeta);
    }
    if (host_out || !cuda_stream) {
        QT_CUDA(cudaStreamSynchronize(s));
        P->err_pending = false;
        return check_error_word(P);
    }
    return QT_OK;
}

int qt_last_imag(qt_plan_t P, double* edge_imag) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P || !edge_imag) return QT_EINVAL;
    if (P->host_only) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    QT_CUDA(cudaStreamSynchronize(P->stream));
    QT_CUDA(cudaDeviceSynchronize());
    QT_CUDA(cudaMemcpy(edge_imag, P->de.zz_imag, sizeof(double) * P->hp.nets.size(), cudaMemcpyDeviceToHost));
    return QT_OK;
}

int qt_sync(qt_plan_t P, void* cuda_stream) {
    if (P && !P->parts.empty()) {
        for (auto& part : P->parts) {
            const int rc = qt_sync(part.get(), cuda_stream);
            if (rc != QT_OK) return rc;
        }
        return QT_OK;
    }
    if (!P) return QT_EINVAL;
    if (P->host_only) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    QT_CUDA(cudaStreamSynchronize(cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : P->stream));
    P->err_pending = false;
    return check_error_word(P);
}

int qt_kernel_time(qt_plan_t P, double* avg_ms, int64_t* launches, int32_t reset) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P) return QT_EINVAL;
    if (P->host_only) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    for (int s = 0; s < kRing; ++s) harvest_slot(P, s);
    if (avg_ms) *avg_ms = P->timed ? P->time_ms / (double)P->timed : 0.0;
    if (launches) *launches = P->timed;
    if (reset) {
        P->time_ms = 0;
        P->timed = 0;
    }
    return QT_OK;
}

int qt_bucket_time(qt_plan_t P, int64_t bucket, int32_t reps, double* avg_ms, double* bytes) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P || !avg_ms || reps < 1 || bucket < 0 || bucket >= (int64_t)P->hp.buckets.size()) return QT_EINVAL;
    if (P->host_only || P->sched != QT_SCHED_PERSISTENT) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    const qt::DBucket& d = P->hp.buckets[bucket];
    // the bucket alone: its tiles spread evenly over every warp of the grid
    const uint32_t gt =
        qt::lone_group_tiles(d.n_tasks, (uint32_t)P->grid * (qt::kPersistentThreads / 32), d.group_tiles);
    std::vector<qt::DRun> groups;
    for (uint32_t c = 0; c < d.n_tasks; c += gt)
        groups.push_back(qt::DRun{(uint32_t)bucket, c, std::min(gt, d.n_tasks - c), d.op_begin, 0, 0, 0, d.n_ops});
    qt::DRun* d_groups = nullptr;
    QT_CUDA(cudaMalloc((void**)&d_groups, groups.size() * sizeof(qt::DRun)));
    cudaError_t e = cudaMemcpy(d_groups, groups.data(), groups.size() * sizeof(qt::DRun), cudaMemcpyHostToDevice);
    qt::DevPlan dp = P->dp;
    dp.runs = d_groups;
    dp.n_static = dp.n_groups = (uint32_t)groups.size();
    dp.isolated = 1;
    cudaEvent_t e0 = P->cap_ev[0], e1 = P->cap_ev[1];
    float total = 0;
    // isolated groups have no producers and notify no consumer: of the
    // counters only the control word (the claim position) needs resetting
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_counters, 0, P->counters_bytes, P->stream);
    if (e == cudaSuccess) e = qt::launch_persistent(P->dtype, P->grid, dp, P->stream);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaMemsetAsync(P->d_counters, 0, sizeof(qt::DControl), P->stream);
        if (e == cudaSuccess) e = qt::launch_persistent(P->dtype, P->grid, dp, P->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&total, e0, e1);
    int32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, &P->dp.ctl->error, sizeof(err), cudaMemcpyDeviceToHost);
    cudaFree(d_groups);
    if (e != cudaSuccess) return cuda_fail(e, "qt_bucket_time", __LINE__);
    if (err != 0) return err;
    *avg_ms = total / reps;
    if (bytes) {
        double b = (double)(1ull << qt::result_bits(d));
        for (uint32_t o = d.op_begin; o < d.op_begin + d.n_ops; ++o) b += std::ldexp(1.0, P->hp.op_rank[o]);
        *bytes = b * (double)P->esize;
    }
    return QT_OK;
}

int qt_trace_counters(qt_plan_t P, uint64_t* totals, int64_t* n_warps) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P || !totals) return QT_EINVAL;
    if (P->host_only || !P->trace) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    QT_CUDA(cudaDeviceSynchronize());
    const size_t nw = (size_t)P->grid * (qt::kPersistentThreads / 32);
    std::vector<uint64_t> buf(nw * qt::kTraceSlots);
    QT_CUDA(cudaMemcpy(buf.data(), P->d_trace, buf.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < qt::kTraceSlots; ++i) totals[i] = 0;
    for (size_t w = 0; w < nw; ++w)
        for (int i = 0; i < qt::kTraceSlots; ++i) totals[i] += buf[w * qt::kTraceSlots + i];
    if (n_warps) *n_warps = (int64_t)nw;
    return QT_OK;
}

int qt_trace_bucket_times(qt_plan_t P, uint64_t* start_end_ns) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P || !start_end_ns) return QT_EINVAL;
    if (P->host_only || !P->trace) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    QT_CUDA(cudaDeviceSynchronize());
    QT_CUDA(cudaMemcpy(start_end_ns, P->d_btimes, P->hp.buckets.size() * 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return QT_OK;
}

int qt_debug_stall_bucket(qt_plan_t P, int64_t bucket) {
    if (P && !P->parts.empty()) return QT_ESTATE;  // a plan that runs in passes: energy and gradient only
    if (!P || bucket < 0 || bucket >= (int64_t)P->hp.buckets.size()) return QT_EINVAL;
    if (P->host_only) return QT_ESTATE;
    QT_CUDA(cudaSetDevice(P->device));
    // the bucket then never counts as complete, so its consumer never starts:
    // one tile more than will ever be written, both in the bucket's own count
    // (the ready queue publishes on it) and in its consumer's operand (the
    // static order's dependency check reads that)
    qt::DBucket d = P->hp.buckets[bucket];
    d.n_tasks += 1;
    QT_CUDA(cudaMemcpy((void*)(P->dp.buckets + bucket), &d, sizeof(d), cudaMemcpyHostToDevice));
    for (size_t i = 0; i < P->hp.operands.size(); ++i)
        if (P->hp.op_src[i] == (int32_t)bucket) {
            qt::DOperand o = P->hp.operands[i];
            o.src_tiles += 1;
            QT_CUDA(cudaMemcpy((void*)(P->dp.ops + i), &o, sizeof(o), cudaMemcpyHostToDevice));
        }
    return QT_OK;
}

void qt_plan_free(qt_plan_t P) {
    if (!P) return;
    if (!P->host_only) {
        cudaSetDevice(P->device);
        if (P->stream) cudaStreamSynchronize(P->stream);
    }
    delete P;
}

const char* qt_error_string(int code) {
    switch (code) {
        case QT_OK: return "ok";
        case QT_EINVAL: return "invalid argument";
        case QT_EWIDTH: return "bucket wider than max_width";
        case QT_ENOMEM: return "out of memory";
        case QT_ECUDA: return "CUDA runtime error";
        case QT_ETIMEOUT: return "kernel dependency wait timed out";
        case QT_EBOUNDS: return "operand index out of bounds";
        case QT_ESTATE: return "call not valid for this plan";
        default: return "unknown error";
    }
}

const char* qt_version(void) { return "qtgb 0.1 sm_103a"; }

const char* qt_last_error_detail(void) { return g_detail; }

}  // extern "C"

// ---------------------------------------------------------------------------
// qt_energy_noalloc: the persistent-kernel evaluation with every piece of
// device memory it needs (plan arrays, counters, intermediate results) taken
// from one statically sized array, so the call itself allocates nothing.

// The only device memory qt_energy_noalloc uses. In host code this name
// denotes a host-side stand-in, not the device array: host code gets the
// device address from cudaGetSymbolAddress (per device, in scratch_setup).
static __device__ __align__(256) unsigned char g_noalloc_scratch[QT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxScratchDevices = 64;
struct ScratchDevice {
    void* base = nullptr;  // device address of g_noalloc_scratch on this device
    int grid[2] = {0, 0};  // persistent grid for complex64 / complex128 (0: not yet set up)
};
std::mutex g_scratch_mu;
ScratchDevice g_scratch_dev[kMaxScratchDevices];

size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of every piece inside the scratch array.
struct ScratchLayout {
    size_t buckets, ops, runs, net_first_root, root_bucket, graph_first_net, unit_list, net_first_factor, factor,
        graph_owned;
    size_t counters, counters_bytes, ctl_bytes, cnt_bytes;
    size_t angles, out, arena, total;
};

ScratchLayout scratch_layout(const qt::HostPlan& hp, size_t esize) {
    ScratchLayout L{};
    size_t at = 0;
    auto take = [&at](size_t bytes) {
        const size_t off = at;
        at += pad256(bytes);
        return off;
    };
    const size_t nb = hp.buckets.size();
    L.buckets = take(nb * sizeof(qt::DBucket));
    L.ops = take((hp.operands.size() + qt::kMaxOps) * sizeof(qt::DOperand));
    L.runs = take(hp.runs.size() * sizeof(qt::DRun));
    L.net_first_root = take(hp.net_first_root.size() * sizeof(uint32_t));
    L.root_bucket = take(hp.root_bucket.size() * sizeof(uint32_t));
    L.graph_first_net = take(hp.graph_first_net.size() * sizeof(int32_t));
    L.unit_list = take(hp.unit_prog.size() * sizeof(qt::URec));
    L.net_first_factor = take(hp.net_first_factor.size() * sizeof(uint32_t));
    L.factor = take(hp.factor.size() * sizeof(uint64_t));
    L.graph_owned = take(hp.graph_owned.size() * sizeof(int32_t));
    L.ctl_bytes = 256;
    L.cnt_bytes = pad256(2 * nb * sizeof(uint32_t));
    L.counters_bytes = L.ctl_bytes + L.cnt_bytes + (size_t)(hp.n_groups - hp.runs.size()) * sizeof(qt::DSlot);
    L.counters = take(L.counters_bytes);
    L.angles = take(sizeof(double) * 2 * hp.graphs.size() * hp.cfg.p);
    L.out = take(sizeof(double) * (2 * hp.nets.size() + hp.graphs.size()));
    L.arena = take((size_t)hp.total_elems * esize);
    L.total = at;
    return L;
}

// Once per device (under a lock, with that device current): the device
// address of the scratch array, and the persistent kernel's shared-memory
// attribute and grid for `dtype`.
int scratch_setup(int dtype, void** base, int* grid) {
    int dev = 0;
    QT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxScratchDevices) {
        std::snprintf(g_detail, sizeof(g_detail), "device %d is beyond the %d devices qt_energy_noalloc supports", dev,
                      kMaxScratchDevices);
        return QT_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchDevice& sd = g_scratch_dev[dev];
    if (!sd.base) {
        void* ptr = nullptr;
        QT_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        sd.base = ptr;
    }
    const int di = dtype == QT_C128 ? 1 : 0;
    if (!sd.grid[di]) {
        int sms = 0;
        QT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int per_sm = qt::persistent_blocks_per_sm(dtype);
        if (per_sm <= 0) {
            std::snprintf(g_detail, sizeof(g_detail), "persistent kernel does not fit an SM (%zu bytes of shared memory)",
                          qt::persistent_smem_bytes(dtype));
            return QT_ECUDA;
        }
        sd.grid[di] = sms * per_sm;
    }
    *base = sd.base;
    *grid = sd.grid[di];
    return QT_OK;
}

}  // namespace

extern "C" {

int qt_energy_noalloc(qt_plan_t P, const double* gammas, const double* betas, double* energies, double* edge_zz,
                      void* cuda_stream) {
    if (!P || !gammas || !betas) return QT_EINVAL;
    const qt::HostPlan& hp = P->hp;
    const ScratchLayout L = scratch_layout(hp, P->esize);
    if (L.total > (size_t)QT_NOALLOC_SCRATCH_BYTES) {
        std::snprintf(g_detail, sizeof(g_detail),
                      "qt_energy_noalloc: the plan needs %zu bytes of device scratch; the static scratch holds %zu",
                      L.total, (size_t)QT_NOALLOC_SCRATCH_BYTES);
        return QT_ENOMEM;
    }
    void* base_v = nullptr;
    int grid = 0;
    int rc = scratch_setup(P->dtype, &base_v, &grid);
    if (rc != QT_OK) return rc;
    char* base = static_cast<char*>(base_v);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int G = (int)hp.graphs.size(), p = hp.cfg.p;
    const size_t n_nets = hp.nets.size();

    // plan arrays (the operand array keeps kMaxOps zeroed entries past its end)
    QT_CUDA(cudaMemcpyAsync(base + L.buckets, hp.buckets.data(), bytes_of(hp.buckets), cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.ops, hp.operands.data(), bytes_of(hp.operands), cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemsetAsync(base + L.ops + bytes_of(hp.operands), 0, qt::kMaxOps * sizeof(qt::DOperand), s));
    if (!hp.runs.empty())
        QT_CUDA(cudaMemcpyAsync(base + L.runs, hp.runs.data(), bytes_of(hp.runs), cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.net_first_root, hp.net_first_root.data(), bytes_of(hp.net_first_root),
                            cudaMemcpyHostToDevice, s));
    if (!hp.root_bucket.empty())
        QT_CUDA(cudaMemcpyAsync(base + L.root_bucket, hp.root_bucket.data(), bytes_of(hp.root_bucket),
                                cudaMemcpyHostToDevice, s));
    static_assert(sizeof(int) == sizeof(int32_t), "graph_first_net is copied as int32");
    QT_CUDA(cudaMemcpyAsync(base + L.graph_first_net, hp.graph_first_net.data(), bytes_of(hp.graph_first_net),
                            cudaMemcpyHostToDevice, s));
    if (!hp.unit_prog.empty())
        QT_CUDA(cudaMemcpyAsync(base + L.unit_list, hp.unit_prog.data(), bytes_of(hp.unit_prog),
                                cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.net_first_factor, hp.net_first_factor.data(), bytes_of(hp.net_first_factor),
                            cudaMemcpyHostToDevice, s));
    if (!hp.factor.empty())
        QT_CUDA(cudaMemcpyAsync(base + L.factor, hp.factor.data(), bytes_of(hp.factor), cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.graph_owned, hp.graph_owned.data(), bytes_of(hp.graph_owned),
                            cudaMemcpyHostToDevice, s));
    // the array keeps the previous call's contents: counters and the queue start at zero
    QT_CUDA(cudaMemsetAsync(base + L.counters, 0, L.counters_bytes, s));
    double* d_angles = reinterpret_cast<double*>(base + L.angles);
    QT_CUDA(cudaMemcpyAsync(d_angles, gammas, sizeof(double) * G * p, cudaMemcpyDefault, s));
    QT_CUDA(cudaMemcpyAsync(d_angles + (size_t)G * p, betas, sizeof(double) * G * p, cudaMemcpyDefault, s));

    qt::DevPlan dp{};
    dp.buckets = reinterpret_cast<const qt::DBucket*>(base + L.buckets);
    dp.ops = reinterpret_cast<const qt::DOperand*>(base + L.ops);
    dp.runs = reinterpret_cast<const qt::DRun*>(base + L.runs);
    dp.unit_prog = reinterpret_cast<const qt::URec*>(base + L.unit_list);
    dp.has_units = hp.n_units > 0 ? 1u : 0u;
    dp.n_static = (uint32_t)hp.runs.size();
    dp.n_groups = (uint32_t)hp.n_groups;
    dp.n_buckets = (uint32_t)hp.buckets.size();
    char* cbase = base + L.counters;
    dp.ctl = reinterpret_cast<qt::DControl*>(cbase);
    dp.tiles_done = reinterpret_cast<uint32_t*>(cbase + L.ctl_bytes);
    dp.prod_done = dp.tiles_done + hp.buckets.size();
    dp.slots = reinterpret_cast<qt::DSlot*>(cbase + L.ctl_bytes + L.cnt_bytes);
    dp.arena = base + L.arena;
    dp.spin_limit = P->spin_limit;

    qt::DevEpilogue de{};
    de.buckets = dp.buckets;
    de.net_first_root = reinterpret_cast<const uint32_t*>(base + L.net_first_root);
    de.root_bucket = reinterpret_cast<const uint32_t*>(base + L.root_bucket);
    de.graph_first_net = reinterpret_cast<const int32_t*>(base + L.graph_first_net);
    de.net_first_factor = reinterpret_cast<const uint32_t*>(base + L.net_first_factor);
    de.factor = reinterpret_cast<const uint64_t*>(base + L.factor);
    de.graph_owned = reinterpret_cast<const int32_t*>(base + L.graph_owned);
    de.n_graphs = G;
    de.arena = dp.arena;
    double* d_out = reinterpret_cast<double*>(base + L.out);
    de.zz = d_out;
    de.zz_imag = d_out + n_nets;
    de.energies = d_out + 2 * n_nets;

    QT_CUDA(qt::launch_leaf_fill(P->dtype, d_angles, G, p, dp.arena, hp.dleaf_off, s));
    QT_CUDA(qt::launch_persistent(P->dtype, grid, dp, s));
    QT_CUDA(qt::launch_epilogue(P->dtype, de, s));
    int32_t err[2] = {0, 0};
    QT_CUDA(cudaMemcpyAsync(err, &dp.ctl->error, sizeof(err), cudaMemcpyDeviceToHost, s));
    QT_CUDA(cudaStreamSynchronize(s));
    if (err[0] != 0) return err[0];
    if (energies) QT_CUDA(cudaMemcpyAsync(energies, de.energies, sizeof(double) * G, cudaMemcpyDefault, s));
    if (edge_zz) QT_CUDA(cudaMemcpyAsync(edge_zz, de.zz, sizeof(double) * n_nets, cudaMemcpyDefault, s));
    QT_CUDA(cudaStreamSynchronize(s));
    return QT_OK;
}

}  // extern "C"
